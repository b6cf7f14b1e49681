// tuner.cu -- the autotuner: search over pass splits, block shapes and twiddle
// modes for one transform size, timed on the device with CUDA events.
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/zkntt.h"
#include "kernels.h"
#include "tuner.h"

namespace zkntt {
namespace {

std::mutex g_mu;
bool g_loaded = false;
std::map<std::tuple<std::string, int, int, int>, TuneEntry> g_cache;

std::string gpu_name() {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    std::string n = prop.name;
    for (char &c : n)
        if (c == '"' || c == '\n') c = '_';
    return n;
}

const char *cache_path() {
    const char *p = getenv("ZKNTT_TUNE_CACHE");
    return (p && *p) ? p : nullptr;
}

// schedules shipped with the library: "zkntt_tuned.jsonl" in the directory of
// the shared library itself (same format as the user cache)
std::string bundled_path() {
    Dl_info info;
    if (dladdr(reinterpret_cast<void *>(&tuner_lookup), &info) == 0 || !info.dli_fname) return "";
    std::string so = info.dli_fname;
    size_t slash = so.rfind('/');
    return (slash == std::string::npos ? std::string(".") : so.substr(0, slash)) + "/zkntt_tuned.jsonl";
}

// one entry per line:
// {"gpu":"NAME","field":F,"log_n":L,"dir":D,"passes":P,"digits":[a,b,c,d],"log_cols":[a,b,c,d],"mode":M,"ilp":I,"ms":T}
void load_file(const char *path);

void load_locked() {
    if (g_loaded) return;
    g_loaded = true;
    const std::string b = bundled_path();
    if (!b.empty()) load_file(b.c_str());
    if (const char *path = cache_path()) load_file(path);  // user entries override
}

void load_file(const char *path) {
    FILE *f = fopen(path, "r");
    if (!f) return;
    char line[1024];
    while (fgets(line, sizeof line, f)) {
        char name[256] = {0};
        int field, L, dir;
        TuneEntry e;
        const char *q = strstr(line, "\"gpu\":\"");
        if (!q) continue;
        q += 7;
        const char *end = strchr(q, '"');
        if (!end || end - q >= 255) continue;
        memcpy(name, q, end - q);
        int n = sscanf(end + 1,
                       ",\"field\":%d,\"log_n\":%d,\"dir\":%d,\"passes\":%d,\"digits\":[%d,%d,%d,%d],"
                       "\"log_cols\":[%d,%d,%d,%d],\"mode\":%d,\"ilp\":%d,\"ms\":%lf",
                       &field, &L, &dir, &e.passes, &e.digits[0], &e.digits[1], &e.digits[2],
                       &e.digits[3], &e.log_cols[0], &e.log_cols[1], &e.log_cols[2], &e.log_cols[3],
                       &e.mode, &e.ilp, &e.ms);
        if (n == 15) g_cache[{std::string(name), field, L, dir}] = e;
    }
    fclose(f);
}

}  // namespace

bool tuner_lookup(int field, int log_n, int dir, TuneEntry *out) {
    std::string name = gpu_name();
    std::lock_guard<std::mutex> lk(g_mu);
    load_locked();
    auto it = g_cache.find({name, field, log_n, dir});
    if (it == g_cache.end()) return false;
    *out = it->second;
    return true;
}

void tuner_store(int field, int log_n, int dir, const TuneEntry &e) {
    std::string name = gpu_name();
    std::lock_guard<std::mutex> lk(g_mu);
    load_locked();
    g_cache[{name, field, log_n, dir}] = e;
    const char *path = cache_path();
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f,
            "{\"gpu\":\"%s\",\"field\":%d,\"log_n\":%d,\"dir\":%d,\"passes\":%d,\"digits\":[%d,%d,%d,%d],"
            "\"log_cols\":[%d,%d,%d,%d],\"mode\":%d,\"ilp\":%d,\"ms\":%.6f}\n",
            name.c_str(), field, log_n, dir, e.passes, e.digits[0], e.digits[1], e.digits[2],
            e.digits[3], e.log_cols[0], e.log_cols[1], e.log_cols[2], e.log_cols[3], e.mode, e.ilp,
            e.ms);
    fclose(f);
}

namespace {

// digit splits of L into p parts in [lo, MAX_DIGIT_BITS], near-balanced
void splits(int L, int p, std::vector<std::vector<int>> &out) {
    std::vector<int> cur(p, 0);
    std::function<void(int, int)> rec = [&](int i, int left) {
        if (i == p - 1) {
            if (left < 3 || left > MAX_DIGIT_BITS) return;
            cur[i] = left;
            int mx = *std::max_element(cur.begin(), cur.end());
            int mn = *std::min_element(cur.begin(), cur.end());
            if (mx - mn <= 3) out.push_back(cur);
            return;
        }
        for (int k = 3; k <= MAX_DIGIT_BITS && k < left; k++) {
            cur[i] = k;
            rec(i + 1, left - k);
        }
    };
    if (p == 1) {
        if (L <= MAX_DIGIT_BITS) out.push_back({L});
        return;
    }
    rec(0, L);
}

}  // namespace
}  // namespace zkntt

using namespace zkntt;

// The tuning input: uniform field elements (SplitMix64 words, rejection-sampled
// below r) rather than zeros, so the candidates are timed on the bit activity --
// and hence the power draw and sustained clock -- of real data.  A block of
// 2^16 elements is drawn on the host and repeated over the vector by
// device-to-device copies.
static zkntt_status fill_uniform(zkntt_field field, void *d, size_t n) {
    uint32_t r[8];
    int s = 0;
    zkntt_status st = zkntt_field_info(field, r, nullptr, &s);
    if (st != ZKNTT_OK) return st;
    int top = 255;
    while (top > 0 && !((r[top / 32] >> (top % 32)) & 1u)) top--;
    const size_t blk = std::min<size_t>(n, size_t(1) << 16);
    std::vector<uint32_t> h(blk * 8);
    uint64_t state = 0x5eed0fba5e11ull;
    auto next = [&state]() {
        uint64_t z = (state += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    for (size_t e = 0; e < blk; e++) {
        uint32_t x[8];
        for (;;) {
            for (int w = 0; w < 4; w++) {
                const uint64_t v = next();
                x[2 * w] = uint32_t(v);
                x[2 * w + 1] = uint32_t(v >> 32);
            }
            for (int b = top + 1; b < 256; b++) x[b / 32] &= ~(1u << (b % 32));
            int i = 7;
            while (i > 0 && x[i] == r[i]) i--;
            if (x[i] < r[i]) break;  // below r: accept
        }
        for (int k = 0; k < 8; k++) h[e * 8 + k] = x[k];
    }
    if (cudaMemcpy(d, h.data(), blk * 32, cudaMemcpyHostToDevice) != cudaSuccess) return ZKNTT_ECUDA;
    for (size_t done = blk; done < n; done *= 2) {
        const size_t c = std::min(done, n - done);
        if (cudaMemcpy(static_cast<char *>(d) + done * 32, d, c * 32, cudaMemcpyDeviceToDevice) !=
            cudaSuccess)
            return ZKNTT_ECUDA;
    }
    return ZKNTT_OK;
}

// Candidate schedules for one digit split: both twiddle modes, variants
// 1 .. TUNED_VARIANTS (6 and 7 were measured slower than 3 and 1 at every size
// and stay explicit options), column caps 3..1.
static void split_candidates(int log_n, const std::vector<int> &d, std::vector<zkntt_plan_options> &out) {
    const int p = int(d.size());
    for (int mode : {ZKNTT_TWIDDLE_PRECOMP, ZKNTT_TWIDDLE_OTF})
        for (int ilp = 1; ilp <= TUNED_VARIANTS; ilp++)
            for (int cap = 3; cap >= 1; cap--) {
                if (p == 1 && (mode == ZKNTT_TWIDDLE_OTF || cap != 3)) continue;
                zkntt_plan_options o;
                memset(&o, 0, sizeof o);
                o.twiddle_mode = mode;
                o.ilp = ilp;
                o.num_passes = p;
                int hi = 0;
                for (int i = 0; i < p; i++) {
                    o.digit_bits[i] = d[i];
                    int span = (i == p - 1) ? hi : (log_n - hi - d[i]);
                    int lc = std::min({cap, MAX_DIGIT_BITS - d[i], span});
                    o.cols_per_cta[i] = 1 << std::max(0, lc);
                    hi += d[i];
                }
                out.push_back(o);
            }
}

extern "C" zkntt_status zkntt_tune(zkntt_field field, int log_n, zkntt_dir dir, int max_candidates,
                                   zkntt_tune_result *best) {
    if (field < 0 || field >= NUM_FIELDS) return ZKNTT_EINVAL;
    if (log_n < 1 || log_n > 28 || max_candidates < 1) return ZKNTT_EINVAL;
    std::vector<std::vector<int>> all_splits;
    int pmin = (log_n + MAX_DIGIT_BITS - 1) / MAX_DIGIT_BITS;
    for (int p = pmin; p <= std::min(4, pmin + 1); p++) splits(log_n, p, all_splits);

    const size_t bytes = size_t(32) << log_n;
    void *in = nullptr, *out = nullptr, *scr = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    zkntt_status result = ZKNTT_OK;
    if (cudaMalloc(&in, bytes) != cudaSuccess || cudaMalloc(&out, bytes) != cudaSuccess ||
        cudaMalloc(&scr, bytes) != cudaSuccess || cudaStreamCreate(&s) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        result = ZKNTT_ENOMEM;
    }
    if (result == ZKNTT_OK) result = fill_uniform(field, in, size_t(1) << log_n);

    // median time of one schedule over `samples` samples; < 0 if it cannot run
    auto time_one = [&](const zkntt_plan_options &o, int samples) -> double {
        zkntt_plan plan = nullptr;
        if (zkntt_plan_create_ex(&plan, field, log_n, dir, nullptr, &o) != ZKNTT_OK) return -1;
        bool ok = true;
        for (int w = 0; w < 2 && ok; w++)
            ok = zkntt_execute_scratch(plan, in, out, scr, bytes, s) == ZKNTT_OK;
        // each sample times `reps` back-to-back executions (at least ~1 ms of
        // work), so small transforms are timed at their throughput rather than
        // at one launch's latency and the events' resolution
        int reps = 1;
        if (ok) {
            cudaEventRecord(e0, s);
            ok = zkntt_execute_scratch(plan, in, out, scr, bytes, s) == ZKNTT_OK;
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float one = 0;
            cudaEventElapsedTime(&one, e0, e1);
            reps = std::max(1, std::min(200, int(1.0f / std::max(one, 1e-3f)) + 1));
        }
        std::vector<float> t;
        for (int r = 0; r < samples && ok; r++) {
            cudaEventRecord(e0, s);
            for (int k = 0; k < reps && ok; k++)
                ok = zkntt_execute_scratch(plan, in, out, scr, bytes, s) == ZKNTT_OK;
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            t.push_back(ms / float(reps));
        }
        zkntt_plan_destroy(plan);
        if (!ok || t.empty()) return -1;
        std::sort(t.begin(), t.end());
        return t[t.size() / 2];
    };

    // Stage 1: every digit split with one representative schedule (precomputed
    // tables; for small sizes the variant with twice the threads and wider
    // tiles, else the 64-register variant with 2-column tiles).
    std::vector<std::pair<double, size_t>> ranked;
    for (size_t si = 0; si < all_splits.size() && result == ZKNTT_OK; si++) {
        std::vector<zkntt_plan_options> c;
        split_candidates(log_n, all_splits[si], c);
        const int want_ilp = log_n <= 16 ? 5 : 3, want_cap = log_n <= 16 ? 2 : 1;
        zkntt_plan_options rep = c.front();
        for (const auto &o : c) {
            int cap = 0;
            for (int i = 0; i < o.num_passes; i++) cap = std::max(cap, o.cols_per_cta[i]);
            if (o.twiddle_mode == ZKNTT_TWIDDLE_PRECOMP && o.ilp == want_ilp &&
                cap <= (1 << want_cap)) {
                rep = o;
                break;
            }
        }
        const double ms = all_splits.size() > 1 ? time_one(rep, 3) : 0.0;
        if (ms >= 0) ranked.push_back({ms, si});
    }
    std::stable_sort(ranked.begin(), ranked.end());
    // Stage 2: every schedule of the best three splits, best split first,
    // within the candidate budget.
    std::vector<zkntt_plan_options> cands;
    for (size_t k = 0; k < ranked.size() && k < 3; k++)
        split_candidates(log_n, all_splits[ranked[k].second], cands);
    if (int(cands.size()) > max_candidates) cands.resize(max_candidates);

    TuneEntry bestE;
    double best_ms = 1e30;
    for (size_t ci = 0; ci < cands.size() && result == ZKNTT_OK; ci++) {
        const double med = time_one(cands[ci], 5);
        if (med < 0) continue;
        if (med < best_ms) {
            best_ms = med;
            bestE.passes = cands[ci].num_passes;
            for (int i = 0; i < 4; i++) {
                bestE.digits[i] = cands[ci].digit_bits[i];
                int c = cands[ci].cols_per_cta[i], l = 0;
                while (c > 1) {
                    c >>= 1;
                    l++;
                }
                bestE.log_cols[i] = i < bestE.passes ? l : -1;
            }
            bestE.mode = cands[ci].twiddle_mode;
            bestE.ilp = cands[ci].ilp;
            bestE.ms = med;
        }
    }
    if (in) cudaFree(in);
    if (out) cudaFree(out);
    if (scr) cudaFree(scr);
    if (s) cudaStreamDestroy(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (result != ZKNTT_OK) return result;
    if (best_ms >= 1e30) return ZKNTT_ECUDA;
    tuner_store(field, log_n, dir, bestE);
    if (best) {
        best->num_passes = bestE.passes;
        for (int i = 0; i < 4; i++) {
            best->digit_bits[i] = bestE.digits[i];
            best->cols_per_cta[i] = bestE.log_cols[i] >= 0 ? (1 << bestE.log_cols[i]) : 0;
        }
        best->twiddle_mode = bestE.mode;
        best->ilp = bestE.ilp;
        best->ms = float(bestE.ms);
    }
    return ZKNTT_OK;
}
