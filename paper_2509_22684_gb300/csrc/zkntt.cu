// zkntt.cu -- host runtime and C ABI of the transform library (include/zkntt.h).
//
// Host side of the method:
//  * field constants derived at start-up from the modulus limbs the kernels are
//    compiled with (R mod r, R^2 mod r, r', roots of unity), using a
//    separated-operand-scanning Montgomery product on 8 x 32-bit limbs;
//  * the planner: the digit split of log_n into passes (four-step / six-step,
//    each digit <= 11 bits so a sub-transform fits one block's shared memory)
//    and the columns per block;
//  * resident twiddle tables per plan, generated on the device;
//  * stream-ordered execution, the persistent batch launch and the Groth16 H
//    sequence (Fig. 2 of the paper).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/zkntt.h"
#include "aux_kernels.cuh"
#include "batch.cuh"
#include "field.cuh"
#include "kernels.h"
#include "ntt_pass.cuh"
#include "tuner.h"

using namespace zkntt;

namespace {

thread_local int g_last_cuda_error = 0;

zkntt_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return ZKNTT_OK;
    g_last_cuda_error = int(e);
    cudaGetLastError();  // clear the sticky-free error state of the runtime
    if (e == cudaErrorMemoryAllocation) return ZKNTT_ENOMEM;
    return ZKNTT_ECUDA;
}

#define ZK_CHECK(call)                              \
    do {                                            \
        zkntt_status _s = from_cuda(call);          \
        if (_s != ZKNTT_OK) return _s;              \
    } while (0)

// ---------------------------------------------------------------------------
// host field arithmetic (Montgomery form, R = 2^256, 8 x 32-bit limbs)
using E8 = std::array<uint32_t, 8>;

struct HostField {
    E8 p{};
    uint32_t rp = 0;   // -p^-1 mod 2^32
    E8 one{};          // R mod p
    E8 r2{};           // R^2 mod p
    uint32_t gen = 0;  // multiplicative generator (plain)
    int s = 0;         // 2-adicity
    E8 gen_m{};        // generator, Montgomery form
    E8 wmax{};         // primitive 2^s-th root, Montgomery form
    bool ok = false;
};

bool geq8(const E8 &a, const E8 &b) {
    for (int i = 7; i >= 0; i--)
        if (a[i] != b[i]) return a[i] > b[i];
    return true;
}

uint32_t add8(E8 &r, const E8 &a, const E8 &b) {
    uint64_t c = 0;
    for (int i = 0; i < 8; i++) {
        c += uint64_t(a[i]) + b[i];
        r[i] = uint32_t(c);
        c >>= 32;
    }
    return uint32_t(c);
}

uint32_t sub8(E8 &r, const E8 &a, const E8 &b) {
    int64_t c = 0;
    for (int i = 0; i < 8; i++) {
        c += int64_t(a[i]) - int64_t(b[i]);
        r[i] = uint32_t(c);
        c >>= 32;  // arithmetic: 0 or -1
    }
    return c ? 1u : 0u;
}

// SOS: full 512-bit product, then eight word-wise reductions
E8 hmul(const HostField &F, const E8 &a, const E8 &b) {
    uint32_t t[17] = {0};
    for (int i = 0; i < 8; i++) {
        uint64_t carry = 0;
        for (int j = 0; j < 8; j++) {
            uint64_t v = uint64_t(a[i]) * b[j] + t[i + j] + carry;
            t[i + j] = uint32_t(v);
            carry = v >> 32;
        }
        t[i + 8] = uint32_t(carry);
    }
    for (int i = 0; i < 8; i++) {
        uint32_t m = t[i] * F.rp;
        uint64_t carry = 0;
        for (int j = 0; j < 8; j++) {
            uint64_t v = uint64_t(m) * F.p[j] + t[i + j] + carry;
            t[i + j] = uint32_t(v);
            carry = v >> 32;
        }
        for (int k = i + 8; carry && k < 17; k++) {
            uint64_t v = uint64_t(t[k]) + carry;
            t[k] = uint32_t(v);
            carry = v >> 32;
        }
    }
    E8 r;
    for (int i = 0; i < 8; i++) r[i] = t[8 + i];
    if (t[16] || geq8(r, F.p)) sub8(r, r, F.p);
    return r;
}

E8 hsub(const HostField &F, const E8 &a, const E8 &b) {
    E8 r;
    if (sub8(r, a, b)) add8(r, r, F.p);
    return r;
}

E8 hpow_words(const HostField &F, const E8 &base, const uint32_t *exp_words, int nwords) {
    E8 acc = F.one, b = base;
    for (int i = 0; i < 32 * nwords; i++) {
        if ((exp_words[i / 32] >> (i % 32)) & 1u) acc = hmul(F, acc, b);
        b = hmul(F, b, b);
    }
    return acc;
}

E8 hpow(const HostField &F, const E8 &base, uint64_t e) {
    uint32_t w[2] = {uint32_t(e), uint32_t(e >> 32)};
    return hpow_words(F, base, w, 2);
}

E8 hinv(const HostField &F, const E8 &a) {
    E8 e, two{};
    two[0] = 2;
    sub8(e, F.p, two);  // Fermat: a^(p-2)
    return hpow_words(F, a, e.data(), 8);
}

E8 hto_mont(const HostField &F, uint64_t v) {
    E8 x{};
    x[0] = uint32_t(v);
    x[1] = uint32_t(v >> 32);
    return hmul(F, x, F.r2);
}

bool is_zero(const E8 &a) {
    for (uint32_t v : a)
        if (v) return false;
    return true;
}

template <class FD>
HostField make_field(uint32_t gen) {
    HostField F;
    F.p = {FD::P0, FD::P1, FD::P2, FD::P3, FD::P4, FD::P5, FD::P6, FD::P7};
    // -p^-1 mod 2^32 by Newton's iteration on the low limb
    uint32_t inv = 1;
    for (int i = 0; i < 5; i++) inv *= 2u - F.p[0] * inv;
    F.rp = 0u - inv;
    // R mod p: 2^256 - p (two's complement), then subtract p until below p
    E8 zero{}, x;
    sub8(x, zero, F.p);
    while (geq8(x, F.p)) sub8(x, x, F.p);
    F.one = x;
    // R^2 mod p: double R mod p 256 times
    for (int i = 0; i < 256; i++) {
        E8 y;
        uint32_t c = add8(y, x, x);
        if (c || geq8(y, F.p)) sub8(y, y, F.p);
        x = y;
    }
    F.r2 = x;
    F.gen = gen;
    E8 pm1, onep{};
    onep[0] = 1;
    sub8(pm1, F.p, onep);
    int s = 0;
    while (((pm1[s / 32] >> (s % 32)) & 1u) == 0) s++;
    F.s = s;
    E8 e{};
    for (int i = 0; i + s < 256; i++)
        if ((pm1[(i + s) / 32] >> ((i + s) % 32)) & 1u) e[i / 32] |= 1u << (i % 32);
    F.gen_m = hto_mont(F, gen);
    F.wmax = hpow_words(F, F.gen_m, e.data(), 8);
    // self-check: the root has order exactly 2^s and r' matches the kernels'
    E8 w = F.wmax;
    for (int i = 0; i < s - 1; i++) w = hmul(F, w, w);
    E8 minus_one = hsub(F, E8{}, F.one);
    F.ok = (w == minus_one) && (F.rp == FD::RP) && (hmul(F, w, w) == F.one);
    return F;
}

const HostField &host_field(int id) {
    static const HostField bls = make_field<FrBLS12_381>(7);
    static const HostField bn = make_field<FrBN254>(5);
    static const HostField bls377 = make_field<FrBLS12_377>(22);
    return id == 0 ? bls : id == 1 ? bn : bls377;
}

const FieldKernels &field_kernels(int id) {
    return id == 0 ? kernels_bls12_381() : id == 1 ? kernels_bn254() : kernels_bls12_377();
}

uint32_t rev_bits(uint32_t x, int bits) {
    uint32_t r = 0;
    for (int i = 0; i < bits; i++) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}

// ---------------------------------------------------------------------------
// Device-side error words: one per stream that ran a persistent batch launch,
// taken from a fixed slab allocated at device set-up (so a launch never
// allocates one, and a capture never sees an allocation for it).  Streams
// beyond the slab share its last word.
constexpr int STATUS_WORDS = 1024;

struct DeviceInfo {
    int sms = 0;
    // batch kernel occupancy per field for 2^(10+i) bytes of shared memory
    int batch_blocks_per_sm[NUM_FIELDS][8] = {};
    bool init = false;
    uint32_t *status_slab = nullptr;             // STATUS_WORDS sticky error words
    std::map<uintptr_t, int> status_of_stream;   // stream handle -> word index
    // the library's own stream-ordered pool for scratch (the device's default
    // pool, which other code in the process shares, is left as it is)
    cudaMemPool_t pool = nullptr;
};

std::mutex g_dev_mu;
std::map<int, DeviceInfo> g_devices;

zkntt_status device_info(DeviceInfo **out) {
    int dev = 0;
    ZK_CHECK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_dev_mu);
    DeviceInfo &d = g_devices[dev];
    if (!d.init) {
        ZK_CHECK(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
        for (int f = 0; f < NUM_FIELDS; f++)
            for (int ilp = 1; ilp <= NUM_VARIANTS; ilp++)
                ZK_CHECK(cudaFuncSetAttribute(field_kernels(f).pass[ilp],
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (ilp == 6 ? 128 : 64) * 1024));
        for (int f = 0; f < NUM_FIELDS; f++) {
            ZK_CHECK(cudaFuncSetAttribute(batch_kernel_ptr(f),
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));
            for (int i = 0; i < 7; i++) {
                ZK_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &d.batch_blocks_per_sm[f][i], batch_kernel_ptr(f), BATCH_THREADS,
                    size_t(1024) << i));
                d.batch_blocks_per_sm[f][i] = std::max(d.batch_blocks_per_sm[f][i], 1);
            }
        }
        ZK_CHECK(cudaMalloc(&d.status_slab, STATUS_WORDS * sizeof(uint32_t)));
        ZK_CHECK(cudaMemset(d.status_slab, 0, STATUS_WORDS * sizeof(uint32_t)));
        // A private pool: freed scratch stays in it between executions (no
        // release threshold), and a block freed on one stream is never handed
        // to another stream behind an inserted wait -- calls on different
        // streams (the host-buffer path, concurrent batches) stay independent;
        // the pool grows instead.
        cudaMemPoolProps props;
        memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        ZK_CHECK(cudaMemPoolCreate(&d.pool, &props));
        uint64_t thr = UINT64_MAX;
        ZK_CHECK(cudaMemPoolSetAttribute(d.pool, cudaMemPoolAttrReleaseThreshold, &thr));
        int no = 0;
        ZK_CHECK(cudaMemPoolSetAttribute(d.pool, cudaMemPoolReuseAllowInternalDependencies, &no));
        d.init = true;
    }
    *out = &d;
    return ZKNTT_OK;
}

// the error word of stream s on the current device (assigned on first use)
uint32_t *status_word(DeviceInfo *d, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_dev_mu);
    const uintptr_t key = reinterpret_cast<uintptr_t>(s);
    auto it = d->status_of_stream.find(key);
    int idx;
    if (it != d->status_of_stream.end()) {
        idx = it->second;
    } else {
        idx = std::min<int>(int(d->status_of_stream.size()), STATUS_WORDS - 1);
        d->status_of_stream[key] = idx;
    }
    return d->status_slab + idx;
}

// Stream-ordered scratch from the library's pool.  Inside a stream capture the
// allocation becomes a graph allocation node (cudaMallocAsync), which draws on
// graph-owned memory rather than on any pool's.
zkntt_status pool_alloc(void **p, size_t bytes, cudaStream_t s) {
    DeviceInfo *dev;
    zkntt_status st = device_info(&dev);
    if (st != ZKNTT_OK) return st;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    ZK_CHECK(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone) return from_cuda(cudaMallocAsync(p, bytes, s));
    return from_cuda(cudaMallocFromPoolAsync(p, bytes, dev->pool, s));
}

}  // namespace

// ---------------------------------------------------------------------------
struct PassPlan {
    int K = 0, lo_bits = 0, hi_bits = 0, log_cols = 0, ilp = 1;
    int threads = 0, grid = 0;
    uint32_t num_tiles = 0;
    size_t smem = 0;
    uint4 *w_stage = nullptr, *tw = nullptr, *w_hi = nullptr, *w_lo = nullptr, *fl = nullptr,
          *fd = nullptr;
    int tw_bits = 0, split_bits = 0;
};

struct zkntt_plan_s {
    int field = 0, log_n = 0, dir = 0, coset = 0, mode = 0, passes = 0, device = 0;
    E8 shift{};
    PassPlan ps[4];
    uint4 *pre = nullptr, *post = nullptr;
    std::vector<void *> allocs;
    size_t table_bytes = 0;
    int extra_scalar = 0;  // 1: an extra constant folded into the output scale
    E8 extra{};
};

namespace {

zkntt_status dalloc(zkntt_plan_s *P, uint4 **out, size_t elems) {
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, elems * 32);
    if (e != cudaSuccess) return from_cuda(e);
    P->allocs.push_back(p);
    P->table_bytes += elems * 32;
    *out = static_cast<uint4 *>(p);
    return ZKNTT_OK;
}

zkntt_status upload(zkntt_plan_s *P, uint4 **out, const std::vector<E8> &v) {
    zkntt_status s = dalloc(P, out, v.size());
    if (s != ZKNTT_OK) return s;
    return from_cuda(cudaMemcpy(*out, v.data(), v.size() * 32, cudaMemcpyHostToDevice));
}

void free_plan(zkntt_plan_s *P) {
    for (void *p : P->allocs) cudaFree(p);
    P->allocs.clear();
    delete P;
}

std::vector<E8> powers(const HostField &F, const E8 &base, size_t count, const E8 &scale) {
    std::vector<E8> v(count);
    E8 cur = scale;
    for (size_t i = 0; i < count; i++) {
        v[i] = cur;
        cur = hmul(F, cur, base);
    }
    return v;
}

int grid_for(size_t work, int per_block, int sms) {
    size_t g = (work + per_block - 1) / per_block;
    size_t cap = size_t(sms) * 8;
    return int(std::max<size_t>(1, std::min(g, cap)));
}

// default digit split and columns (the tuner may override both)
void default_digits(int L, int *passes, int k[4]) {
    if (L <= MAX_DIGIT_BITS) {
        *passes = 1;
        k[0] = L;
    } else if (L <= 2 * MAX_DIGIT_BITS) {
        *passes = 2;
        k[0] = (L + 1) / 2;
        k[1] = L - k[0];
    } else {
        *passes = 3;
        k[0] = (L + 2) / 3;
        k[1] = (L - k[0] + 1) / 2;
        k[2] = L - k[0] - k[1];
    }
}

// interleaved butterflies per thread in the stage loop (planner default)
constexpr int DEFAULT_ILP = 1;

int default_log_cols(int K, int span_bits) {
    // tile of C x 2^K elements, at most 2^11 elements (64 KiB); C <= 8 and
    // C <= the number of columns the pass has (2^span_bits)
    int lc = std::min(3, MAX_DIGIT_BITS - K);
    return std::max(0, std::min(lc, span_bits));
}

zkntt_status launch_gen_twiddle(int field, uint4 *out, int K, int lo_bits, const uint4 *w_hi,
                                const uint4 *w_lo, int split, const uint4 *fl, const uint4 *fd,
                                int sms) {
    const FieldKernels &kk = field_kernels(field);
    uint32_t uK = K, ulo = lo_bits, usp = split;
    void *args[] = {&out, &uK, &ulo, &w_hi, &w_lo, &usp, &fl, &fd};
    size_t total = size_t(1) << (K + lo_bits);
    return from_cuda(cudaLaunchKernel(kk.gen_twiddle, dim3(grid_for(total, 256, sms)), dim3(256),
                                      args, 0, nullptr));
}

zkntt_status launch_gen_powers(int field, uint4 *out, uint32_t count, const uint4 *hi,
                               const uint4 *lo, int split, int sms) {
    const FieldKernels &kk = field_kernels(field);
    uint32_t usp = split;
    void *args[] = {&out, &count, &hi, &lo, &usp};
    return from_cuda(cudaLaunchKernel(kk.gen_powers, dim3(grid_for(count, 256, sms)), dim3(256),
                                      args, 0, nullptr));
}

// split tables for base^e, e < 2^bits: lo[x] = base^x * scale, hi[y] = base^(y 2^split)
zkntt_status split_tables(zkntt_plan_s *P, const HostField &F, const E8 &base, int bits,
                          const E8 &scale, uint4 **hi, uint4 **lo, int *split) {
    int sp = (bits + 1) / 2;
    *split = sp;
    zkntt_status s = upload(P, lo, powers(F, base, size_t(1) << sp, scale));
    if (s != ZKNTT_OK) return s;
    E8 step = hpow(F, base, uint64_t(1) << sp);
    return upload(P, hi, powers(F, step, size_t(1) << (bits - sp), F.one));
}

zkntt_status build_plan(zkntt_plan_s *P, const zkntt_plan_options *opts) {
    const HostField &F = host_field(P->field);
    if (!F.ok) return ZKNTT_ECUDA;
    DeviceInfo *dev;
    zkntt_status st = device_info(&dev);
    if (st != ZKNTT_OK) return st;
    ZK_CHECK(cudaGetDevice(&P->device));
    const int L = P->log_n;
    const bool inverse = P->dir == ZKNTT_INVERSE;
    const bool coset = P->coset != 0;

    // ---- schedule
    int k[4] = {0, 0, 0, 0}, cols[4] = {-1, -1, -1, -1};
    int mode = ZKNTT_TWIDDLE_AUTO;
    int ilp = DEFAULT_ILP;
    default_digits(L, &P->passes, k);
    // tuned schedules (shipped with the library or from ZKNTT_TUNE_CACHE) are
    // used unless the caller opts out (use_tuner < 0) or forces a split
    const bool explicit_split = opts && opts->num_passes > 0;
    if (!explicit_split && !(opts && opts->use_tuner < 0)) {
        TuneEntry te;
        if (tuner_lookup(P->field, L, P->dir, &te)) {
            P->passes = te.passes;
            for (int i = 0; i < 4; i++) {
                k[i] = te.digits[i];
                cols[i] = te.log_cols[i];
            }
            mode = te.mode;
            if (te.ilp >= 1 && te.ilp <= NUM_VARIANTS) ilp = te.ilp;
        }
    }
    if (opts && opts->num_passes > 0) {
        if (opts->num_passes > 4) return ZKNTT_EINVAL;
        int sum = 0;
        for (int i = 0; i < opts->num_passes; i++) {
            if (opts->digit_bits[i] < 1 || opts->digit_bits[i] > MAX_DIGIT_BITS) return ZKNTT_EINVAL;
            sum += opts->digit_bits[i];
        }
        if (sum != L) return ZKNTT_EINVAL;
        P->passes = opts->num_passes;
        for (int i = 0; i < 4; i++) {
            k[i] = i < P->passes ? opts->digit_bits[i] : 0;
            cols[i] = -1;
        }
    }
    if (opts && opts->twiddle_mode) mode = opts->twiddle_mode;
    if (opts && opts->ilp) {
        if (opts->ilp < 1 || opts->ilp > NUM_VARIANTS) return ZKNTT_EINVAL;
        ilp = opts->ilp;
    }
    const int p = P->passes;
    if (mode == ZKNTT_TWIDDLE_AUTO && p > 1) {
        // Precomputed inter-pass tables (pass i: 2^(K_i + lo_bits_i) entries;
        // pass 1's is n entries) unless they would not fit beside the input,
        // output and scratch vectors in the device memory free now: then the
        // split-exponent tables (about 2 sqrt(n_i) entries) instead.
        size_t fr = 0, tot = 0;
        ZK_CHECK(cudaMemGetInfo(&fr, &tot));
        size_t tables = 0;
        for (int i = 0, hb = 0; i < p - 1; i++) {
            hb += k[i];
            tables += size_t(32) << (L - hb + k[i]);
        }
        const size_t vectors = 3 * (size_t(32) << L);
        if (tables + vectors > fr) mode = ZKNTT_TWIDDLE_OTF;
    }
    if (mode != ZKNTT_TWIDDLE_OTF) mode = ZKNTT_TWIDDLE_PRECOMP;
    P->mode = mode;

    // ---- scalars
    E8 w = hpow(F, F.wmax, uint64_t(1) << (F.s - L));  // w_n
    if (inverse) w = hinv(F, w);
    const E8 ninv = hinv(F, hto_mont(F, uint64_t(1) << L));
    const E8 g = P->shift;
    const E8 ginv = coset ? hinv(F, g) : F.one;
    E8 out_scale = inverse ? ninv : F.one;  // folded into pass 0 (p > 1) or post (p == 1)
    if (P->extra_scalar) out_scale = hmul(F, out_scale, P->extra);

    int hi_bits = 0;
    for (int i = 0; i < p; i++) {
        PassPlan &ps = P->ps[i];
        ps.K = k[i];
        ps.hi_bits = hi_bits;
        ps.lo_bits = L - hi_bits - k[i];
        hi_bits += k[i];
        const bool last = (i == p - 1);
        const int span = last ? ps.hi_bits : ps.lo_bits;
        int lc = default_log_cols(ps.K, span);
        // keep at least four tiles per SM so the persistent grid fills the GPU
        while (lc > 0 && ((L - ps.K - lc) < 0 || (uint64_t(1) << (L - ps.K - lc)) < uint64_t(4) * dev->sms))
            lc--;
        if (opts && opts->cols_per_cta[i] > 0) {
            int c = opts->cols_per_cta[i], l = 0;
            while ((1 << l) < c) l++;
            if ((1 << l) != c || l > 3 || l > span || (ps.K + l) > MAX_DIGIT_BITS) return ZKNTT_EINVAL;
            lc = l;
        } else if (cols[i] >= 0 && cols[i] <= std::min(3, span) && ps.K + cols[i] <= MAX_DIGIT_BITS) {
            lc = cols[i];
        }
        ps.log_cols = lc;
        ps.ilp = ilp;
        ps.num_tiles = last ? (uint32_t(1) << (ps.hi_bits - lc))
                            : (uint32_t(1) << (ps.hi_bits + ps.lo_bits - lc));
        ps.threads = int(pass_threads_for(uint32_t(ps.K), uint32_t(lc), ilp));
        ps.smem = size_t(32) << (ps.K + lc);
        if (ilp == 6) ps.smem *= 2;  // two tile buffers
        int nb = 0;
        ZK_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &nb, field_kernels(P->field).pass[ps.ilp], ps.threads, ps.smem));
        nb = std::max(nb, 1);
        ps.grid = int(std::min<uint64_t>(ps.num_tiles, uint64_t(nb) * dev->sms));

        // sub-transform twiddles, stage-major: stage s holds w_N^(j 2^s) for
        // j < N / 2^(s+1) at offset N - 2^(K-s)
        const E8 wn_i = hpow(F, w, uint64_t(1) << ps.hi_bits);          // root of order n_i
        const E8 wN = hpow(F, wn_i, uint64_t(1) << ps.lo_bits);         // root of order N_i
        {
            const size_t N = size_t(1) << ps.K;
            std::vector<E8> all = powers(F, wN, std::max<size_t>(1, N / 2), F.one);
            std::vector<E8> st_tab;
            st_tab.reserve(N);
            for (int sidx = 0; sidx < ps.K; sidx++)
                for (size_t j = 0; j < (N >> (sidx + 1)); j++) st_tab.push_back(all[j << sidx]);
            st = upload(P, &ps.w_stage, st_tab);
            if (st != ZKNTT_OK) return st;
        }

        // per-row coset-inverse factor for this digit: g^-(rev(d) * 2^hi_bits)
        std::vector<E8> phi;
        if (coset && inverse) {
            const E8 gstep = hpow(F, ginv, uint64_t(1) << ps.hi_bits);
            std::vector<E8> pw = powers(F, gstep, size_t(1) << ps.K, F.one);
            phi.resize(pw.size());
            for (uint32_t d = 0; d < pw.size(); d++) phi[d] = pw[rev_bits(d, ps.K)];
        }
        if (!last) {
            ps.tw_bits = ps.K + ps.lo_bits;
            const E8 scale = (i == 0) ? out_scale : F.one;
            st = split_tables(P, F, wn_i, ps.tw_bits, scale, &ps.w_hi, &ps.w_lo, &ps.split_bits);
            if (st != ZKNTT_OK) return st;
            if (i == 0 && coset && !inverse) {
                // column factor g^lo, lo < 2^lo_bits
                uint4 *ghi, *glo;
                int gsp;
                st = split_tables(P, F, g, ps.lo_bits, F.one, &ghi, &glo, &gsp);
                if (st != ZKNTT_OK) return st;
                st = dalloc(P, &ps.fl, size_t(1) << ps.lo_bits);
                if (st != ZKNTT_OK) return st;
                st = launch_gen_powers(P->field, ps.fl, uint32_t(1) << ps.lo_bits, ghi, glo, gsp, dev->sms);
                if (st != ZKNTT_OK) return st;
            }
            if (!phi.empty()) {
                st = upload(P, &ps.fd, phi);
                if (st != ZKNTT_OK) return st;
            }
            if (mode == ZKNTT_TWIDDLE_PRECOMP) {
                st = dalloc(P, &ps.tw, size_t(1) << (ps.K + ps.lo_bits));
                if (st != ZKNTT_OK) return st;
                st = launch_gen_twiddle(P->field, ps.tw, ps.K, ps.lo_bits, ps.w_hi, ps.w_lo,
                                        ps.split_bits, ps.fl, ps.fd, dev->sms);
                if (st != ZKNTT_OK) return st;
            }
        } else {
            // output scale on the last pass: coset-inverse row factor, and for a
            // single pass also n^-1 and any extra constant
            const bool need_scalar = (p == 1) && !(out_scale == F.one);
            if (!phi.empty() || need_scalar) {
                const size_t N = size_t(1) << ps.K;
                std::vector<E8> q(N, p == 1 ? out_scale : F.one);
                if (!phi.empty())
                    for (size_t d = 0; d < N; d++) q[d] = hmul(F, q[d], phi[d]);
                st = upload(P, &P->post, q);
                if (st != ZKNTT_OK) return st;
            }
        }
        if (i == 0 && coset && !inverse) {
            // input row factor (g^(2^lo_bits))^d
            const E8 gs = hpow(F, g, uint64_t(1) << ps.lo_bits);
            st = upload(P, &P->pre, powers(F, gs, size_t(1) << ps.K, F.one));
            if (st != ZKNTT_OK) return st;
        }
    }
    // tables are generated on the legacy stream; make them visible to all streams
    return from_cuda(cudaDeviceSynchronize());
}

PassArgs pass_args(const zkntt_plan_s *P, int i, const void *in, void *out) {
    const PassPlan &ps = P->ps[i];
    PassArgs a;
    memset(&a, 0, sizeof a);
    a.in = static_cast<const uint4 *>(in);
    a.out = static_cast<uint4 *>(out);
    a.w_stage = ps.w_stage;
    a.K = uint32_t(ps.K);
    a.tw = ps.tw;
    a.w_hi = ps.w_hi;
    a.w_lo = ps.w_lo;
    a.fl = ps.fl;
    a.fd = ps.fd;
    a.pre = (i == 0) ? P->pre : nullptr;
    a.post = (i == P->passes - 1) ? P->post : nullptr;
    a.pw_b = nullptr;
    a.pw_c = nullptr;
    a.lo_bits = ps.lo_bits;
    a.hi_bits = ps.hi_bits;
    a.tw_bits = ps.tw_bits;
    a.split_bits = ps.split_bits;
    a.log_cols = ps.log_cols;
    a.last = (i == P->passes - 1);
    a.otf = (P->mode == ZKNTT_TWIDDLE_OTF);
    a.num_tiles = ps.num_tiles;
    return a;
}

bool valid_field(int field) { return field >= 0 && field < NUM_FIELDS; }

bool bad_ptr(const void *p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 31u); }

bool partial_overlap(const void *a, const void *b, size_t bytes) {
    uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    if (x == y) return false;
    return x < y + bytes && y < x + bytes;
}

// [a, a + na) and [b, b + nb) share at least one byte
bool ranges_overlap(const void *a, size_t na, const void *b, size_t nb) {
    uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}

// A plan's tables live on the device it was created on: executing it while
// another device is current would pair them with that device's stream and
// scratch.  EINVAL (nothing enqueued) when the current device differs;
// ECUDA when the current device cannot be read.
zkntt_status check_plan_device(const zkntt_plan_s *P) {
    int cur = 0;
    ZK_CHECK(cudaGetDevice(&cur));
    return cur == P->device ? ZKNTT_OK : ZKNTT_EINVAL;
}

zkntt_status run_passes(const zkntt_plan_s *P, const void *in, void *out, void *scratch,
                        cudaStream_t s) {
    const FieldKernels &kk = field_kernels(P->field);
    for (int i = 0; i < P->passes; i++) {
        const void *src = (i == 0) ? in : scratch;
        void *dst = (i == P->passes - 1) ? out : scratch;
        PassArgs a = pass_args(P, i, src, dst);
        void *args[] = {&a};
        const PassPlan &ps = P->ps[i];
        if (i == 0 || ps.ilp == 2) {
            // the first pass is ordered after all earlier work on the stream
            // (which may write `in`); plans of the two-butterfly variant keep
            // plain launches throughout (measured 1-7% slower as dependents)
            ZK_CHECK(cudaLaunchKernel(kk.pass[ps.ilp], dim3(ps.grid), dim3(ps.threads), args, ps.smem, s));
            continue;
        }
        // later passes depend only on the pass before: a programmatic
        // dependent launch overlaps their launch with its tail (the kernel
        // waits for the previous pass's completion before any memory access)
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(ps.grid);
        cfg.blockDim = dim3(ps.threads);
        cfg.dynamicSmemBytes = ps.smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        ZK_CHECK(cudaLaunchKernelExC(&cfg, kk.pass[ps.ilp], args));
    }
    return ZKNTT_OK;
}

// Scratch for zkntt_execute_noalloc: a file-scope device array, so that entry
// point never allocates.  In host code `g_noalloc_scratch` only stands for the
// symbol; its device address comes from cudaGetSymbolAddress, looked up once
// per device (with that device current) and kept in a fixed table.
static __device__ __align__(256) unsigned char g_noalloc_scratch[ZKNTT_NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// (called with the plan's device current: check_plan_device has passed)
zkntt_status noalloc_scratch(int dev, void **out) {
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return ZKNTT_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        ZK_CHECK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return ZKNTT_OK;
}

size_t scratch_bytes_of(const zkntt_plan_s *P) {
    return P->passes > 1 ? (size_t(32) << P->log_n) : 0;
}

zkntt_status create_plan(zkntt_plan *out, zkntt_field field, int log_n, zkntt_dir dir,
                         const uint32_t *coset_shift, const zkntt_plan_options *opts,
                         const E8 *extra) {
    if (!out) return ZKNTT_EINVAL;
    if (!valid_field(field)) return ZKNTT_EINVAL;
    if (dir != ZKNTT_FORWARD && dir != ZKNTT_INVERSE) return ZKNTT_EINVAL;
    const HostField &F = host_field(field);
    if (log_n < 1 || log_n > F.s) return ZKNTT_EINVAL;
    // A transform of 2^33 or more elements needs at least 2 x 2^33 x 32 bytes
    // (the vector and its scratch, 512 GiB): more than any device holds.
    if (log_n > 32) return ZKNTT_ENOMEM;
    if (opts && (opts->twiddle_mode < 0 || opts->twiddle_mode > 2)) return ZKNTT_EINVAL;
    zkntt_plan_s *P = new (std::nothrow) zkntt_plan_s;
    if (!P) return ZKNTT_ENOMEM;
    P->field = field;
    P->log_n = log_n;
    P->dir = dir;
    if (coset_shift) {
        for (int i = 0; i < 8; i++) P->shift[i] = coset_shift[i];
        if (is_zero(P->shift) || geq8(P->shift, F.p)) {
            delete P;
            return ZKNTT_EINVAL;
        }
        P->coset = 1;
    }
    if (extra) {
        P->extra_scalar = 1;
        P->extra = *extra;
    }
    zkntt_status s = build_plan(P, opts);
    if (s != ZKNTT_OK) {
        free_plan(P);
        return s;
    }
    *out = P;
    return ZKNTT_OK;
}

// ---------------------------------------------------------------------------
// batch construction
struct JobSpec {
    const zkntt_plan_s *plan;
    const void *in;
    void *out;
    void *scratch;
    const void *pw_b = nullptr, *pw_c = nullptr;  // fused pointwise on the first pass
    int level0 = 0;                               // level of the job's first pass
    int deps[3] = {-1, -1, -1};                   // jobs whose last pass must finish first
};

// One persistent launch over jobs of one field (job_ids: completion-word index
// of each job).
zkntt_status launch_batch_field(const std::vector<JobSpec> &jobs, cudaStream_t s,
                                unsigned long long timeout_ns, uint32_t *flags, uint32_t epoch,
                                const std::vector<uint32_t> &job_ids) {
    DeviceInfo *dev;
    zkntt_status st = device_info(&dev);
    if (st != ZKNTT_OK) return st;
    const int field = jobs.empty() ? 0 : jobs[0].plan->field;
    struct SegTmp {
        int job, pass, level;
    };
    std::vector<SegTmp> segs;
    for (int j = 0; j < int(jobs.size()); j++)
        for (int i = 0; i < jobs[j].plan->passes; i++) segs.push_back({j, i, jobs[j].level0 + i});
    std::stable_sort(segs.begin(), segs.end(),
                     [](const SegTmp &a, const SegTmp &b) { return a.level < b.level; });
    if (segs.size() > size_t(BATCH_MAX_SEGMENTS)) return ZKNTT_EUNSUPPORTED;
    std::map<std::pair<int, int>, int> index;
    for (int k = 0; k < int(segs.size()); k++) index[{segs[k].job, segs[k].pass}] = k;
    // The batch kernel runs 256 threads a block whatever the tile, so a tile of
    // C x 2^K elements with C x 2^K / 4 < 256 leaves threads idle.  Each pass
    // therefore takes the widest tile up to 2^BATCH_TILE_BITS elements (32 KiB,
    // so four blocks fit an SM's shared memory; an 11-bit digit keeps its
    // 2^11-element tile), narrowed toward the plan's own width only while the
    // pass has fewer tiles than one wave of resident blocks (the plan's tables
    // do not depend on the tile width).
    const uint64_t wave = uint64_t(dev->sms) * BATCH_WAVE_BLOCKS;
    auto batch_log_cols = [&](const zkntt_plan_s *P, int i) {
        const PassPlan &ps = P->ps[i];
        const int span = (i == P->passes - 1) ? ps.hi_bits : ps.lo_bits;
        const int cap = std::max(BATCH_TILE_BITS, ps.K);
        int lc = std::max(0, std::min({3, cap - ps.K, span}));
        while (lc > ps.log_cols && (uint64_t(1) << (P->log_n - ps.K - lc)) < wave) lc--;
        return lc;
    };
    auto batch_tiles = [&](const zkntt_plan_s *P, int i) {
        return uint32_t(1) << (P->log_n - P->ps[i].K - batch_log_cols(P, i));
    };

    BatchTable *tab = new (std::nothrow) BatchTable;
    if (!tab) return ZKNTT_ENOMEM;
    memset(tab, 0, sizeof *tab);
    tab->nseg = uint32_t(segs.size());
    tab->timeout_ns = timeout_ns;
    tab->flags = flags;
    tab->epoch = epoch;
    uint32_t item = 0;
    for (int k = 0; k < int(segs.size()); k++) {
        const JobSpec &J = jobs[segs[k].job];
        const zkntt_plan_s *P = J.plan;
        const int i = segs[k].pass;
        const void *src = (i == 0) ? J.in : J.scratch;
        void *dst = (i == P->passes - 1) ? J.out : J.scratch;
        BatchSeg &sg = tab->seg[k];
        sg.a = pass_args(P, i, src, dst);
        sg.a.log_cols = uint32_t(batch_log_cols(P, i));
        sg.a.num_tiles = batch_tiles(P, i);
        if (i == 0) {
            sg.a.pw_b = static_cast<const uint4 *>(J.pw_b);
            sg.a.pw_c = static_cast<const uint4 *>(J.pw_c);
        }
        sg.K = uint32_t(P->ps[i].K);
        sg.first_item = item;
        sg.ntiles = sg.a.num_tiles;
        sg.job = job_ids[segs[k].job];
        sg.signal = (flags && i == P->passes - 1) ? 1u : 0u;
        item += sg.a.num_tiles;
        for (int d = 0; d < 3; d++) {
            sg.dep[d] = -1;
            sg.dep_tiles[d] = 0;
        }
        if (i > 0) {
            int dk = index[{segs[k].job, i - 1}];
            sg.dep[0] = dk;
            sg.dep_tiles[0] = batch_tiles(jobs[segs[k].job].plan, i - 1);
        } else {
            for (int d = 0; d < 3; d++) {
                int dj = J.deps[d];
                if (dj < 0) continue;
                const zkntt_plan_s *DP = jobs[dj].plan;
                int dk = index[{dj, DP->passes - 1}];
                sg.dep[d] = dk;
                sg.dep_tiles[d] = batch_tiles(DP, DP->passes - 1);
            }
        }
        // every dependency must point to an earlier segment of the work list:
        // that ordering is what makes the persistent schedule deadlock-free
        for (int d = 0; d < 3; d++) {
            if (sg.dep[d] >= k) {
                delete tab;
                return ZKNTT_EINVAL;
            }
        }
    }
    tab->total_items = item;

    uint32_t *ctrl = nullptr;
    const size_t words = 2 + segs.size();
    st = pool_alloc(reinterpret_cast<void **>(&ctrl), words * 4, s);
    if (st != ZKNTT_OK) {
        delete tab;
        return st;
    }
    cudaError_t e = cudaMemsetAsync(ctrl, 0, words * 4, s);
    if (e == cudaSuccess) {
        // shared memory for the largest tile of the launch; occupancy comes from
        // the table built at device set-up (no query here: this path must stay
        // legal inside a stream capture)
        size_t smem = 1024;
        for (int k = 0; k < int(segs.size()); k++)
            smem = std::max(smem, size_t(32) << (tab->seg[k].a.K + tab->seg[k].a.log_cols));
        int si = 0;
        while ((size_t(1024) << si) < smem) si++;
        smem = size_t(1024) << si;
        // Resident blocks: at most what fits, and no more than splits the
        // widest dependency level into whole, equal waves -- a level of T tiles
        // over G blocks otherwise ends in a partial wave with most SMs idle
        // while the next level waits on it.
        uint32_t grid = std::min<uint32_t>(item, uint32_t(dev->batch_blocks_per_sm[field][si]) *
                                                     uint32_t(dev->sms));
        std::map<int, uint32_t> per_level;
        for (int k = 0; k < int(segs.size()); k++) per_level[segs[k].level] += tab->seg[k].ntiles;
        uint32_t widest = 0;
        for (const auto &kv : per_level) widest = std::max(widest, kv.second);
        if (grid > 0 && widest > 0) {
            const uint32_t waves = (widest + grid - 1) / grid;
            grid = std::min(grid, std::max<uint32_t>((widest + waves - 1) / waves,
                                                     std::min<uint32_t>(item, dev->sms)));
        }
        uint32_t *done = ctrl + 2;
        uint32_t *status = status_word(dev, s);
        void *args[] = {tab, &ctrl, &done, &status};
        if (e == cudaSuccess && grid > 0)
            e = cudaLaunchKernel(batch_kernel_ptr(field), dim3(grid), dim3(BATCH_THREADS), args,
                                 smem, s);
    }
    cudaError_t e2 = cudaFreeAsync(ctrl, s);
    delete tab;
    if (e != cudaSuccess) return from_cuda(e);
    return from_cuda(e2);
}

// Jobs of several fields run as one persistent launch per field, in order of
// each field's first job, on stream s (a dependency must stay within a field).
zkntt_status launch_batch(const std::vector<JobSpec> &jobs, cudaStream_t s,
                          unsigned long long timeout_ns, uint32_t *flags = nullptr,
                          uint32_t epoch = 0, const std::vector<uint32_t> *job_ids = nullptr) {
    std::vector<int> order;  // fields in order of first appearance
    for (const JobSpec &J : jobs)
        if (std::find(order.begin(), order.end(), J.plan->field) == order.end())
            order.push_back(J.plan->field);
    for (int f : order) {
        std::vector<JobSpec> sub;
        std::vector<uint32_t> ids;
        std::vector<int> local(jobs.size(), -1);
        for (int j = 0; j < int(jobs.size()); j++) {
            if (jobs[j].plan->field != f) continue;
            local[j] = int(sub.size());
            sub.push_back(jobs[j]);
            ids.push_back(job_ids ? (*job_ids)[j] : uint32_t(j));
        }
        for (JobSpec &J : sub)
            for (int d = 0; d < 3; d++) {
                if (J.deps[d] < 0) continue;
                if (local[J.deps[d]] < 0) return ZKNTT_EINVAL;  // dependency across fields
                J.deps[d] = local[J.deps[d]];
            }
        zkntt_status st = launch_batch_field(sub, s, timeout_ns, flags, epoch, ids);
        if (st != ZKNTT_OK) return st;
    }
    return ZKNTT_OK;
}

unsigned long long batch_timeout_ns() {
    const char *v = getenv("ZKNTT_BATCH_TIMEOUT_MS");
    unsigned long long ms = v ? strtoull(v, nullptr, 10) : 2000ull;
    if (ms == 0) ms = 2000;
    return ms * 1000000ull;
}

// Groth16 plans per (field, log_n).  Separate form (the sequence as stated):
// iNTT, coset NTT, coset iNTT.  Fused form: cosetNTT_g(iNTT(a)) is computed as
// NTT(cosetINTT_{g^-1}(a)) -- the inverse's output scale g^j then rides the
// store of its last pass and the forward transform needs no input scale -- and
// the final coset iNTT carries (g^n - 1)^-1 in its output scale.
struct G16Plans {
    zkntt_plan intt = nullptr, cntt = nullptr, cintt = nullptr, cintt_z = nullptr;
    zkntt_plan intt_gj = nullptr, ntt = nullptr;
    E8 zinv{};
};
std::mutex g_g16_mu;
std::map<std::pair<int, std::pair<int, int>>, G16Plans> g_g16;

zkntt_status g16_plans(int field, int log_n, G16Plans **out) {
    int dev = 0;
    ZK_CHECK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_g16_mu);
    G16Plans &G = g_g16[{dev, {field, log_n}}];
    if (!G.intt) {
        const HostField &F = host_field(field);
        const E8 g = F.gen_m;
        E8 gn = hpow(F, g, uint64_t(1) << log_n);
        G.zinv = hinv(F, hsub(F, gn, F.one));
        zkntt_status s;
        zkntt_plan_options o;
        memset(&o, 0, sizeof o);
        o.use_tuner = 1;
        if ((s = create_plan(&G.intt, zkntt_field(field), log_n, ZKNTT_INVERSE, nullptr, &o, nullptr)) ||
            (s = create_plan(&G.cntt, zkntt_field(field), log_n, ZKNTT_FORWARD, g.data(), &o, nullptr)) ||
            (s = create_plan(&G.cintt, zkntt_field(field), log_n, ZKNTT_INVERSE, g.data(), &o, nullptr)) ||
            (s = create_plan(&G.cintt_z, zkntt_field(field), log_n, ZKNTT_INVERSE, g.data(), &o, &G.zinv)) ||
            (s = create_plan(&G.intt_gj, zkntt_field(field), log_n, ZKNTT_INVERSE, hinv(F, g).data(), &o,
                             nullptr)) ||
            (s = create_plan(&G.ntt, zkntt_field(field), log_n, ZKNTT_FORWARD, nullptr, &o, nullptr))) {
            for (zkntt_plan *q : {&G.intt, &G.cntt, &G.cintt, &G.cintt_z, &G.intt_gj, &G.ntt})
                if (*q) {
                    free_plan(*q);
                    *q = nullptr;
                }
            return s;
        }
    }
    *out = &G;
    return ZKNTT_OK;
}

zkntt_status launch_pointwise(int field, const void *a, const void *b, const void *c,
                              const void *z_dev, void *h, size_t n, cudaStream_t s) {
    DeviceInfo *dev;
    zkntt_status st = device_info(&dev);
    if (st != ZKNTT_OK) return st;
    void *args[] = {&a, &b, &c, &z_dev, &h, &n};
    return from_cuda(cudaLaunchKernel(field_kernels(field).pointwise,
                                      dim3(grid_for(n, 256, dev->sms)), dim3(256), args, 0, s));
}

}  // namespace

// ===========================================================================
// C ABI
extern "C" {

zkntt_status zkntt_plan_create(zkntt_plan *out, zkntt_field field, int log_n, zkntt_dir dir,
                               const uint32_t *coset_shift) {
    return create_plan(out, field, log_n, dir, coset_shift, nullptr, nullptr);
}

zkntt_status zkntt_plan_create_ex(zkntt_plan *out, zkntt_field field, int log_n, zkntt_dir dir,
                                  const uint32_t *coset_shift, const zkntt_plan_options *opts) {
    return create_plan(out, field, log_n, dir, coset_shift, opts, nullptr);
}

zkntt_status zkntt_plan_destroy(zkntt_plan plan) {
    if (plan) free_plan(plan);
    return ZKNTT_OK;
}

zkntt_status zkntt_plan_scratch_bytes(zkntt_plan plan, size_t *bytes) {
    if (!plan || !bytes) return ZKNTT_EINVAL;
    *bytes = scratch_bytes_of(plan);
    return ZKNTT_OK;
}

zkntt_status zkntt_plan_describe(zkntt_plan plan, int *num_passes, int digit_bits[4],
                                 int *twiddle_mode, size_t *table_bytes) {
    if (!plan) return ZKNTT_EINVAL;
    if (num_passes) *num_passes = plan->passes;
    if (digit_bits)
        for (int i = 0; i < 4; i++) digit_bits[i] = i < plan->passes ? plan->ps[i].K : 0;
    if (twiddle_mode) *twiddle_mode = plan->mode;
    if (table_bytes) *table_bytes = plan->table_bytes;
    return ZKNTT_OK;
}

zkntt_status zkntt_execute_scratch(zkntt_plan plan, const void *d_in, void *d_out, void *d_scratch,
                                   size_t scratch_bytes, void *stream) {
    if (!plan || bad_ptr(d_in) || bad_ptr(d_out)) return ZKNTT_EINVAL;
    if (zkntt_status dc = check_plan_device(plan)) return dc;
    const size_t bytes = size_t(32) << plan->log_n;
    if (partial_overlap(d_in, d_out, bytes)) return ZKNTT_EINVAL;
    const size_t need = scratch_bytes_of(plan);
    if (need) {
        if (bad_ptr(d_scratch) || scratch_bytes < need) return ZKNTT_EINVAL;
        if (ranges_overlap(d_scratch, need, d_in, bytes) || ranges_overlap(d_scratch, need, d_out, bytes))
            return ZKNTT_EINVAL;
    }
    return run_passes(plan, d_in, d_out, d_scratch, static_cast<cudaStream_t>(stream));
}

zkntt_status zkntt_execute(zkntt_plan plan, const void *d_in, void *d_out, void *stream) {
    if (!plan || bad_ptr(d_in) || bad_ptr(d_out)) return ZKNTT_EINVAL;
    if (zkntt_status dc = check_plan_device(plan)) return dc;
    const size_t bytes = size_t(32) << plan->log_n;
    if (partial_overlap(d_in, d_out, bytes)) return ZKNTT_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t need = scratch_bytes_of(plan);
    void *scratch = nullptr;
    if (need) {
        zkntt_status sa = pool_alloc(&scratch, need, s);
        if (sa != ZKNTT_OK) return sa;
    }
    zkntt_status st = run_passes(plan, d_in, d_out, scratch, s);
    if (scratch) {
        zkntt_status st2 = from_cuda(cudaFreeAsync(scratch, s));
        if (st == ZKNTT_OK) st = st2;
    }
    return st;
}

zkntt_status zkntt_execute_host(zkntt_plan plan, const void *h_in, void *h_out, void *stream) {
    if (!plan || !h_in || !h_out) return ZKNTT_EINVAL;
    if (zkntt_status dc = check_plan_device(plan)) return dc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = size_t(32) << plan->log_n;
    const size_t need = scratch_bytes_of(plan);
    char *buf = nullptr;
    zkntt_status sa = pool_alloc(reinterpret_cast<void **>(&buf), bytes + need, s);
    if (sa != ZKNTT_OK) return sa;
    zkntt_status st = from_cuda(cudaMemcpyAsync(buf, h_in, bytes, cudaMemcpyHostToDevice, s));
    if (st == ZKNTT_OK) st = run_passes(plan, buf, buf, need ? buf + bytes : nullptr, s);
    if (st == ZKNTT_OK) st = from_cuda(cudaMemcpyAsync(h_out, buf, bytes, cudaMemcpyDeviceToHost, s));
    zkntt_status st2 = from_cuda(cudaFreeAsync(buf, s));
    return st != ZKNTT_OK ? st : st2;
}

zkntt_status zkntt_execute_host_buffered(zkntt_plan plan, const void *h_in, void *h_out,
                                         void *d_work, size_t work_bytes, void *stream) {
    if (!plan || !h_in || !h_out || bad_ptr(d_work)) return ZKNTT_EINVAL;
    if (zkntt_status dc = check_plan_device(plan)) return dc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = size_t(32) << plan->log_n;
    const size_t need = scratch_bytes_of(plan);
    if (work_bytes < bytes + need) return ZKNTT_EINVAL;
    char *buf = static_cast<char *>(d_work);
    zkntt_status st = from_cuda(cudaMemcpyAsync(buf, h_in, bytes, cudaMemcpyHostToDevice, s));
    if (st == ZKNTT_OK) st = run_passes(plan, buf, buf, need ? buf + bytes : nullptr, s);
    if (st == ZKNTT_OK) st = from_cuda(cudaMemcpyAsync(h_out, buf, bytes, cudaMemcpyDeviceToHost, s));
    return st;
}

zkntt_status zkntt_execute_noalloc(zkntt_plan plan, const void *d_in, void *d_out, void *stream) {
    if (!plan || bad_ptr(d_in) || bad_ptr(d_out)) return ZKNTT_EINVAL;
    if (zkntt_status dc = check_plan_device(plan)) return dc;
    const size_t bytes = size_t(32) << plan->log_n;
    if (partial_overlap(d_in, d_out, bytes)) return ZKNTT_EINVAL;
    const size_t need = scratch_bytes_of(plan);
    if (need > ZKNTT_NOALLOC_SCRATCH_BYTES) return ZKNTT_EINVAL;
    void *scratch = nullptr;
    if (need) {
        zkntt_status st = noalloc_scratch(plan->device, &scratch);
        if (st != ZKNTT_OK) return st;
    }
    return run_passes(plan, d_in, d_out, scratch, static_cast<cudaStream_t>(stream));
}

zkntt_status zkntt_execute_batch(const zkntt_plan *plans, const zkntt_io *ptrs, int count,
                                 void *stream) {
    if (count < 0 || (count > 0 && (!plans || !ptrs))) return ZKNTT_EINVAL;
    if (count == 0) return ZKNTT_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    size_t scratch_total = 0;
    for (int j = 0; j < count; j++) {
        if (!plans[j] || bad_ptr(ptrs[j].d_in) || bad_ptr(ptrs[j].d_out)) return ZKNTT_EINVAL;
        if (zkntt_status dc = check_plan_device(plans[j])) return dc;
        const size_t bytes = size_t(32) << plans[j]->log_n;
        if (partial_overlap(ptrs[j].d_in, ptrs[j].d_out, bytes)) return ZKNTT_EINVAL;
        scratch_total += scratch_bytes_of(plans[j]);
    }
    char *scratch = nullptr;
    if (scratch_total) {
        zkntt_status sa = pool_alloc(reinterpret_cast<void **>(&scratch), scratch_total, s);
        if (sa != ZKNTT_OK) return sa;
    }
    std::vector<JobSpec> jobs(count);
    size_t off = 0;
    for (int j = 0; j < count; j++) {
        jobs[j].plan = plans[j];
        jobs[j].in = ptrs[j].d_in;
        jobs[j].out = ptrs[j].d_out;
        jobs[j].scratch = scratch_bytes_of(plans[j]) ? scratch + off : nullptr;
        off += scratch_bytes_of(plans[j]);
    }
    // chunk so that each launch stays within the segment table
    zkntt_status st = ZKNTT_OK;
    size_t b = 0;
    while (b < jobs.size() && st == ZKNTT_OK) {
        size_t e = b, segs = 0;
        while (e < jobs.size() && segs + jobs[e].plan->passes <= size_t(BATCH_MAX_SEGMENTS)) {
            segs += jobs[e].plan->passes;
            e++;
        }
        std::vector<JobSpec> chunk(jobs.begin() + b, jobs.begin() + e);
        st = launch_batch(chunk, s, batch_timeout_ns());
        b = e;
    }
    if (scratch) {
        zkntt_status st2 = from_cuda(cudaFreeAsync(scratch, s));
        if (st == ZKNTT_OK) st = st2;
    }
    return st;
}

zkntt_status zkntt_execute_batch_signal(const zkntt_plan *plans, const zkntt_io *ptrs, int count,
                                        uint32_t *d_flags, uint32_t epoch, void *stream) {
    if (count < 0 || (count > 0 && (!plans || !ptrs || !d_flags))) return ZKNTT_EINVAL;
    if (count == 0) return ZKNTT_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    size_t scratch_total = 0;
    for (int j = 0; j < count; j++) {
        if (!plans[j] || bad_ptr(ptrs[j].d_in) || bad_ptr(ptrs[j].d_out)) return ZKNTT_EINVAL;
        if (zkntt_status dc = check_plan_device(plans[j])) return dc;
        const size_t bytes = size_t(32) << plans[j]->log_n;
        if (partial_overlap(ptrs[j].d_in, ptrs[j].d_out, bytes)) return ZKNTT_EINVAL;
        scratch_total += scratch_bytes_of(plans[j]);
    }
    // shortest transforms first, each transform's passes back to back
    std::vector<int> order(count);
    for (int j = 0; j < count; j++) order[j] = j;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return plans[a]->log_n < plans[b]->log_n; });
    char *scratch = nullptr;
    if (scratch_total) {
        zkntt_status sa = pool_alloc(reinterpret_cast<void **>(&scratch), scratch_total, s);
        if (sa != ZKNTT_OK) return sa;
    }
    zkntt_status st = ZKNTT_OK;
    size_t off = 0, b = 0;
    while (b < order.size() && st == ZKNTT_OK) {
        std::vector<JobSpec> chunk;
        std::vector<uint32_t> ids;
        size_t segs = 0;
        int level = 0;
        while (b < order.size() && segs + plans[order[b]]->passes <= size_t(BATCH_MAX_SEGMENTS)) {
            const int j = order[b];
            JobSpec J;
            J.plan = plans[j];
            J.in = ptrs[j].d_in;
            J.out = ptrs[j].d_out;
            J.scratch = scratch_bytes_of(plans[j]) ? scratch + off : nullptr;
            J.level0 = level;
            off += scratch_bytes_of(plans[j]);
            level += plans[j]->passes;
            segs += plans[j]->passes;
            chunk.push_back(J);
            ids.push_back(uint32_t(j));
            b++;
        }
        st = launch_batch(chunk, s, batch_timeout_ns(), d_flags, epoch, &ids);
    }
    if (scratch) {
        zkntt_status st2 = from_cuda(cudaFreeAsync(scratch, s));
        if (st == ZKNTT_OK) st = st2;
    }
    return st;
}

zkntt_status zkntt_flags_create(int count, uint32_t **host_view, uint32_t **device_view) {
    if (count < 1 || !host_view || !device_view) return ZKNTT_EINVAL;
    void *h = nullptr, *d = nullptr;
    ZK_CHECK(cudaHostAlloc(&h, size_t(count) * 4, cudaHostAllocMapped));
    memset(h, 0, size_t(count) * 4);
    cudaError_t e = cudaHostGetDevicePointer(&d, h, 0);
    if (e != cudaSuccess) {
        cudaFreeHost(h);
        return from_cuda(e);
    }
    *host_view = static_cast<uint32_t *>(h);
    *device_view = static_cast<uint32_t *>(d);
    return ZKNTT_OK;
}

zkntt_status zkntt_flags_destroy(uint32_t *host_view) {
    if (!host_view) return ZKNTT_OK;
    return from_cuda(cudaFreeHost(host_view));
}

zkntt_status zkntt_groth16_h(zkntt_field field, int log_n, const void *d_a, const void *d_b,
                             const void *d_c, void *d_h, void *d_scratch, void *stream) {
    return zkntt_groth16_h_ex(field, log_n, d_a, d_b, d_c, d_h, d_scratch, 1, stream);
}

zkntt_status zkntt_groth16_h_ex(zkntt_field field, int log_n, const void *d_a, const void *d_b,
                                const void *d_c, void *d_h, void *d_scratch, int fused, void *stream) {
    if (!valid_field(field)) return ZKNTT_EINVAL;
    if (log_n < 1 || log_n > 28) return ZKNTT_EINVAL;
    if (bad_ptr(d_a) || bad_ptr(d_b) || bad_ptr(d_c) || bad_ptr(d_h) || bad_ptr(d_scratch))
        return ZKNTT_EINVAL;
    const size_t bytes = size_t(32) << log_n;
    char *S = static_cast<char *>(d_scratch);
    for (const void *q : {d_a, d_b, d_c, (const void *)d_h})
        if (ranges_overlap(q, bytes, S, 3 * bytes)) return ZKNTT_EINVAL;
    for (const void *q : {d_a, d_b, d_c})
        if (ranges_overlap(q, bytes, d_h, bytes)) return ZKNTT_EINVAL;
    G16Plans *G;
    zkntt_status st = g16_plans(field, log_n, &G);
    if (st != ZKNTT_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *S0 = S, *S1 = S + bytes, *S2 = S + 2 * bytes;
    const void *in[3] = {d_a, d_b, d_c};
    void *sv[3] = {S0, S1, S2};
    if (!fused) {
        for (int k = 0; k < 3; k++)
            if ((st = zkntt_execute(G->intt, in[k], sv[k], s))) return st;
        for (int k = 0; k < 3; k++)
            if ((st = zkntt_execute(G->cntt, sv[k], sv[k], s))) return st;
        uint4 *z = nullptr;
        zkntt_status sa = pool_alloc(reinterpret_cast<void **>(&z), 32, s);
        if (sa != ZKNTT_OK) return sa;
        st = from_cuda(cudaMemcpyAsync(z, G->zinv.data(), 32, cudaMemcpyHostToDevice, s));
        if (st == ZKNTT_OK) st = launch_pointwise(field, S0, S1, S2, z, d_h, size_t(1) << log_n, s);
        zkntt_status st2 = from_cuda(cudaFreeAsync(z, s));
        if (st != ZKNTT_OK) return st;
        if (st2 != ZKNTT_OK) return st2;
        return zkntt_execute(G->cintt, d_h, d_h, s);
    }
    // fused: one persistent launch over the dependency graph
    //   jobs 0-2: cosetINTT_{g^-1}(a|b|c) -> S0|S1|S2   levels 0 .. p-1
    //   jobs 3-5: NTT in place on S0|S1|S2              levels p .. 2p-1
    //   job 6:    cosetINTT_g(S0*S1 - S2) * zinv -> h   levels 2p .. 3p-1
    const size_t per = scratch_bytes_of(G->ntt);
    char *ps = nullptr;
    if (per) {
        zkntt_status sa = pool_alloc(reinterpret_cast<void **>(&ps), 7 * per, s);
        if (sa != ZKNTT_OK) return sa;
    }
    std::vector<JobSpec> jobs(7);
    const int p1 = G->intt_gj->passes, p2 = G->ntt->passes;
    for (int k = 0; k < 3; k++) {
        jobs[k].plan = G->intt_gj;
        jobs[k].in = in[k];
        jobs[k].out = sv[k];
        jobs[k].level0 = 0;
        jobs[3 + k].plan = G->ntt;
        jobs[3 + k].in = sv[k];
        jobs[3 + k].out = sv[k];
        jobs[3 + k].level0 = p1;
        jobs[3 + k].deps[0] = k;
    }
    jobs[6].plan = G->cintt_z;
    jobs[6].in = S0;
    jobs[6].out = d_h;
    jobs[6].pw_b = S1;
    jobs[6].pw_c = S2;
    jobs[6].level0 = p1 + p2;
    jobs[6].deps[0] = 3;
    jobs[6].deps[1] = 4;
    jobs[6].deps[2] = 5;
    for (int j = 0; j < 7; j++) jobs[j].scratch = per ? ps + j * per : nullptr;
    st = launch_batch(jobs, s, batch_timeout_ns());
    if (ps) {
        zkntt_status st2 = from_cuda(cudaFreeAsync(ps, s));
        if (st == ZKNTT_OK) st = st2;
    }
    return st;
}

struct zkntt_graph_s {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

zkntt_status zkntt_groth16_graph_create(zkntt_graph *out, zkntt_field field, int log_n,
                                        const void *d_a, const void *d_b, const void *d_c, void *d_h,
                                        void *d_scratch, void *stream) {
    if (!out) return ZKNTT_EINVAL;
    if (!valid_field(field)) return ZKNTT_EINVAL;
    if (log_n < 1 || log_n > 28) return ZKNTT_EINVAL;
    if (!stream) return ZKNTT_EINVAL;  // the legacy default stream cannot be captured
    // everything that allocates or synchronises happens before the capture
    G16Plans *G;
    zkntt_status st = g16_plans(field, log_n, &G);
    if (st != ZKNTT_OK) return st;
    DeviceInfo *dev;
    st = device_info(&dev);
    if (st != ZKNTT_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    zkntt_graph_s *g = new (std::nothrow) zkntt_graph_s;
    if (!g) return ZKNTT_ENOMEM;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        delete g;
        return from_cuda(e);
    }
    st = zkntt_groth16_h_ex(field, log_n, d_a, d_b, d_c, d_h, d_scratch, 1, stream);
    e = cudaStreamEndCapture(s, &g->graph);
    if (st == ZKNTT_OK && e == cudaSuccess)
        e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (st != ZKNTT_OK || e != cudaSuccess) {
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return st != ZKNTT_OK ? st : from_cuda(e);
    }
    *out = g;
    return ZKNTT_OK;
}

zkntt_status zkntt_graph_launch(zkntt_graph graph, void *stream) {
    if (!graph || !graph->exec) return ZKNTT_EINVAL;
    return from_cuda(cudaGraphLaunch(graph->exec, static_cast<cudaStream_t>(stream)));
}

zkntt_status zkntt_graph_destroy(zkntt_graph graph) {
    if (!graph) return ZKNTT_OK;
    if (graph->exec) cudaGraphExecDestroy(graph->exec);
    if (graph->graph) cudaGraphDestroy(graph->graph);
    delete graph;
    return ZKNTT_OK;
}

const char *zkntt_status_str(zkntt_status status) {
    switch (status) {
        case ZKNTT_OK: return "ok";
        case ZKNTT_EINVAL: return "invalid argument";
        case ZKNTT_ENOMEM: return "out of device memory";
        case ZKNTT_ECUDA: return "CUDA error";
        case ZKNTT_ETIMEOUT: return "device-side wait timed out";
        case ZKNTT_EUNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

zkntt_status zkntt_last_cuda_error(int *err) {
    if (!err) return ZKNTT_EINVAL;
    *err = g_last_cuda_error;
    return ZKNTT_OK;
}

zkntt_status zkntt_sync_status(void *stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ZK_CHECK(cudaStreamSynchronize(s));
    DeviceInfo *dev;
    zkntt_status st = device_info(&dev);
    if (st != ZKNTT_OK) return st;
    uint32_t *w = status_word(dev, s);
    uint32_t word = 0;
    ZK_CHECK(cudaMemcpy(&word, w, 4, cudaMemcpyDeviceToHost));
    if (word) {
        ZK_CHECK(cudaMemset(w, 0, 4));
        if (word & BATCH_STATUS_TIMEOUT) return ZKNTT_ETIMEOUT;
        return ZKNTT_ECUDA;
    }
    return ZKNTT_OK;
}

zkntt_status zkntt_inject_timeout(int timeout_ms, void *stream) {
    if (timeout_ms < 1 || timeout_ms > 10000) return ZKNTT_EINVAL;
    DeviceInfo *dev;
    zkntt_status st = device_info(&dev);
    if (st != ZKNTT_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    BatchTable *tab = new (std::nothrow) BatchTable;
    if (!tab) return ZKNTT_ENOMEM;
    memset(tab, 0, sizeof *tab);
    // one segment with one tile that waits for its own completion: the wait can
    // only end by the time limit, and the tile body never runs
    tab->nseg = 1;
    tab->total_items = 1;
    tab->timeout_ns = (unsigned long long)timeout_ms * 1000000ull;
    tab->seg[0].K = 4;
    tab->seg[0].first_item = 0;
    tab->seg[0].dep[0] = 0;
    tab->seg[0].dep[1] = tab->seg[0].dep[2] = -1;
    tab->seg[0].dep_tiles[0] = 1;
    uint32_t *ctrl = nullptr;
    st = pool_alloc(reinterpret_cast<void **>(&ctrl), 3 * 4, s);
    if (st != ZKNTT_OK) {
        delete tab;
        return st;
    }
    cudaError_t e = cudaMemsetAsync(ctrl, 0, 3 * 4, s);
    if (e == cudaSuccess) {
        uint32_t *done = ctrl + 2;
        uint32_t *status = status_word(dev, s);
        void *args[] = {tab, &ctrl, &done, &status};
        e = cudaLaunchKernel(batch_kernel_ptr(0), dim3(1), dim3(BATCH_THREADS), args, 64 * 1024, s);
    }
    if (ctrl) cudaFreeAsync(ctrl, s);
    delete tab;
    return from_cuda(e);
}

zkntt_status zkntt_selftest_timeout(int timeout_ms, void *stream) {
    zkntt_status st = zkntt_inject_timeout(timeout_ms, stream);
    if (st != ZKNTT_OK) return st;
    return zkntt_sync_status(stream);
}

zkntt_status zkntt_selftest_device_check(int *checked, int *rejected) {
    if (!checked || !rejected) return ZKNTT_EINVAL;
    *checked = *rejected = 0;
    int cur = 0;
    ZK_CHECK(cudaGetDevice(&cur));
    // a real plan and real buffers of 16 elements: were a check missing, the
    // call would run a valid transform on them
    zkntt_plan real = nullptr;
    zkntt_status st = create_plan(&real, ZKNTT_BLS12_381_FR, 4, ZKNTT_FORWARD, nullptr, nullptr, nullptr);
    if (st != ZKNTT_OK) return st;
    char *buf = nullptr;
    st = from_cuda(cudaMalloc(&buf, 4 * 512));
    if (st != ZKNTT_OK) {
        free_plan(real);
        return st;
    }
    char *hbuf = nullptr;
    st = from_cuda(cudaMallocHost(&hbuf, 2 * 512));
    if (st != ZKNTT_OK) {
        cudaFree(buf);
        free_plan(real);
        return st;
    }
    zkntt_plan_s *fake = new (std::nothrow) zkntt_plan_s;
    if (!fake) {
        cudaFreeHost(hbuf);
        cudaFree(buf);
        free_plan(real);
        return ZKNTT_ENOMEM;
    }
    *fake = *real;
    fake->allocs.clear();       // the tables belong to `real`
    fake->device = cur + 1;     // as if created on another device
    zkntt_plan plans[1] = {fake};
    zkntt_io io[1] = {{buf, buf + 512}};
    uint32_t *flags = reinterpret_cast<uint32_t *>(buf + 3 * 512);
    const zkntt_status got[] = {
        zkntt_execute(fake, buf, buf + 512, nullptr),
        zkntt_execute_scratch(fake, buf, buf + 512, buf + 1024, 512, nullptr),
        zkntt_execute_host(fake, hbuf, hbuf + 512, nullptr),
        zkntt_execute_host_buffered(fake, hbuf, hbuf + 512, buf, 2048, nullptr),
        zkntt_execute_noalloc(fake, buf, buf + 512, nullptr),
        zkntt_execute_batch(plans, io, 1, nullptr),
        zkntt_execute_batch_signal(plans, io, 1, flags, 1, nullptr),
    };
    for (zkntt_status g : got) {
        (*checked)++;
        if (g == ZKNTT_EINVAL) (*rejected)++;
    }
    delete fake;
    st = from_cuda(cudaDeviceSynchronize());
    cudaFreeHost(hbuf);
    cudaFree(buf);
    free_plan(real);
    return st;
}

zkntt_status zkntt_scale_powers(zkntt_field field, const void *d_x, void *d_out, size_t n,
                                const uint32_t *c_mont, const uint32_t *base_mont, void *stream) {
    if (!valid_field(field) || !c_mont || !base_mont) return ZKNTT_EINVAL;
    if (n == 0) return ZKNTT_OK;
    if (bad_ptr(d_x) || bad_ptr(d_out)) return ZKNTT_EINVAL;
    if (partial_overlap(d_x, d_out, n * 32)) return ZKNTT_EINVAL;
    const HostField &F = host_field(field);
    E8 c, base;
    for (int i = 0; i < 8; i++) {
        c[i] = c_mont[i];
        base[i] = base_mont[i];
    }
    if (geq8(c, F.p) || geq8(base, F.p)) return ZKNTT_EINVAL;
    DeviceInfo *dev;
    zkntt_status st = device_info(&dev);
    if (st != ZKNTT_OK) return st;
    int bits = 0;
    while ((size_t(1) << bits) < n) bits++;
    const int sp = (bits + 1) / 2;
    // lo[t] = c base^t (t < 2^sp), hi[u] = base^(u 2^sp) (u < 2^(bits - sp))
    std::vector<E8> tab = powers(F, base, size_t(1) << sp, c);
    const std::vector<E8> hi = powers(F, hpow(F, base, uint64_t(1) << sp), size_t(1) << (bits - sp), F.one);
    tab.insert(tab.end(), hi.begin(), hi.end());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint4 *d_tab = nullptr;
    st = pool_alloc(reinterpret_cast<void **>(&d_tab), tab.size() * 32, s);
    if (st != ZKNTT_OK) return st;
    // pageable source: the copy is staged before the call returns
    st = from_cuda(cudaMemcpyAsync(d_tab, tab.data(), tab.size() * 32, cudaMemcpyHostToDevice, s));
    if (st == ZKNTT_OK) {
        const uint4 *lo_t = d_tab, *hi_t = d_tab + 2 * (size_t(1) << sp);
        uint32_t usp = uint32_t(sp);
        void *args[] = {&d_x, &d_out, &n, &hi_t, &lo_t, &usp};
        st = from_cuda(cudaLaunchKernel(field_kernels(field).scale_powers,
                                        dim3(grid_for(n, 256, dev->sms)), dim3(256), args, 0, s));
    }
    zkntt_status st2 = from_cuda(cudaFreeAsync(d_tab, s));
    return st != ZKNTT_OK ? st : st2;
}

zkntt_status zkntt_block_dft(zkntt_field field, int log_g, size_t b, const void *d_in, void *d_out,
                             int inverse, void *stream) {
    if (!valid_field(field) || log_g < 1 || log_g > 3) return ZKNTT_EINVAL;
    if (b == 0) return ZKNTT_OK;
    if (bad_ptr(d_in) || bad_ptr(d_out)) return ZKNTT_EINVAL;
    const size_t G = size_t(1) << log_g;
    if (partial_overlap(d_in, d_out, G * b * 32)) return ZKNTT_EINVAL;
    const HostField &F = host_field(field);
    if (!F.ok) return ZKNTT_ECUDA;
    DeviceInfo *dev;
    zkntt_status st = device_info(&dev);
    if (st != ZKNTT_OK) return st;
    // w of order G (w_max^(2^(s - g)), or its inverse) and its first powers
    E8 w = hpow(F, F.wmax, uint64_t(1) << (F.s - log_g));
    if (inverse) w = hinv(F, w);
    BlockTw tw;
    memset(&tw, 0, sizeof tw);
    E8 cur = F.one;
    for (size_t k = 0; k < G / 2; k++) {
        memcpy(tw.w[k], cur.data(), 32);
        cur = hmul(F, cur, w);
    }
    void *args[] = {&d_in, &d_out, &b, &tw};
    return from_cuda(cudaLaunchKernel(field_kernels(field).block_dft[log_g],
                                      dim3(grid_for(b, 128, dev->sms)), dim3(128), args, 0,
                                      static_cast<cudaStream_t>(stream)));
}

zkntt_status zkntt_pool_info(size_t *reserved_bytes, size_t *used_bytes) {
    if (!reserved_bytes || !used_bytes) return ZKNTT_EINVAL;
    DeviceInfo *dev;
    zkntt_status st = device_info(&dev);
    if (st != ZKNTT_OK) return st;
    uint64_t r = 0, u = 0;
    ZK_CHECK(cudaMemPoolGetAttribute(dev->pool, cudaMemPoolAttrReservedMemCurrent, &r));
    ZK_CHECK(cudaMemPoolGetAttribute(dev->pool, cudaMemPoolAttrUsedMemCurrent, &u));
    *reserved_bytes = size_t(r);
    *used_bytes = size_t(u);
    return ZKNTT_OK;
}

zkntt_status zkntt_imadbench(int mode, int blocks, int threads, int iters, void *d_sink,
                             void *stream) {
    if (mode < 0 || mode > 4) return ZKNTT_EINVAL;
    if (blocks < 1 || threads < 32 || threads > 1024 || iters < 1 || !d_sink) return ZKNTT_EINVAL;
    void *args[] = {&mode, &iters, &d_sink};
    return from_cuda(cudaLaunchKernel(imadbench_kernel_ptr(), dim3(blocks), dim3(threads), args, 0,
                                      static_cast<cudaStream_t>(stream)));
}

zkntt_status zkntt_field_info(zkntt_field field, uint32_t modulus[8], uint32_t generator_mont[8],
                              int *two_adicity) {
    if (!valid_field(field)) return ZKNTT_EINVAL;
    const HostField &F = host_field(field);
    if (!F.ok) return ZKNTT_ECUDA;
    if (modulus) memcpy(modulus, F.p.data(), 32);
    if (generator_mont) memcpy(generator_mont, F.gen_m.data(), 32);
    if (two_adicity) *two_adicity = F.s;
    return ZKNTT_OK;
}

zkntt_status zkntt_field_op(zkntt_field field, int op, const void *d_a, const void *d_b, void *d_c,
                            size_t n, void *stream) {
    if (!valid_field(field)) return ZKNTT_EINVAL;
    if (op < 0 || op > 3) return ZKNTT_EINVAL;
    if (n == 0) return ZKNTT_OK;
    if (bad_ptr(d_a) || bad_ptr(d_b) || bad_ptr(d_c)) return ZKNTT_EINVAL;
    DeviceInfo *dev;
    zkntt_status st = device_info(&dev);
    if (st != ZKNTT_OK) return st;
    void *args[] = {&op, &d_a, &d_b, &d_c, &n};
    return from_cuda(cudaLaunchKernel(field_kernels(field).field_op, dim3(grid_for(n, 256, dev->sms)),
                                      dim3(256), args, 0, static_cast<cudaStream_t>(stream)));
}

zkntt_status zkntt_pointwise(zkntt_field field, const void *d_a, const void *d_b, const void *d_c,
                             const uint32_t *z_mont, void *d_h, size_t n, void *stream) {
    if (!valid_field(field)) return ZKNTT_EINVAL;
    if (!z_mont) return ZKNTT_EINVAL;
    if (n == 0) return ZKNTT_OK;
    if (bad_ptr(d_a) || bad_ptr(d_b) || bad_ptr(d_c) || bad_ptr(d_h)) return ZKNTT_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *z = nullptr;
    zkntt_status sa = pool_alloc(&z, 32, s);
    if (sa != ZKNTT_OK) return sa;
    zkntt_status st = from_cuda(cudaMemcpyAsync(z, z_mont, 32, cudaMemcpyHostToDevice, s));
    if (st == ZKNTT_OK) st = launch_pointwise(field, d_a, d_b, d_c, z, d_h, n, s);
    zkntt_status st2 = from_cuda(cudaFreeAsync(z, s));
    return st != ZKNTT_OK ? st : st2;
}

zkntt_status zkntt_mulbench(zkntt_field field, int blocks, int threads, int iters, void *d_sink,
                            void *stream) {
    if (!valid_field(field)) return ZKNTT_EINVAL;
    if (blocks < 1 || threads < 32 || threads > 256 || iters < 1 || !d_sink) return ZKNTT_EINVAL;
    void *args[] = {&iters, &d_sink};
    return from_cuda(cudaLaunchKernel(field_kernels(field).mulbench, dim3(blocks), dim3(threads),
                                      args, 0, static_cast<cudaStream_t>(stream)));
}

}  // extern "C"
