// ntt_pass.cuh -- one pass of the multi-pass NTT for sm_103a.
//
// Decomposition (the four-step identity applied recursively; Section II-B of
// the paper notes that a block NTT is bounded by shared memory and that groups
// of stages may be run together):
//   n = 2^L is split into digits k_1 + ... + k_p = L (top digit first).  Pass i
//   treats the vector as columns: for fixed (hi, lo) the N = 2^K elements at
//       q = (hi * N + d) * 2^lo_bits + lo,   d = 0..N-1
//   form one sub-transform.  It is computed by radix-2 decimation-in-frequency
//   stages (output position d then holds frequency rev(d)) and, for every pass
//   but the last, multiplied by the inter-pass twiddle w_{n_i}^(lo * rev(d)),
//   n_i = N * 2^lo_bits.  After the last pass the value at position q is
//   output bitrev_L(q); the last pass writes it there directly, so the result
//   is in natural order without a permutation pass.
//
// Inside a thread block: a tile of C columns x N rows (C consecutive lo values,
// or for the last pass C blocks whose bit-reversed indices are consecutive, so
// the scattered writes form C*32-byte runs) is copied into shared memory with
// cp.async.  Stages 0..K-3 run as a loop: each thread takes butterflies
// (x, y) -> (x + y, (x - y) w) from shared memory and writes them back, so the
// loop body holds a single inlined Montgomery product and stays resident in
// the instruction cache.  The difference x - y is formed as x + r - y with no
// conditional correction: it only feeds the product, as its limb-scanned
// operand, which may be any value below 2^256 (the product's output is
// canonical either way).  The last two stages run as one radix-4 step per
// thread on four neighbouring rows, and the scaled elements are then written
// to global memory.  All sizes (K, C, the stride) are runtime values: one
// kernel per field serves every digit size.
//
// Shared memory holds each element as two 16-byte halves in separate arrays.
// The slot of (column c, row d) is c*N + (d ^ s) with
//   s = (7 if bit 3 of d is set) ^ (c << (3 - log2 C))   (low three bits),
// which keeps the butterfly accesses of every stage (pairs at distance 1, 2, 4
// and >= 8), the column-major copies and the row-major copies free of bank
// conflicts.
//
// Fused per-element factors (one Montgomery product each, only when present):
//   pre[d]          first pass, on input row d (coset forward shift powers)
//   pw_b, pw_c      first pass, x <- x * pw_b[q] - pw_c[q] (Groth16 pointwise)
//   tw[d][lo]       inter-pass twiddles, precomputed, or formed on the fly from
//                   split-exponent tables (w_hi, w_lo) and optional per-column
//                   (fl) and per-row (fd) factors
//   post[d]         last pass, on output position d (inverse / coset scales)
#pragma once
#include <cstdint>

#include "field.cuh"

namespace zkntt {

struct PassArgs {
    const uint4 *in;
    uint4 *out;
    const uint4 *w_stage; // per stage s: w_N^(j 2^s), j < N/2^(s+1), at offset N - 2^(K-s)
    const uint4 *tw;      // precomputed inter-pass twiddles [N][2^lo_bits] (row-major by d)
    const uint4 *w_hi;    // on-the-fly: w^((e >> split_bits) << split_bits)
    const uint4 *w_lo;    // on-the-fly: w^(e & (2^split_bits - 1)) (times any folded scalar)
    const uint4 *fl;      // on-the-fly: per-column factor (may be null)
    const uint4 *fd;      // on-the-fly: per-row factor (may be null)
    const uint4 *pre;     // first pass input scale by row (may be null)
    const uint4 *post;    // last pass output scale by position (may be null)
    const uint4 *pw_b;    // fused Groth16 pointwise: x <- x * pw_b[q] - pw_c[q] on load
    const uint4 *pw_c;    //   (first pass only; both null otherwise)
    uint32_t K;           // log2 of the sub-transform size N
    uint32_t lo_bits;     // log2 of this digit's stride
    uint32_t hi_bits;     // bits above this digit
    uint32_t tw_bits;     // on-the-fly: log2 n_i (exponents are taken mod n_i)
    uint32_t split_bits;  // on-the-fly: width of the low exponent table
    uint32_t log_cols;    // log2 C
    uint32_t last;        // 1: last pass (bit-reversed scatter to natural order)
    uint32_t otf;         // 1: form inter-pass twiddles on the fly
    uint32_t num_tiles;   // tiles in this pass
};

__device__ __forceinline__ uint32_t brev_bits(uint32_t x, uint32_t bits) {
    return bits == 0 ? 0u : (__brev(x) >> (32 - bits));
}

// swizzled shared-memory slot of element (column c, row d)
__device__ __forceinline__ uint32_t smem_slot(uint32_t c, uint32_t d, uint32_t K, uint32_t lc) {
    if (K < 3) return (c << K) + d;
    uint32_t s = ((((d >> 3) & 1u) * 7u) ^ (c << (3 - lc))) & 7u;
    return (c << K) + (d ^ s);
}

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}

// the same with the shared-memory destination as a 32-bit shared address
__device__ __forceinline__ void cp_async16_sa(uint32_t s, const void *gmem_src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// wait until at most N committed groups of this thread's copies are pending
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ void lds_elem(uint32_t x[8], const uint4 *s_lo, const uint4 *s_hi,
                                         uint32_t slot) {
    uint4 v0 = s_lo[slot], v1 = s_hi[slot];
    x[0] = v0.x; x[1] = v0.y; x[2] = v0.z; x[3] = v0.w;
    x[4] = v1.x; x[5] = v1.y; x[6] = v1.z; x[7] = v1.w;
}

__device__ __forceinline__ void sts_elem(uint4 *s_lo, uint4 *s_hi, uint32_t slot,
                                         const uint32_t x[8]) {
    s_lo[slot] = make_uint4(x[0], x[1], x[2], x[3]);
    s_hi[slot] = make_uint4(x[4], x[5], x[6], x[7]);
}

// Global index of tile element (row d, column cc) before (src) and after (dst)
// the pass.
__device__ __forceinline__ size_t tile_src(const PassArgs &a, uint32_t tile, uint32_t d,
                                           uint32_t cc) {
    if (!a.last) {
        const uint32_t lo_tiles_bits = a.lo_bits - a.log_cols;
        const size_t hi = tile >> lo_tiles_bits;
        const size_t lo0 = size_t(tile & ((1u << lo_tiles_bits) - 1u)) << a.log_cols;
        return ((hi << a.K | d) << a.lo_bits) + lo0 + cc;
    }
    const uint32_t b = (tile << a.log_cols) + cc;
    return (size_t(brev_bits(b, a.hi_bits)) << a.K) + d;
}

__device__ __forceinline__ size_t tile_dst(const PassArgs &a, uint32_t tile, uint32_t d,
                                           uint32_t cc) {
    if (!a.last) return tile_src(a, tile, d, cc);
    return (size_t(brev_bits(d, a.K)) << a.hi_bits) + (size_t(tile) << a.log_cols) + cc;
}

// Output factor of row position d in column cc: the inter-pass twiddle (times
// folded factors) or the last pass's post scale.  Returns false when there is
// no factor.
template <class F>
__device__ __forceinline__ bool out_factor(uint32_t f[8], const PassArgs &a, uint32_t tile,
                                           uint32_t d, uint32_t cc) {
    if (a.last) {
        if (!a.post) return false;
        ldg_elem(f, a.post + 2 * size_t(d));
        return true;
    }
    const uint32_t lo_tiles_bits = a.lo_bits - a.log_cols;
    const uint32_t lo = ((tile & ((1u << lo_tiles_bits) - 1u)) << a.log_cols) + cc;
    if (!a.otf) {
        ldg_elem(f, a.tw + 2 * ((size_t(d) << a.lo_bits) + lo));
        return true;
    }
    // lo < 2^lo_bits and rev(d) < 2^K, so e < 2^tw_bits = n_i: no reduction
    // (and no overflow: tw_bits <= 32)
    const uint32_t e = lo * brev_bits(d, a.K);
    uint32_t g[8];
    ldg_elem(f, a.w_hi + 2 * size_t(e >> a.split_bits));
    ldg_elem(g, a.w_lo + 2 * size_t(e & ((1u << a.split_bits) - 1u)));
    mul_call<F>(f, f, g);
    if (a.fl) {
        ldg_elem(g, a.fl + 2 * size_t(lo));
        mul_call<F>(f, f, g);
    }
    if (a.fd) {
        ldg_elem(g, a.fd + 2 * size_t(d));
        mul_call<F>(f, f, g);
    }
    return true;
}

// Issue (without waiting) the 16-byte copies of one tile into shared memory:
// 8 lanes copy the low halves of 8 elements, the next 8 lanes their high
// halves (tiles under 8 elements: element-major); columns fastest for strided
// passes, rows fastest for the last.
__device__ __forceinline__ void issue_tile_load(const PassArgs &a, uint4 *smem, uint32_t tile,
                                                uint32_t nthreads) {
    const uint32_t K = a.K, lc = a.log_cols;
    const uint32_t N = 1u << K, C = 1u << lc, CN = C << K;
    uint4 *s_lo = smem, *s_hi = smem + CN;
    const uint32_t tid = threadIdx.x;
    if (tid >= nthreads) return;
    if (CN >= 64 && (nthreads & 15u) == 0 && (nthreads & (nthreads - 1u)) == 0 && nthreads <= 2 * CN) {
        // Every thread makes 2 C N / nthreads copies of one half (the lane's
        // bit 3) of elements e0, e0 + E, e0 + 2E, ... (E = nthreads / 2); in
        // a strided pass they share a column and step by a fixed row count,
        // so the source address steps by a fixed stride and only the shared
        // slot is formed per copy.
        const uint32_t half = (tid >> 3) & 1u;
        const uint32_t e0 = (tid & 7u) | ((tid >> 4) << 3);
        const uint32_t E = nthreads >> 1, iters = (2 * CN) / nthreads;
        const uint32_t sbase =
            static_cast<uint32_t>(__cvta_generic_to_shared(half ? s_hi : s_lo));
        if (!a.last) {
            const uint32_t cc = e0 & (C - 1), dstep = E >> lc;
            uint32_t d = e0 >> lc;
            const uint4 *src = a.in + 2 * tile_src(a, tile, d, cc) + half;
            const size_t sstep = size_t(2 * dstep) << a.lo_bits;
            if ((dstep & 15u) == 0) {
                // rows d, d + dstep, ... agree in their low four bits, so they
                // share the swizzle term and their slots step by dstep too
                uint32_t sa = sbase + 16u * smem_slot(cc, d, K, lc);
                for (uint32_t k = 0; k < iters; k++, sa += 16u * dstep, src += sstep)
                    cp_async16_sa(sa, src);
            } else {
                for (uint32_t k = 0; k < iters; k++, d += dstep, src += sstep)
                    cp_async16_sa(sbase + 16u * smem_slot(cc, d, K, lc), src);
            }
        } else if (E < N) {
            // last pass, rows fastest: N / E copies in one column (rows e0,
            // e0 + E, ...; e0 < E), then the next column
            const uint32_t per = N / E;
            for (uint32_t cc = 0; cc < C; cc++) {
                const uint4 *row = a.in + 2 * tile_src(a, tile, 0, cc) + half;
                for (uint32_t j = 0, d = e0; j < per; j++, d += E)
                    cp_async16_sa(sbase + 16u * smem_slot(cc, d, K, lc), row + 2 * d);
            }
        } else {
            uint32_t e = e0;
            for (uint32_t k = 0; k < iters; k++, e += E) {
                const uint32_t d = e & (N - 1), cc = e >> K;
                cp_async16_sa(sbase + 16u * smem_slot(cc, d, K, lc),
                              a.in + 2 * tile_src(a, tile, d, cc) + half);
            }
        }
        return;
    }
    const bool grouped = CN >= 8;
    for (uint32_t u = tid; u < 2 * CN; u += nthreads) {
        const uint32_t e = grouped ? ((u & 7u) | ((u >> 4) << 3)) : (u >> 1);
        const uint32_t half = grouped ? ((u >> 3) & 1u) : (u & 1u);
        uint32_t d, cc;
        if (a.last) { d = e & (N - 1); cc = e >> K; }
        else        { cc = e & (C - 1); d = e >> lc; }
        const size_t g = tile_src(a, tile, d, cc);
        cp_async16((half ? s_hi : s_lo) + smem_slot(cc, d, K, lc), a.in + 2 * g + half);
    }
}

// Process one tile with `nthreads` threads of the block (threads at or beyond
// nthreads only take part in the barriers).  PRELOADED: the caller has
// already copied the tile into `smem` and synchronised the block.  PAIR: let a
// thread's two butterflies of one row pair share their twiddle (below).
template <class F, int ILP, bool PRELOADED = false, bool SHFL = false, bool PAIR = true>
__device__ __forceinline__ void run_tile(const PassArgs &a, uint4 *smem, uint32_t tile,
                                         uint32_t nthreads) {
    const uint32_t K = a.K, lc = a.log_cols;
    const uint32_t N = 1u << K;
    const uint32_t C = 1u << lc;
    const uint32_t CN = C << K;
    uint4 *s_lo = smem;
    uint4 *s_hi = smem + CN;
    const uint32_t tid = threadIdx.x;
    const bool active = tid < nthreads;

    // ---- load (columns fastest for strided passes, rows fastest for the last)
    if (PRELOADED) {
    } else if (!a.pre && !a.pw_b) {
        issue_tile_load(a, smem, tile, nthreads);
        cp_async_wait_all();
    } else {
        for (uint32_t e = tid; active && e < CN; e += nthreads) {
            uint32_t d, cc;
            if (a.last) { d = e & (N - 1); cc = e >> K; }
            else        { cc = e & (C - 1); d = e >> lc; }
            const size_t g = tile_src(a, tile, d, cc);
            uint32_t x[8], f[8];
            ld_elem_cg(x, a.in + 2 * g);
            if (a.pw_b) {
                ld_elem_cg(f, a.pw_b + 2 * g);
                mul_call<F>(x, x, f);
                ld_elem_cg(f, a.pw_c + 2 * g);
                sub<F>(x, x, f);
            }
            if (a.pre) {
                ldg_elem(f, a.pre + 2 * size_t(d));
                mul_call<F>(x, x, f);
            }
            sts_elem(s_lo, s_hi, smem_slot(cc, d, K, lc), x);
        }
    }
    if (!PRELOADED) __syncthreads();

    // ---- stages 0 .. K-3: radix-2 butterflies through shared memory.  Each
    // thread takes ILP independent butterflies per step (every thread owns at
    // least two per stage: nthreads <= C*N/4), so the carry chains and loads of
    // one overlap with the other's product.
    // SHFL: the stages with pair distance 16, 8 and 4 run in registers with
    // warp shuffles (below) instead of through shared memory
    const bool shfl_tail = SHFL && K >= 6 && nthreads >= 32;
    // (K < 3: no loop stages; K - 2 must not wrap around)
    const uint32_t s_end = shfl_tail ? K - 5 : (K > 2 ? K - 2 : 0u);
    for (uint32_t s = 0; s < s_end; s++) {
        const uint32_t lh = K - 1 - s;
        const uint32_t h = 1u << lh;
        const uint4 *ws = a.w_stage + 2 * size_t(N - 2 * h);
        // slot of row i0 + h from that of row i0 (bit lh of i0 is clear): the
        // swizzle term changes only when lh = 3
        const uint32_t step = K < 3 ? h : (h ^ (lh == 3 ? 7u : 0u));
        if constexpr (ILP == 0) {
            // software-pipelined: the product of one butterfly overlaps the
            // loads and add/subtract of the next (every thread owns >= 2)
            uint32_t x[8], t[8], w[8], s0, s1;
            auto prepare = [&](uint32_t bk, uint32_t px[8], uint32_t pt[8], uint32_t pw[8],
                               uint32_t &q0, uint32_t &q1) {
                const uint32_t cc = bk >> (K - 1);
                const uint32_t b = bk & ((N >> 1) - 1);
                const uint32_t j = b & (h - 1);
                const uint32_t i0 = ((b >> lh) << (lh + 1)) | j;
                q0 = smem_slot(cc, i0, K, lc);
                q1 = q0 ^ step;
                uint32_t py[8];
                lds_elem(px, s_lo, s_hi, q0);
                lds_elem(py, s_lo, s_hi, q1);
                ldg_elem(pw, ws + 2 * size_t(j));
                sub_lazy<F>(pt, px, py);
                add<F>(px, px, py);
            };
            if (active) prepare(tid, x, t, w, s0, s1);
            for (uint32_t bg = tid; active && bg < (CN >> 1); bg += nthreads) {
                const uint32_t nb = bg + nthreads;
                uint32_t x2[8], t2[8], w2[8], n0 = 0, n1 = 0;
                if (nb < (CN >> 1)) prepare(nb, x2, t2, w2, n0, n1);
                uint32_t y[8];
                mul<F>(y, w, t);
                sts_elem(s_lo, s_hi, s0, x);
                sts_elem(s_lo, s_hi, s1, y);
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    x[k] = x2[k];
                    t[k] = t2[k];
                    w[k] = w2[k];
                }
                s0 = n0;
                s1 = n1;
            }
        } else if (PAIR && ILP == 1 && lc >= 1 && (CN >> 1) == 2 * nthreads) {
            // Each thread owns two butterflies, bk = tid and tid + C N/4: the
            // same row pair in columns cc and cc + C/2, so one twiddle serves
            // both and the second pair's slot is the first's moved by C/2
            // columns, its swizzle term flipped in bit 2.
            if (active) {
                const uint32_t cc = tid >> (K - 1);
                const uint32_t b = tid & ((N >> 1) - 1);
                const uint32_t j = b & (h - 1);
                const uint32_t i0 = ((b >> lh) << (lh + 1)) | j;
                const uint32_t q0 = smem_slot(cc, i0, K, lc);
                const uint32_t q0b = (q0 + ((C >> 1) << K)) ^ (K >= 3 ? 4u : 0u);
                uint32_t w[8];
                ldg_elem(w, ws + 2 * size_t(j));
#pragma unroll
                for (int q = 0; q < 2; q++) {
                    const uint32_t a0 = q ? q0b : q0;
                    uint32_t x[8], y[8], t[8];
                    lds_elem(x, s_lo, s_hi, a0);
                    lds_elem(y, s_lo, s_hi, a0 ^ step);
                    sub_lazy<F>(t, x, y);
                    add<F>(x, x, y);
                    mul<F>(y, w, t);
                    sts_elem(s_lo, s_hi, a0, x);
                    sts_elem(s_lo, s_hi, a0 ^ step, y);
                }
            }
        } else {
        for (uint32_t bg = tid; active && bg < (CN >> 1); bg += ILP * nthreads) {
            constexpr int IL = ILP > 0 ? ILP : 1;
            uint32_t x[IL][8], y[IL][8], w[IL][8], t[IL][8], s0[IL], s1[IL];
#pragma unroll
            for (int k = 0; k < IL; k++) {
                const uint32_t bk = bg + k * nthreads;
                const uint32_t cc = bk >> (K - 1);
                const uint32_t b = bk & ((N >> 1) - 1);
                const uint32_t j = b & (h - 1);
                const uint32_t i0 = ((b >> lh) << (lh + 1)) | j;
                s0[k] = smem_slot(cc, i0, K, lc);
                s1[k] = s0[k] ^ step;
                lds_elem(x[k], s_lo, s_hi, s0[k]);
                lds_elem(y[k], s_lo, s_hi, s1[k]);
                ldg_elem(w[k], ws + 2 * size_t(j));
            }
#pragma unroll
            for (int k = 0; k < IL; k++) {
                sub_lazy<F>(t[k], x[k], y[k]);
                add<F>(x[k], x[k], y[k]);
            }
#pragma unroll
            for (int k = 0; k < IL; k++) mul<F>(y[k], w[k], t[k]);
#pragma unroll
            for (int k = 0; k < IL; k++) {
                sts_elem(s_lo, s_hi, s0[k], x[k]);
                sts_elem(s_lo, s_hi, s1[k], y[k]);
            }
        }
        }
        __syncthreads();
    }

    if constexpr (SHFL) {
        if (shfl_tail) {
            // A warp holds the 64 rows of one group (2 per lane) for the stages
            // with pair distance h = 16, 8, 4.  At distance 2^lh lane L holds
            // the pair (d, d + 2^lh), d = L with a zero inserted at bit lh; for
            // the next distance, lanes L and L ^ 2^(lh-1) exchange one element
            // (the one the partner's next pair needs) with 8 shuffles.
            const uint32_t lane = tid & 31u, warp = tid >> 5, nwarps = nthreads >> 5;
            const uint32_t groups = CN >> 6;
            for (uint32_t gi = warp; active && gi < groups; gi += nwarps) {
                const uint32_t cc = gi >> (K - 6), base = (gi & ((N >> 6) - 1)) << 6;
                uint32_t d0 = ((lane >> 4) << 5) | (lane & 15u);
                uint32_t x[8], y[8];
                lds_elem(x, s_lo, s_hi, smem_slot(cc, base + d0, K, lc));
                lds_elem(y, s_lo, s_hi, smem_slot(cc, base + d0 + 16, K, lc));
                for (uint32_t lh = 4; lh >= 2; lh--) {
                    const uint32_t h = 1u << lh;
                    uint32_t w[8], t[8];
                    ldg_elem(w, a.w_stage + 2 * (size_t(N - 2 * h) + (d0 & (h - 1))));
                    sub_lazy<F>(t, x, y);
                    add<F>(x, x, y);
                    mul<F>(y, w, t);
                    if (lh > 2) {
                        const uint32_t m = h >> 1;
                        const bool beta = (lane >> (lh - 1)) & 1u;
#pragma unroll
                        for (int k = 0; k < 8; k++) {
                            const uint32_t r = __shfl_xor_sync(0xffffffffu, beta ? x[k] : y[k], m);
                            if (beta) x[k] = r;
                            else y[k] = r;
                        }
                        d0 = ((lane >> (lh - 1)) << lh) | (lane & (m - 1));
                    }
                }
                sts_elem(s_lo, s_hi, smem_slot(cc, base + d0, K, lc), x);
                sts_elem(s_lo, s_hi, smem_slot(cc, base + d0 + 4, K, lc), y);
            }
            __syncthreads();
        }
    }

    // ---- last two stages as radix-4 on rows d0..d0+3 (columns fastest)
    if (K >= 2) {
        uint32_t w4[8];
        ldg_elem(w4, a.w_stage + 2 * size_t(N - 3));  // w_N^(2^(K-2)) = w_4
        for (uint32_t qd = tid; active && qd < (CN >> 2); qd += nthreads) {
            const uint32_t cc = qd & (C - 1);
            const uint32_t d0 = (qd >> lc) << 2;
            uint32_t x0[8], x1[8], x2[8], x3[8], t[8];
            // rows d0 + i (d0 a multiple of 4) share the swizzle term: their
            // slots are the first one's with i in the low two bits
            const uint32_t s0 = smem_slot(cc, d0, K, lc), s1 = s0 ^ 1u, s2 = s0 ^ 2u, s3 = s0 ^ 3u;
            lds_elem(x0, s_lo, s_hi, s0);
            lds_elem(x1, s_lo, s_hi, s1);
            lds_elem(x2, s_lo, s_hi, s2);
            lds_elem(x3, s_lo, s_hi, s3);
            // stage K-2: pairs (0,2) with twiddle 1, (1,3) with w_4
            sub<F>(t, x0, x2);
            add<F>(x0, x0, x2);
#pragma unroll
            for (int k = 0; k < 8; k++) x2[k] = t[k];
            sub_lazy<F>(t, x1, x3);
            add<F>(x1, x1, x3);
            mul<F>(x3, w4, t);
            // stage K-1: pairs (0,1), (2,3), twiddle 1
            sub<F>(t, x0, x1);
            add<F>(x0, x0, x1);
#pragma unroll
            for (int k = 0; k < 8; k++) x1[k] = t[k];
            sub<F>(t, x2, x3);
            add<F>(x2, x2, x3);
            sts_elem(s_lo, s_hi, s0, x0);
            sts_elem(s_lo, s_hi, s1, x1);
            sts_elem(s_lo, s_hi, s2, x2);
            sts_elem(s_lo, s_hi, s3, t);
        }
    } else {
        // N = 2: one radix-2 butterfly per column
        for (uint32_t cc = tid; active && cc < C; cc += nthreads) {
            uint32_t x0[8], x1[8], t[8];
            const uint32_t s0 = smem_slot(cc, 0, K, lc), s1 = smem_slot(cc, 1, K, lc);
            lds_elem(x0, s_lo, s_hi, s0);
            lds_elem(x1, s_lo, s_hi, s1);
            sub<F>(t, x0, x1);
            add<F>(x0, x0, x1);
            sts_elem(s_lo, s_hi, s0, x0);
            sts_elem(s_lo, s_hi, s1, t);
        }
    }
    __syncthreads();

    // ---- scale and store (columns fastest: C-element runs in global memory)
    for (uint32_t e = tid; active && e < CN; e += nthreads) {
        const uint32_t cc = e & (C - 1), d = e >> lc;
        uint32_t x[8], f[8];
        lds_elem(x, s_lo, s_hi, smem_slot(cc, d, K, lc));
        if (out_factor<F>(f, a, tile, d, cc)) mul<F>(x, x, f);
        st_elem(a.out + 2 * tile_dst(a, tile, d, cc), x);
    }
    __syncthreads();
}

// threads per block for a tile of C x 2^K elements: one per radix-4 group,
// at most 256
__host__ __device__ constexpr uint32_t pass_threads(uint32_t K, uint32_t lc) {
    return ((K >= 2 ? (1u << (K + lc - 2)) : (1u << lc)) < 256u)
               ? (K >= 2 ? (1u << (K + lc - 2)) : (1u << lc))
               : 256u;
}

// threads per block for schedule variant v: variant 5 doubles the count (one
// butterfly per thread per stage), still at most 256
__host__ __device__ constexpr uint32_t pass_threads_for(uint32_t K, uint32_t lc, int v) {
    return v == 5 && K >= 2 && pass_threads(K, lc) < 256u ? 2u * pass_threads(K, lc)
                                                           : pass_threads(K, lc);
}

// Schedule variants (the plan's `ilp` option):
//   1: one butterfly per thread per stage step, registers for 3 blocks of 256
//   2: two interleaved butterflies per thread, registers for 2 blocks
//   3: one butterfly per thread, registers for 4 blocks (tiles of <= 1024
//      elements so four fit in shared memory)
//   4: software-pipelined stage loop (the product of one butterfly overlaps
//      the loads and add/subtract of the next), registers for 2 blocks
//   5: as 3 with twice the threads per tile (one butterfly per thread per
//      stage; half the threads idle in the radix-4 epilogue): more warps in
//      flight for transforms too small to fill the GPU
//   6: as 3 with two tile buffers: the next tile's loads overlap this tile's
//      stages (twice the shared memory per block)
//   7: as 1 with the stages of pair distance 16, 8 and 4 in registers, the
//      partners exchanged by warp shuffles (digits of 6 bits or more)
template <int V> struct PassVariant;
template <> struct PassVariant<1> { static constexpr int ILP = 1, MIN_BLOCKS = 3; };
template <> struct PassVariant<2> { static constexpr int ILP = 2, MIN_BLOCKS = 2; };
template <> struct PassVariant<3> { static constexpr int ILP = 1, MIN_BLOCKS = 4; };
template <> struct PassVariant<4> { static constexpr int ILP = 0, MIN_BLOCKS = 2; };  // pipelined
template <> struct PassVariant<5> { static constexpr int ILP = 1, MIN_BLOCKS = 4; };  // 2x threads
template <> struct PassVariant<6> { static constexpr int ILP = 1, MIN_BLOCKS = 4; };  // 2 buffers
template <> struct PassVariant<7> { static constexpr int ILP = 1, MIN_BLOCKS = 3; };  // shuffles

template <class F, int V>
__global__ void __launch_bounds__(256, PassVariant<V>::MIN_BLOCKS) ntt_pass_kernel(const PassArgs a) {
    extern __shared__ uint4 smem[];
    // Passes after the first are launched as programmatic dependents of the
    // pass before, and wait here until that pass has completed and its writes
    // are visible (launched without that attribute, the wait returns at once).
    // A block lets the next pass launch when it starts its last tile, so the
    // next pass's blocks take SM places only as this grid winds down.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (V != 6 || a.pre || a.pw_b) {
        for (uint32_t tile = blockIdx.x; tile < a.num_tiles; tile += gridDim.x) {
            if (tile + gridDim.x >= a.num_tiles)
                asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
            run_tile<F, PassVariant<V>::ILP, false, V == 7>(a, smem, tile, blockDim.x);
        }
        return;
    }
    // Variant 6: two tile buffers.  The copies of the block's next tile are in
    // flight (cp.async group) while the current tile's stages run, so a tile's
    // load latency overlaps the previous tile's arithmetic within the block.
    // The buffer a load goes to was last used by the tile before, which ended
    // with a block barrier.
    const uint32_t CN = 1u << (a.K + a.log_cols);
    uint32_t tile = blockIdx.x;
    if (tile >= a.num_tiles) return;
    issue_tile_load(a, smem, tile, blockDim.x);
    cp_async_commit();
    uint32_t cur = 0;
    for (; tile < a.num_tiles; tile += gridDim.x) {
        const uint32_t next = tile + gridDim.x;
        if (next >= a.num_tiles) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        if (next < a.num_tiles) {
            issue_tile_load(a, smem + (cur ^ 1u) * 2 * CN, next, blockDim.x);
            cp_async_commit();
            cp_async_wait_group<1>();
        } else {
            cp_async_wait_group<0>();
        }
        __syncthreads();
        run_tile<F, 1, true>(a, smem + cur * 2 * CN, tile, blockDim.x);
        cur ^= 1u;
    }
}

}  // namespace zkntt
