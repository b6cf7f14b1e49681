// ntt_pass.cuh -- one pass of the multi-pass NTT for sm_103a.
//
// Decomposition (the four-step identity, applied recursively; Section II-B of
// the paper notes that a block NTT is bounded by shared memory and that
// "different stages can be processed in batches"):
//   n = 2^L is split into digits k_1 + ... + k_p = L (top digit first).  Pass i
//   treats the vector as columns: for fixed (hi, lo) the N_i = 2^k_i elements
//   at  q = (hi * N_i + d) * 2^lo_bits + lo,  d = 0..N_i-1
//   form one sub-transform.  It is computed in place by radix-2
//   decimation-in-frequency stages (output position d holds frequency
//   rev(d)), then, for every pass but the last, multiplied by the inter-pass
//   twiddle  w_{n_i}^(lo * rev(d))  with n_i = N_i * 2^lo_bits.  After the last
//   pass the value at position q is output bitrev_L(q); the last pass writes
//   it there directly, so the result is in natural order with no separate
//   permutation pass.
//
// Inside a thread block: a tile of C columns x N rows (C consecutive lo values,
// or for the last pass C blocks whose bit-reversed indices are consecutive so
// the scattered writes form C*32-byte runs) is copied into shared memory with
// cp.async, then processed in rounds of three radix-2 stages: each thread holds
// 8 elements in registers (radix-8), exchanges go through shared memory.
// Shared memory holds the tile as two 16-byte halves per element in separate
// arrays, XOR-swizzled so both the copy and the round access patterns are free
// of bank conflicts.
//
// Fused per-element factors (each one Montgomery product, only when present):
//   pre[d]   first pass, on input row d    (coset forward shift powers)
//   tw       inter-pass twiddles, precomputed table [lo][d] or formed on the
//            fly from split-exponent tables (w_hi, w_lo) and optional per-column
//            (fl) and per-row (fd) factors
//   post[d]  last pass, on output position d  (inverse / coset inverse scales)
#pragma once
#include <cstdint>

#include "field.cuh"

namespace zkntt {

struct PassArgs {
    const uint4 *in;
    uint4 *out;
    const uint4 *w_sub;   // w_N^e for e in [0, N/2) (w_N^-e for inverse plans)
    const uint4 *tw;      // precomputed inter-pass twiddles [2^lo_bits][N], position order
    const uint4 *w_hi;    // on-the-fly: w^(e >> split_bits << split_bits) table
    const uint4 *w_lo;    // on-the-fly: w^(e & (2^split_bits - 1)) table
    const uint4 *fl;      // on-the-fly: per-column factor (may be null)
    const uint4 *fd;      // on-the-fly: per-row factor (may be null)
    const uint4 *pre;     // first pass input scale by row (may be null)
    const uint4 *post;    // last pass output scale by position (may be null)
    const uint4 *pw_b;    // fused Groth16 pointwise: x <- x * pw_b[q] - pw_c[q] on load
    const uint4 *pw_c;    //   (first pass only; both null otherwise)
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

// swizzled shared-memory slot of element (column c, row d); N >= 8
template <int K>
__device__ __forceinline__ uint32_t smem_slot(uint32_t c, uint32_t d, uint32_t log_cols) {
    if constexpr (K < 3) {
        return (c << K) + d;
    } else {
        uint32_t sw = ((d >> 3) ^ (c << (3 - log_cols))) & 7u;
        return (c << K) + (d ^ sw);
    }
}

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// position of the m-th held element: the held window of H bits starts at b0
template <int H>
__device__ __forceinline__ uint32_t held_index(uint32_t t, int b0, int m) {
    return ((t >> b0) << (b0 + H)) | (uint32_t(m) << b0) | (t & ((1u << b0) - 1u));
}

// inter-pass twiddle for column lo and row position d (non-last pass)
template <class F, int K>
__device__ __forceinline__ void inter_twiddle(uint32_t w[8], const PassArgs &a, uint32_t lo,
                                              uint32_t d) {
    if (!a.otf) {
        ldg_elem(w, a.tw + 2 * ((size_t(lo) << K) + d));
        return;
    }
    uint32_t e = (lo * brev_bits(d, K)) & ((1u << a.tw_bits) - 1u);
    uint32_t w1[8];
    ldg_elem(w, a.w_hi + 2 * size_t(e >> a.split_bits));
    ldg_elem(w1, a.w_lo + 2 * size_t(e & ((1u << a.split_bits) - 1u)));
    mul_call<F>(w, w, w1);
    if (a.fl) {
        ldg_elem(w1, a.fl + 2 * size_t(lo));
        mul_call<F>(w, w, w1);
    }
    if (a.fd) {
        ldg_elem(w1, a.fd + 2 * size_t(d));
        mul_call<F>(w, w, w1);
    }
}

// One round: up to three DIF stages on the held window of each thread.
__device__ __forceinline__ size_t tile_src(const PassArgs &a, int K, uint32_t tile, uint32_t d,
                                           uint32_t cc);

template <class F, int K, int R>
__device__ __forceinline__ void dif_round(uint4 *s_lo, uint4 *s_hi, const PassArgs &a,
                                          uint32_t c, uint32_t t, uint32_t lo, uint32_t tile) {
    constexpr int H = K < 3 ? K : 3;
    constexpr int E = 1 << H;
    constexpr int ROUNDS = (K + 2) / 3;
    constexpr int BT = K - 1 - 3 * R;                  // first stage bit of this round
    constexpr int NST = (K - 3 * R) < 3 ? (K - 3 * R) : 3;
    constexpr int B0 = (BT - H + 1) > 0 ? (BT - H + 1) : 0;

    uint32_t x[E][8];
    uint32_t pos[E];
#pragma unroll
    for (int m = 0; m < E; m++) {
        pos[m] = held_index<H>(t, B0, m);
        uint32_t slot = smem_slot<K>(c, pos[m], a.log_cols);
        uint4 v0 = s_lo[slot], v1 = s_hi[slot];
        x[m][0] = v0.x; x[m][1] = v0.y; x[m][2] = v0.z; x[m][3] = v0.w;
        x[m][4] = v1.x; x[m][5] = v1.y; x[m][6] = v1.z; x[m][7] = v1.w;
    }
    if (R == 0 && a.pw_b) {
        // Groth16 step H = A * B - C on the coset, fused into the load of A
#pragma unroll
        for (int m = 0; m < E; m++) {
            size_t g = tile_src(a, K, tile, pos[m], c);
            uint32_t f[8];
            ld_elem_cg(f, a.pw_b + 2 * g);
            mul_call<F>(x[m], x[m], f);
            ld_elem_cg(f, a.pw_c + 2 * g);
            sub<F>(x[m], x[m], f);
        }
    }
    if (R == 0 && a.pre) {
#pragma unroll
        for (int m = 0; m < E; m++) {
            uint32_t f[8];
            ldg_elem(f, a.pre + 2 * size_t(pos[m]));
            mul_call<F>(x[m], x[m], f);
        }
    }
#pragma unroll
    for (int s = 0; s < NST; s++) {
        const int b = BT - s;      // stage on index bit b: pairs at distance 2^b
        const int lb = b - B0;     // that bit inside the held window
#pragma unroll
        for (int m = 0; m < E; m++) {
            if (m & (1 << lb)) continue;
            const int m2 = m | (1 << lb);
            uint32_t diff[8];
            sub<F>(diff, x[m], x[m2]);
            add<F>(x[m], x[m], x[m2]);
            // twiddle w_N^((i mod 2^b) * 2^(K-1-b)); statically 1 when every
            // index bit below b is held and zero
            const bool trivial = (B0 == 0) && ((m & ((1 << b) - 1)) == 0);
            if (trivial) {
#pragma unroll
                for (int j = 0; j < 8; j++) x[m2][j] = diff[j];
            } else {
                uint32_t e = (pos[m] & ((1u << b) - 1u)) << (K - 1 - b);
                uint32_t w[8];
                ldg_elem(w, a.w_sub + 2 * size_t(e));
                mul<F>(x[m2], diff, w);
            }
        }
    }
    if (R == ROUNDS - 1) {
        if (!a.last) {
#pragma unroll
            for (int m = 0; m < E; m++) {
                uint32_t w[8];
                inter_twiddle<F, K>(w, a, lo, pos[m]);
                mul<F>(x[m], x[m], w);
            }
        } else if (a.post) {
#pragma unroll
            for (int m = 0; m < E; m++) {
                uint32_t f[8];
                ldg_elem(f, a.post + 2 * size_t(pos[m]));
                mul_call<F>(x[m], x[m], f);
            }
        }
    }
#pragma unroll
    for (int m = 0; m < E; m++) {
        uint32_t slot = smem_slot<K>(c, pos[m], a.log_cols);
        s_lo[slot] = make_uint4(x[m][0], x[m][1], x[m][2], x[m][3]);
        s_hi[slot] = make_uint4(x[m][4], x[m][5], x[m][6], x[m][7]);
    }
}

template <class F, int K, int R>
__device__ __forceinline__ void dif_rounds(uint4 *s_lo, uint4 *s_hi, const PassArgs &a,
                                           uint32_t c, uint32_t t, uint32_t lo, uint32_t tile,
                                           bool active) {
    constexpr int ROUNDS = (K + 2) / 3;
    if constexpr (R < ROUNDS) {
        if (active) dif_round<F, K, R>(s_lo, s_hi, a, c, t, lo, tile);
        __syncthreads();
        dif_rounds<F, K, R + 1>(s_lo, s_hi, a, c, t, lo, tile, active);
    }
}

// Global index of tile element (row d, column cc).
__device__ __forceinline__ size_t tile_src(const PassArgs &a, int K, uint32_t tile, uint32_t d,
                                           uint32_t cc) {
    if (!a.last) {
        uint32_t lo_tiles_bits = a.lo_bits - a.log_cols;
        size_t hi = tile >> lo_tiles_bits;
        size_t lo0 = size_t(tile & ((1u << lo_tiles_bits) - 1u)) << a.log_cols;
        return ((hi << K | d) << a.lo_bits) + lo0 + cc;
    }
    uint32_t b = (tile << a.log_cols) + cc;
    return (size_t(brev_bits(b, a.hi_bits)) << K) + d;
}

__device__ __forceinline__ size_t tile_dst(const PassArgs &a, int K, uint32_t tile, uint32_t d,
                                           uint32_t cc) {
    if (!a.last) return tile_src(a, K, tile, d, cc);
    return (size_t(brev_bits(d, K)) << a.hi_bits) + (size_t(tile) << a.log_cols) + cc;
}

// Process one tile (load, rounds, store) with the block's threads.
template <class F, int K>
__device__ __forceinline__ void run_tile(const PassArgs &a, uint4 *smem, uint32_t tile) {
    constexpr int N = 1 << K;
    constexpr int H = K < 3 ? K : 3;
    constexpr int T = N >> H;
    const uint32_t C = 1u << a.log_cols;
    uint4 *s_lo = smem;
    uint4 *s_hi = smem + (C << K);
    const uint32_t nthreads = C * T;  // threads with work; blockDim.x may be larger
    const uint32_t tid = threadIdx.x;
    const bool active = tid < nthreads;
    const uint32_t units = 2u * (C << K);

    // load: 16-byte units; 8 lanes copy the low halves of 8 elements, the next 8
    // lanes their high halves (unit u covers element e and half, a bijection
    // onto the tile's 2 * C * N units).  Non-last passes walk columns fastest (C
    // contiguous elements per row); the last pass walks rows fastest (its
    // columns are contiguous blocks).
    // (tiles of fewer than 8 elements use plain element-major order)
    const bool grouped = (C << K) >= 8;
    for (uint32_t u = tid; active && u < units; u += nthreads) {
        uint32_t e = grouped ? ((u & 7u) | ((u >> 4) << 3)) : (u >> 1);
        uint32_t half = grouped ? ((u >> 3) & 1u) : (u & 1u);
        uint32_t d, cc;
        if (a.last) { d = e & (N - 1); cc = e >> K; }
        else        { cc = e & (C - 1); d = e >> a.log_cols; }
        size_t g = tile_src(a, K, tile, d, cc);
        uint4 *dst = (half ? s_hi : s_lo) + smem_slot<K>(cc, d, a.log_cols);
        cp_async16(dst, a.in + 2 * g + half);
    }
    cp_async_wait_all();
    __syncthreads();

    const uint32_t c = tid / T, t = tid % T;
    uint32_t lo = 0;
    if (!a.last) {
        uint32_t lo_tiles_bits = a.lo_bits - a.log_cols;
        lo = ((tile & ((1u << lo_tiles_bits) - 1u)) << a.log_cols) + c;
    }
    dif_rounds<F, K, 0>(s_lo, s_hi, a, c, t, lo, tile, active);

    // store: columns fastest, so the last pass's bit-reversed scatter writes
    // runs of C consecutive outputs
    for (uint32_t u = tid; active && u < units; u += nthreads) {
        uint32_t e = grouped ? ((u & 7u) | ((u >> 4) << 3)) : (u >> 1);
        uint32_t half = grouped ? ((u >> 3) & 1u) : (u & 1u);
        uint32_t cc = e & (C - 1), d = e >> a.log_cols;
        size_t g = tile_dst(a, K, tile, d, cc);
        const uint4 *src = (half ? s_hi : s_lo) + smem_slot<K>(cc, d, a.log_cols);
        a.out[2 * g + half] = *src;
    }
    __syncthreads();
}

template <class F, int K>
__global__ void __launch_bounds__(256, 2) ntt_pass_kernel(const PassArgs a) {
    extern __shared__ uint4 smem[];
    for (uint32_t tile = blockIdx.x; tile < a.num_tiles; tile += gridDim.x)
        run_tile<F, K>(a, smem, tile);
}

}  // namespace zkntt
