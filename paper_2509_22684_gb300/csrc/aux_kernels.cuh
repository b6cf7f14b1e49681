// aux_kernels.cuh -- table generation, elementwise field kernels and the
// integer-pipe calibration kernel.
#pragma once
#include <cstdint>

#include "field.cuh"
#include "ntt_pass.cuh"

namespace zkntt {

// out[i] = hi[i >> split] * lo[i & (2^split - 1)]: the powers b^i from two
// small tables (b^(i_hi * 2^split) and b^i_lo)
template <class F>
__global__ void gen_powers_kernel(uint4 *out, uint32_t count, const uint4 *hi, const uint4 *lo,
                                  uint32_t split) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        uint32_t a[8], b[8];
        ldg_elem(a, hi + 2 * size_t(i >> split));
        ldg_elem(b, lo + 2 * size_t(i & ((1u << split) - 1u)));
        mul<F>(a, a, b);
        st_elem(out + 2 * size_t(i), a);
    }
}

// Inter-pass twiddle table, row-major by position d (so a tile of consecutive
// columns lo reads consecutive entries):
//   out[d * 2^lo_bits + lo] = w^(lo * rev_K(d)) * fl[lo] * fd[d]
// with w^e = w_hi[e >> split] * w_lo[e & mask] (any scalar factor folded into
// w_lo by the host).  fl / fd may be null.
template <class F>
__global__ void gen_twiddle_kernel(uint4 *out, uint32_t K, uint32_t lo_bits, const uint4 *w_hi,
                                   const uint4 *w_lo, uint32_t split, const uint4 *fl,
                                   const uint4 *fd) {
    const size_t total = size_t(1) << (lo_bits + K);
    for (size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
         idx += size_t(gridDim.x) * blockDim.x) {
        uint32_t d = uint32_t(idx >> lo_bits);
        uint32_t lo = uint32_t(idx & ((size_t(1) << lo_bits) - 1));
        uint32_t e = lo * brev_bits(d, K);  // < 2^(lo_bits + K)
        uint32_t a[8], b[8];
        ldg_elem(a, w_hi + 2 * size_t(e >> split));
        ldg_elem(b, w_lo + 2 * size_t(e & ((1u << split) - 1u)));
        mul<F>(a, a, b);
        if (fl) {
            ldg_elem(b, fl + 2 * size_t(lo));
            mul<F>(a, a, b);
        }
        if (fd) {
            ldg_elem(b, fd + 2 * size_t(d));
            mul<F>(a, a, b);
        }
        st_elem(out + 2 * idx, a);
    }
}

// out[i] = x[i] * hi[i >> split] * lo[i & (2^split - 1)]: with lo[t] = c base^t
// and hi[u] = base^(u 2^split) this is x[i] * c * base^i
template <class F>
__global__ void scale_powers_kernel(const uint4 *x, uint4 *out, size_t n, const uint4 *hi,
                                    const uint4 *lo, uint32_t split) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += size_t(gridDim.x) * blockDim.x) {
        uint32_t v[8], a[8], b[8];
        ldg_elem(a, hi + 2 * (i >> split));
        ldg_elem(b, lo + 2 * (i & ((size_t(1) << split) - 1)));
        mul<F>(a, a, b);
        ldg_elem(v, x + 2 * i);
        mul<F>(v, a, v);
        st_elem(out + 2 * i, v);
    }
}

// Powers w^k (k < 4) of the root used by the G-point transforms below
// (Montgomery form), passed by value.
struct BlockTw {
    uint32_t w[4][8];
};

// G-point transforms over whole blocks: for every column i < b,
//   out[k * b + i] = sum_r in[r * b + i] w^(r k)      (r, k < G; w of order G)
// by radix-2 decimation in frequency in registers (G/2 log2 G butterflies, the
// j = 0 ones without a product), then the bit-reversed positions written back
// in natural order.  One thread per column; each thread reads its whole
// column before writing, so in == out is allowed.
template <class F, int G>
__global__ void __launch_bounds__(128) block_dft_kernel(const uint4 *in, uint4 *out, size_t b,
                                                        const BlockTw tw) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < b;
         i += size_t(gridDim.x) * blockDim.x) {
        uint32_t v[G][8];
#pragma unroll
        for (int r = 0; r < G; r++) ldg_elem(v[r], in + 2 * (size_t(r) * b + i));
#pragma unroll
        for (int h = G / 2; h >= 1; h >>= 1) {
#pragma unroll
            for (int g0 = 0; g0 < G; g0 += 2 * h) {
#pragma unroll
                for (int j = 0; j < h; j++) {
                    uint32_t t[8];
                    if (j == 0) {
                        sub<F>(t, v[g0], v[g0 + h]);
                    } else {
                        sub_lazy<F>(t, v[g0 + j], v[g0 + j + h]);
                    }
                    add<F>(v[g0 + j], v[g0 + j], v[g0 + j + h]);
                    if (j == 0) {
#pragma unroll
                        for (int l = 0; l < 8; l++) v[g0 + h][l] = t[l];
                    } else {
                        mul<F>(v[g0 + j + h], tw.w[j * (G / (2 * h))], t);
                    }
                }
            }
        }
#pragma unroll
        for (int p = 0; p < G; p++) {
            int q = 0;
#pragma unroll
            for (int bit = 1; bit < G; bit <<= 1) q = (q << 1) | ((p & bit) ? 1 : 0);
            st_elem(out + 2 * (size_t(q) * b + i), v[p]);
        }
    }
}

// c = op(a, b) elementwise: 0 mul, 1 add, 2 sub
template <class F>
__global__ void field_op_kernel(int op, const uint4 *a, const uint4 *b, uint4 *c, size_t n) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += size_t(gridDim.x) * blockDim.x) {
        uint32_t x[8], y[8], z[8];
        ldg_elem(x, a + 2 * i);
        ldg_elem(y, b + 2 * i);
        if (op == 0) mul<F>(z, x, y);
        else if (op == 1) add<F>(z, x, y);
        else if (op == 2) sub<F>(z, x, y);
        else sub_lazy<F>(z, x, y);
        st_elem(c + 2 * i, z);
    }
}

// Groth16 pointwise on the coset: h = (a * b - c) * z
template <class F>
__global__ void pointwise_kernel(const uint4 *a, const uint4 *b, const uint4 *c, const uint4 *z,
                                 uint4 *h, size_t n) {
    uint32_t zz[8];
    ldg_elem(zz, z);
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += size_t(gridDim.x) * blockDim.x) {
        uint32_t x[8], y[8], w[8];
        ldg_elem(x, a + 2 * i);
        ldg_elem(y, b + 2 * i);
        mul<F>(x, x, y);
        ldg_elem(w, c + 2 * i);
        sub<F>(x, x, w);
        mul<F>(x, x, zz);
        st_elem(h + 2 * i, x);
    }
}

// Calibration: four independent chains of Montgomery products per thread, all
// in registers; one checksum word per thread keeps the work live.
template <class F>
__global__ void __launch_bounds__(256) mulbench_kernel(int iters, uint32_t *sink) {
    uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t x0[8], x1[8], x2[8], x3[8], y[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
        // small distinct canonical values (top limb cleared keeps them below r)
        uint32_t v = tid * 0x9E3779B9u + j * 0x85EBCA6Bu;
        x0[j] = v;
        x1[j] = v ^ 0x5bd1e995u;
        x2[j] = v + 0x27d4eb2fu;
        x3[j] = v * 3u + 1u;
        y[j] = v ^ 0xc2b2ae35u;
    }
    x0[7] = x1[7] = x2[7] = x3[7] = y[7] = 0;
    for (int it = 0; it < iters; it++) {
        mul<F>(x0, x0, y);
        mul<F>(x1, x1, y);
        mul<F>(x2, x2, y);
        mul<F>(x3, x3, y);
    }
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) acc ^= x0[j] ^ x1[j] ^ x2[j] ^ x3[j];
    sink[tid] = acc;
}

}  // namespace zkntt
