// batch.cu -- the persistent batch kernel (one instantiation per field, every digit size).
#include "batch.cuh"
#include "kernels.h"

namespace zkntt {

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// ctrl[0]: next work item, ctrl[1]: abort word; done[s]: tiles retired per
// segment; status: sticky per-device error word read by the host.  Thread 0
// claims the block's next work item while the current tile is processed, so
// the atomic's round trip is hidden behind the tile; the claimed index waits in
// shared memory, which keeps the tile routine's register budget (64, for four
// blocks of 256 per SM) free of bookkeeping.  One kernel per field: the tile
// routine is inlined and its constants are immediates.
template <class F>
__global__ void __launch_bounds__(BATCH_THREADS, BATCH_MIN_BLOCKS)
    batch_kernel(const __grid_constant__ BatchTable tab, uint32_t *ctrl, uint32_t *done,
                 uint32_t *status) {
    extern __shared__ uint4 smem[];
    __shared__ uint32_t s_item, s_seg, s_stop, s_next;
    if (threadIdx.x == 0) s_next = atomicAdd(&ctrl[0], 1u);
    for (;;) {
        if (threadIdx.x == 0) {
            uint32_t stop = 0, segi = 0;
            const uint32_t item = s_next;
            if (item >= tab.total_items || *(volatile uint32_t *)&ctrl[1]) {
                stop = 1;
            } else {
                s_next = atomicAdd(&ctrl[0], 1u);  // claim ahead
                uint32_t lo = 0, hi = tab.nseg;    // last segment with first_item <= item
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (tab.seg[mid].first_item <= item) lo = mid;
                    else hi = mid;
                }
                segi = lo;
                const BatchSeg &sg = tab.seg[segi];
                for (int k = 0; k < 3 && !stop; k++) {
                    if (sg.dep[k] < 0) continue;
                    const uint32_t *cnt = done + sg.dep[k];
                    if (ld_acquire(cnt) >= sg.dep_tiles[k]) continue;
                    const unsigned long long t0 = global_ns();
                    while (ld_acquire(cnt) < sg.dep_tiles[k]) {
                        if (*(volatile uint32_t *)&ctrl[1]) { stop = 1; break; }
                        if (global_ns() - t0 > tab.timeout_ns) {
                            atomicExch(&ctrl[1], 1u);
                            atomicOr(status, BATCH_STATUS_TIMEOUT);
                            stop = 1;
                            break;
                        }
                        __nanosleep(256);
                    }
                }
            }
            s_item = item;
            s_seg = segi;
            s_stop = stop;
        }
        __syncthreads();
        if (s_stop) break;
        const BatchSeg &sg = tab.seg[s_seg];
        const uint32_t tile = s_item - sg.first_item;
        // one butterfly per thread per stage (as pass variant 5): small tiles
        // keep twice the threads of the block busy
        const uint32_t nt = pass_threads_for(sg.a.K, sg.a.log_cols, 5);
        // with the shared-twiddle pairing (one twiddle load for a thread's two
        // butterflies of a stage): the fused Groth16 sequences run 1-3% faster
        // from 2^16 up
#ifndef ZKNTT_BATCH_PAIR
#define ZKNTT_BATCH_PAIR 1
#endif
        run_tile<F, 1, false, false, ZKNTT_BATCH_PAIR>(sg.a, smem, tile, nt < BATCH_THREADS ? nt : BATCH_THREADS);
        // run_tile ends with a block barrier: every store of the tile is issued
        if (threadIdx.x == 0) {
            __threadfence();
            const uint32_t retired = atomicAdd(&done[s_seg], 1u) + 1u;
            if (sg.signal && retired == sg.ntiles && tab.flags) {
                // the transform's last tile: publish its completion to the host
                __threadfence_system();
                asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(tab.flags + sg.job),
                             "r"(tab.epoch)
                             : "memory");
            }
        }
    }
}

// Calibration of the 32-bit integer multiply-add rate (the peak the transform's
// roofline is quoted against) and of the multiply forms a Montgomery product
// is built from.  Every thread runs eight independent register chains of
//   mode 0: mad.lo.u32   x = lo(x * y) + z
//   mode 1: mad.wide.u32 x = lo(x) * y + x               (64-bit addend)
//   mode 2: mul.wide.u32 x = lo(x) * y                    (no addend)
//   mode 3: mad.hi.u32   x = hi(x * y) + z
//   mode 4: mad.lo.cc.u32 / madc.hi.u32 pair (x, c) = (lo(x y) + z, hi(x y) + carry):
//           two instructions per step
// Each chain's next step depends on its previous one, so nothing can be
// folded away; a checksum per thread keeps the chains live.  Count: 8 * iters
// steps per thread (16 * iters instructions in mode 4).
__global__ void __launch_bounds__(1024) imadbench_kernel(int mode, int iters, uint32_t *sink) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t y = tid * 0x9E3779B9u + 0x7f4a7c15u, z = tid ^ 0x85ebca6bu;
    uint32_t acc = 0;
    if (mode == 0 || mode == 3) {
        uint32_t x[8];
#pragma unroll
        for (int k = 0; k < 8; k++) x[k] = tid + 0x1000193u * k;
        if (mode == 0) {
            for (int it = 0; it < iters; it++) {
#pragma unroll
                for (int k = 0; k < 8; k++)
                    asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[k]) : "r"(y), "r"(z));
            }
        } else {
            for (int it = 0; it < iters; it++) {
#pragma unroll
                for (int k = 0; k < 8; k++)
                    asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(x[k]) : "r"(y), "r"(z));
            }
        }
#pragma unroll
        for (int k = 0; k < 8; k++) acc ^= x[k];
    } else if (mode == 1 || mode == 2) {
        uint64_t x[8];
#pragma unroll
        for (int k = 0; k < 8; k++) x[k] = tid + 0x1000193ull * k;
        if (mode == 1) {
            for (int it = 0; it < iters; it++) {
#pragma unroll
                for (int k = 0; k < 8; k++)
                    asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(x[k]) : "r"(uint32_t(x[k])), "r"(y));
            }
        } else {
            for (int it = 0; it < iters; it++) {
#pragma unroll
                for (int k = 0; k < 8; k++)
                    asm volatile("mul.wide.u32 %0, %1, %2;" : "=l"(x[k]) : "r"(uint32_t(x[k]) ^ uint32_t(x[k] >> 32)), "r"(y));
            }
        }
#pragma unroll
        for (int k = 0; k < 8; k++) acc ^= uint32_t(x[k]) ^ uint32_t(x[k] >> 32);
    } else {
        uint32_t x[8], c[8];
#pragma unroll
        for (int k = 0; k < 8; k++) {
            x[k] = tid + 0x1000193u * k;
            c[k] = 0;
        }
        for (int it = 0; it < iters; it++) {
#pragma unroll
            for (int k = 0; k < 8; k++)
                asm volatile("mad.lo.cc.u32 %0, %0, %2, %3;\n\t"
                             "madc.hi.u32 %1, %0, %2, %1;"
                             : "+r"(x[k]), "+r"(c[k])
                             : "r"(y), "r"(z));
        }
#pragma unroll
        for (int k = 0; k < 8; k++) acc ^= x[k] ^ c[k];
    }
    sink[tid] = acc;
}

const void *imadbench_kernel_ptr() { return (const void *)&imadbench_kernel; }

const void *batch_kernel_ptr(int field) {
    if (field == 1) return (const void *)&batch_kernel<FrBN254>;
    if (field == 2) return (const void *)&batch_kernel<FrBLS12_377>;
    return (const void *)&batch_kernel<FrBLS12_381>;
}

}  // namespace zkntt
