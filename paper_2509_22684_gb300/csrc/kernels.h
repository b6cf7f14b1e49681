// kernels.h -- per-field table of kernel entry points, filled by the
// field-specific translation units and used by the host runtime.
#pragma once
#include <cstdint>

namespace zkntt {

constexpr int MAX_DIGIT_BITS = 11;  // largest sub-transform a block holds (2^11 x 32 B = 64 KiB)
constexpr int MAX_TILE_BITS = 11;   // tiles hold at most 2^11 elements (C x 2^K)

struct FieldKernels {
    const void *pass[8];  // ntt_pass_kernel<F, V> at index V = 1..7 (digit size is a runtime argument)
    const void *gen_powers;
    const void *gen_twiddle;
    const void *field_op;
    const void *pointwise;
    const void *mulbench;
    const void *scale_powers;
    const void *block_dft[4];  // block_dft_kernel<F, 2^g> at index g = 1..3
};

const FieldKernels &kernels_bls12_381();
const FieldKernels &kernels_bn254();
const FieldKernels &kernels_bls12_377();

// fields with kernels, ids 0 .. NUM_FIELDS - 1 (the zkntt_field values)
constexpr int NUM_FIELDS = 3;
// pass-kernel schedule variants, 1 .. NUM_VARIANTS (the plan's `ilp` option)
constexpr int NUM_VARIANTS = 7;
// variants the autotuner tries (1 .. TUNED_VARIANTS)
constexpr int TUNED_VARIANTS = 5;
const void *batch_kernel_ptr(int field);
// the 32-bit multiply-add rate calibration kernel (field-independent)
const void *imadbench_kernel_ptr();

}  // namespace zkntt
