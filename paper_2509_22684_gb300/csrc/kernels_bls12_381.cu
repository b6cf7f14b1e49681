// kernels_bls12_381.cu -- kernel instantiations for the bls12_381 scalar field.
#include "aux_kernels.cuh"
#include "kernels.h"
#include "ntt_pass.cuh"

namespace zkntt {

const FieldKernels &kernels_bls12_381() {
    using F = FrBLS12_381;
    static const FieldKernels k = {
        {nullptr, (const void *)&ntt_pass_kernel<F, 1>, (const void *)&ntt_pass_kernel<F, 2>,
         (const void *)&ntt_pass_kernel<F, 3>, (const void *)&ntt_pass_kernel<F, 4>,
         (const void *)&ntt_pass_kernel<F, 5>, (const void *)&ntt_pass_kernel<F, 6>,
         (const void *)&ntt_pass_kernel<F, 7>},
        (const void *)&gen_powers_kernel<F>,
        (const void *)&gen_twiddle_kernel<F>,
        (const void *)&field_op_kernel<F>,
        (const void *)&pointwise_kernel<F>,
        (const void *)&mulbench_kernel<F>,
        (const void *)&scale_powers_kernel<F>,
        {nullptr, (const void *)&block_dft_kernel<F, 2>, (const void *)&block_dft_kernel<F, 4>,
         (const void *)&block_dft_kernel<F, 8>},
    };
    return k;
}

}  // namespace zkntt
