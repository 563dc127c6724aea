// fftconv_lg8.cu -- the FP32 pass kernels for transforms of 256 points with
// the length fixed at compile time (see FixedPassKernels in fftconv.cu).
#define SG_FFTCONV_KERNELS_ONLY
#include "fftconv.cu"

namespace sg {
FixedPassKernels fixed_pass_kernels_lg8() { return make_fixed_pass_kernels<8>(); }
}  // namespace sg
