// fftconv_df.cu -- the passes of the compensated FP32 plans (SG_F32X2):
// fftconv.cu's run-time-length kernels instantiated on double-float values
// (sg_df.cuh), and the conversions between the API's FP64 fields and the
// double-float working fields.
#define SG_FFTCONV_DF
#include "fftconv.cu"

namespace sg {

// x -> (fl(x), fl(x - fl(x))): the nearest double-float, exact to about 2^-48
__global__ void __launch_bounds__(256) k_to_df(const double* __restrict__ in, dfloat* __restrict__ out, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double x = in[i];
        const float h = __double2float_rn(x);
        out[i] = dfloat(h, __double2float_rn(x - (double)h));
    }
}
__global__ void __launch_bounds__(256) k_from_df(const dfloat* __restrict__ in, double* __restrict__ out, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = df_to_double(in[i]);
}

static int conv_grid(size_t n, int sms)
{
    const size_t blocks = (n + 255) / 256;
    const size_t cap = (size_t)sms * 8;
    return (int)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

cudaError_t launch_to_df(const double* in, dfloat* out, size_t n, int sms, cudaStream_t st)
{
    k_to_df<<<conv_grid(n, sms), 256, 0, st>>>(in, out, n);
    return cudaGetLastError();
}
cudaError_t launch_from_df(const dfloat* in, double* out, size_t n, int sms, cudaStream_t st)
{
    k_from_df<<<conv_grid(n, sms), 256, 0, st>>>(in, out, n);
    return cudaGetLastError();
}

template cudaError_t launch_forward<dfloat>(const PlanView&, const dfloat*, dfloat*, dfloat*, cudaStream_t,
                                            cudaEvent_t*, bool);
template cudaError_t launch_backward<dfloat>(const PlanView&, const dfloat*, const dfloat*, dfloat*, cudaStream_t,
                                             cudaEvent_t*);
template cudaError_t launch_spectra<dfloat2>(const PlanView&, const double*, const double*, double2*, dfloat2*,
                                             dfloat2*, cudaStream_t);
}  // namespace sg
