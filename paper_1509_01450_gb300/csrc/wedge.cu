// wedge.cu -- the origin wedge's contribution per step (Sec. 3.2.1: the
// cells [0, r_in] x one azimuthal cell below the grid, and the third terms
// of Eq. 27-29, single sums over the wedge cells).
//
// Per target row i the wedge term is two phi-convolutions: of the wedge
// densities sigma_w with W[i, .] and of the grid's first row sigma_0 with
// V[i, .] (the wedge's radial slope is one-sided toward that row); the
// builder stores their phi-spectra as real tables tab[t][m][i] (t = Wr,
// Wphi, Vr, Vphi, the azimuthal ones as -i times the stored value).  In the
// column spectra of the passes (mode-major, rows i of mode m contiguous)
// the forward update is a rank-2 update of each mode's column,
//   B[m][i] += wpre[i] (Wr[m][i] s^_w + Vr[m][i] a_0),
//   C[m][i] += wpre[i] (-i) (Wphi[m][i] s^_w + Vphi[m][i] a_0),
// with s^_w the phi-DFT of sigma_w and a_0 = A[m][0] / wpre[0] that of
// sigma_0, applied between the column pass and the inverse-row pass.  Mode 0
// packs (DC, Nyquist) as the passes do: real parts use the m = 0 tables,
// imaginary parts the m = N_phi/2 ones, and the azimuthal terms vanish.
// The adjoint forms the transposed sums t(m) per mode, adds the V part to
// row 0 of the backward column spectra and returns gsigma_w as the inverse
// phi-DFT of the W part.  The DFTs of the one wedge row run in FP64 from
// the FP64 twiddle table (N_phi^2 / 2 products: negligible next to a pass).
#include "sg_internal.cuh"

namespace sg {

__device__ __forceinline__ double blk_sum(double v, double* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < nw; w++) s += red[w];
    return s;
}

template <typename T>
__global__ void __launch_bounds__(256) k_wedge_fwd(const typename CX<T>::t* __restrict__ A, typename CX<T>::t* B,
                                                   typename CX<T>::t* C, const T* __restrict__ sigw,
                                                   const T* __restrict__ tab, const T* __restrict__ wpre,
                                                   const double2* __restrict__ tw64, int nu, int nphi)
{
    typedef typename CX<T>::t V;
    __shared__ double red[8];
    const int m = blockIdx.x, half = nphi / 2, stride = SG_NMAX / nphi;
    const long tsz = (long)(half + 1) * nu;
    // s^_w(m) = sum_j sigma_w[j] e^{-2 pi i m j / N_phi}; mode 0: (DC, Nyquist)
    double sx = 0.0, sy = 0.0;
    for (int j = threadIdx.x; j < nphi; j += blockDim.x) {
        const double v = (double)sigw[j];
        if (m == 0) {
            sx += v;
            sy += (j & 1) ? -v : v;
        } else {
            const double2 w = tw64[(long)((m * j) & (nphi - 1)) * stride];
            sx += v * w.x;
            sy += v * w.y;
        }
    }
    sx = blk_sum(sx, red);
    sy = blk_sum(sy, red);
    const V a = A[(size_t)m * nu];
    const double i0 = 1.0 / (double)wpre[0];
    const double ax = a.x * i0, ay = a.y * i0;
    const T* Wr = tab + 0 * tsz + (long)m * nu;
    const T* Wp = tab + 1 * tsz + (long)m * nu;
    const T* Vr = tab + 2 * tsz + (long)m * nu;
    const T* Vp = tab + 3 * tsz + (long)m * nu;
    const T* WrN = tab + 0 * tsz + (long)half * nu;  // Nyquist (mode 0 only)
    const T* VrN = tab + 2 * tsz + (long)half * nu;
    for (int i = threadIdx.x; i < nu; i += blockDim.x) {
        const double w = (double)wpre[i];
        V b = B[(size_t)m * nu + i];
        if (m == 0) {
            b.x += (T)(w * ((double)Wr[i] * sx + (double)Vr[i] * ax));
            b.y += (T)(w * ((double)WrN[i] * sy + (double)VrN[i] * ay));
        } else {
            b.x += (T)(w * ((double)Wr[i] * sx + (double)Vr[i] * ax));
            b.y += (T)(w * ((double)Wr[i] * sy + (double)Vr[i] * ay));
            // -i (p s) = p (s.y - i s.x)
            const double px = (double)Wp[i] * sx + (double)Vp[i] * ax, py = (double)Wp[i] * sy + (double)Vp[i] * ay;
            V c = C[(size_t)m * nu + i];
            c.x += (T)(w * py);
            c.y -= (T)(w * px);
            C[(size_t)m * nu + i] = c;
        }
        B[(size_t)m * nu + i] = b;
    }
}

// The transpose: with A, C the column spectra of the weighted seeds gF_r,
// gF_phi and B the backward column pass's result,
//   t_W(m) = sum_i wpre[i] (Wr[m][i] A[m][i] + i Wphi[m][i] C[m][i]),  t_V likewise,
//   B[m][0] += t_V(m) / wpre[0],   tw[m] = t_W(m).
template <typename T>
__global__ void __launch_bounds__(256) k_wedge_bwd(const typename CX<T>::t* __restrict__ A,
                                                   const typename CX<T>::t* __restrict__ C, typename CX<T>::t* B,
                                                   const T* __restrict__ tab, const T* __restrict__ wpre,
                                                   double2* __restrict__ tw_out, int nu, int nphi)
{
    typedef typename CX<T>::t V;
    __shared__ double red[8];
    const int m = blockIdx.x, half = nphi / 2;
    const long tsz = (long)(half + 1) * nu;
    const T* Wr = tab + 0 * tsz + (long)m * nu;
    const T* Wp = tab + 1 * tsz + (long)m * nu;
    const T* Vr = tab + 2 * tsz + (long)m * nu;
    const T* Vp = tab + 3 * tsz + (long)m * nu;
    const T* WrN = tab + 0 * tsz + (long)half * nu;
    const T* VrN = tab + 2 * tsz + (long)half * nu;
    double wx = 0, wy = 0, vx = 0, vy = 0;
    for (int i = threadIdx.x; i < nu; i += blockDim.x) {
        const double w = (double)wpre[i];
        const V a = A[(size_t)m * nu + i];
        if (m == 0) {
            wx += w * (double)Wr[i] * a.x;
            wy += w * (double)WrN[i] * a.y;
            vx += w * (double)Vr[i] * a.x;
            vy += w * (double)VrN[i] * a.y;
        } else {
            const V c = C[(size_t)m * nu + i];
            // i p c = p (-c.y + i c.x)
            wx += w * ((double)Wr[i] * a.x - (double)Wp[i] * c.y);
            wy += w * ((double)Wr[i] * a.y + (double)Wp[i] * c.x);
            vx += w * ((double)Vr[i] * a.x - (double)Vp[i] * c.y);
            vy += w * ((double)Vr[i] * a.y + (double)Vp[i] * c.x);
        }
    }
    wx = blk_sum(wx, red);
    wy = blk_sum(wy, red);
    vx = blk_sum(vx, red);
    vy = blk_sum(vy, red);
    if (threadIdx.x == 0) {
        const double i0 = 1.0 / (double)wpre[0];
        V b = B[(size_t)m * nu];
        b.x += (T)(vx * i0);
        b.y += (T)(vy * i0);
        B[(size_t)m * nu] = b;
        tw_out[m] = make_double2(wx, wy);
    }
}

// gsigma_w[j] = sum over all modes of t(m) e^{+2 pi i m j / N_phi} for the
// real sequence whose half spectrum t holds (mode 0 packed (DC, Nyquist)).
template <typename T>
__global__ void k_wedge_idft(const double2* __restrict__ t, const double2* __restrict__ tw64, T* __restrict__ gsw,
                             int nphi)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x, half = nphi / 2, stride = SG_NMAX / nphi;
    if (j >= nphi) return;
    const double2 t0 = t[0];
    double s = t0.x + ((j & 1) ? -t0.y : t0.y), r = 0.0;
    for (int m = 1; m < half; m++) {
        const double2 w = tw64[(long)((m * j) & (nphi - 1)) * stride];  // e^{-i theta}
        const double2 v = t[m];
        r += v.x * w.x + v.y * w.y;  // Re(v e^{+i theta})
    }
    gsw[j] = (T)(s + 2.0 * r);
}

template <typename T>
cudaError_t launch_wedge(const PlanView& p, bool adjoint, cudaStream_t st)
{
    typedef typename CX<T>::t V;
    if (adjoint) {
        if (!p.gsigw) return cudaErrorInvalidValue;
        k_wedge_bwd<T><<<p.nphi / 2, 256, 0, st>>>((const V*)p.wa, (const V*)p.wc, (V*)p.wb, (const T*)p.wtab,
                                                   (const T*)p.wpre, (double2*)p.wtmp, p.nu, p.nphi);
        k_wedge_idft<T><<<(p.nphi + 255) / 256, 256, 0, st>>>((const double2*)p.wtmp, (const double2*)p.tw64,
                                                              (T*)p.gsigw, p.nphi);
    } else {
        if (!p.sigw) return cudaErrorInvalidValue;
        k_wedge_fwd<T><<<p.nphi / 2, 256, 0, st>>>((const V*)p.wa, (V*)p.wb, (V*)p.wc, (const T*)p.sigw,
                                                   (const T*)p.wtab, (const T*)p.wpre, (const double2*)p.tw64,
                                                   p.nu, p.nphi);
    }
    return cudaGetLastError();
}
template cudaError_t launch_wedge<float>(const PlanView&, bool, cudaStream_t);
template cudaError_t launch_wedge<double>(const PlanView&, bool, cudaStream_t);

}  // namespace sg
