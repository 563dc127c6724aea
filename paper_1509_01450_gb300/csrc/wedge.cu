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
// sigma_0, applied between the column pass and the inverse-row pass by
// k_wedge_fwd, or, for FP32 columns of 16 points per thread, inside the
// forward column pass with s^_w formed ahead by k_wedge_dft.  Mode 0
// packs (DC, Nyquist) as the passes do: real parts use the m = 0 tables,
// imaginary parts the m = N_phi/2 ones, and the azimuthal terms vanish.
// The adjoint forms the transposed sums t(m) per mode, adds the V part to
// row 0 of the backward column spectra and returns gsigma_w as the inverse
// phi-DFT of the W part.  All arithmetic is in the plan's dtype with the
// plan's twiddle table (GB300's FP64 rate would make FP64 sums here cost
// more than a pass); the direct DFTs of the one wedge row take N_phi^2 / 2
// products, spread over one block per mode (forward) or per output (adjoint).
#include "sg_internal.cuh"

namespace sg {

// e^{-2 pi i (a b mod N) / N} from the plan's table (length SG_NMAX)
template <typename V>
__device__ __forceinline__ V tw_at(const V* tw, long a, long b, int nphi)
{
    return tw[((a * b) & (nphi - 1)) * (SG_NMAX / nphi)];
}

// sum_j x[j] e^{-2 pi i m j / N} over this thread's j = threadIdx.x + k
// blockDim.x: the twiddle advances by a product per step (two table loads
// per thread instead of one scattered load per term)
template <typename T, typename V>
__device__ __forceinline__ void dft_partial(const T* __restrict__ x, const V* __restrict__ tw, int m, int nphi,
                                            T& sx, T& sy)
{
    V w = tw_at(tw, m, threadIdx.x, nphi);
    const V st = tw_at(tw, m, blockDim.x, nphi);
    for (int j = threadIdx.x; j < nphi; j += blockDim.x) {
        const T v = x[j];
        sx += v * w.x;
        sy += v * w.y;
        w = V{w.x * st.x - w.y * st.y, w.x * st.y + w.y * st.x};
    }
}

template <typename T>
__device__ __forceinline__ T blk_sum(T v, T* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += sg_shfl_xor(v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    T s = 0;
    for (int w = 0; w < nw; w++) s += red[w];
    return s;
}

// ps: element stride (in complex values) of B and C: 1, or 2 in the pair layout
template <typename T>
__global__ void __launch_bounds__(256) k_wedge_fwd(const typename CX<T>::t* __restrict__ A, typename CX<T>::t* B,
                                                   typename CX<T>::t* C, const T* __restrict__ sigw,
                                                   const T* __restrict__ tab, const T* __restrict__ wpre,
                                                   const typename CX<T>::t* __restrict__ tw, int nu, int nphi, int ps)
{
    typedef typename CX<T>::t V;
    __shared__ T red[8];
    const int m = blockIdx.x, half = nphi / 2;
    const long tsz = (long)(half + 1) * nu;
    // s^_w(m) = sum_j sigma_w[j] e^{-2 pi i m j / N_phi}; mode 0: (DC, Nyquist)
    T sx = 0, sy = 0;
    if (m == 0) {
        for (int j = threadIdx.x; j < nphi; j += blockDim.x) {
            const T v = sigw[j];
            sx += v;
            sy += (j & 1) ? -v : v;
        }
    } else {
        dft_partial(sigw, tw, m, nphi, sx, sy);
    }
    sx = blk_sum(sx, red);
    sy = blk_sum(sy, red);
    const V a = A[(size_t)m * nu];
    const T i0 = (T)1 / wpre[0];
    const T ax = a.x * i0, ay = a.y * i0;
    const T* Wr = tab + 0 * tsz + (long)m * nu;
    const T* Wp = tab + 1 * tsz + (long)m * nu;
    const T* Vr = tab + 2 * tsz + (long)m * nu;
    const T* Vp = tab + 3 * tsz + (long)m * nu;
    const T* WrN = tab + 0 * tsz + (long)half * nu;  // Nyquist (mode 0 only)
    const T* VrN = tab + 2 * tsz + (long)half * nu;
    for (int i = threadIdx.x; i < nu; i += blockDim.x) {
        const T w = wpre[i];
        V b = B[((size_t)m * nu + i) * ps];
        if (m == 0) {
            b.x += w * (Wr[i] * sx + Vr[i] * ax);
            b.y += w * (WrN[i] * sy + VrN[i] * ay);
        } else {
            b.x += w * (Wr[i] * sx + Vr[i] * ax);
            b.y += w * (Wr[i] * sy + Vr[i] * ay);
            // -i (p s) = p (s.y - i s.x)
            const T px = Wp[i] * sx + Vp[i] * ax, py = Wp[i] * sy + Vp[i] * ay;
            V c = C[((size_t)m * nu + i) * ps];
            c.x += w * py;
            c.y -= w * px;
            C[((size_t)m * nu + i) * ps] = c;
        }
        B[((size_t)m * nu + i) * ps] = b;
    }
}

// The transpose: with A, C the column spectra of the weighted seeds gF_r,
// gF_phi and B the backward column pass's result,
//   t_W(m) = sum_i wpre[i] (Wr[m][i] A[m][i] + i Wphi[m][i] C[m][i]),  t_V likewise,
//   B[m][0] += t_V(m) / wpre[0],   tw[m] = t_W(m).
// ps: element stride (in complex values) of A and C: 1, or 2 in the pair layout
template <typename T>
__global__ void __launch_bounds__(256) k_wedge_bwd(const typename CX<T>::t* __restrict__ A,
                                                   const typename CX<T>::t* __restrict__ C, typename CX<T>::t* B,
                                                   const T* __restrict__ tab, const T* __restrict__ wpre,
                                                   typename CX<T>::t* __restrict__ t_out, int nu, int nphi, int ps)
{
    typedef typename CX<T>::t V;
    __shared__ T red[8];
    const int m = blockIdx.x, half = nphi / 2;
    const long tsz = (long)(half + 1) * nu;
    const T* Wr = tab + 0 * tsz + (long)m * nu;
    const T* Wp = tab + 1 * tsz + (long)m * nu;
    const T* Vr = tab + 2 * tsz + (long)m * nu;
    const T* Vp = tab + 3 * tsz + (long)m * nu;
    const T* WrN = tab + 0 * tsz + (long)half * nu;
    const T* VrN = tab + 2 * tsz + (long)half * nu;
    T wx = 0, wy = 0, vx = 0, vy = 0;
    for (int i = threadIdx.x; i < nu; i += blockDim.x) {
        const T w = wpre[i];
        const V a = A[((size_t)m * nu + i) * ps];
        if (m == 0) {
            wx += w * Wr[i] * a.x;
            wy += w * WrN[i] * a.y;
            vx += w * Vr[i] * a.x;
            vy += w * VrN[i] * a.y;
        } else {
            const V c = C[((size_t)m * nu + i) * ps];
            // i p c = p (-c.y + i c.x)
            wx += w * (Wr[i] * a.x - Wp[i] * c.y);
            wy += w * (Wr[i] * a.y + Wp[i] * c.x);
            vx += w * (Vr[i] * a.x - Vp[i] * c.y);
            vy += w * (Vr[i] * a.y + Vp[i] * c.x);
        }
    }
    wx = blk_sum(wx, red);
    wy = blk_sum(wy, red);
    vx = blk_sum(vx, red);
    vy = blk_sum(vy, red);
    if (threadIdx.x == 0) {
        const T i0 = (T)1 / wpre[0];
        V b = B[(size_t)m * nu];
        b.x += vx * i0;
        b.y += vy * i0;
        B[(size_t)m * nu] = b;
        t_out[m] = V{wx, wy};
    }
}

// gsigma_w[j] = sum over all modes of t(m) e^{+2 pi i m j / N_phi} for the
// real sequence whose half spectrum t holds (mode 0 packed (DC, Nyquist)):
// one block per output j, the modes split over its threads.
template <typename T>
__global__ void __launch_bounds__(256) k_wedge_idft(const typename CX<T>::t* __restrict__ t,
                                                    const typename CX<T>::t* __restrict__ tw, T* __restrict__ gsw,
                                                    int nphi)
{
    typedef typename CX<T>::t V;
    __shared__ T red[8];
    const int j = blockIdx.x, half = nphi / 2;
    T r = 0;
    V w = tw_at(tw, 1 + threadIdx.x, j, nphi);  // e^{-i theta}, theta = 2 pi m j / N
    const V st = tw_at(tw, blockDim.x, j, nphi);
    for (int m = 1 + threadIdx.x; m < half; m += blockDim.x) {
        const V v = t[m];
        r += v.x * w.x + v.y * w.y;  // Re(v e^{+i theta})
        w = V{w.x * st.x - w.y * st.y, w.x * st.y + w.y * st.x};
    }
    r = blk_sum(r, red);
    if (threadIdx.x == 0) {
        const V t0 = t[0];
        gsw[j] = t0.x + ((j & 1) ? -t0.y : t0.y) + 2 * r;
    }
}

// s^_w(m) for every mode, for the update fused into the forward column
// pass: one block per mode, mode 0 packed (DC, Nyquist).
template <typename T>
__global__ void __launch_bounds__(256) k_wedge_dft(const T* __restrict__ sigw, const typename CX<T>::t* __restrict__ tw,
                                                   typename CX<T>::t* __restrict__ swh, int nphi)
{
    typedef typename CX<T>::t V;
    __shared__ T red[8];
    const int m = blockIdx.x;
    T sx = 0, sy = 0;
    if (m == 0) {
        for (int j = threadIdx.x; j < nphi; j += blockDim.x) {
            const T v = sigw[j];
            sx += v;
            sy += (j & 1) ? -v : v;
        }
    } else {
        dft_partial(sigw, tw, m, nphi, sx, sy);
    }
    sx = blk_sum(sx, red);
    sy = blk_sum(sy, red);
    if (threadIdx.x == 0) swh[m] = V{sx, sy};
}

template <typename T>
cudaError_t launch_wedge_dft(const PlanView& p, cudaStream_t st)
{
    typedef typename CX<T>::t V;
    if (!p.sigw) return cudaErrorInvalidValue;
    k_wedge_dft<T><<<p.nphi / 2, 256, 0, st>>>((const T*)p.sigw, (const V*)p.tw, (V*)p.wtmp, p.nphi);
    return cudaGetLastError();
}
template cudaError_t launch_wedge_dft<float>(const PlanView&, cudaStream_t);
template cudaError_t launch_wedge_dft<double>(const PlanView&, cudaStream_t);
template cudaError_t launch_wedge_dft<dfloat>(const PlanView&, cudaStream_t);

template <typename T>
cudaError_t launch_wedge(const PlanView& p, bool adjoint, cudaStream_t st)
{
    typedef typename CX<T>::t V;
    // the pair layout: wb holds (B, C) forward and (A, C) in the adjoint, wa the adjoint's B
    const int ps = p.pairs ? 2 : 1;
    V* const X = (V*)p.wb;
    V* const Y = p.pairs ? (V*)p.wb + 1 : (V*)p.wc;
    if (adjoint) {
        if (!p.gsigw) return cudaErrorInvalidValue;
        k_wedge_bwd<T><<<p.nphi / 2, 256, 0, st>>>(p.pairs ? X : (const V*)p.wa, Y, p.pairs ? (V*)p.wa : X,
                                                   (const T*)p.wtab, (const T*)p.wpre, (V*)p.wtmp, p.nu, p.nphi, ps);
        k_wedge_idft<T><<<p.nphi, 256, 0, st>>>((const V*)p.wtmp, (const V*)p.tw, (T*)p.gsigw, p.nphi);
    } else {
        if (!p.sigw) return cudaErrorInvalidValue;
        k_wedge_fwd<T><<<p.nphi / 2, 256, 0, st>>>((const V*)p.wa, X, Y, (const T*)p.sigw, (const T*)p.wtab,
                                                   (const T*)p.wpre, (const V*)p.tw, p.nu, p.nphi, ps);
    }
    return cudaGetLastError();
}
template cudaError_t launch_wedge<float>(const PlanView&, bool, cudaStream_t);
template cudaError_t launch_wedge<double>(const PlanView&, bool, cudaStream_t);
template cudaError_t launch_wedge<dfloat>(const PlanView&, bool, cudaStream_t);

}  // namespace sg
