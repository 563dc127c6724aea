// fftconv.cu -- FFT convolution passes of the thin-disk force (sm_103a).
//
// The forces are the convolution (zero-padded to L = 2 N_u rows in u,
// periodic in phi) of the weighted density w = sigma beta^{p i} with the
// weighted kernel spectra Khat (built once, kbuild.cu), evaluated in three
// passes per direction:
//
//  forward  P1 rows   : R2C along phi of w (two rows per complex FFT),
//                       half spectra to the column-block buffer A
//  forward  P2 columns: per phi-mode: zero-padded FFT of length L, times
//                       Khat_r and Khat_phi, two inverse FFTs, crop to N_u
//                       rows; written row-major to B (r) and C (phi)
//  forward  P3 rows   : one inverse FFT of Z = F_r + i F_phi per row,
//                       scaled by beta^{-p i}
//  backward P1b rows  : FFT of (gF_r + i gF_phi) beta^{-p i}, split into the
//                       two half spectra (column-block buffers A and C)
//  backward P2b cols  : FFT of both columns, times conj(Khat), summed, one
//                       inverse FFT, crop; row-major to B
//  backward P3b rows  : inverse real FFT of two rows at once, times beta^{p i}
//
// Half spectra along phi keep modes 0..N_phi/2-1, with the real DC and
// Nyquist values packed into mode 0 as (DC, Nyquist).  The column-block
// layout stores mode m of row i at ((m / CB) N_u + i) CB + m mod CB, so a
// column block is contiguous for P2 and a row writes CB-wide chunks.
//
// Khat storage (per mode m = 0..N_phi/2, stride KS = N_u + 2): kappa =
// 0..N_u of the L-point spectrum; Khat_r is Hermitian in kappa
// (Khat_r[L - kappa] = conj Khat_r[kappa]) and Khat_phi anti-Hermitian.
// Khat_phi vanishes at modes 0 and N_phi/2 (odd kernel).
#include "sg_internal.cuh"

namespace sg {

// ---------------------------------------------------------------------------
// Kernel spectrum at index kappa in [0, L) from the symmetry-reduced store
// ---------------------------------------------------------------------------
template <typename V>
__device__ __forceinline__ V khat_r(const V* __restrict__ K, int kappa, int L, int nu)
{
    return kappa <= nu ? __ldg(&K[kappa]) : cconj(__ldg(&K[L - kappa]));
}
template <typename V>
__device__ __forceinline__ V khat_p(const V* __restrict__ K, int kappa, int L, int nu)
{
    if (kappa <= nu) return __ldg(&K[kappa]);
    V a = __ldg(&K[L - kappa]);
    return V{-a.x, a.y};  // -conj
}

// ===========================================================================
// Forward P1: rows (i0, i1) packed as z = w_i0 + i w_i1, FFT along phi,
// split X_i0[m] = (Z[m] + conj Z[N-m]) / 2, X_i1[m] = (Z[m] - conj Z[N-m]) / 2i.
// ===========================================================================
template <typename T, int E>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 256 : 512) k_fwd_rows(const T* __restrict__ sigma, const T* __restrict__ wpre,
                                                  typename CX<T>::t* __restrict__ A, int nu, int nphi, int log2n,
                                                  int cb, const typename CX<T>::t* __restrict__ tw)
{
    typedef typename CX<T>::t V;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* small = reinterpret_cast<V*>(smraw);
    const int N = nphi, NT = N / E;
    const int slot = threadIdx.x / NT, t = threadIdx.x % NT;
    const int slots = blockDim.x / NT;
    V* sm = small + slot * sg_padded(N);
    const int pair = blockIdx.x * slots + slot;
    const bool live = pair < nu / 2;
    const int i0 = 2 * (live ? pair : 0), i1 = i0 + 1;
    const T w0 = wpre[i0], w1 = wpre[i1];
    V v[E];
#pragma unroll
    for (int e = 0; e < E; e++) {
        const int n = t + e * NT;
        v[e] = V{sigma[(size_t)i0 * N + n] * w0, sigma[(size_t)i1 * N + n] * w1};
    }
    sg_fft<E, -1>(v, sm, N, log2n, t, tw);
#pragma unroll
    for (int e = 0; e < E; e++) sm[sg_pad(t + e * NT)] = v[e];
    __syncthreads();
    if (!live) return;
    const T h = (T)0.5;
#pragma unroll
    for (int e = 0; e < E / 2; e++) {
        const int m = t + e * NT;
        V z = v[e], zc = cconj(sm[sg_pad((N - m) & (N - 1))]);
        V x0, x1;
        if (m == 0) {
            const V zn = sm[sg_pad(N / 2)];
            x0 = V{z.x, zn.x};
            x1 = V{z.y, zn.y};
        } else {
            x0 = cscale(cadd(z, zc), h);
            V d = csub(z, zc);
            x1 = V{d.y * h, -d.x * h};  // d / 2i
        }
        const size_t blk = (size_t)(m / cb) * nu;
        A[(blk + i0) * cb + (m % cb)] = x0;
        A[(blk + i1) * cb + (m % cb)] = x1;
    }
}

// ===========================================================================
// Forward P2: one phi-mode column per slot.
// ===========================================================================
template <typename T, int E>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 256 : 512) k_fwd_cols(const typename CX<T>::t* __restrict__ A,
                                                  const typename CX<T>::t* __restrict__ Kr,
                                                  const typename CX<T>::t* __restrict__ Kp,
                                                  typename CX<T>::t* __restrict__ Br,
                                                  typename CX<T>::t* __restrict__ Cp, int nu, int nphi, int log2L,
                                                  int cb, const typename CX<T>::t* __restrict__ tw)
{
    typedef typename CX<T>::t V;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* small = reinterpret_cast<V*>(smraw);
    const int L = 2 * nu, NT = L / E, half = nphi / 2, KS = nu + 2;
    const int slot = threadIdx.x / NT, t = threadIdx.x % NT;
    const int slots = blockDim.x / NT;
    V* sm = small + slot * sg_padded(L);
    const int m0 = blockIdx.x * slots + slot;
    const bool live = m0 < half;
    const int m = live ? m0 : 0;
    const size_t blk = (size_t)(m / cb) * nu;
    const int cm = m % cb;
    V v[E], x[E];
#pragma unroll
    for (int e = 0; e < E; e++) {
        const int i = t + e * NT;
        v[e] = (e < E / 2) ? A[(blk + i) * cb + cm] : V{0, 0};  // rows >= nu are the zero pad
    }
    sg_fft<E, -1>(v, sm, L, log2L, t, tw);
#pragma unroll
    for (int e = 0; e < E; e++) x[e] = v[e];
    const V* kr = Kr + (size_t)m * KS;
    const V* kp = Kp + (size_t)m * KS;
    // every slot takes the same branch only if the block holds one column,
    // so the packed mode-0 column uses block-wide exchanges unconditionally
    // in the block that contains it
    const bool packed_block = (blockIdx.x == 0);
    if (packed_block) {
#pragma unroll
        for (int e = 0; e < E; e++) sm[sg_pad(t + e * NT)] = x[e];
        __syncthreads();
        if (m == 0) {
            // x holds the FFT of (DC + i Nyquist); separate the two real
            // sequences and apply the kernels of modes 0 and N_phi/2
            const V* krn = Kr + (size_t)half * KS;
            const float hf = 0.5f;
#pragma unroll
            for (int e = 0; e < E; e++) {
                const int k = t + e * NT;
                V z = x[e], zc = cconj(sm[sg_pad((L - k) & (L - 1))]);
                V a = cscale(cadd(z, zc), (T)hf);
                V d = csub(z, zc);
                V b = V{d.y * (T)hf, -d.x * (T)hf};
                v[e] = cadd(cmul(a, khat_r(kr, k, L, nu)), cmuli(cmul(b, khat_r(krn, k, L, nu))));
            }
        } else {
#pragma unroll
            for (int e = 0; e < E; e++) v[e] = cmul(x[e], khat_r(kr, t + e * NT, L, nu));
        }
    } else {
#pragma unroll
        for (int e = 0; e < E; e++) v[e] = cmul(x[e], khat_r(kr, t + e * NT, L, nu));
    }
    sg_fft<E, +1>(v, sm, L, log2L, t, tw);
    if (live) {
#pragma unroll
        for (int e = 0; e < E / 2; e++) Br[(size_t)(t + e * NT) * half + m] = v[e];
    }
    if (m == 0) {
#pragma unroll
        for (int e = 0; e < E; e++) v[e] = V{0, 0};
    } else {
#pragma unroll
        for (int e = 0; e < E; e++) v[e] = cmul(x[e], khat_p(kp, t + e * NT, L, nu));
    }
    sg_fft<E, +1>(v, sm, L, log2L, t, tw);
    if (live) {
#pragma unroll
        for (int e = 0; e < E / 2; e++) Cp[(size_t)(t + e * NT) * half + m] = v[e];
    }
}

// ===========================================================================
// Forward P3: row i, Zhat = Fhat_r + i Fhat_phi (Hermitian halves expanded),
// inverse FFT, F_r = Re, F_phi = Im, times beta^{-p i}.
// ===========================================================================
template <typename T, int E>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 256 : 512) k_fwd_rows_inv(const typename CX<T>::t* __restrict__ Br,
                                                      const typename CX<T>::t* __restrict__ Cp,
                                                      const T* __restrict__ wpost, T* __restrict__ Fr,
                                                      T* __restrict__ Fp, int nu, int nphi, int log2n,
                                                      const typename CX<T>::t* __restrict__ tw)
{
    typedef typename CX<T>::t V;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* small = reinterpret_cast<V*>(smraw);
    const int N = nphi, NT = N / E, half = N / 2;
    const int slot = threadIdx.x / NT, t = threadIdx.x % NT;
    const int slots = blockDim.x / NT;
    V* sm = small + slot * sg_padded(N);
    const int i0 = blockIdx.x * slots + slot;
    const bool live = i0 < nu;
    const int i = live ? i0 : 0;
    const V* br = Br + (size_t)i * half;
    const V* cp = Cp + (size_t)i * half;
    V v[E];
#pragma unroll
    for (int e = 0; e < E; e++) {
        const int n = t + e * NT;
        V z;
        if (e < E / 2) {
            if (n == 0) {
                z = V{br[0].x, 0};
            } else {
                const V a = br[n], b = cp[n];
                z = V{a.x - b.y, a.y + b.x};  // a + i b
            }
        } else {
            if (n == half) {
                z = V{br[0].y, 0};
            } else {
                const V a = br[N - n], b = cp[N - n];
                z = V{a.x + b.y, -a.y + b.x};  // conj a + i conj b
            }
        }
        v[e] = z;
    }
    sg_fft<E, +1>(v, sm, N, log2n, t, tw);
    if (!live) return;
    const T w = wpost[i];
#pragma unroll
    for (int e = 0; e < E; e++) {
        const int n = t + e * NT;
        Fr[(size_t)i * N + n] = v[e].x * w;
        Fp[(size_t)i * N + n] = v[e].y * w;
    }
}

// ===========================================================================
// Backward P1b: row i, z = (gF_r + i gF_phi) beta^{-p i}, FFT, split into
// the half spectra of gF_r (-> A) and gF_phi (-> C), column-block layout.
// ===========================================================================
template <typename T, int E>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 256 : 512) k_bwd_rows(const T* __restrict__ gr, const T* __restrict__ gp,
                                                  const T* __restrict__ wpost, typename CX<T>::t* __restrict__ A,
                                                  typename CX<T>::t* __restrict__ C, int nu, int nphi, int log2n,
                                                  int cb, const typename CX<T>::t* __restrict__ tw)
{
    typedef typename CX<T>::t V;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* small = reinterpret_cast<V*>(smraw);
    const int N = nphi, NT = N / E;
    const int slot = threadIdx.x / NT, t = threadIdx.x % NT;
    const int slots = blockDim.x / NT;
    V* sm = small + slot * sg_padded(N);
    const int i0 = blockIdx.x * slots + slot;
    const bool live = i0 < nu;
    const int i = live ? i0 : 0;
    const T w = wpost[i];
    V v[E];
#pragma unroll
    for (int e = 0; e < E; e++) {
        const int n = t + e * NT;
        v[e] = V{gr[(size_t)i * N + n] * w, gp[(size_t)i * N + n] * w};
    }
    sg_fft<E, -1>(v, sm, N, log2n, t, tw);
#pragma unroll
    for (int e = 0; e < E; e++) sm[sg_pad(t + e * NT)] = v[e];
    __syncthreads();
    if (!live) return;
    const T h = (T)0.5;
#pragma unroll
    for (int e = 0; e < E / 2; e++) {
        const int m = t + e * NT;
        V z = v[e], zc = cconj(sm[sg_pad((N - m) & (N - 1))]);
        V x0, x1;
        if (m == 0) {
            const V zn = sm[sg_pad(N / 2)];
            x0 = V{z.x, zn.x};
            x1 = V{z.y, zn.y};
        } else {
            x0 = cscale(cadd(z, zc), h);
            V d = csub(z, zc);
            x1 = V{d.y * h, -d.x * h};
        }
        const size_t idx = ((size_t)(m / cb) * nu + i) * cb + (m % cb);
        A[idx] = x0;
        C[idx] = x1;
    }
}

// ===========================================================================
// Backward P2b: column m: FFT of both zero-padded columns, times conj(Khat),
// summed, inverse FFT, crop; row-major to B.
// ===========================================================================
template <typename T, int E>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 256 : 512) k_bwd_cols(const typename CX<T>::t* __restrict__ A,
                                                  const typename CX<T>::t* __restrict__ C,
                                                  const typename CX<T>::t* __restrict__ Kr,
                                                  const typename CX<T>::t* __restrict__ Kp,
                                                  typename CX<T>::t* __restrict__ B, int nu, int nphi, int log2L,
                                                  int cb, const typename CX<T>::t* __restrict__ tw)
{
    typedef typename CX<T>::t V;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* small = reinterpret_cast<V*>(smraw);
    const int L = 2 * nu, NT = L / E, half = nphi / 2, KS = nu + 2;
    const int slot = threadIdx.x / NT, t = threadIdx.x % NT;
    const int slots = blockDim.x / NT;
    V* sm = small + slot * sg_padded(L);
    const int m0 = blockIdx.x * slots + slot;
    const bool live = m0 < half;
    const int m = live ? m0 : 0;
    const size_t blk = (size_t)(m / cb) * nu;
    const int cm = m % cb;
    const V* kr = Kr + (size_t)m * KS;
    const V* kp = Kp + (size_t)m * KS;
    V v[E], y[E];
#pragma unroll
    for (int e = 0; e < E; e++) v[e] = (e < E / 2) ? A[(blk + t + e * NT) * cb + cm] : V{0, 0};
    sg_fft<E, -1>(v, sm, L, log2L, t, tw);
    const bool packed_block = (blockIdx.x == 0);
    if (packed_block) {
#pragma unroll
        for (int e = 0; e < E; e++) sm[sg_pad(t + e * NT)] = v[e];
        __syncthreads();
        if (m == 0) {
            const V* krn = Kr + (size_t)half * KS;
#pragma unroll
            for (int e = 0; e < E; e++) {
                const int k = t + e * NT;
                V z = v[e], zc = cconj(sm[sg_pad((L - k) & (L - 1))]);
                V a = cscale(cadd(z, zc), (T)0.5);
                V d = csub(z, zc);
                V b = V{d.y * (T)0.5, -d.x * (T)0.5};
                y[e] = cadd(cmul(a, cconj(khat_r(kr, k, L, nu))), cmuli(cmul(b, cconj(khat_r(krn, k, L, nu)))));
            }
        } else {
#pragma unroll
            for (int e = 0; e < E; e++) y[e] = cmul(v[e], cconj(khat_r(kr, t + e * NT, L, nu)));
        }
    } else {
#pragma unroll
        for (int e = 0; e < E; e++) y[e] = cmul(v[e], cconj(khat_r(kr, t + e * NT, L, nu)));
    }
#pragma unroll
    for (int e = 0; e < E; e++) v[e] = (e < E / 2) ? C[(blk + t + e * NT) * cb + cm] : V{0, 0};
    sg_fft<E, -1>(v, sm, L, log2L, t, tw);
    if (m != 0) {
#pragma unroll
        for (int e = 0; e < E; e++) y[e] = cadd(y[e], cmul(v[e], cconj(khat_p(kp, t + e * NT, L, nu))));
    }
    sg_fft<E, +1>(y, sm, L, log2L, t, tw);
    if (live) {
#pragma unroll
        for (int e = 0; e < E / 2; e++) B[(size_t)(t + e * NT) * half + m] = y[e];
    }
}

// ===========================================================================
// Backward P3b: rows (i0, i1): Zhat = S_i0 + i S_i1 with S the Hermitian
// extension of each half spectrum; inverse FFT gives rows i0 (Re), i1 (Im).
// ===========================================================================
template <typename T, int E>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 256 : 512) k_bwd_rows_inv(const typename CX<T>::t* __restrict__ B,
                                                      const T* __restrict__ wpre, T* __restrict__ gs, int nu,
                                                      int nphi, int log2n, const typename CX<T>::t* __restrict__ tw)
{
    typedef typename CX<T>::t V;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* small = reinterpret_cast<V*>(smraw);
    const int N = nphi, NT = N / E, half = N / 2;
    const int slot = threadIdx.x / NT, t = threadIdx.x % NT;
    const int slots = blockDim.x / NT;
    V* sm = small + slot * sg_padded(N);
    const int pair = blockIdx.x * slots + slot;
    const bool live = pair < nu / 2;
    const int i0 = 2 * (live ? pair : 0), i1 = i0 + 1;
    const V* b0 = B + (size_t)i0 * half;
    const V* b1 = B + (size_t)i1 * half;
    V v[E];
#pragma unroll
    for (int e = 0; e < E; e++) {
        const int n = t + e * NT;
        V s0, s1;
        if (e < E / 2) {
            if (n == 0) {
                s0 = V{b0[0].x, 0};
                s1 = V{b1[0].x, 0};
            } else {
                s0 = b0[n];
                s1 = b1[n];
            }
        } else {
            if (n == half) {
                s0 = V{b0[0].y, 0};
                s1 = V{b1[0].y, 0};
            } else {
                s0 = cconj(b0[N - n]);
                s1 = cconj(b1[N - n]);
            }
        }
        v[e] = cadd(s0, cmuli(s1));
    }
    sg_fft<E, +1>(v, sm, N, log2n, t, tw);
    if (!live) return;
    const T w0 = wpre[i0], w1 = wpre[i1];
#pragma unroll
    for (int e = 0; e < E; e++) {
        const int n = t + e * NT;
        gs[(size_t)i0 * N + n] = v[e].x * w0;
        gs[(size_t)i1 * N + n] = v[e].y * w1;
    }
}

// ===========================================================================
// Spectra (FP64): rows kk of the cyclic weighted kernels, z = Kr + i Kphi,
// FFT along q; Re of the even part and Im of the odd part, transposed to
// W[m][kk] for m = 0..N_phi/2.
// ===========================================================================
template <int E>
__global__ void __launch_bounds__(512) k_spec_rows(const double* __restrict__ kr, const double* __restrict__ kp,
                                                   double2* __restrict__ W, int L, int nphi, int log2n,
                                                   const double2* __restrict__ tw)
{
    typedef double2 V;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* small = reinterpret_cast<V*>(smraw);
    const int N = nphi, NT = N / E;
    const int slot = threadIdx.x / NT, t = threadIdx.x % NT;
    const int slots = blockDim.x / NT;
    V* sm = small + slot * sg_padded(N);
    const int r0 = blockIdx.x * slots + slot;
    const bool live = r0 < L;
    const int kk = live ? r0 : 0;
    V v[E];
#pragma unroll
    for (int e = 0; e < E; e++) {
        const int q = t + e * NT;
        v[e] = V{kr[(size_t)kk * N + q], kp[(size_t)kk * N + q]};
    }
    sg_fft<E, -1>(v, sm, N, log2n, t, tw);
#pragma unroll
    for (int e = 0; e < E; e++) sm[sg_pad(t + e * NT)] = v[e];
    __syncthreads();
    if (!live) return;
#pragma unroll
    for (int e = 0; e <= E / 2; e++) {
        const int m = t + e * NT;
        if (m > N / 2) break;
        const V z = sm[sg_pad(m)], zc = sm[sg_pad((N - m) & (N - 1))];
        // even part (Kr): (z + conj zc)/2, real; odd part (Kphi): (z - conj zc)/(2i), imaginary
        W[(size_t)m * L + kk] = V{0.5 * (z.x + zc.x), -0.5 * (z.x - zc.x)};
    }
}

// Columns: per mode m, FFT along kk of W[m][.] = Ktilde_r + i Im Ktilde_phi;
// Khat_r = (Z + conj Zc)/2, Khat_phi = i (Z - conj Zc)/(2i) = (Z - conj Zc)/2,
// kappa = 0..N_u, rounded to the working dtype.
template <int E, typename VO>
__global__ void __launch_bounds__(512) k_spec_cols(const double2* __restrict__ W, VO* __restrict__ Kr,
                                                   VO* __restrict__ Kp, int nu, int nphi, int log2L,
                                                   const double2* __restrict__ tw)
{
    typedef double2 V;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* small = reinterpret_cast<V*>(smraw);
    const int L = 2 * nu, NT = L / E, KS = nu + 2;
    const int slot = threadIdx.x / NT, t = threadIdx.x % NT;
    const int slots = blockDim.x / NT;
    V* sm = small + slot * sg_padded(L);
    const int m0 = blockIdx.x * slots + slot;
    const bool live = m0 <= nphi / 2;
    const int m = live ? m0 : 0;
    V v[E];
#pragma unroll
    for (int e = 0; e < E; e++) v[e] = W[(size_t)m * L + t + e * NT];
    sg_fft<E, -1>(v, sm, L, log2L, t, tw);
#pragma unroll
    for (int e = 0; e < E; e++) sm[sg_pad(t + e * NT)] = v[e];
    __syncthreads();
    if (!live) return;
    typedef decltype(VO().x) TO;
#pragma unroll
    for (int e = 0; e <= E / 2; e++) {
        const int k = t + e * NT;
        if (k > nu) break;
        const V z = sm[sg_pad(k)], zc = sm[sg_pad((L - k) & (L - 1))];
        const V a = V{0.5 * (z.x + zc.x), 0.5 * (z.y - zc.y)};
        const V b = V{0.5 * (z.x - zc.x), 0.5 * (z.y + zc.y)};
        Kr[(size_t)m * KS + k] = VO{(TO)a.x, (TO)a.y};
        Kp[(size_t)m * KS + k] = VO{(TO)b.x, (TO)b.y};
    }
}

// ===========================================================================
// Host launchers
// ===========================================================================
struct Shape {
    int E, NT, slots, threads;
    size_t smem;
};

template <typename V>
static Shape shape_for(int n, int min_threads)
{
    Shape s;
    s.E = n >= 16 ? 16 : n;
    s.NT = n / s.E;
    s.slots = s.NT >= min_threads ? 1 : min_threads / s.NT;
    s.threads = s.NT * s.slots;
    s.smem = (size_t)s.slots * sg_padded(n) * sizeof(V);
    return s;
}

template <typename K>
static cudaError_t set_smem(K kernel, size_t smem)
{
    if (smem > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

#define SG_DISPATCH_E(E, ...)                   \
    do {                                        \
        if ((E) == 16) {                        \
            constexpr int EE = 16;              \
            __VA_ARGS__;                        \
        } else if ((E) == 8) {                  \
            constexpr int EE = 8;               \
            __VA_ARGS__;                        \
        } else {                                \
            constexpr int EE = 4;               \
            __VA_ARGS__;                        \
        }                                       \
    } while (0)

template <typename T>
cudaError_t launch_forward(const PlanView& p, const T* sigma, T* Fr, T* Fp, cudaStream_t st, cudaEvent_t* ev)
{
    typedef typename CX<T>::t V;
    const V* tw = (const V*)p.tw;
    V* A = (V*)p.wa;
    V* B = (V*)p.wb;
    V* C = (V*)p.wc;
    const int ln = sg_ilog2(p.nphi), lL = sg_ilog2(2 * p.nu);
    cudaError_t err;
    if (ev && (err = cudaEventRecord(ev[0], st)) != cudaSuccess) return err;
    {
        Shape s = shape_for<V>(p.nphi, 64);
        const int grid = (p.nu / 2 + s.slots - 1) / s.slots;
        SG_DISPATCH_E(s.E, {
            auto k = k_fwd_rows<T, EE>;
            if ((err = set_smem(k, s.smem)) != cudaSuccess) return err;
            k<<<grid, s.threads, s.smem, st>>>(sigma, (const T*)p.wpre, A, p.nu, p.nphi, ln, p.cb, tw);
        });
    }
    if (ev && (err = cudaEventRecord(ev[1], st)) != cudaSuccess) return err;
    {
        Shape s = shape_for<V>(2 * p.nu, 64);
        const int grid = (p.nphi / 2 + s.slots - 1) / s.slots;
        SG_DISPATCH_E(s.E, {
            auto k = k_fwd_cols<T, EE>;
            if ((err = set_smem(k, s.smem)) != cudaSuccess) return err;
            k<<<grid, s.threads, s.smem, st>>>(A, (const V*)p.kr, (const V*)p.kp, B, C, p.nu, p.nphi, lL, p.cb, tw);
        });
    }
    if (ev && (err = cudaEventRecord(ev[2], st)) != cudaSuccess) return err;
    {
        Shape s = shape_for<V>(p.nphi, 64);
        const int grid = (p.nu + s.slots - 1) / s.slots;
        SG_DISPATCH_E(s.E, {
            auto k = k_fwd_rows_inv<T, EE>;
            if ((err = set_smem(k, s.smem)) != cudaSuccess) return err;
            k<<<grid, s.threads, s.smem, st>>>(B, C, (const T*)p.wpost, Fr, Fp, p.nu, p.nphi, ln, tw);
        });
    }
    if (ev && (err = cudaEventRecord(ev[3], st)) != cudaSuccess) return err;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_backward(const PlanView& p, const T* gr, const T* gp, T* gs, cudaStream_t st)
{
    typedef typename CX<T>::t V;
    const V* tw = (const V*)p.tw;
    V* A = (V*)p.wa;
    V* B = (V*)p.wb;
    V* C = (V*)p.wc;
    const int ln = sg_ilog2(p.nphi), lL = sg_ilog2(2 * p.nu);
    cudaError_t err;
    {
        Shape s = shape_for<V>(p.nphi, 64);
        const int grid = (p.nu + s.slots - 1) / s.slots;
        SG_DISPATCH_E(s.E, {
            auto k = k_bwd_rows<T, EE>;
            if ((err = set_smem(k, s.smem)) != cudaSuccess) return err;
            k<<<grid, s.threads, s.smem, st>>>(gr, gp, (const T*)p.wpost, A, C, p.nu, p.nphi, ln, p.cb, tw);
        });
    }
    {
        Shape s = shape_for<V>(2 * p.nu, 64);
        const int grid = (p.nphi / 2 + s.slots - 1) / s.slots;
        SG_DISPATCH_E(s.E, {
            auto k = k_bwd_cols<T, EE>;
            if ((err = set_smem(k, s.smem)) != cudaSuccess) return err;
            k<<<grid, s.threads, s.smem, st>>>(A, C, (const V*)p.kr, (const V*)p.kp, B, p.nu, p.nphi, lL, p.cb, tw);
        });
    }
    {
        Shape s = shape_for<V>(p.nphi, 64);
        const int grid = (p.nu / 2 + s.slots - 1) / s.slots;
        SG_DISPATCH_E(s.E, {
            auto k = k_bwd_rows_inv<T, EE>;
            if ((err = set_smem(k, s.smem)) != cudaSuccess) return err;
            k<<<grid, s.threads, s.smem, st>>>(B, (const T*)p.wpre, gs, p.nu, p.nphi, ln, tw);
        });
    }
    return cudaGetLastError();
}

template <typename VO>
cudaError_t launch_spectra(const PlanView& p, const double* nsr, const double* nsp, double2* W, VO* Kr, VO* Kp,
                           cudaStream_t st)
{
    const double2* tw = (const double2*)p.tw64;
    const int L = 2 * p.nu;
    const int ln = sg_ilog2(p.nphi), lL = sg_ilog2(L);
    cudaError_t err;
    {
        Shape s = shape_for<double2>(p.nphi, 64);
        const int grid = (L + s.slots - 1) / s.slots;
        SG_DISPATCH_E(s.E, {
            auto k = k_spec_rows<EE>;
            if ((err = set_smem(k, s.smem)) != cudaSuccess) return err;
            k<<<grid, s.threads, s.smem, st>>>(nsr, nsp, W, L, p.nphi, ln, tw);
        });
    }
    {
        Shape s = shape_for<double2>(L, 64);
        const int grid = (p.nphi / 2 + 1 + s.slots - 1) / s.slots;
        SG_DISPATCH_E(s.E, {
            auto k = k_spec_cols<EE, VO>;
            if ((err = set_smem(k, s.smem)) != cudaSuccess) return err;
            k<<<grid, s.threads, s.smem, st>>>(W, Kr, Kp, p.nu, p.nphi, lL, tw);
        });
    }
    return cudaGetLastError();
}

template cudaError_t launch_forward<float>(const PlanView&, const float*, float*, float*, cudaStream_t, cudaEvent_t*);
template cudaError_t launch_forward<double>(const PlanView&, const double*, double*, double*, cudaStream_t,
                                              cudaEvent_t*);
template cudaError_t launch_backward<float>(const PlanView&, const float*, const float*, float*, cudaStream_t);
template cudaError_t launch_backward<double>(const PlanView&, const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_spectra<float2>(const PlanView&, const double*, const double*, double2*, float2*,
                                            float2*, cudaStream_t);
template cudaError_t launch_spectra<double2>(const PlanView&, const double*, const double*, double2*, double2*,
                                             double2*, cudaStream_t);

}  // namespace sg
