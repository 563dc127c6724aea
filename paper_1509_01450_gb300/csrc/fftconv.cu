// fftconv.cu -- FFT convolution passes of the thin-disk force (sm_103a).
//
// The forces are the convolution (zero-padded to L = 2 N_u rows in u,
// periodic in phi) of the weighted density w = sigma beta^{p i} with the
// weighted kernel spectra Khat (built once, kbuild.cu), evaluated in three
// passes per direction:
//
//  forward  P1 rows   : R2C along phi of w (two rows per complex FFT),
//                       half spectra to A
//  forward  P2 columns: one phi-mode column per block: the column and both
//                       kernel spectra arrive by bulk asynchronous copy
//                       (TMA) into shared memory; zero-padded FFT of length
//                       L, times Khat_r and Khat_phi, two inverse FFTs, crop
//                       to N_u rows, to B (r) and C (phi)
//  forward  P3 rows   : one inverse FFT of Z = F_r + i F_phi per row,
//                       scaled by beta^{-p i}
//  backward P1b rows  : FFT of (gF_r + i gF_phi) beta^{-p i}, split into the
//                       two half spectra (A and C)
//  backward P2b cols  : FFT of both columns, times conj(Khat), summed, one
//                       inverse FFT, crop, to B
//  backward P3b rows  : inverse real FFT of two rows at once, times beta^{p i}
//
// Half spectra along phi keep modes 0..N_phi/2-1, with the real DC and
// Nyquist values packed into mode 0 as (DC, Nyquist).  A, B and C are all
// mode-major, X[m N_u + i]: a column pass reads and writes whole contiguous
// columns, and the row passes move them through shared memory in 16-byte
// units (stage_load / stage_store).
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
// the same from a copy in shared memory
template <typename V>
__device__ __forceinline__ V khat_r_s(const V* K, int kappa, int L, int nu)
{
    return kappa <= nu ? K[kappa] : cconj(K[L - kappa]);
}
template <typename V>
__device__ __forceinline__ V khat_p_s(const V* K, int kappa, int L, int nu)
{
    if (kappa <= nu) return K[kappa];
    const V a = K[L - kappa];
    return V{-a.x, a.y};
}

// shared-memory carve-up of the column kernels (16-byte aligned regions)
__host__ __device__ __forceinline__ size_t sg_align16(size_t b) { return (b + 15) & ~(size_t)15; }

// Twiddle source of one thread's transforms: FP32 transforms with 16
// elements per thread keep their pass twiddles in registers (loaded once per
// kernel); the others read the table in every pass.
template <int E, typename V>
struct Twd {
    const V* tab;
    SgTwid<V> h;
};
template <int E, typename V>
__device__ __forceinline__ Twd<E, V> make_twd(int log2N, int t, const V* __restrict__ tab)
{
    Twd<E, V> w;
    w.tab = tab;
    if constexpr (E == 16 && sizeof(V) == 8) w.h = sg_fft_twiddles(log2N, t, tab);
    return w;
}
template <int E, int DIR, typename V>
__device__ __forceinline__ void fft(V (&v)[E], V* sm, int N, int log2N, int t, const Twd<E, V>& w)
{
    if constexpr (E == 16 && sizeof(V) == 8)
        sg_fft<E, DIR>(v, sm, N, log2N, t, w.h);
    else
        sg_fft<E, DIR>(v, sm, N, log2N, t, w.tab);
}

// ===========================================================================
// Mode-major half spectra X[m N_u + i] and the row passes.  A block of R
// consecutive rows (R a power of two) moves its part of X through shared
// memory staged as S[m R + r], so that every global access is a 16-byte unit
// (two FP32 complex values or one FP64) and a block's units of one mode are
// adjacent (R = 4 FP32 rows fill a 32-byte sector).
// ===========================================================================
template <typename V>
__device__ __forceinline__ void stage_store(V* __restrict__ X, const V* S, int nu, int half, int ib, int R)
{
    const uint64_t keep = sg_policy_evict_last();  // the next pass reads X from L2
    if (R * (int)sizeof(V) >= 16) {
        constexpr int VPU = 16 / sizeof(V);
        const int U = R / VPU, lgU = __ffs(U) - 1;
        for (int u = threadIdx.x; u < half * U; u += blockDim.x) {
            const int m = u >> lgU, r = (u & (U - 1)) * VPU;
            if (ib + r < nu)
                sg_st_hint(reinterpret_cast<float4*>(X + (size_t)m * nu + ib + r),
                           *reinterpret_cast<const float4*>(S + m * R + r), keep);
        }
    } else if (ib < nu) {  // R = 1, FP32
        for (int m = threadIdx.x; m < half; m += blockDim.x) sg_st_hint(X + (size_t)m * nu + ib, S[m], keep);
    }
}

// stage_load only issues asynchronous copies: complete them with
// sg_cp_async_wait_all() and __syncthreads() before reading S.
template <typename V>
__device__ __forceinline__ void stage_load(V* S, const V* __restrict__ X, int nu, int half, int ib, int R)
{
    const uint64_t drop = sg_policy_evict_first();  // X is consumed here
    if (R * (int)sizeof(V) >= 16) {
        constexpr int VPU = 16 / sizeof(V);
        const int U = R / VPU, lgU = __ffs(U) - 1;
        for (int u = threadIdx.x; u < half * U; u += blockDim.x) {
            const int m = u >> lgU, r = (u & (U - 1)) * VPU;
            if (ib + r < nu) sg_cp_async16(S + m * R + r, X + (size_t)m * nu + ib + r, drop);
        }
    } else if (ib < nu) {
        for (int m = threadIdx.x; m < half; m += blockDim.x) sg_cp_async8(S + m, X + (size_t)m * nu + ib, drop);
    }
}

// ===========================================================================
// Forward P1: rows (i0, i1) packed as z = w_i0 + i w_i1, FFT along phi,
// split X_i0[m] = (Z[m] + conj Z[N-m]) / 2, X_i1[m] = (Z[m] - conj Z[N-m]) / 2i,
// staged and stored mode-major (R = 2 slots rows per block).
// ===========================================================================
template <typename T, int E>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 256 : 512) k_fwd_rows(const T* __restrict__ sigma, const T* __restrict__ wpre,
                                                  typename CX<T>::t* __restrict__ A, int nu, int nphi, int log2n,
                                                  const typename CX<T>::t* __restrict__ tw)
{
    typedef typename CX<T>::t V;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* small = reinterpret_cast<V*>(smraw);
    const int N = nphi, NT = N / E, half = N / 2;
    const int slot = threadIdx.x / NT, t = threadIdx.x % NT;
    const Twd<E, V> twd = make_twd<E>(log2n, t, tw);
    const int slots = blockDim.x / NT;
    V* sm = small + slot * sg_padded(N);
    const int pair = blockIdx.x * slots + slot;
    const bool live = pair < nu / 2;
    const int i0 = 2 * (live ? pair : 0), i1 = i0 + 1;
    const T w0 = wpre[i0], w1 = wpre[i1];
    const uint64_t stream = sg_policy_evict_first();
    V v[E];
#pragma unroll
    for (int e = 0; e < E; e++) {
        const int n = t + e * NT;
        v[e] = V{sg_ld_hint(sigma + (size_t)i0 * N + n, stream) * w0, sg_ld_hint(sigma + (size_t)i1 * N + n, stream) * w1};
    }
    fft<E, -1>(v, sm, N, log2n, t, twd);
#pragma unroll
    for (int e = 0; e < E; e++) sm[sg_pad(t + e * NT)] = v[e];
    __syncthreads();
    const T h = (T)0.5;
    V x0[E / 2], x1[E / 2];
#pragma unroll
    for (int e = 0; e < E / 2; e++) {
        const int m = t + e * NT;
        const V z = v[e], zc = cconj(sm[sg_pad((N - m) & (N - 1))]);
        if (m == 0) {
            const V zn = sm[sg_pad(N / 2)];
            x0[e] = V{z.x, zn.x};
            x1[e] = V{z.y, zn.y};
        } else {
            x0[e] = cscale(cadd(z, zc), h);
            const V d = csub(z, zc);
            x1[e] = V{d.y * h, -d.x * h};  // d / 2i
        }
    }
    __syncthreads();  // every mirror read is done: the buffers become the stage
    const int R = 2 * slots;
    if (live) {
#pragma unroll
        for (int e = 0; e < E / 2; e++) {
            V* d = small + (t + e * NT) * R + 2 * slot;
            d[0] = x0[e];
            d[1] = x1[e];
        }
    }
    __syncthreads();
    stage_store(A, small, nu, half, blockIdx.x * R, R);
}

// ===========================================================================
// Forward P2: one phi-mode column m per block.  Shared memory: the FFT
// exchange buffer (its first N_u entries double as the landing area of the
// column), then Khat_r[m] and Khat_phi[m] (for m = 0: Khat_r of modes 0 and
// N_phi/2), which are later reused to park the phi product.
// ===========================================================================
template <typename T>
__host__ __device__ __forceinline__ size_t cols_smem_bytes(int nu)
{
    typedef typename CX<T>::t V;
    const int L = 2 * nu, KS = nu + 2;
    return sg_align16(sg_padded(L) * sizeof(V)) + 2 * (size_t)KS * sizeof(V);
}

// NTB: the block size the kernel is compiled for (L / E threads); FP32
// blocks of 256 threads are held to SG_COLS_MINB per SM (3: registers <= 80,
// which the shared memory of N_u = 2048 also allows)
#ifndef SG_COLS_MINB
#define SG_COLS_MINB 3
#endif
#define SG_COLS_BOUNDS(T, NTB) __launch_bounds__(NTB, (sizeof(T) == 4 && NTB == 256) ? SG_COLS_MINB : 1)

template <typename T, int E, int NTB>
__global__ void SG_COLS_BOUNDS(T, NTB) k_fwd_cols(const typename CX<T>::t* __restrict__ A,
                                                  const typename CX<T>::t* __restrict__ Kr,
                                                  const typename CX<T>::t* __restrict__ Kp,
                                                  typename CX<T>::t* __restrict__ Br,
                                                  typename CX<T>::t* __restrict__ Cp, int nu, int nphi, int log2L,
                                                  const typename CX<T>::t* __restrict__ tw, int* err)
{
    typedef typename CX<T>::t V;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ __align__(8) uint64_t bar[2];  // [0]: the column, [1]: the spectra
    const int L = 2 * nu, NT = L / E, half = nphi / 2, KS = nu + 2;
    const int t = threadIdx.x;
    const int m = blockIdx.x;
    V* sm = reinterpret_cast<V*>(smraw);
    V* ks = reinterpret_cast<V*>(smraw + sg_align16(sg_padded(L) * sizeof(V)));  // 2 KS entries
    V* kr_s = ks;
    V* kp_s = ks + KS;
    if (t == 0) {
        sg_mbar_init(&bar[0], 1);
        sg_mbar_init(&bar[1], 1);
    }
    __syncthreads();
    if (t == 0) {
        const uint32_t ab = (uint32_t)(nu * sizeof(V)), kb = (uint32_t)(KS * sizeof(V));
        const uint64_t drop = sg_policy_evict_first();
        sg_mbar_expect_tx(&bar[0], ab);
        sg_bulk_g2s_hint(sm, A + (size_t)m * nu, ab, &bar[0], drop);
        sg_mbar_expect_tx(&bar[1], 2 * kb);
        sg_bulk_g2s_hint(kr_s, Kr + (size_t)m * KS, kb, &bar[1], drop);
        // mode 0 holds (DC, Nyquist): bring the Nyquist mode's Khat_r instead
        // of Khat_phi, which vanishes at both
        sg_bulk_g2s_hint(kp_s, (m == 0 ? Kr + (size_t)half * KS : Kp + (size_t)m * KS), kb, &bar[1], drop);
    }
    const Twd<E, V> twd = make_twd<E>(log2L, t, tw);
    const uint64_t keep = sg_policy_evict_last();  // the row pass reads B and C from L2
    // inputs that never arrive: leave (all threads together) after a last wait for the spectra
    if (__syncthreads_or(!sg_mbar_wait_bounded(&bar[0], 0, err, 1))) {
        sg_mbar_wait_bounded(&bar[1], 0, err, 1);
        return;
    }
    V v[E];
#pragma unroll
    for (int e = 0; e < E; e++) v[e] = (e < E / 2) ? sm[t + e * NT] : V{0, 0};  // rows >= nu: zero pad
    fft<E, -1>(v, sm, L, log2L, t, twd);  // the spectra land meanwhile
    if (__syncthreads_or(!sg_mbar_wait_bounded(&bar[1], 0, err, 1))) return;
    if (m == 0) {
        // v holds the FFT of (DC + i Nyquist): separate the two real
        // sequences and apply the kernels of modes 0 and N_phi/2
#pragma unroll
        for (int e = 0; e < E; e++) sm[sg_pad(t + e * NT)] = v[e];
        __syncthreads();
        V y[E];
#pragma unroll
        for (int e = 0; e < E; e++) {
            const int k = t + e * NT;
            const V z = v[e], zc = cconj(sm[sg_pad((L - k) & (L - 1))]);
            const V a = cscale(cadd(z, zc), (T)0.5);
            const V d = csub(z, zc);
            const V b = V{d.y * (T)0.5, -d.x * (T)0.5};
            y[e] = cadd(cmul(a, khat_r_s(kr_s, k, L, nu)), cmuli(cmul(b, khat_r_s(kp_s, k, L, nu))));
        }
        fft<E, +1>(y, sm, L, log2L, t, twd);
#pragma unroll
        for (int e = 0; e < E / 2; e++) {
            sg_st_hint(Br + t + e * NT, y[e], keep);
            sg_st_hint(Cp + t + e * NT, V{0, 0}, keep);
        }
        return;
    }
    // phi product into the (now free) exchange buffer, r product in place
#pragma unroll
    for (int e = 0; e < E; e++) {
        const int k = t + e * NT;
        sm[sg_pad(k)] = cmul(v[e], khat_p_s(kp_s, k, L, nu));
        v[e] = cmul(v[e], khat_r_s(kr_s, k, L, nu));
    }
    __syncthreads();  // every read of the spectra is done
#pragma unroll
    for (int e = 0; e < E; e++) ks[t + e * NT] = sm[sg_pad(t + e * NT)];  // park the phi product
    fft<E, +1>(v, sm, L, log2L, t, twd);
#pragma unroll
    for (int e = 0; e < E / 2; e++) sg_st_hint(Br + (size_t)m * nu + t + e * NT, v[e], keep);
#pragma unroll
    for (int e = 0; e < E; e++) v[e] = ks[t + e * NT];
    fft<E, +1>(v, sm, L, log2L, t, twd);
#pragma unroll
    for (int e = 0; e < E / 2; e++) sg_st_hint(Cp + (size_t)m * nu + t + e * NT, v[e], keep);
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
    const Twd<E, V> twd = make_twd<E>(log2n, t, tw);
    const int slots = blockDim.x / NT;
    V* sm = small + slot * sg_padded(N);
    const int i0 = blockIdx.x * slots + slot;
    const bool live = i0 < nu;
    const int i = live ? i0 : 0;
    // stage rows [ib, ib + R) of both half spectra: Sb[m R + r], Sc[m R + r]
    const int R = slots, ib = blockIdx.x * slots;
    V* Sb = small;
    V* Sc = small + (size_t)R * half;
    stage_load(Sb, Br, nu, half, ib, R);
    stage_load(Sc, Cp, nu, half, ib, R);
    sg_cp_async_wait_all();
    __syncthreads();
    V v[E];
#pragma unroll
    for (int e = 0; e < E; e++) {
        const int n = t + e * NT;
        V z;
        if (e < E / 2) {
            if (n == 0) {
                z = V{Sb[slot].x, 0};
            } else {
                const V a = Sb[n * R + slot], b = Sc[n * R + slot];
                z = V{a.x - b.y, a.y + b.x};  // a + i b
            }
        } else {
            if (n == half) {
                z = V{Sb[slot].y, 0};
            } else {
                const V a = Sb[(N - n) * R + slot], b = Sc[(N - n) * R + slot];
                z = V{a.x + b.y, -a.y + b.x};  // conj a + i conj b
            }
        }
        v[e] = z;
    }
    fft<E, +1>(v, sm, N, log2n, t, twd);  // its first exchange waits for every thread's stage reads
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
// the half spectra of gF_r (-> A) and gF_phi (-> C), mode-major.
// ===========================================================================
template <typename T, int E>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 256 : 512) k_bwd_rows(const T* __restrict__ gr, const T* __restrict__ gp,
                                                  const T* __restrict__ wpost, typename CX<T>::t* __restrict__ A,
                                                  typename CX<T>::t* __restrict__ C, int nu, int nphi, int log2n,
                                                  const typename CX<T>::t* __restrict__ tw)
{
    typedef typename CX<T>::t V;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* small = reinterpret_cast<V*>(smraw);
    const int N = nphi, NT = N / E;
    const int slot = threadIdx.x / NT, t = threadIdx.x % NT;
    const Twd<E, V> twd = make_twd<E>(log2n, t, tw);
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
    fft<E, -1>(v, sm, N, log2n, t, twd);
#pragma unroll
    for (int e = 0; e < E; e++) sm[sg_pad(t + e * NT)] = v[e];
    __syncthreads();
    const T h = (T)0.5;
    V x0[E / 2], x1[E / 2];
#pragma unroll
    for (int e = 0; e < E / 2; e++) {
        const int m = t + e * NT;
        const V z = v[e], zc = cconj(sm[sg_pad((N - m) & (N - 1))]);
        if (m == 0) {
            const V zn = sm[sg_pad(N / 2)];
            x0[e] = V{z.x, zn.x};
            x1[e] = V{z.y, zn.y};
        } else {
            x0[e] = cscale(cadd(z, zc), h);
            const V d = csub(z, zc);
            x1[e] = V{d.y * h, -d.x * h};
        }
    }
    __syncthreads();  // mirror reads done: the buffers become the stages of A and C
    const int R = slots, half = N / 2;
    V* Sa = small;
    V* Sc = small + (size_t)R * half;
    if (live) {
#pragma unroll
        for (int e = 0; e < E / 2; e++) {
            Sa[(t + e * NT) * R + slot] = x0[e];
            Sc[(t + e * NT) * R + slot] = x1[e];
        }
    }
    __syncthreads();
    stage_store(A, Sa, nu, half, blockIdx.x * R, R);
    stage_store(C, Sc, nu, half, blockIdx.x * R, R);
}

// ===========================================================================
// Backward P2b: column m: FFT of both zero-padded columns, times conj(Khat),
// summed, inverse FFT, crop, to B.  Shared memory: exchange
// buffer (first N_u entries: landing area of the A column), the C column,
// Khat_r[m] and Khat_phi[m] (m = 0: Khat_r of modes 0 and N_phi/2).
// ===========================================================================
template <typename T>
__host__ __device__ __forceinline__ size_t bcols_smem_bytes(int nu)
{
    typedef typename CX<T>::t V;
    const int L = 2 * nu, KS = nu + 2;
    return sg_align16(sg_padded(L) * sizeof(V)) + (size_t)nu * sizeof(V) + 2 * (size_t)KS * sizeof(V);
}

template <typename T, int E, int NTB>
__global__ void SG_COLS_BOUNDS(T, NTB) k_bwd_cols(const typename CX<T>::t* __restrict__ A,
                                                  const typename CX<T>::t* __restrict__ C,
                                                  const typename CX<T>::t* __restrict__ Kr,
                                                  const typename CX<T>::t* __restrict__ Kp,
                                                  typename CX<T>::t* __restrict__ B, int nu, int nphi, int log2L,
                                                  const typename CX<T>::t* __restrict__ tw, int* err)
{
    typedef typename CX<T>::t V;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ __align__(8) uint64_t bar[2];  // [0]: the A column, [1]: the C column and the spectra
    const int L = 2 * nu, NT = L / E, half = nphi / 2, KS = nu + 2;
    const int t = threadIdx.x;
    const int m = blockIdx.x;
    V* sm = reinterpret_cast<V*>(smraw);
    V* cs = reinterpret_cast<V*>(smraw + sg_align16(sg_padded(L) * sizeof(V)));  // nu entries
    V* kr_s = cs + nu;
    V* kp_s = kr_s + KS;
    if (t == 0) {
        sg_mbar_init(&bar[0], 1);
        sg_mbar_init(&bar[1], 1);
    }
    __syncthreads();
    if (t == 0) {
        const uint32_t ab = (uint32_t)(nu * sizeof(V)), kb = (uint32_t)(KS * sizeof(V));
        const uint64_t drop = sg_policy_evict_first();
        sg_mbar_expect_tx(&bar[0], ab);
        sg_bulk_g2s_hint(sm, A + (size_t)m * nu, ab, &bar[0], drop);
        sg_mbar_expect_tx(&bar[1], ab + 2 * kb);
        sg_bulk_g2s_hint(cs, C + (size_t)m * nu, ab, &bar[1], drop);
        sg_bulk_g2s_hint(kr_s, Kr + (size_t)m * KS, kb, &bar[1], drop);
        sg_bulk_g2s_hint(kp_s, (m == 0 ? Kr + (size_t)half * KS : Kp + (size_t)m * KS), kb, &bar[1], drop);
    }
    const Twd<E, V> twd = make_twd<E>(log2L, t, tw);
    const uint64_t keep = sg_policy_evict_last();
    if (__syncthreads_or(!sg_mbar_wait_bounded(&bar[0], 0, err, 1))) {
        sg_mbar_wait_bounded(&bar[1], 0, err, 1);
        return;
    }
    V v[E], y[E];
#pragma unroll
    for (int e = 0; e < E; e++) v[e] = (e < E / 2) ? sm[t + e * NT] : V{0, 0};
    fft<E, -1>(v, sm, L, log2L, t, twd);
    if (__syncthreads_or(!sg_mbar_wait_bounded(&bar[1], 0, err, 1))) return;
    if (m == 0) {
#pragma unroll
        for (int e = 0; e < E; e++) sm[sg_pad(t + e * NT)] = v[e];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; e++) {
            const int k = t + e * NT;
            const V z = v[e], zc = cconj(sm[sg_pad((L - k) & (L - 1))]);
            const V a = cscale(cadd(z, zc), (T)0.5);
            const V d = csub(z, zc);
            const V b = V{d.y * (T)0.5, -d.x * (T)0.5};
            y[e] = cadd(cmul(a, cconj(khat_r_s(kr_s, k, L, nu))), cmuli(cmul(b, cconj(khat_r_s(kp_s, k, L, nu)))));
        }
    } else {
#pragma unroll
        for (int e = 0; e < E; e++) y[e] = cmul(v[e], cconj(khat_r_s(kr_s, t + e * NT, L, nu)));
#pragma unroll
        for (int e = 0; e < E; e++) v[e] = (e < E / 2) ? cs[t + e * NT] : V{0, 0};
        fft<E, -1>(v, sm, L, log2L, t, twd);
#pragma unroll
        for (int e = 0; e < E; e++) y[e] = cadd(y[e], cmul(v[e], cconj(khat_p_s(kp_s, t + e * NT, L, nu))));
    }
    fft<E, +1>(y, sm, L, log2L, t, twd);
#pragma unroll
    for (int e = 0; e < E / 2; e++) sg_st_hint(B + (size_t)m * nu + t + e * NT, y[e], keep);
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
    const Twd<E, V> twd = make_twd<E>(log2n, t, tw);
    const int slots = blockDim.x / NT;
    V* sm = small + slot * sg_padded(N);
    const int pair = blockIdx.x * slots + slot;
    const bool live = pair < nu / 2;
    const int i0 = 2 * (live ? pair : 0), i1 = i0 + 1;
    // stage rows [ib, ib + R) of B as Sb[m R + r]; this pair is r = 2 slot, 2 slot + 1
    const int R = 2 * slots, ib = blockIdx.x * R;
    V* Sb = small;
    stage_load(Sb, B, nu, half, ib, R);
    sg_cp_async_wait_all();
    __syncthreads();
    const V* b0 = Sb + 2 * slot;
    const V* b1 = b0 + 1;
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
                s0 = b0[n * R];
                s1 = b1[n * R];
            }
        } else {
            if (n == half) {
                s0 = V{b0[0].y, 0};
                s1 = V{b1[0].y, 0};
            } else {
                s0 = cconj(b0[(N - n) * R]);
                s1 = cconj(b1[(N - n) * R]);
            }
        }
        v[e] = cadd(s0, cmuli(s1));
    }
    fft<E, +1>(v, sm, N, log2n, t, twd);
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

// Dynamic shared memory above the 48 KB default needs an opt-in; carveout
// asks for the largest shared-memory split of L1 (several blocks of a
// shared-memory-heavy kernel per SM).
template <typename K>
static cudaError_t set_smem(K kernel, size_t smem, bool carveout = false)
{
    cudaError_t e = cudaSuccess;
    if (smem > 48 * 1024) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && carveout)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
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
        Shape s = shape_for<V>(p.nphi, sizeof(T) == 8 ? 64 : 512);
        const int grid = (p.nu / 2 + s.slots - 1) / s.slots;
        SG_DISPATCH_E(s.E, {
            auto k = k_fwd_rows<T, EE>;
            if ((err = set_smem(k, s.smem)) != cudaSuccess) return err;
            k<<<grid, s.threads, s.smem, st>>>(sigma, (const T*)p.wpre, A, p.nu, p.nphi, ln, tw);
        });
    }
    if (ev && (err = cudaEventRecord(ev[1], st)) != cudaSuccess) return err;
    {
        const int L = 2 * p.nu, E = L >= 16 ? 16 : L;
        const size_t smem = cols_smem_bytes<T>(p.nu);
        SG_DISPATCH_E(E, {
            auto k = k_fwd_cols<T, EE, 256>;
            if constexpr (sizeof(T) == 4)  // FP64 columns are at most 256 threads
                if (L / EE > 256) k = k_fwd_cols<T, EE, 512>;
            if ((err = set_smem(k, smem, true)) != cudaSuccess) return err;
            k<<<p.nphi / 2, L / EE, smem, st>>>(A, (const V*)p.kr, (const V*)p.kp, B, C, p.nu, p.nphi, lL, tw, p.err);
        });
    }
    if (ev && (err = cudaEventRecord(ev[2], st)) != cudaSuccess) return err;
    {
        Shape s = shape_for<V>(p.nphi, sizeof(T) == 8 ? 64 : 512);
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
        Shape s = shape_for<V>(p.nphi, sizeof(T) == 8 ? 64 : 512);
        const int grid = (p.nu + s.slots - 1) / s.slots;
        SG_DISPATCH_E(s.E, {
            auto k = k_bwd_rows<T, EE>;
            if ((err = set_smem(k, s.smem)) != cudaSuccess) return err;
            k<<<grid, s.threads, s.smem, st>>>(gr, gp, (const T*)p.wpost, A, C, p.nu, p.nphi, ln, tw);
        });
    }
    {
        const int L = 2 * p.nu, E = L >= 16 ? 16 : L;
        const size_t smem = bcols_smem_bytes<T>(p.nu);
        SG_DISPATCH_E(E, {
            auto k = k_bwd_cols<T, EE, 256>;
            if constexpr (sizeof(T) == 4)  // FP64 columns are at most 256 threads
                if (L / EE > 256) k = k_bwd_cols<T, EE, 512>;
            if ((err = set_smem(k, smem, true)) != cudaSuccess) return err;
            k<<<p.nphi / 2, L / EE, smem, st>>>(A, C, (const V*)p.kr, (const V*)p.kp, B, p.nu, p.nphi, lL, tw, p.err);
        });
    }
    {
        Shape s = shape_for<V>(p.nphi, sizeof(T) == 8 ? 64 : 512);
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
