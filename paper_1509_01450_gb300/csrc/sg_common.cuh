// sg_common.cuh -- shared device helpers of the GB300 thin-disk force library:
// complex arithmetic on float2/double2 and a register-resident Stockham FFT.
//
// FFT engine.  A transform of length N = 2^m is held by NT = N / E threads,
// E = min(16, N) elements each: thread t owns x[t + e NT], e = 0..E-1, on
// entry and X[t + e NT] on exit (natural order, strided).  The passes are
// Stockham autosort passes (Cooley-Tukey decimation in time with the
// reordering folded into the exchange): one optional radix-2/4/8 pass first,
// then radix-16 passes, all butterflies in registers, exchanges through a
// padded shared-memory buffer of N + N/16 elements.  Twiddles come from a
// table tw[j] = exp(-2 pi i j / SG_NMAX) in global memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define SG_NMAX 16384  // longest transform length; twiddle table length

template <typename T>
struct CX;
template <>
struct CX<float> {
    typedef float2 t;
};
template <>
struct CX<double> {
    typedef double2 t;
};

template <typename V>
__device__ __forceinline__ V cadd(V a, V b) { return V{a.x + b.x, a.y + b.y}; }
template <typename V>
__device__ __forceinline__ V csub(V a, V b) { return V{a.x - b.x, a.y - b.y}; }
template <typename V>
__device__ __forceinline__ V cmul(V a, V b) { return V{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
template <typename V>
__device__ __forceinline__ V cconj(V a) { return V{a.x, -a.y}; }
template <typename V, typename T>
__device__ __forceinline__ V cscale(V a, T s) { return V{a.x * s, a.y * s}; }
// multiply by i: (x + iy) i = -y + ix
template <typename V>
__device__ __forceinline__ V cmuli(V a) { return V{-a.y, a.x}; }

__host__ __device__ __forceinline__ int sg_pad(int i) { return i + (i >> 4); }
__host__ __device__ __forceinline__ int sg_padded(int n) { return n + (n >> 4) + 1; }

// e^{DIR 2 pi i j / M} from the table (stride NMAX / M folded into idx)
template <int DIR, typename V>
__device__ __forceinline__ V sg_tw(const V* __restrict__ tw, int idx)
{
    V w = __ldg(&tw[idx]);
    if (DIR > 0) w.y = -w.y;
    return w;
}

// ---------------------------------------------------------------------------
// Butterflies in registers: natural-order DFT of R points, sign DIR.
// ---------------------------------------------------------------------------
template <int DIR, typename V>
__device__ __forceinline__ V sg_mulw4(V a)  // a * e^{DIR i pi / 2} = a * (DIR i)
{
    return DIR > 0 ? V{-a.y, a.x} : V{a.y, -a.x};
}

template <int DIR, typename V>
__device__ __forceinline__ void sg_dft2(V* a)
{
    V t = a[0];
    a[0] = cadd(t, a[1]);
    a[1] = csub(t, a[1]);
}

template <int DIR, typename V>
__device__ __forceinline__ void sg_dft4v(V& a0, V& a1, V& a2, V& a3)
{
    V t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3);
    V t3 = sg_mulw4<DIR>(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

template <int DIR, typename V>
__device__ __forceinline__ void sg_dft4(V* a) { sg_dft4v<DIR>(a[0], a[1], a[2], a[3]); }

// multiply by e^{DIR i pi k / 4}, k = 1, 3  (r = sqrt(2)/2)
template <int DIR, int K, typename V>
__device__ __forceinline__ V sg_mulw8(V a)
{
    typedef decltype(a.x) T;
    const T r = (T)0.70710678118654752440084436210484904;
    if (K == 1) return V{r * (a.x - DIR * a.y), r * (a.y + DIR * a.x)};
    return V{r * (-a.x - DIR * a.y), r * (-a.y + DIR * a.x)};  // K == 3
}

template <int DIR, typename V>
__device__ __forceinline__ void sg_dft8(V* a)
{
    // even / odd halves, then combine with w8^k
    sg_dft4v<DIR>(a[0], a[2], a[4], a[6]);
    sg_dft4v<DIR>(a[1], a[3], a[5], a[7]);
    V o1 = sg_mulw8<DIR, 1>(a[3]);
    V o2 = sg_mulw4<DIR>(a[5]);
    V o3 = sg_mulw8<DIR, 3>(a[7]);
    V e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6], o0 = a[1];
    a[0] = cadd(e0, o0);
    a[4] = csub(e0, o0);
    a[1] = cadd(e1, o1);
    a[5] = csub(e1, o1);
    a[2] = cadd(e2, o2);
    a[6] = csub(e2, o2);
    a[3] = cadd(e3, o3);
    a[7] = csub(e3, o3);
}

// e^{DIR 2 pi i j / 16}, j = 0..9, as compile-time constants
template <int DIR, int J, typename V>
__device__ __forceinline__ V sg_mulw16(V a)
{
    typedef decltype(a.x) T;
    // cos and sin of 2 pi j / 16
    const T C1 = (T)0.92387953251128675612818318939678829;  // cos(pi/8)
    const T S1 = (T)0.38268343236508977172845998403039887;  // sin(pi/8)
    const T R2 = (T)0.70710678118654752440084436210484904;
    T c, s;
    switch (J) {
        case 0: return a;
        case 1: c = C1; s = S1; break;
        case 2: c = R2; s = R2; break;
        case 3: c = S1; s = C1; break;
        case 4: return sg_mulw4<DIR>(a);
        case 5: c = -S1; s = C1; break;
        case 6: c = -R2; s = R2; break;
        case 7: c = -C1; s = S1; break;
        case 8: return V{-a.x, -a.y};
        case 9: c = -C1; s = -S1; break;
        default: c = 1; s = 0; break;
    }
    s = DIR * s;
    return V{a.x * c - a.y * s, a.x * s + a.y * c};
}

template <int DIR, typename V>
__device__ __forceinline__ void sg_dft16(V* a)
{
    // n = n1 + 4 n2: DFT-4 over n2, twiddle w16^{n1 k2}, DFT-4 over n1,
    // output index k2 + 4 k1.
    sg_dft4v<DIR>(a[0], a[4], a[8], a[12]);
    sg_dft4v<DIR>(a[1], a[5], a[9], a[13]);
    sg_dft4v<DIR>(a[2], a[6], a[10], a[14]);
    sg_dft4v<DIR>(a[3], a[7], a[11], a[15]);
    // a[n1 + 4 k2] now holds B[n1][k2]
    a[5] = sg_mulw16<DIR, 1>(a[5]);
    a[9] = sg_mulw16<DIR, 2>(a[9]);
    a[13] = sg_mulw16<DIR, 3>(a[13]);
    a[6] = sg_mulw16<DIR, 2>(a[6]);
    a[10] = sg_mulw16<DIR, 4>(a[10]);
    a[14] = sg_mulw16<DIR, 6>(a[14]);
    a[7] = sg_mulw16<DIR, 3>(a[7]);
    a[11] = sg_mulw16<DIR, 6>(a[11]);
    a[15] = sg_mulw16<DIR, 9>(a[15]);
    // DFT-4 over n1 for each k2: inputs a[4 k2 + n1], outputs X[k2 + 4 k1]
    sg_dft4v<DIR>(a[0], a[1], a[2], a[3]);
    sg_dft4v<DIR>(a[4], a[5], a[6], a[7]);
    sg_dft4v<DIR>(a[8], a[9], a[10], a[11]);
    sg_dft4v<DIR>(a[12], a[13], a[14], a[15]);
    // a[4 k2 + k1] holds X[k2 + 4 k1]: transpose the 4 x 4 block
    V t;
    t = a[1]; a[1] = a[4]; a[4] = t;
    t = a[2]; a[2] = a[8]; a[8] = t;
    t = a[3]; a[3] = a[12]; a[12] = t;
    t = a[6]; a[6] = a[9]; a[9] = t;
    t = a[7]; a[7] = a[13]; a[13] = t;
    t = a[11]; a[11] = a[14]; a[14] = t;
}

template <int R, int DIR, typename V>
__device__ __forceinline__ void sg_dft(V* a)
{
    if (R == 2) sg_dft2<DIR>(a);
    if (R == 4) sg_dft4<DIR>(a);
    if (R == 8) sg_dft8<DIR>(a);
    if (R == 16) sg_dft16<DIR>(a);
}

// ---------------------------------------------------------------------------
// Stockham passes.  Butterfly b (0 <= b < N/R) of a pass with sub-transform
// length Ns reads x[b + r N/R], multiplies by w_{Ns R}^{r (b mod Ns)}, does a
// radix-R DFT and writes y[(b - b mod Ns) R + b mod Ns + r Ns].  Thread t does
// the butterflies b = t + s NT, s < E/R, on registers e = s + r E/R.
// ---------------------------------------------------------------------------
template <int R, int E, int DIR, typename V>
__device__ __forceinline__ void sg_pass_compute(V (&v)[E], int t, int NT, int Ns, const V* __restrict__ tw)
{
#pragma unroll
    for (int s = 0; s < E / R; s++) {
        V a[R];
#pragma unroll
        for (int r = 0; r < R; r++) a[r] = v[s + r * (E / R)];
        if (Ns > 1) {
            const int k = (t + s * NT) & (Ns - 1);
            const int stride = SG_NMAX / (Ns * R);
#pragma unroll
            for (int r = 1; r < R; r++) a[r] = cmul(a[r], sg_tw<DIR>(tw, r * k * stride));
        }
        sg_dft<R, DIR>(a);
#pragma unroll
        for (int r = 0; r < R; r++) v[s + r * (E / R)] = a[r];
    }
}

template <int R, int E, typename V>
__device__ __forceinline__ void sg_pass_store(const V (&v)[E], V* sm, int t, int NT, int Ns)
{
#pragma unroll
    for (int s = 0; s < E / R; s++) {
        const int b = t + s * NT;
        const int k = b & (Ns - 1);
        const int base = (b - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; r++) sm[sg_pad(base + r * Ns)] = v[s + r * (E / R)];
    }
}

template <int R, int E, typename V>
__device__ __forceinline__ void sg_pass_load(V (&v)[E], const V* sm, int t, int NT, int N)
{
#pragma unroll
    for (int s = 0; s < E / R; s++) {
        const int b = t + s * NT;
#pragma unroll
        for (int r = 0; r < R; r++) v[s + r * (E / R)] = sm[sg_pad(b + r * (N / R))];
    }
}

// Whole transform.  All threads of the block must call it together (it uses
// __syncthreads); sm is this transform's exchange buffer (sg_padded(N)
// elements).  On exit the buffer is free for reuse.
template <int E, int DIR, typename V>
__device__ __forceinline__ void sg_fft(V (&v)[E], V* sm, int N, int log2N, int t, const V* __restrict__ tw)
{
    const int NT = N / E;
    if (E < 16) {  // N == E: one pass in registers
        sg_pass_compute<E, E, DIR>(v, t, NT, 1, tw);
        return;
    }
    const int rem = log2N & 3;
    int n16 = log2N >> 2;
    int Rprev, Ns;
    if (rem == 1) {
        sg_pass_compute<2, E, DIR>(v, t, NT, 1, tw);
        Rprev = 2;
    } else if (rem == 2) {
        sg_pass_compute<4, E, DIR>(v, t, NT, 1, tw);
        Rprev = 4;
    } else if (rem == 3) {
        sg_pass_compute<8, E, DIR>(v, t, NT, 1, tw);
        Rprev = 8;
    } else {
        sg_pass_compute<16, E, DIR>(v, t, NT, 1, tw);
        Rprev = 16;
        n16--;
    }
    Ns = 1;
    for (int p = 0; p < n16; p++) {
        if (p == 0) __syncthreads();  // the caller may have just read sm
        if (Rprev == 2)
            sg_pass_store<2, E>(v, sm, t, NT, Ns);
        else if (Rprev == 4)
            sg_pass_store<4, E>(v, sm, t, NT, Ns);
        else if (Rprev == 8)
            sg_pass_store<8, E>(v, sm, t, NT, Ns);
        else
            sg_pass_store<16, E>(v, sm, t, NT, Ns);
        Ns *= Rprev;
        __syncthreads();
        sg_pass_load<16, E>(v, sm, t, NT, N);
        __syncthreads();
        sg_pass_compute<16, E, DIR>(v, t, NT, Ns, tw);
        Rprev = 16;
    }
}

// launch-shape helpers shared by the host code
__host__ __device__ __forceinline__ int sg_ilog2(int n)
{
    int l = 0;
    while ((1 << l) < n) l++;
    return l;
}
