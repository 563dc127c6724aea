// sg_common.cuh -- shared device helpers of the GB300 thin-disk force library:
// complex arithmetic on float2/double2; a register-resident Stockham FFT for
// one transform, or for two FP32 transforms in lockstep on the paired f32x2
// instructions (C2, sg_fft_pair); bulk and tensor copies through the TMA
// unit with bounded mbarrier waits; L2 eviction policies.
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
#include <cuda.h>  // CUtensorMap (the descriptor type only; no driver calls here)
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "sg_df.cuh"

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
template <>
struct CX<dfloat> {  // the compensated plans' double-float values (sg_df.cuh)
    typedef dfloat2 t;
};

// read-only loads; the 16-byte double-float pairs have their own overloads
template <typename V>
__device__ __forceinline__ V sg_ldg(const V* p)
{
    return __ldg(p);
}
// warp sums (the double-float values shuffle their two halves)
__device__ __forceinline__ float sg_shfl_xor(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double sg_shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ dfloat sg_shfl_xor(dfloat v, int o) { return df_shfl_xor(v, o); }

// Products and multiply-adds with their rounding stated: one rounding per
// product (sg_mul) or per fused multiply-add (sg_fma), whatever code they are
// inlined into, so that every kernel that runs a transform rounds it the
// same way (the library is built without implicit contraction of a * b + c).
template <typename T>
__device__ __forceinline__ T sg_mul(T a, T b) { return a * b; }
template <typename T>
__device__ __forceinline__ T sg_fma(T a, T b, T c) { return a * b + c; }  // double-float: its own operators
template <>
__device__ __forceinline__ float sg_mul<float>(float a, float b) { return __fmul_rn(a, b); }
template <>
__device__ __forceinline__ float sg_fma<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <>
__device__ __forceinline__ double sg_mul<double>(double a, double b) { return __dmul_rn(a, b); }
template <>
__device__ __forceinline__ double sg_fma<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename V>
__device__ __forceinline__ V cadd(V a, V b) { return V{a.x + b.x, a.y + b.y}; }
template <typename V>
__device__ __forceinline__ V csub(V a, V b) { return V{a.x - b.x, a.y - b.y}; }
template <typename V>
__device__ __forceinline__ V cmul(V a, V b)
{
    return V{sg_fma(a.x, b.x, -sg_mul(a.y, b.y)), sg_fma(a.x, b.y, sg_mul(a.y, b.x))};
}
template <typename V>
__device__ __forceinline__ V cconj(V a) { return V{a.x, -a.y}; }
template <typename V, typename T>
__device__ __forceinline__ V cscale(V a, T s)
{
    typedef decltype(a.x) R;
    return V{sg_mul(a.x, (R)s), sg_mul(a.y, (R)s)};
}
// multiply by i: (x + iy) i = -y + ix
template <typename V>
__device__ __forceinline__ V cmuli(V a) { return V{-a.y, a.x}; }

__host__ __device__ __forceinline__ int sg_pad(int i) { return i + (i >> 4); }
__host__ __device__ __forceinline__ int sg_padded(int n) { return n + (n >> 4) + 1; }

// e^{DIR 2 pi i j / M} from the table (stride NMAX / M folded into idx)
template <int DIR, typename V>
__device__ __forceinline__ V sg_tw(const V* __restrict__ tw, int idx)
{
    V w = sg_ldg(&tw[idx]);
    if (DIR > 0) w.y = -w.y;
    return w;
}

// ---------------------------------------------------------------------------
// Barriers of one transform's threads: the whole block (SgSyncBlock), or only
// the n threads of one slot (named barrier id, n a multiple of 32), so that
// the slots of a block run their transforms independently.
// ---------------------------------------------------------------------------
struct SgSyncBlock {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct SgSyncSlot {
    int id, n;  // id 0: the whole block
    __device__ __forceinline__ void operator()() const
    {
        if (id == 0)
            __syncthreads();
        else
            asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
    }
};

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
    if (K == 1) return V{sg_mul(r, a.x - DIR * a.y), sg_mul(r, a.y + DIR * a.x)};
    return V{sg_mul(r, -a.x - DIR * a.y), sg_mul(r, -a.y + DIR * a.x)};  // K == 3
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
    return V{sg_fma(a.x, c, -sg_mul(a.y, s)), sg_fma(a.x, s, sg_mul(a.y, c))};
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

// The butterflies of a first pass whose inputs r >= R/2 are zero (the
// zero-padded half of a transform): the same outputs, without the
// additions of zeros (which IEEE signed zeros keep the compiler from
// folding).  a4 below is the pair (a0, a1) of a 4-point DFT with a2 = a3 = 0.
// x + DIR i d and x - DIR i d, the factor folded into the additions
template <int DIR, typename V>
__device__ __forceinline__ V cadd_i(V x, V d)
{
    return DIR > 0 ? V{x.x - d.y, x.y + d.x} : V{x.x + d.y, x.y - d.x};
}
template <int DIR, typename V>
__device__ __forceinline__ V csub_i(V x, V d)
{
    return DIR > 0 ? V{x.x + d.y, x.y - d.x} : V{x.x - d.y, x.y + d.x};
}

template <int DIR, typename V>
__device__ __forceinline__ void sg_dft4v_zh(V& a0, V& a1, V& a2, V& a3)
{
    const V b0 = a0, b1 = a1;
    a0 = cadd(b0, b1);
    a2 = csub(b0, b1);
    a1 = cadd_i<DIR>(b0, b1);
    a3 = csub_i<DIR>(b0, b1);
}

template <int R, int DIR, typename V>
__device__ __forceinline__ void sg_dft_zh(V* a)
{
    if (R == 2) a[1] = a[0];
    if (R == 4) sg_dft4v_zh<DIR>(a[0], a[1], a[2], a[3]);
    if (R == 8) {
        // sg_dft8 with a4..a7 = 0: the two 4-point halves are (a0, a2) and (a1, a3)
        V e0 = a[0], e2 = a[2], o1 = a[1], o3 = a[3];
        sg_dft4v_zh<DIR>(e0, e2, a[4], a[6]);
        a[0] = e0;
        a[2] = e2;
        sg_dft4v_zh<DIR>(o1, o3, a[5], a[7]);
        a[1] = o1;
        a[3] = o3;
        const V q1 = sg_mulw8<DIR, 1>(a[3]);
        const V d2 = a[5];
        const V q3 = sg_mulw8<DIR, 3>(a[7]);
        const V f0 = a[0], f1 = a[2], f2_ = a[4], f3 = a[6], g0 = a[1];
        a[0] = cadd(f0, g0);
        a[4] = csub(f0, g0);
        a[1] = cadd(f1, q1);
        a[5] = csub(f1, q1);
        a[2] = cadd_i<DIR>(f2_, d2);
        a[6] = csub_i<DIR>(f2_, d2);
        a[3] = cadd(f3, q3);
        a[7] = csub(f3, q3);
    }
    if (R == 16) {
        // sg_dft16 with a8..a15 = 0: its first four 4-point DFTs lose half their terms
        sg_dft4v_zh<DIR>(a[0], a[4], a[8], a[12]);
        sg_dft4v_zh<DIR>(a[1], a[5], a[9], a[13]);
        sg_dft4v_zh<DIR>(a[2], a[6], a[10], a[14]);
        sg_dft4v_zh<DIR>(a[3], a[7], a[11], a[15]);
        a[5] = sg_mulw16<DIR, 1>(a[5]);
        a[9] = sg_mulw16<DIR, 2>(a[9]);
        a[13] = sg_mulw16<DIR, 3>(a[13]);
        a[6] = sg_mulw16<DIR, 2>(a[6]);
        a[10] = sg_mulw16<DIR, 4>(a[10]);
        a[14] = sg_mulw16<DIR, 6>(a[14]);
        a[7] = sg_mulw16<DIR, 3>(a[7]);
        a[11] = sg_mulw16<DIR, 6>(a[11]);
        a[15] = sg_mulw16<DIR, 9>(a[15]);
        sg_dft4v<DIR>(a[0], a[1], a[2], a[3]);
        sg_dft4v<DIR>(a[4], a[5], a[6], a[7]);
        sg_dft4v<DIR>(a[8], a[9], a[10], a[11]);
        sg_dft4v<DIR>(a[12], a[13], a[14], a[15]);
        V t;
        t = a[1]; a[1] = a[4]; a[4] = t;
        t = a[2]; a[2] = a[8]; a[8] = t;
        t = a[3]; a[3] = a[12]; a[12] = t;
        t = a[6]; a[6] = a[9]; a[9] = t;
        t = a[7]; a[7] = a[13]; a[13] = t;
        t = a[11]; a[11] = a[14]; a[14] = t;
    }
}

// The untwiddled first pass (Ns = 1) of a transform whose thread elements
// e >= E/2 are zero: butterfly s takes v[s + r E/R], zero for r >= R/2.
template <int R, int E, int DIR, typename V>
__device__ __forceinline__ void sg_pass_first_zh(V (&v)[E])
{
#pragma unroll
    for (int s = 0; s < E / R; s++) {
        V a[R];
#pragma unroll
        for (int r = 0; r < R / 2; r++) a[r] = v[s + r * (E / R)];
        sg_dft_zh<R, DIR>(a);
#pragma unroll
        for (int r = 0; r < R; r++) v[s + r * (E / R)] = a[r];
    }
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
// Twiddles w^r, r = 1..R-1, of a butterfly from w = w^1 alone: a product
// tree of depth <= 4 (w^2 = w w, w^3 = w^2 w, w^4 = w^2 w^2, ...), so each
// power carries a few roundings instead of costing a table load.
template <int R, typename V>
__device__ __forceinline__ void sg_twiddle_powers(V* a, V w1)
{
    V w[R];
    w[1] = w1;
    if (R > 2) w[2] = cmul(w1, w1);
    if (R > 3) w[3] = cmul(w[2], w1);
    if (R > 4) {
        w[4] = cmul(w[2], w[2]);
        w[5] = cmul(w[4], w1);
        w[6] = cmul(w[4], w[2]);
        w[7] = cmul(w[4], w[3]);
    }
    if (R > 8) {
        w[8] = cmul(w[4], w[4]);
#pragma unroll
        for (int r = 9; r < 16; r++) w[r] = cmul(w[8], w[r - 8]);
    }
#pragma unroll
    for (int r = 1; r < R; r++) a[r] = cmul(a[r], w[r]);
}

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
            if (sizeof(a[0].x) == 4) {
                // FP32: one table load, the other powers by multiplication
                sg_twiddle_powers<R>(a, sg_tw<DIR>(tw, k * stride));
            } else {
                // FP64 arithmetic is the scarce resource: load every power
#pragma unroll
                for (int r = 1; r < R; r++) a[r] = cmul(a[r], sg_tw<DIR>(tw, r * k * stride));
            }
        }
        sg_dft<R, DIR>(a);
#pragma unroll
        for (int r = 0; r < R; r++) v[s + r * (E / R)] = a[r];
    }
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (TMA, cp.async.bulk) into shared memory, completed
// on an mbarrier.  Addresses and sizes must be multiples of 16 bytes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t sg_smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void sg_mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sg_smem_u32(bar)), "r"(count) : "memory");
    // make the initialised barrier visible to the asynchronous (bulk copy) proxy
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void sg_mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sg_smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool sg_mbar_try_wait(uint64_t* bar, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(sg_smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t sg_globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------------------
// Checked builds (-DSG_DEBUG): before each global copy, store or tensor-copy
// coordinate of the pass kernels, SG_IF_OK tests that the access stays
// inside its buffer (and, for shared-memory ends, inside the block's dynamic
// shared memory, 16-byte aligned).  A failed test sets bit SG_FLAG_BOUNDS of
// the plan's flag word, records the site's number in the word after it (the
// first failure wins) and skips the access; sg_plan_check then reports
// SG_ERR_BOUNDS.  A skipped copy leaves its barrier short, so the pass's
// bounded wait gives up as well.  In ordinary builds SG_IF_OK(c, err, site)
// expands to nothing and the guarded statement always runs.
// ---------------------------------------------------------------------------
#define SG_FLAG_BOUNDS 2
__host__ __device__ __forceinline__ bool sg_in(long long off, long long len, long long extent)
{
    return off >= 0 && len >= 0 && off + len <= extent;
}
__device__ __forceinline__ uint32_t sg_dyn_smem_bytes()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}
// [dst, dst + bytes) inside the dynamic shared memory that starts at base, 16-byte aligned
__device__ __forceinline__ bool sg_smem_in(const void* base, const void* dst, uint32_t bytes)
{
    const long long off = (long long)sg_smem_u32(dst) - (long long)sg_smem_u32(base);
    return (sg_smem_u32(dst) & 15) == 0 && sg_in(off, bytes, sg_dyn_smem_bytes());
}
#ifdef SG_DEBUG
static __device__ __noinline__ bool sg_dbg_fail(int* err, int site)
{
    if (err) {
        atomicOr(err, SG_FLAG_BOUNDS);
        atomicCAS(err + 1, 0, site);
    }
    return false;
}
#define SG_IF_OK(cond, err, site) if ((cond) || sg_dbg_fail((err), (site)))
#else
#define SG_IF_OK(cond, err, site)
#endif

// Prefetch of a contiguous range into L2 (no shared memory, no completion):
// address and size multiples of 16 bytes
__device__ __forceinline__ void sg_prefetch_l2(const void* src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Bulk copy with an L2 eviction-priority policy (sg_policy_*).
__device__ __forceinline__ void sg_bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                                 uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            sg_smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(sg_smem_u32(bar)), "l"(policy)
        : "memory");
}

// ---------------------------------------------------------------------------
// Tensor (tiled) and bulk copies through the TMA unit.  Shared-memory ends of
// tensor copies are 128-byte aligned; every copy's global start obeys the
// 16-byte rule (inner coordinate x element size a multiple of 16).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void sg_tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar,
                                               uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(sg_smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(sg_smem_u32(bar)), "l"(policy)
        : "memory");
}
__device__ __forceinline__ void sg_tma_store_2d(const CUtensorMap* map, int x, int y, const void* src, uint64_t policy)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group.L2::cache_hint [%0, {%1, %2}], [%3], %4;" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(sg_smem_u32(src)), "l"(policy)
                 : "memory");
}
__device__ __forceinline__ void sg_bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// wait until the bulk stores issued by this thread have read their shared memory
__device__ __forceinline__ void sg_bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// order this thread's generic shared-memory accesses with later asynchronous-proxy ones
__device__ __forceinline__ void sg_fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Programmatic dependent launch: a pass lets the next one launch early
// (its blocks are placed once every block of this grid has started) and
// waits for the previous pass's results only where it reads them.  Both are
// no-ops for launches without the programmatic-serialization attribute.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void sg_grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void sg_grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------------------
// L2 eviction priorities.  The half-spectrum intermediates are written by one
// pass and read, transposed, by the next; they are kept in L2 (evict_last)
// while the streamed inputs (density, kernel spectra, consumed intermediates)
// are marked evict_first.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t sg_policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t sg_policy_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void sg_st_hint(float2* a, float2 v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(a), "f"(v.x), "f"(v.y), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void sg_st_hint(double2* a, double2 v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(a), "d"(v.x), "d"(v.y), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void sg_st_hint(float4* a, float4 v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(a), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void sg_st_hint(dfloat2* a, dfloat2 v, uint64_t pol)
{
    sg_st_hint(reinterpret_cast<float4*>(a), make_float4(v.x.hi, v.x.lo, v.y.hi, v.y.lo), pol);
}
__device__ __forceinline__ void sg_st_hint(dfloat* a, dfloat v, uint64_t pol)
{
    sg_st_hint(reinterpret_cast<float2*>(a), make_float2(v.hi, v.lo), pol);
}
// 32 bytes (a whole L2 sector) from one thread: a, then b; p 32-byte aligned
__device__ __forceinline__ void sg_st256_hint(float* p, float4 a, float4 b, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8}, %9;" ::"l"(p), "f"(a.x),
                 "f"(a.y), "f"(a.z), "f"(a.w), "f"(b.x), "f"(b.y), "f"(b.z), "f"(b.w), "l"(pol)
                 : "memory");
}
// read-only loads (data not written during the kernel)
__device__ __forceinline__ float4 sg_ld_hint(const float4* a, uint64_t pol)
{
    float4 r;
    asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
        : "l"(a), "l"(pol));
    return r;
}
__device__ __forceinline__ float2 sg_ld_hint(const float2* a, uint64_t pol)
{
    float2 r;
    asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(r.x), "=f"(r.y) : "l"(a), "l"(pol));
    return r;
}
__device__ __forceinline__ double2 sg_ld_hint(const double2* a, uint64_t pol)
{
    double2 r;
    asm("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(r.x), "=d"(r.y) : "l"(a), "l"(pol));
    return r;
}
__device__ __forceinline__ float sg_ld_hint(const float* a, uint64_t pol)
{
    float r;
    asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(r) : "l"(a), "l"(pol));
    return r;
}
__device__ __forceinline__ double sg_ld_hint(const double* a, uint64_t pol)
{
    double r;
    asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(r) : "l"(a), "l"(pol));
    return r;
}
__device__ __forceinline__ dfloat2 sg_ld_hint(const dfloat2* a, uint64_t pol)
{
    const float4 v = sg_ld_hint(reinterpret_cast<const float4*>(a), pol);
    return dfloat2{dfloat(v.x, v.y), dfloat(v.z, v.w)};
}
__device__ __forceinline__ dfloat sg_ld_hint(const dfloat* a, uint64_t pol)
{
    const float2 v = sg_ld_hint(reinterpret_cast<const float2*>(a), pol);
    return dfloat(v.x, v.y);
}

// Asynchronous global -> shared copies of 16 (or 8) bytes (cp.async), with
// an L2 policy; complete them with sg_cp_async_wait_all and a block barrier.
__device__ __forceinline__ void sg_cp_async16(void* dst, const void* src, uint64_t policy)
{
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(sg_smem_u32(dst)), "l"(src),
                 "l"(policy)
                 : "memory");
}
__device__ __forceinline__ void sg_cp_async8(void* dst, const void* src, uint64_t policy)
{
    asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 8, %2;" ::"r"(sg_smem_u32(dst)), "l"(src),
                 "l"(policy)
                 : "memory");
}
__device__ __forceinline__ void sg_cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Wait for phase `phase` of the barrier, giving up after a time budget (or
// an iteration cap, whichever comes first).  The budget of the first wait,
// `limit`, comes from the flag block (sg_wait_budget: nanoseconds, about a
// second unless a test sets it; 0 gives up at once).  On that timeout the error flag gets
// `code`, a second wait of the full default budget gives the copies in
// flight the time to land (no block leaves with copies still writing its
// shared memory), and the call returns false: the caller then leaves the
// block early (uniformly, via __syncthreads_or) and the host reads the flag.
// Returns true when the data arrived in time.
#define SG_WAIT_NS 1000000000ull
#define SG_WAIT_ITERS (1 << 24)
__device__ __forceinline__ bool sg_mbar_wait_once(uint64_t* bar, uint32_t phase, unsigned long long limit_ns)
{
    if (limit_ns == 0) return false;
    const uint64_t t0 = sg_globaltimer_ns();
    for (int it = 0; it < SG_WAIT_ITERS; it++) {
        if (sg_mbar_try_wait(bar, phase)) return true;
        if ((it & 255) == 255 && sg_globaltimer_ns() - t0 > limit_ns) break;
    }
    return false;
}
// the first-wait budget of the plan's flag block; read once per kernel
__device__ __forceinline__ unsigned long long sg_wait_budget(const int* err)
{
    return err ? __ldg(reinterpret_cast<const unsigned long long*>(err + 2)) : SG_WAIT_NS;
}
// landed (if given): whether the phase completed after all, during the one
// more second that a wait which gave up allows the copies still in flight
__device__ __forceinline__ bool sg_mbar_wait_bounded(uint64_t* bar, uint32_t phase, int* err, int code,
                                                     unsigned long long limit, bool* landed = nullptr)
{
    if (sg_mbar_wait_once(bar, phase, limit)) {
        if (landed) *landed = true;
        return true;
    }
    if (err) atomicOr(err, code);
    const bool late = sg_mbar_wait_once(bar, phase, SG_WAIT_NS);
    if (landed) *landed = late;
    return false;
}

template <int R, int E, typename V>
__device__ __forceinline__ void sg_pass_store(const V (&v)[E], V* sm, int t, int NT, int Ns)
{
#pragma unroll
    for (int s = 0; s < E / R; s++) {
        const int b = t + s * NT;
        const int k = b & (Ns - 1);
        const int base = (b - k) * R + k;
        if (Ns == 1 || (Ns & 15) == 0) {
            // the padding commutes with the stride: pad(base + r Ns) =
            // pad(base) + r (Ns + Ns/16) for Ns a multiple of 16, and
            // pad(base) + r for Ns = 1 (R divides 16, so base..base+R-1 stay
            // in one 16-element group): one index computation per butterfly
            V* p = sm + sg_pad(base);
            const int st = Ns == 1 ? 1 : Ns + (Ns >> 4);
#pragma unroll
            for (int r = 0; r < R; r++) p[r * st] = v[s + r * (E / R)];
        } else {
#pragma unroll
            for (int r = 0; r < R; r++) sm[sg_pad(base + r * Ns)] = v[s + r * (E / R)];
        }
    }
}

template <int R, int E, typename V>
__device__ __forceinline__ void sg_pass_load(V (&v)[E], const V* sm, int t, int NT, int N)
{
    const int M = N / R;
#pragma unroll
    for (int s = 0; s < E / R; s++) {
        const int b = t + s * NT;
        if ((M & 15) == 0) {  // as in sg_pass_store: pad(b + r M) = pad(b) + r (M + M/16)
            const V* p = sm + sg_pad(b);
            const int st = M + (M >> 4);
#pragma unroll
            for (int r = 0; r < R; r++) v[s + r * (E / R)] = p[r * st];
        } else {
#pragma unroll
            for (int r = 0; r < R; r++) v[s + r * (E / R)] = sm[sg_pad(b + r * M)];
        }
    }
}

// Whole transform.  All threads of the block must call it together (it uses
// __syncthreads); sm is this transform's exchange buffer (sg_padded(N)
// elements).  On exit the buffer is free for reuse.
template <int E, int DIR, typename V, typename Sync = SgSyncBlock>
__device__ __forceinline__ void sg_fft(V (&v)[E], V* sm, int N, int log2N, int t, const V* __restrict__ tw,
                                       const Sync& sync = Sync())
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
        if (p == 0) sync();  // the caller may have just read sm
        if (Rprev == 2)
            sg_pass_store<2, E>(v, sm, t, NT, Ns);
        else if (Rprev == 4)
            sg_pass_store<4, E>(v, sm, t, NT, Ns);
        else if (Rprev == 8)
            sg_pass_store<8, E>(v, sm, t, NT, Ns);
        else
            sg_pass_store<16, E>(v, sm, t, NT, Ns);
        Ns *= Rprev;
        sync();
        sg_pass_load<16, E>(v, sm, t, NT, N);
        sync();
        sg_pass_compute<16, E, DIR>(v, t, NT, Ns, tw);
        Rprev = 16;
    }
}

// ---------------------------------------------------------------------------
// The same transform with its twiddles held in registers (E == 16): each of
// a thread's radix-16 passes after the first needs one base twiddle
// w = e^{-2 pi i k / (16 Ns)}, k = t mod Ns, whose powers the pass forms by
// multiplication.  sg_fft_twiddles loads those (at most three) bases once;
// every transform of that length in the kernel then reuses them, in either
// direction, with no further table loads.
// ---------------------------------------------------------------------------
template <typename V>
struct SgTwid {
    V w[3];
};

template <typename V>
__device__ __forceinline__ SgTwid<V> sg_fft_twiddles(int log2N, int t, const V* __restrict__ tw)
{
    SgTwid<V> r;
    const int rem = log2N & 3;
    const int n16 = (log2N >> 2) - (rem == 0 ? 1 : 0);
    int Ns = rem == 0 ? 16 : (1 << rem);
#pragma unroll
    for (int p = 0; p < 3; p++) {
        r.w[p] = V{1, 0};
        if (p < n16) r.w[p] = sg_ldg(&tw[(t & (Ns - 1)) * (SG_NMAX / (Ns * 16))]);
        Ns *= 16;
    }
    return r;
}

template <int DIR, typename V>
__device__ __forceinline__ void sg_pass16_tw(V (&v)[16], V w)
{
    if (DIR > 0) w = cconj(w);
    sg_twiddle_powers<16>(v, w);
    sg_dft<16, DIR>(v);
}

// ZH: the thread elements e >= E/2 are zero on entry (a zero-padded half);
// the first pass skips their terms
template <int E, int DIR, int LG = 0, bool ZH = false, typename V, typename Sync = SgSyncBlock>
__device__ __forceinline__ void sg_fft(V (&v)[E], V* sm, int N_, int log2N_, int t, const SgTwid<V>& tws,
                                       const Sync& sync = Sync())
{
    static_assert(E == 16, "register twiddles need 16 elements per thread");
    // LG > 0: the length 2^LG is a compile-time constant, so every exchange
    // index and stride folds into immediates and the passes unroll
    const int N = LG > 0 ? (1 << LG) : N_, log2N = LG > 0 ? LG : log2N_;
    const int NT = N / E;
    const int rem = log2N & 3;
    const int n16 = (log2N >> 2) - (rem == 0 ? 1 : 0);
    const V* none = nullptr;
    if constexpr (ZH) {
        if (rem == 1)
            sg_pass_first_zh<2, E, DIR>(v);
        else if (rem == 2)
            sg_pass_first_zh<4, E, DIR>(v);
        else if (rem == 3)
            sg_pass_first_zh<8, E, DIR>(v);
        else
            sg_pass_first_zh<16, E, DIR>(v);
    } else if (rem == 1)
        sg_pass_compute<2, E, DIR>(v, t, NT, 1, none);
    else if (rem == 2)
        sg_pass_compute<4, E, DIR>(v, t, NT, 1, none);
    else if (rem == 3)
        sg_pass_compute<8, E, DIR>(v, t, NT, 1, none);
    else
        sg_pass_compute<16, E, DIR>(v, t, NT, 1, none);
    if (n16 == 0) return;
    sync();  // the caller may have just read sm
    if (rem == 1)
        sg_pass_store<2, E>(v, sm, t, NT, 1);
    else if (rem == 2)
        sg_pass_store<4, E>(v, sm, t, NT, 1);
    else if (rem == 3)
        sg_pass_store<8, E>(v, sm, t, NT, 1);
    else
        sg_pass_store<16, E>(v, sm, t, NT, 1);
    auto pass = [&](int p) {
        const int Ns = p > 0 ? (rem == 0 ? 16 : (1 << rem)) << (4 * (p - 1)) : 1;  // stride of pass p's stores
        if (p > 0) sg_pass_store<16, E>(v, sm, t, NT, Ns);
        sync();
        sg_pass_load<16, E>(v, sm, t, NT, N);
        sync();
        sg_pass16_tw<DIR>(v, p == 0 ? tws.w[0] : (p == 1 ? tws.w[1] : tws.w[2]));
    };
    if constexpr (LG > 0) {
#pragma unroll
        for (int p = 0; p < n16; p++) pass(p);
    } else {
        // the radix-16 passes share one copy of their code (a small
        // instruction footprint matters more here than the loop overhead)
#pragma unroll 1
        for (int p = 0; p < n16; p++) pass(p);
    }
}

// ---------------------------------------------------------------------------
// Two FP32 transforms in lockstep.  F2 holds two floats in one 64-bit
// register pair, and its arithmetic uses the paired FP32 instructions of
// sm_100 and later (add/sub/mul/fma .f32x2): one instruction does the same
// operation for both transforms.  C2 holds element e of both transforms:
// real parts in x, imaginary parts in y.  Every step of a transform is the
// same for the two, so nothing is ever moved between the lanes.
// ---------------------------------------------------------------------------
struct F2 {
    unsigned long long v;
};
__device__ __forceinline__ F2 f2(float a, float b)
{
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}
// the halves of a pair (f2 packs its first value into the low 32 bits)
__device__ __forceinline__ float f2_lo(F2 a) { return __uint_as_float((unsigned)(a.v & 0xffffffffull)); }
__device__ __forceinline__ float f2_hi(F2 a) { return __uint_as_float((unsigned)(a.v >> 32)); }
__device__ __forceinline__ F2 operator+(F2 a, F2 b)
{
    F2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 operator-(F2 a, F2 b)
{
    F2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b)
{
    F2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 f2_fma(F2 a, F2 b, F2 c)  // a b + c
{
    F2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}

struct __align__(16) C2 {
    F2 x, y;
};
__device__ __forceinline__ C2 c2(float2 a, float2 b) { return C2{f2(a.x, b.x), f2(a.y, b.y)}; }
__device__ __forceinline__ float2 c2_lo(C2 a) { return make_float2(f2_lo(a.x), f2_lo(a.y)); }
__device__ __forceinline__ float2 c2_hi(C2 a) { return make_float2(f2_hi(a.x), f2_hi(a.y)); }
__device__ __forceinline__ C2 c2_bcast(float2 w) { return C2{f2(w.x, w.x), f2(w.y, w.y)}; }
__device__ __forceinline__ C2 cadd(C2 a, C2 b) { return C2{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ C2 csub(C2 a, C2 b) { return C2{a.x - b.x, a.y - b.y}; }
// (a.x + i a.y)(b.x + i b.y): five paired instructions for the two products
__device__ __forceinline__ C2 cmul(C2 a, C2 b) { return C2{a.x * b.x - a.y * b.y, f2_fma(a.x, b.y, a.y * b.x)}; }

template <int DIR>
__device__ __forceinline__ void sg_dft4v(C2& a0, C2& a1, C2& a2, C2& a3)
{
    // as the scalar one, with the factor DIR i of the odd difference folded
    // into the final additions (no negation instructions)
    const C2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), d = csub(a1, a3);
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    if (DIR > 0) {  // t3 = i d = (-d.y, d.x)
        a1 = C2{t1.x - d.y, t1.y + d.x};
        a3 = C2{t1.x + d.y, t1.y - d.x};
    } else {  // t3 = -i d = (d.y, -d.x)
        a1 = C2{t1.x + d.y, t1.y - d.x};
        a3 = C2{t1.x - d.y, t1.y + d.x};
    }
}

// (a.x + i a.y)(c + i s) with c, s the same in both lanes: four paired
// instructions, the real part's negated product taken from -s
__device__ __forceinline__ C2 cmul_cs(C2 a, F2 c, F2 s, F2 ns) { return C2{f2_fma(a.x, c, a.y * ns), f2_fma(a.x, s, a.y * c)}; }

// a times the twiddle w shared by both lanes (its parts broadcast to the two
// lanes; the sign of -w.y flipped in the integer unit)
__device__ __forceinline__ C2 cmul_b(C2 a, float2 w)
{
    const float nwy = __int_as_float(__float_as_int(w.y) ^ (int)0x80000000);
    return cmul_cs(a, f2(w.x, w.x), f2(w.y, w.y), f2(nwy, nwy));
}

// e^{DIR 2 pi i j / 16} a for the constant twiddles of the radix-16 butterfly
template <int DIR, int J>
__device__ __forceinline__ C2 sg_mulw16(C2 a)
{
    const float C1 = 0.92387953251128675613f, S1 = 0.38268343236508977173f, R2 = 0.70710678118654752440f;
    float c = 1.f, s = 0.f;
    switch (J) {
        case 1: c = C1; s = S1; break;
        case 2: c = R2; s = R2; break;
        case 3: c = S1; s = C1; break;
        case 6: c = -R2; s = R2; break;
        case 9: c = -C1; s = -S1; break;
        default: break;
    }
    s = DIR * s;
    if (J == 0) return a;
    if (J == 4) {  // times DIR i: one negation
        const F2 z = f2(0.f, 0.f);
        return DIR > 0 ? C2{z - a.y, a.x} : C2{a.y, z - a.x};
    }
    return cmul_cs(a, f2(c, c), f2(s, s), f2(-s, -s));
}

// v[r] *= w^r (r = 1..15) for two transforms sharing the twiddle w: the
// powers come from the same product tree as sg_twiddle_powers, in scalar
// FP32 (one lane's work, not two), and multiply both lanes by cmul_b
__device__ __forceinline__ void sg_twiddle_powers_b(C2 (&v)[16], float2 w1)
{
    float2 w[16];
    w[1] = w1;
    w[2] = cmul(w1, w1);
    w[3] = cmul(w[2], w1);
    w[4] = cmul(w[2], w[2]);
    w[5] = cmul(w[4], w1);
    w[6] = cmul(w[4], w[2]);
    w[7] = cmul(w[4], w[3]);
    w[8] = cmul(w[4], w[4]);
#pragma unroll
    for (int r = 9; r < 16; r++) w[r] = cmul(w[8], w[r - 8]);
#pragma unroll
    for (int r = 1; r < 16; r++) v[r] = cmul_b(v[r], w[r]);
}

// e^{DIR i pi k / 4} a, k = 1, 3, for the radix-8 butterfly
template <int DIR, int K>
__device__ __forceinline__ C2 sg_mulw8(C2 a)
{
    const float r = 0.70710678118654752440f;
    const F2 rr = f2(r, r), nr = f2(-r, -r);
    if (K == 1) return DIR > 0 ? C2{(a.x - a.y) * rr, (a.y + a.x) * rr} : C2{(a.x + a.y) * rr, (a.y - a.x) * rr};
    return DIR > 0 ? C2{(a.x + a.y) * nr, (a.x - a.y) * rr} : C2{(a.x - a.y) * nr, (a.x + a.y) * nr};
}

template <int DIR>
__device__ __forceinline__ void sg_dft8(C2* a)
{
    sg_dft4v<DIR>(a[0], a[2], a[4], a[6]);
    sg_dft4v<DIR>(a[1], a[3], a[5], a[7]);
    const C2 o1 = sg_mulw8<DIR, 1>(a[3]);
    const C2 o3 = sg_mulw8<DIR, 3>(a[7]);
    const C2 e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6], o0 = a[1], d = a[5];
    a[0] = cadd(e0, o0);
    a[4] = csub(e0, o0);
    a[1] = cadd(e1, o1);
    a[5] = csub(e1, o1);
    if (DIR > 0) {  // o2 = i d
        a[2] = C2{e2.x - d.y, e2.y + d.x};
        a[6] = C2{e2.x + d.y, e2.y - d.x};
    } else {
        a[2] = C2{e2.x + d.y, e2.y - d.x};
        a[6] = C2{e2.x - d.y, e2.y + d.x};
    }
    a[3] = cadd(e3, o3);
    a[7] = csub(e3, o3);
}

// Two transforms of length N (E = 16 points per thread each), twiddles from
// the registers of sg_fft_twiddles (the same for both).  Same exchange
// pattern as sg_fft; sm holds sg_padded(N) C2 elements (16 bytes each).
template <int DIR, int LG = 0, bool ZH = false, typename Sync = SgSyncBlock>
__device__ __forceinline__ void sg_fft_pair(C2 (&v)[16], C2* sm, int N_, int log2N_, int t,
                                            const SgTwid<float2>& tws, const Sync& sync = Sync())
{
    constexpr int E = 16;
    const int N = LG > 0 ? (1 << LG) : N_, log2N = LG > 0 ? LG : log2N_;  // as in sg_fft
    const int NT = N / E;
    const int rem = log2N & 3;
    const int n16 = (log2N >> 2) - (rem == 0 ? 1 : 0);
    auto first = [&](auto Rc) {
        constexpr int R = decltype(Rc)::value;
        if constexpr (ZH) {  // elements e >= 8 are zero (see sg_fft)
            sg_pass_first_zh<R, E, DIR>(v);
            return;
        }
#pragma unroll
        for (int s = 0; s < E / R; s++) {
            C2 a[R];
#pragma unroll
            for (int r = 0; r < R; r++) a[r] = v[s + r * (E / R)];
            sg_dft<R, DIR>(a);
#pragma unroll
            for (int r = 0; r < R; r++) v[s + r * (E / R)] = a[r];
        }
    };
    if (rem == 1)
        first(std::integral_constant<int, 2>());
    else if (rem == 2)
        first(std::integral_constant<int, 4>());
    else if (rem == 3)
        first(std::integral_constant<int, 8>());
    else
        first(std::integral_constant<int, 16>());
    if (n16 == 0) return;
    sync();  // the caller may have just read sm
    if (rem == 1)
        sg_pass_store<2, E>(v, sm, t, NT, 1);
    else if (rem == 2)
        sg_pass_store<4, E>(v, sm, t, NT, 1);
    else if (rem == 3)
        sg_pass_store<8, E>(v, sm, t, NT, 1);
    else
        sg_pass_store<16, E>(v, sm, t, NT, 1);
    auto pass = [&](int p) {
        const int Ns = p > 0 ? (rem == 0 ? 16 : (1 << rem)) << (4 * (p - 1)) : 1;
        if (p > 0) sg_pass_store<16, E>(v, sm, t, NT, Ns);
        sync();
        sg_pass_load<16, E>(v, sm, t, NT, N);
        sync();
        float2 w = p == 0 ? tws.w[0] : (p == 1 ? tws.w[1] : tws.w[2]);
        if (DIR > 0) w.y = -w.y;
        sg_twiddle_powers_b(v, w);
        sg_dft<16, DIR>(v);
    };
    if constexpr (LG > 0) {
#pragma unroll
        for (int p = 0; p < n16; p++) pass(p);
    } else {
#pragma unroll 1
        for (int p = 0; p < n16; p++) pass(p);
    }
}

// launch-shape helpers shared by the host code
__host__ __device__ __forceinline__ int sg_ilog2(int n)
{
    int l = 0;
    while ((1 << l) < n) l++;
    return l;
}
