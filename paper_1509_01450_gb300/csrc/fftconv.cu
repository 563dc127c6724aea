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
//
// Plans with one-sided radial edge slopes add a rank-4 update per mode
// after P2 (inside P2 for FP32 with 16 points per thread) and its transpose
// after P2b.  FP32 transforms of 2^8 .. 2^13 points run instances with the
// length fixed at compile time, compiled in fftconv_lg<LG>.cu.
#include <map>
#include <mutex>
#include <tuple>

#include <nvtx3/nvToolsExt.h>

#include "sg_internal.cuh"

namespace sg {

// ---------------------------------------------------------------------------
// Kernel spectrum at index kappa in [0, L) from the symmetry-reduced store
// (a copy of one mode's row in shared memory): Khat_r is Hermitian in kappa,
// Khat_phi anti-Hermitian
// ---------------------------------------------------------------------------
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

// Khat_r and Khat_phi at the frequency k = t + e NT of a column transform
// with E points per thread (L = E NT): the lower half of the e's lies below
// N_u and the upper half at or above it (N_u itself only at t = 0,
// e = E/2), so with e unrolled the mirror test costs nothing.
template <int E, typename V>
__device__ __forceinline__ void khat_at(const V* kr, const V* kp, int t, int e, int NT, V& a, V& b)
{
    if (e < E / 2) {
        a = kr[t + e * NT];
        b = kp[t + e * NT];
        return;
    }
    const int j = (E - e) * NT - t;  // L - k
    a = kr[j];
    b = kp[j];
    if (e > E / 2 || t != 0) {
        a.y = -a.y;  // Khat_r(L - k) = conj Khat_r(k)
        b.x = -b.x;  // Khat_phi(L - k) = -conj Khat_phi(k)
    }
}

// coefficients of the one-sided edge-slope update: [a][b], the slope change
// of source row a in {-1, 0, N_u-1, N_u} per weighted sigma of row b in
// {0, 1, N_u-2, N_u-1}
template <typename T>
struct EdgeCoef {
    T c[16];
};

// The origin wedge's update fused into the forward column pass: the wedge
// row's phi-spectrum per mode (swh, written by k_wedge_dft before the row
// pass) and the plan's wedge tables [4][N_phi/2 + 1][N_u] (Wr, Wphi, Vr, Vphi).
template <typename T>
struct WedgeArgs {
    const typename CX<T>::t* swh;
    const T* tab;
};

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
// LG > 0: the transform length 2^LG is fixed at compile time (FP32, 16
// points per thread), see sg_fft
// ZH: the thread elements e >= E/2 are zero (register-twiddle transforms
// skip their terms in the first pass)
template <int E, int DIR, int LG = 0, bool ZH = false, typename V, typename Sync = SgSyncBlock>
__device__ __forceinline__ void fft(V (&v)[E], V* sm, int N, int log2N, int t, const Twd<E, V>& w,
                                    const Sync& sync = Sync())
{
    if constexpr (E == 16 && sizeof(V) == 8)
        sg_fft<E, DIR, LG, ZH>(v, sm, N, log2N, t, w.h, sync);
    else
        sg_fft<E, DIR>(v, sm, N, log2N, t, w.tab, sync);
}

// The slot barrier of a row pass: a named barrier per slot when the slots
// are whole warps and few enough (ids 1..8), else the whole block.
__device__ __forceinline__ SgSyncSlot slot_sync(int slot, int NT, int slots)
{
    return (NT >= 64 && slots <= 8) ? SgSyncSlot{slot + 1, NT} : SgSyncSlot{0, 0};
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
// Row passes: persistent blocks over row blocks of R consecutive rows, with
// two shared-memory buffers: while one block of rows is transformed in one
// buffer (its FFT exchanges included), the inputs of the block after it
// arrive in the other.  Whole rows (density, adjoint seeds) come by one bulk
// copy; the mode-major spectra come and go by 2-D tensor copies (boxes of
// R rows x MB modes, staged as S[m R + r]) when the plan has tensor maps
// for them (use_map), else by cp.async gathers and 16-byte stores.  Results
// that are whole rows leave by bulk stores (use_map) or direct stores.
// ===========================================================================
// elements (V) of one row-pass buffer: the FFT exchange areas of all slots,
// rounded to 128 bytes
template <typename V>
__host__ __device__ __forceinline__ size_t row_buf_elems(int N, int slots)
{
    const size_t per = 128 / sizeof(V);
    return ((size_t)slots * sg_padded(N) + per - 1) / per * per;
}
// Row blocks cycle through a ring of SG_RING buffers: the inputs of block
// j + 1 land in one buffer while block j is transformed in the next, and
// the bulk stores out of block j - 1's buffer finish reading it meanwhile.
#define SG_RING 3
// dynamic shared memory of a row pass: the ring plus alignment slack
template <typename V>
__host__ __device__ __forceinline__ size_t row_smem_bytes(int N, int slots)
{
    return SG_RING * row_buf_elems<V>(N, slots) * sizeof(V) + 128;
}
// two adjacent complex values in one 16-byte access (FP32; FP64 takes two)
__device__ __forceinline__ void ld_pair(const float2* p, float2& a, float2& b)
{
    const float4 q = *reinterpret_cast<const float4*>(p);
    a = make_float2(q.x, q.y);
    b = make_float2(q.z, q.w);
}
__device__ __forceinline__ void ld_pair(const double2* p, double2& a, double2& b)
{
    a = p[0];
    b = p[1];
}
__device__ __forceinline__ void st_pair(float2* p, float2 a, float2 b)
{
    *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st_pair(double2* p, double2 a, double2 b)
{
    p[0] = a;
    p[1] = b;
}
__device__ __forceinline__ void ld_pair(const dfloat2* p, dfloat2& a, dfloat2& b)
{
    a = p[0];
    b = p[1];
}
__device__ __forceinline__ void st_pair(dfloat2* p, dfloat2 a, dfloat2 b)
{
    p[0] = a;
    p[1] = b;
}

// p advanced to the next multiple of A bytes of the shared window.  The
// offset is added to the shared-memory pointer itself: a pointer rebuilt from
// an integer would be generic, and every access through it would take the
// L1TEX path (long-scoreboard waits) instead of a shared-memory instruction.
template <unsigned A = 128>
__device__ __forceinline__ unsigned char* align_smem(unsigned char* p)
{
    return p + ((A - (sg_smem_u32(p) & (A - 1))) & (A - 1));
}
__device__ __forceinline__ unsigned char* align128(unsigned char* p) { return align_smem<128>(p); }
// modes per tensor-copy box
__host__ __device__ __forceinline__ int row_box_modes(int half) { return half < 256 ? half : 256; }

__device__ __forceinline__ void sg_cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most the latest bulk-store group of this thread is still reading shared memory
__device__ __forceinline__ void sg_bulk_wait_read_prev() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }

// Split Z = FFT(z_a + i z_b) of two real sequences into their half spectra
// X_a[m], X_b[m] (m = t + e NT < N/2; mode 0 packs (DC, Nyquist)).  sm is
// the slot's exchange area, free on entry; every thread of the slot calls.
template <int E, typename V, typename T>
__device__ __forceinline__ void split_real_pair(const V (&v)[E], V* sm, int N, int t, V (&xa)[E / 2], V (&xb)[E / 2],
                                                const SgSyncSlot& sync)
{
    const int NT = N / E;
#pragma unroll
    for (int e = 0; e < E; e++) sm[sg_pad(t + e * NT)] = v[e];
    sync();
    const T h = (T)0.5;
#pragma unroll
    for (int e = 0; e < E / 2; e++) {
        const int m = t + e * NT;
        const V z = v[e], zc = cconj(sm[sg_pad((N - m) & (N - 1))]);
        if (m == 0) {
            const V zn = sm[sg_pad(N / 2)];
            xa[e] = V{z.x, zn.x};
            xb[e] = V{z.y, zn.y};
        } else {
            xa[e] = cscale(cadd(z, zc), h);
            const V d = csub(z, zc);
            xb[e] = V{d.y * h, -d.x * h};  // d / 2i
        }
    }
    sync();  // every mirror read is done: the slot's area is free
}

// Tensor stores of a staged mode-major block S[m R + r], box j issued by
// lane j mod 32 of the calling warp (each lane then commits its own group).
template <typename V>
__device__ __forceinline__ void stage_store_map(const CUtensorMap* map, const V* S, int half, int ib, int R, int lane,
                                                int* err, const void* smbase)
{
    constexpr int c = sizeof(V) / 8;  // 8-byte elements per complex value
    const int MB = row_box_modes(half);
    const uint64_t keep = sg_policy_evict_last();  // the next pass reads it from L2
    for (int j = lane; j < half / MB; j += 32)
        SG_IF_OK(((c * ib) & 1) == 0 && ib >= 0 && sg_smem_in(smbase, S + (size_t)j * MB * R, MB * R * sizeof(V)), err,
                 502)
        sg_tma_store_2d(map, c * ib, j * MB, S + (size_t)j * MB * R, keep);
}
// Tensor loads of a mode-major block into S[m R + r], completing on bar
// (whose expected bytes the caller has set); box j issued by lane j mod 32.
template <typename V>
__device__ __forceinline__ void stage_load_map(V* S, const CUtensorMap* map, int half, int ib, int R, uint64_t* bar,
                                               int lane, int* err, const void* smbase)
{
    constexpr int c = sizeof(V) / 8;
    const int MB = row_box_modes(half);
    const uint64_t drop = sg_policy_evict_first();
    for (int j = lane; j < half / MB; j += 32)
        SG_IF_OK(((c * ib) & 1) == 0 && sg_smem_in(smbase, S + (size_t)j * MB * R, MB * R * sizeof(V)), err, 601)
        sg_tma_load_2d(S + (size_t)j * MB * R, map, c * ib, j * MB, bar, drop);
}

// Common prologue of the mbarrier-fed row passes: barriers initialised and
// the first row block requested.  Returns through the loop helpers below.
#define SG_ROWS_BARRIER_INIT()                      \
    if (threadIdx.x == 0)                           \
        for (int q = 0; q < SG_RING; q++) sg_mbar_init(&bar[q], 1); \
    __syncthreads()

// ===========================================================================
// Forward P1: rows (i0, i1) packed as z = w_i0 + i w_i1, FFT along phi,
// split into X_i0, X_i1, staged and stored mode-major.  Each slot takes one
// pair of a row block (R = 2 slots rows).  Shared memory: the output stage
// S[m R + r], the input stage (the block's density rows, one bulk copy) and
// the slots' exchange areas: once the pair is in registers the input stage
// takes the next block's rows, and the output stage is only written again
// after its tensor stores have read it.
// ===========================================================================
template <typename V>
__host__ __device__ __forceinline__ size_t rows_fwd_smem_bytes(int N, int slots)
{
    // output stage R half = slots N, input stage R N reals = slots N, exchange areas
    return ((size_t)2 * slots * N + (size_t)slots * sg_padded(N)) * sizeof(V) + 128;
}

template <typename T, int E, int NTB, int LG = 0>
__global__ void __launch_bounds__(NTB, (sizeof(T) == 4 && NTB == 256) ? 2 : 1) k_fwd_rows(const T* __restrict__ sigma, const T* __restrict__ wpre,
                                                  typename CX<T>::t* __restrict__ A, int nu, int nphi, int log2n,
                                                  const typename CX<T>::t* __restrict__ tw, int* err,
                                                  const __grid_constant__ CUtensorMap mapA, int use_map, int direct)
{
    const unsigned long long wlim = sg_wait_budget(err);  // read once, early
    if constexpr (LG > 0) {  // the length is a compile-time constant
        nphi = 1 << LG;
        log2n = LG;
    }
    typedef typename CX<T>::t V;
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ __align__(8) uint64_t bar;
    const int N = nphi, NT = N / E, half = N / 2;
    const int slot = threadIdx.x / NT, t = threadIdx.x % NT;
    const int slots = blockDim.x / NT;
    const int R = 2 * slots, nblk = (nu + R - 1) / R;
    const int lane = threadIdx.x & 31;
    V* const So = reinterpret_cast<V*>(align128(smraw));        // output stage, R half
    T* const Si = reinterpret_cast<T*>(So + (size_t)slots * N);  // input rows, R N reals
    V* const sm = So + (size_t)2 * slots * N + (size_t)slot * sg_padded(N);
    const Twd<E, V> twd = make_twd<E>(log2n, t, tw);
    const SgSyncSlot ssync = slot_sync(slot, NT, slots);
    if (threadIdx.x == 0) sg_mbar_init(&bar, 1);
    __syncthreads();
    auto issue = [&](int rb) {  // thread 0
        const int rows = min(R, nu - rb * R);
        const uint32_t bytes = (uint32_t)((size_t)rows * N * sizeof(T));
        sg_mbar_expect_tx(&bar, bytes);
        SG_IF_OK(rows > 0 && sg_smem_in(smraw, Si, bytes), err, 501)
        sg_bulk_g2s_hint(Si, sigma + (size_t)rb * R * N, bytes, &bar, sg_policy_evict_first());
    };
    sg_grid_dep_launch();
    sg_grid_dep_wait();  // sigma may come from the previous kernel on the stream
    // direct: sigma is read straight from memory the GPU reaches only by
    // plain loads (pinned host memory), without the bulk copies
    if (!direct && threadIdx.x == 0 && blockIdx.x < nblk) issue(blockIdx.x);
    int it = 0;
    for (int rb = blockIdx.x; rb < nblk; rb += gridDim.x, it++) {
        const bool more = rb + (int)gridDim.x < nblk;
        if (!direct && __syncthreads_or(!sg_mbar_wait_bounded(&bar, it & 1, err, 1, wlim))) {
            if (use_map && threadIdx.x < 32) sg_bulk_wait_read();
            return;  // inputs never arrived
        }
        const int pair = rb * slots + slot;
        const bool live = pair < nu / 2;
        const int i0 = 2 * (live ? pair : 0);
        const T w0 = wpre[i0], w1 = wpre[i0 + 1];
        const T* rows = direct ? sigma + (size_t)i0 * N : Si + (size_t)(2 * slot) * N;
        V v[E];
#pragma unroll
        for (int e = 0; e < E; e++) {
            const int n = t + e * NT;
            v[e] = V{rows[n] * w0, rows[N + n] * w1};
        }
        __syncthreads();  // the input stage is read: it takes the next block's rows
        if (!direct && threadIdx.x == 0 && more) {
            sg_fence_proxy_async();
            issue(rb + gridDim.x);
        }
        fft<E, -1, LG>(v, sm, N, log2n, t, twd, ssync);
        V x0[E / 2], x1[E / 2];
        split_real_pair<E, V, T>(v, sm, N, t, x0, x1, ssync);
        if (use_map && threadIdx.x < 32) sg_bulk_wait_read();  // the last tensor stores have read So
        __syncthreads();
        if (live) {
#pragma unroll
            for (int e = 0; e < E / 2; e++) {
                st_pair(So + (t + e * NT) * R + 2 * slot, x0[e], x1[e]);
            }
        }
        if (use_map) sg_fence_proxy_async();
        __syncthreads();
        if (!use_map) {
            stage_store(A, So, nu, half, rb * R, R);
        } else if (threadIdx.x < 32) {
            stage_store_map(&mapA, So, half, rb * R, R, lane, err, smraw);
            sg_bulk_commit();
        }
    }
    if (use_map && threadIdx.x < 32) sg_bulk_wait_read();
}

// ===========================================================================
// Forward P2: one phi-mode column m per block.  Shared memory: the FFT
// exchange buffer (its first N_u entries double as the landing area of the
// column), then Khat_r[m] and Khat_phi[m] (for m = 0: Khat_r of modes 0 and
// N_phi/2).  FP32 with 16 points per thread: the two inverse transforms run
// in lockstep on paired FP32 instructions, F_r's in the low lanes and
// F_phi's in the high ones, through an exchange area of C2 elements over
// the whole block of shared memory (entered once every spectrum read is
// done).  Otherwise: the phi product is parked over the spectra and the
// inverse transforms run one after the other.
// ===========================================================================
template <typename T>
__host__ __device__ __forceinline__ size_t cols_smem_bytes(int nu)
{
    typedef typename CX<T>::t V;
    const int L = 2 * nu, KS = nu + 2;
    const size_t b = sg_align16(sg_padded(L) * sizeof(V)) + 2 * (size_t)KS * sizeof(V);
    if (sizeof(T) == 4 && L >= 16) {  // the paired inverse transforms' exchange area (C2 elements)
        const size_t pb = sg_padded(L) * sizeof(C2);
        return pb > b ? pb : b;
    }
    return b;
}

// NTB: the block size the kernel is compiled for (L / E threads); FP32
// blocks of 256 threads are compiled for SG_COLS_MINB per SM (2: up to 128
// registers, no spills; 3 would fit the shared memory of N_u = 2048 but
// forces spills)
#ifndef SG_COLS_MINB
#define SG_COLS_MINB 2
#endif
#define SG_COLS_BOUNDS(T, NTB) __launch_bounds__(NTB, (sizeof(T) == 4 && NTB == 256) ? SG_COLS_MINB : 1)
// the forward column pass with its length fixed at 4096: 80 registers fit
// three blocks per SM (the shared memory of N_u = 2048 allows three)
#define SG_FCOLS_BOUNDS(T, NTB, LG, EDGE) \
    __launch_bounds__(NTB, (sizeof(T) == 4 && NTB == 256) ? ((LG == 12 && !EDGE) ? 3 : SG_COLS_MINB) : 1)

// EDGE (FP32, 16 points per thread): the one-sided edge-slope update of
// k_edge_fwd is applied here, before the stores: the mode's two rows of the
// edge tables (gr and gp; for mode 0 gr of modes 0 and N_phi/2) arrive with
// the spectra into an area after the exchange area, and s^_a comes from the
// four edge rows of the landed column.  egr, egp, wpre and ecoef are unused
// otherwise.  WEDGE (with EDGE): the origin wedge's rank-2 update of
// k_wedge_fwd is added in the same place, its table rows read straight from
// global memory by the threads that own the rows, s^_w from swh and a_0 from
// row 0 of the landed column.
// The FP32 forward column transform of mode m (16 points per thread, N_T =
// 2 N_u / 16 threads t): the zero-padded forward FFT of the N_u values in
// sm, the products with both kernel spectra (kr_s, kp_s in shared memory;
// wait_spectra() waits for them and returns false if they never arrive),
// and both inverse transforms paired in w, their exchanges in xarea.  The
// column pass runs one mode per block; the batched kernel (SLOTTED) runs
// several modes of one disk side by side in a block, each on its own
// shared memory, with every barrier taken by the whole block.
template <int LG, bool SLOTTED, typename WaitFn>
__device__ __forceinline__ bool fwd_cols_math(float2 (&v)[16], float2* sm, const float2* kr_s, const float2* kp_s,
                                              C2* xarea, int m, int t, int nu, int log2L,
                                              const Twd<16, float2>& twd, WaitFn wait_spectra, C2 (&w)[16])
{
    typedef float2 V;
    typedef float T;
    constexpr int E = 16;
    const int L = 2 * nu, NT = L / E;
    fft<E, -1, LG, true>(v, sm, L, log2L, t, twd);  // rows >= N_u are zero; the spectra land meanwhile
    if (!wait_spectra()) return false;
    if constexpr (SLOTTED) {  // the barrier below is the whole block's
        if (m == 0)
#pragma unroll
            for (int e = 0; e < E; e++) sm[sg_pad(t + e * NT)] = v[e];
        __syncthreads();
    } else if (m == 0) {
#pragma unroll
        for (int e = 0; e < E; e++) sm[sg_pad(t + e * NT)] = v[e];
        __syncthreads();
    }
    if (m == 0) {
        // v holds the FFT of (DC + i Nyquist): separate the two real
        // sequences and apply the kernels of modes 0 and N_phi/2; the phi
        // force of both modes vanishes
#pragma unroll
        for (int e = 0; e < E; e++) {
            const int k = t + e * NT;
            const V z = v[e], zc = cconj(sm[sg_pad((L - k) & (L - 1))]);
            const V a = cscale(cadd(z, zc), (T)0.5);
            const V d = csub(z, zc);
            const V b = V{sg_mul(d.y, (T)0.5), sg_mul(-d.x, (T)0.5)};
            w[e] = c2(cadd(cmul(a, khat_r_s(kr_s, k, L, nu)), cmuli(cmul(b, khat_r_s(kp_s, k, L, nu)))), V{0, 0});
        }
    } else {
#pragma unroll
        for (int e = 0; e < E; e++) {
            V a, b;
            khat_at<E>(kr_s, kp_s, t, e, NT, a, b);
            w[e] = c2(cmul(v[e], a), cmul(v[e], b));
        }
    }
    // both inverse transforms; their first exchange waits for every spectrum read
    sg_fft_pair<+1, LG>(w, xarea, L, log2L, t, twd.h);
    return true;
}

template <typename T, int E, int NTB, int LG = 0, bool EDGE = false, bool WEDGE = false>
__global__ void SG_FCOLS_BOUNDS(T, NTB, LG, EDGE) k_fwd_cols(const typename CX<T>::t* __restrict__ A,
                                                  const typename CX<T>::t* __restrict__ Kr,
                                                  const typename CX<T>::t* __restrict__ Kp,
                                                  typename CX<T>::t* __restrict__ Br,
                                                  typename CX<T>::t* __restrict__ Cp, int nu, int nphi, int log2L,
                                                  const typename CX<T>::t* __restrict__ tw, int* err,
                                                  const T* __restrict__ egr, const T* __restrict__ egp,
                                                  const T* __restrict__ wpre, EdgeCoef<T> ecoef, WedgeArgs<T> wdg)
{
    const unsigned long long wlim = sg_wait_budget(err);  // read once, early
    if constexpr (LG > 0) {  // the length is a compile-time constant
        nu = 1 << (LG - 1);
        log2L = LG;
    }
    typedef typename CX<T>::t V;
    extern __shared__ __align__(128) unsigned char smraw[];
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
    const uint32_t ab = (uint32_t)(nu * sizeof(V)), kb = (uint32_t)(KS * sizeof(V));
    const uint64_t drop = sg_policy_evict_first();
    const int GS = sg_edge_stride(nu, sizeof(T));
    const uint32_t gb = (uint32_t)(GS * sizeof(T));
    T* const g_s = reinterpret_cast<T*>(smraw + cols_smem_bytes<T>(nu));  // EDGE: 2 GS entries
    if (t == 0) {
        // the spectra (written only by the build) before the previous pass ends
        sg_mbar_expect_tx(&bar[1], 2 * kb + (EDGE ? 2 * gb : 0));
        // spectra [N_phi/2 + 1][KS], edge tables [N_phi/2 + 1][GS]
        SG_IF_OK(m < half && sg_smem_in(smraw, kr_s, 2 * kb), err, 301) {
            sg_bulk_g2s_hint(kr_s, Kr + (size_t)m * KS, kb, &bar[1], drop);
            // mode 0 holds (DC, Nyquist): bring the Nyquist mode's Khat_r
            // instead of Khat_phi, which vanishes at both
            sg_bulk_g2s_hint(kp_s, (m == 0 ? Kr + (size_t)half * KS : Kp + (size_t)m * KS), kb, &bar[1], drop);
        }
        if constexpr (EDGE) {  // likewise the edge tables' rows
            SG_IF_OK(m < half && sg_smem_in(smraw, g_s, 2 * gb), err, 302) {
                sg_bulk_g2s_hint(g_s, egr + (size_t)m * GS, gb, &bar[1], drop);
                sg_bulk_g2s_hint(g_s + GS, (m == 0 ? egr + (size_t)half * GS : egp + (size_t)m * GS), gb, &bar[1],
                                 drop);
            }
        }
    }
    sg_grid_dep_launch();
    sg_grid_dep_wait();  // A is the previous pass's result
    if (t == 0) {
        sg_mbar_expect_tx(&bar[0], ab);
        SG_IF_OK(sg_in((long long)m * nu, nu, (long long)half * nu) && sg_smem_in(smraw, sm, ab), err, 303)
        sg_bulk_g2s_hint(sm, A + (size_t)m * nu, ab, &bar[0], drop);
    }
    const Twd<E, V> twd = make_twd<E>(log2L, t, tw);
    const uint64_t keep = sg_policy_evict_last();  // the row pass reads B and C from L2
    // inputs that never arrive: leave (all threads together) after a last wait for the spectra
    if (__syncthreads_or(!sg_mbar_wait_bounded(&bar[0], 0, err, 1, wlim))) {
        sg_mbar_wait_bounded(&bar[1], 0, err, 1, wlim);
        return;
    }
    V v[E];
#pragma unroll
    for (int e = 0; e < E; e++) v[e] = (e < E / 2) ? sm[t + e * NT] : V{0, 0};  // rows >= nu: zero pad
    __shared__ V es[6];  // EDGE: s^_a; WEDGE: a_0 and s^_w in es[4], es[5]
    if constexpr (EDGE) {
        if (t == 0) {  // read before the transform's first exchange (behind its first barrier)
            const V ab4[4] = {sm[0], sm[1], sm[nu - 2], sm[nu - 1]};
            if constexpr (WEDGE) {
                const T i0 = (T)1 / wpre[0];
                es[4] = V{ab4[0].x * i0, ab4[0].y * i0};
                es[5] = wdg.swh[m];
            }
#pragma unroll
            for (int a = 0; a < 4; a++) {
                V acc{0, 0};
#pragma unroll
                for (int b = 0; b < 4; b++) acc = V{acc.x + ecoef.c[4 * a + b] * ab4[b].x, acc.y + ecoef.c[4 * a + b] * ab4[b].y};
                es[a] = acc;
            }
        }
    }
    if constexpr (sizeof(T) == 4 && E == 16) {
        C2 w[E];  // (Y_r, Y_phi) of each frequency, paired
        const auto wait_spectra = [&] { return !__syncthreads_or(!sg_mbar_wait_bounded(&bar[1], 0, err, 1, wlim)); };
        if (!fwd_cols_math<LG, false>(v, sm, kr_s, kp_s, reinterpret_cast<C2*>(smraw), m, t, nu, log2L, twd,
                                      wait_spectra, w))
            return;
        if constexpr (EDGE) {
            // row i: += wpre[i] sum_a (gr[i - a] s^_a, -i gp[i - a] s^_a), i - a + N_u
            // = i + 1 + N_u, i + N_u, i + 1, i for a = -1, 0, N_u - 1, N_u
            const T* g0 = g_s;
            const T* g1 = g_s + GS;
#pragma unroll
            for (int e = 0; e < E / 2; e++) {
                const int i = t + e * NT;
                const int idx[4] = {i + 1 + nu, i + nu, i + 1, i};
                const T wi = wpre[i];
                V dr{0, 0}, dq{0, 0};
#pragma unroll
                for (int a = 0; a < 4; a++) {
                    const V sa = es[a];
                    const T x0 = g0[idx[a]], x1 = g1[idx[a]];
                    if (m == 0) {  // DC spectrum on the real parts, Nyquist on the imaginary ones
                        dr.x += x0 * sa.x;
                        dr.y += x1 * sa.y;
                    } else {
                        dr.x += x0 * sa.x;
                        dr.y += x0 * sa.y;
                        dq.x += x1 * sa.y;  // -i gp s = gp (s.y - i s.x)
                        dq.y -= x1 * sa.x;
                    }
                }
                if constexpr (WEDGE) {
                    // += (Wr s^_w + Vr a_0, -i (Wphi s^_w + Vphi a_0)); mode 0: Nyquist tables on .y
                    const long tsz = (long)(half + 1) * nu;
                    SG_IF_OK(sg_in((long long)half * nu + i, 1, tsz), err, 304) {}
                    const V a0 = es[4], sw = es[5];
                    const T* tb = wdg.tab + (long)m * nu + i;
                    const T wr = tb[0], wp = tb[tsz], vr = tb[2 * tsz], vp = tb[3 * tsz];
                    if (m == 0) {
                        const T* tn = wdg.tab + (long)half * nu + i;
                        dr.x += wr * sw.x + vr * a0.x;
                        dr.y += tn[0] * sw.y + tn[2 * tsz] * a0.y;
                    } else {
                        dr.x += wr * sw.x + vr * a0.x;
                        dr.y += wr * sw.y + vr * a0.y;
                        dq.x += wp * sw.y + vp * a0.y;
                        dq.y -= wp * sw.x + vp * a0.x;
                    }
                }
                w[e] = C2{w[e].x + f2(wi * dr.x, wi * dq.x), w[e].y + f2(wi * dr.y, wi * dq.y)};
            }
        }
        if constexpr (LG > 0) {
            // the pair layout: {B, C} of each row in 16 bytes (Br holds the pairs)
            float4* P = reinterpret_cast<float4*>(Br) + (size_t)m * nu;
#pragma unroll
            for (int e = 0; e < E / 2; e++)  // crop to N_u rows
                SG_IF_OK(sg_in((long long)m * nu + t + e * NT, 1, (long long)half * nu), err, 305)
                sg_st_hint(P + t + e * NT, make_float4(f2_lo(w[e].x), f2_lo(w[e].y), f2_hi(w[e].x), f2_hi(w[e].y)),
                           keep);
        } else {
#pragma unroll
            for (int e = 0; e < E / 2; e++) {  // crop to N_u rows
                SG_IF_OK(sg_in((long long)m * nu + t + e * NT, 1, (long long)half * nu), err, 306) {
                    sg_st_hint(Br + (size_t)m * nu + t + e * NT, c2_lo(w[e]), keep);
                    sg_st_hint(Cp + (size_t)m * nu + t + e * NT, c2_hi(w[e]), keep);
                }
            }
        }
        return;
    } else {
    // Three transforms share one copy of the FFT code: the forward one, then
    // the two inverse ones as conj(FFT(conj Y)).
#pragma unroll 1
    for (int pass = 0; pass < 3; pass++) {
        fft<E, -1, LG>(v, sm, L, log2L, t, twd);  // pass 0: the spectra land meanwhile
        if (pass == 0) {
            if (__syncthreads_or(!sg_mbar_wait_bounded(&bar[1], 0, err, 1, wlim))) return;
            if (m == 0) {
                // v holds the FFT of (DC + i Nyquist): separate the two real
                // sequences and apply the kernels of modes 0 and N_phi/2; the
                // phi force of both modes vanishes
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
                    v[e] = cconj(cadd(cmul(a, khat_r_s(kr_s, k, L, nu)), cmuli(cmul(b, khat_r_s(kp_s, k, L, nu)))));
                }
                __syncthreads();  // every read of the spectra is done
#pragma unroll
                for (int e = 0; e < E; e++) ks[t + e * NT] = V{0, 0};
            } else {
                // conj of the phi product parked in the exchange buffer, then
                // copied over the spectra; conj of the r product in place
#pragma unroll
                for (int e = 0; e < E; e++) {
                    const int k = t + e * NT;
                    sm[sg_pad(k)] = cconj(cmul(v[e], khat_p_s(kp_s, k, L, nu)));
                    v[e] = cconj(cmul(v[e], khat_r_s(kr_s, k, L, nu)));
                }
                __syncthreads();  // every read of the spectra is done
#pragma unroll
                for (int e = 0; e < E; e++) ks[t + e * NT] = sm[sg_pad(t + e * NT)];
            }
        } else {
            V* out = (pass == 1 ? Br : Cp) + (size_t)m * nu;
#pragma unroll
            for (int e = 0; e < E / 2; e++)  // crop to N_u rows
                SG_IF_OK(sg_in((long long)m * nu + t + e * NT, 1, (long long)half * nu), err, 307)
                sg_st_hint(out + t + e * NT, cconj(v[e]), keep);
            if (pass == 1) {
#pragma unroll
                for (int e = 0; e < E; e++) v[e] = ks[t + e * NT];
            }
        }
    }
    }
}

// ===========================================================================
// Forward P3: row i, Zhat = Fhat_r + i Fhat_phi (Hermitian halves expanded),
// inverse FFT, F_r = Re, F_phi = Im, times beta^{-p i}.  Each slot takes two
// rows of a row block (R = 2 slots rows).  FP32 with 16 points per thread:
// both rows go through one paired transform whose exchange areas lie over
// the stage of the block's B and C rows (S[m R + r], C after B); the next
// block's rows are requested after the transform, while this block's
// forces are stored.  Otherwise the rows go one after the other with
// exchange areas apart from the stage, which takes the next block's inputs
// (tensor copies, or cp.async gathers without maps) during the second FFT.
// ===========================================================================
template <typename V>
__host__ __device__ __forceinline__ size_t rows_inv_smem_bytes(int N, int slots)
{
    const size_t stage = (size_t)2 * slots * N * sizeof(V);  // B and C, R = 2 slots rows
    if (sizeof(V) == 8 && N >= 16) {  // FP32, 16 points per thread: paired areas over the stage
        const size_t pa = (size_t)slots * sg_padded(N) * sizeof(C2);
        return (pa > stage ? pa : stage) + 128;
    }
    return stage + (size_t)slots * sg_padded(N) * sizeof(V) + 128;
}

template <typename T, int E, int NTB, int LG = 0>
__global__ void __launch_bounds__(NTB, (sizeof(T) == 4 && NTB == 256) ? 2 : 1) k_fwd_rows_inv(const typename CX<T>::t* __restrict__ Br,
                                                      const typename CX<T>::t* __restrict__ Cp,
                                                      const T* __restrict__ wpost, T* __restrict__ Fr,
                                                      T* __restrict__ Fp, int nu, int nphi, int log2n,
                                                      const typename CX<T>::t* __restrict__ tw, int* err,
                                                      const __grid_constant__ CUtensorMap mapB,
                                                      const __grid_constant__ CUtensorMap mapC, int use_map)
{
    const unsigned long long wlim = sg_wait_budget(err);  // read once, early
    if constexpr (LG > 0) {  // the length is a compile-time constant
        nphi = 1 << LG;
        log2n = LG;
    }
    typedef typename CX<T>::t V;
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ __align__(8) uint64_t bar;
    const int N = nphi, NT = N / E, half = N / 2;
    const int slot = threadIdx.x / NT, t = threadIdx.x % NT;
    const int slots = blockDim.x / NT;
    const int R = 2 * slots, nblk = (nu + R - 1) / R;
    const int lane = threadIdx.x & 31;
    V* const Sb = reinterpret_cast<V*>(align128(smraw));
    V* const Sc = Sb + (size_t)R * half;
    V* const sm = Sc + (size_t)R * half + (size_t)slot * sg_padded(N);  // this slot's exchange area
    const Twd<E, V> twd = make_twd<E>(log2n, t, tw);
    const SgSyncSlot ssync = slot_sync(slot, NT, slots);
    if (threadIdx.x == 0) sg_mbar_init(&bar, 1);
    __syncthreads();
    auto issue = [&](int rb) {  // use_map: warp 0; else every thread
        if (use_map) {
            if (lane == 0) sg_mbar_expect_tx(&bar, (uint32_t)(2 * (size_t)half * R * sizeof(V)));
            __syncwarp();
            stage_load_map(Sb, &mapB, half, rb * R, R, &bar, lane, err, smraw);
            stage_load_map(Sc, &mapC, half, rb * R, R, &bar, lane, err, smraw);
        } else {
            stage_load(Sb, Br, nu, half, rb * R, R);
            stage_load(Sc, Cp, nu, half, rb * R, R);
            sg_cp_async_commit();
        }
    };
    sg_grid_dep_launch();
    sg_grid_dep_wait();  // B and C are the previous pass's results
    if (blockIdx.x < nblk && (!use_map || threadIdx.x < 32)) issue(blockIdx.x);
    int it = 0;
    for (int rb = blockIdx.x; rb < nblk; rb += gridDim.x, it++) {
        const bool more = rb + (int)gridDim.x < nblk;
        if (use_map) {
            if (__syncthreads_or(!sg_mbar_wait_bounded(&bar, it & 1, err, 1, wlim))) return;  // inputs never arrived
        } else {
            asm volatile("cp.async.wait_all;" ::: "memory");
            __syncthreads();
        }
        // Z of row r of the block at frequency n = t + e NT, from the stage
        auto zrow = [&](int r, int e) -> V {
            const int n = t + e * NT;
            if (e < E / 2) {
                if (n == 0) return V{Sb[r].x, 0};
                const V a = Sb[n * R + r], b = Sc[n * R + r];
                return V{a.x - b.y, a.y + b.x};  // a + i b
            }
            if (n == half) return V{Sb[r].y, 0};
            const V a = Sb[(N - n) * R + r], b = Sc[(N - n) * R + r];
            return V{a.x + b.y, -a.y + b.x};  // conj a + i conj b
        };
        if constexpr (sizeof(T) == 4 && E == 16) {
            // both rows of the slot in one paired transform, its exchange
            // area laid over the stage once every stage read is done
            // the slot's rows r0, r0 + 1 are adjacent in the stage: one
            // 16-byte read gives both, and Z = B + i C (or its mirror
            // conj B + i conj C) of both rows is two paired operations
            C2 w[E];
            const int r0 = 2 * slot;
#pragma unroll
            for (int e = 0; e < E; e++) {
                const int n = t + e * NT;
                const F2 zero = f2(0.f, 0.f);
                if (e < E / 2 && n == 0) {
                    const float4 b = *reinterpret_cast<const float4*>(Sb + r0);
                    w[e] = C2{f2(b.x, b.z), zero};
                } else if (e >= E / 2 && n == half) {
                    const float4 b = *reinterpret_cast<const float4*>(Sb + r0);
                    w[e] = C2{f2(b.y, b.w), zero};
                } else {
                    const int mo = (e < E / 2 ? n : N - n) * R + r0;
                    const float4 a = *reinterpret_cast<const float4*>(Sb + mo);
                    const float4 b = *reinterpret_cast<const float4*>(Sc + mo);
                    if (e < E / 2)
                        w[e] = C2{f2(a.x, a.z) - f2(b.y, b.w), f2(a.y, a.w) + f2(b.x, b.z)};
                    else
                        w[e] = C2{f2(a.x, a.z) + f2(b.y, b.w), f2(b.x, b.z) - f2(a.y, a.w)};
                }
            }
            __syncthreads();
            sg_fft_pair<+1, LG>(w, reinterpret_cast<C2*>(Sb) + (size_t)slot * sg_padded(N), N, log2n, t, twd.h, ssync);
            __syncthreads();  // every slot is done with its area: the stage takes the next block's rows
            if (more && (!use_map || threadIdx.x < 32)) {
                if (use_map) sg_fence_proxy_async();
                issue(rb + gridDim.x);
            }
#pragma unroll 1
            for (int h = 0; h < 2; h++) {
                const int i = rb * R + 2 * slot + h;
                if (i < nu) {
                    const T wt = wpost[i];
#pragma unroll
                    for (int e = 0; e < E; e++) {
                        const int n = t + e * NT;
                        const V z = h ? c2_hi(w[e]) : c2_lo(w[e]);
                        Fr[(size_t)i * N + n] = z.x * wt;
                        Fp[(size_t)i * N + n] = z.y * wt;
                    }
                }
            }
        } else {
#pragma unroll 1
            for (int h = 0; h < 2; h++) {
                const int r = 2 * slot + h;  // row of the block
                V v[E];
#pragma unroll
                for (int e = 0; e < E; e++) {
                    const int n = t + e * NT;
                    V z;
                    if (e < E / 2) {
                        if (n == 0) {
                            z = V{Sb[r].x, 0};
                        } else {
                            const V a = Sb[n * R + r], b = Sc[n * R + r];
                            z = V{a.x - b.y, a.y + b.x};  // a + i b
                        }
                    } else {
                        if (n == half) {
                            z = V{Sb[r].y, 0};
                        } else {
                            const V a = Sb[(N - n) * R + r], b = Sc[(N - n) * R + r];
                            z = V{a.x + b.y, -a.y + b.x};  // conj a + i conj b
                        }
                    }
                    v[e] = z;
                }
                if (h == 1) {
                    __syncthreads();  // the stage is read: it takes the next block's rows
                    if (more && (!use_map || threadIdx.x < 32)) {
                        if (use_map) sg_fence_proxy_async();
                        issue(rb + gridDim.x);
                    }
                }
                fft<E, +1, LG>(v, sm, N, log2n, t, twd, ssync);
                const int i = rb * R + r;
                if (i < nu) {
                    const T w = wpost[i];
#pragma unroll
                    for (int e = 0; e < E; e++) {
                        const int n = t + e * NT;
                        Fr[(size_t)i * N + n] = v[e].x * w;
                        Fp[(size_t)i * N + n] = v[e].y * w;
                    }
                }
            }
        }
    }
    if (!use_map) asm volatile("cp.async.wait_all;" ::: "memory");
}

// ===========================================================================
// One-sided radial slopes at the first and last rows (radial_edges = 1).
// Against the ghost-row slopes of the convolution, the radial slope terms of
// Eq. 28 / A9 change only for the source rows a in {-1, 0, N_u-1, N_u}:
//   dF_i = sum_a beta^{i-a} K^{.,r}[i - a, .] (*)_phi s_a,
// where s_a = r_a (delta_a^onesided - delta_a^ghost) is a combination of
// sigma's rows {0, 1, N_u-2, N_u-1} (zero for the ghost rows' one-sided
// counterparts, which do not exist).  Per phi mode that is a rank-4 update of
// the column: in the weighted frame of the passes
//   B[m][i] += wpre[i] sum_a gr_m[i - a] s^_a,  C[m][i] += wpre[i] sum_a (-i gp_m[i - a]) s^_a,
// with s^_a = sum_b coef[a][b] A[m][b] (coef holds the 1 / wpre[b]).  Mode 0
// packs (DC, Nyquist): its real parts use the DC spectra, its imaginary parts
// the Nyquist ones, and both azimuthal spectra vanish there.
// ===========================================================================
// ps: element stride (in complex values) of B and C: 1, or 2 in the pair layout
template <typename T>
__global__ void __launch_bounds__(256) k_edge_fwd(const typename CX<T>::t* __restrict__ A, typename CX<T>::t* B,
                                                  typename CX<T>::t* C, const T* __restrict__ gr,
                                                  const T* __restrict__ gp, const T* __restrict__ wpre,
                                                  EdgeCoef<T> coef, int nu, int nphi, int ps)
{
    typedef typename CX<T>::t V;
    const int m = blockIdx.x, half = nphi / 2, K = sg_edge_stride(nu, sizeof(T));
    const int brow[4] = {0, 1, nu - 2, nu - 1};
    V ab[4], sa[4];
#pragma unroll
    for (int b = 0; b < 4; b++) ab[b] = A[(size_t)m * nu + brow[b]];
#pragma unroll
    for (int a = 0; a < 4; a++) {
        sa[a] = V{0, 0};
#pragma unroll
        for (int b = 0; b < 4; b++) sa[a] = V{sa[a].x + coef.c[4 * a + b] * ab[b].x, sa[a].y + coef.c[4 * a + b] * ab[b].y};
    }
    // k + N_u = i - a + N_u for a = -1, 0, N_u - 1, N_u
    const T* g0 = gr + (size_t)m * K;
    const T* gN = gr + (size_t)half * K;  // Nyquist (mode 0 only)
    const T* p0 = gp + (size_t)m * K;
    for (int i = threadIdx.x; i < nu; i += blockDim.x) {
        const int idx[4] = {i + 1 + nu, i + nu, i + 1, i};
        const T w = wpre[i];
        V dr{0, 0}, dp{0, 0};
        if (m == 0) {
#pragma unroll
            for (int a = 0; a < 4; a++) {
                dr.x += g0[idx[a]] * sa[a].x;
                dr.y += gN[idx[a]] * sa[a].y;
            }
        } else {
#pragma unroll
            for (int a = 0; a < 4; a++) {
                dr.x += g0[idx[a]] * sa[a].x;
                dr.y += g0[idx[a]] * sa[a].y;
                dp.x += p0[idx[a]] * sa[a].y;  // -i gp s = gp (s.y - i s.x)
                dp.y -= p0[idx[a]] * sa[a].x;
            }
            V c = C[((size_t)m * nu + i) * ps];
            C[((size_t)m * nu + i) * ps] = V{c.x + w * dp.x, c.y + w * dp.y};
        }
        V b = B[((size_t)m * nu + i) * ps];
        B[((size_t)m * nu + i) * ps] = V{b.x + w * dr.x, b.y + w * dr.y};
    }
}

// The transpose for the adjoint: with A, C the column spectra of the weighted
// seeds gF_r, gF_phi (the backward row pass's outputs) and B the backward
// column pass's result,
//   t_a = sum_i wpre[i] (gr_m[i - a] A[m][i] + i gp_m[i - a] C[m][i]),
//   B[m][b] += sum_a coef[a][b] t_a   for b in {0, 1, N_u-2, N_u-1}.
// ps: element stride (in complex values) of A and C: 1, or 2 in the pair layout
template <typename T>
__global__ void __launch_bounds__(256) k_edge_bwd(const typename CX<T>::t* __restrict__ A,
                                                  const typename CX<T>::t* __restrict__ C, typename CX<T>::t* B,
                                                  const T* __restrict__ gr, const T* __restrict__ gp,
                                                  const T* __restrict__ wpre, EdgeCoef<T> coef, int nu, int nphi,
                                                  int ps)
{
    typedef typename CX<T>::t V;
    __shared__ T red[8][8];
    const int m = blockIdx.x, half = nphi / 2, K = sg_edge_stride(nu, sizeof(T));
    const T* g0 = gr + (size_t)m * K;
    const T* gN = gr + (size_t)half * K;
    const T* p0 = gp + (size_t)m * K;
    T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // t_a = (acc[2a], acc[2a + 1])
    for (int i = threadIdx.x; i < nu; i += blockDim.x) {
        const int idx[4] = {i + 1 + nu, i + nu, i + 1, i};
        const T w = wpre[i];
        const V a = A[((size_t)m * nu + i) * ps];
        if (m == 0) {
#pragma unroll
            for (int q = 0; q < 4; q++) {
                acc[2 * q] += w * g0[idx[q]] * a.x;
                acc[2 * q + 1] += w * gN[idx[q]] * a.y;
            }
        } else {
            const V c = C[((size_t)m * nu + i) * ps];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const T r = w * g0[idx[q]], p = w * p0[idx[q]];
                acc[2 * q] += r * a.x - p * c.y;  // i gp c = gp (-c.y + i c.x)
                acc[2 * q + 1] += r * a.y + p * c.x;
            }
        }
    }
#pragma unroll
    for (int v = 0; v < 8; v++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[v] += sg_shfl_xor(acc[v], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int v = 0; v < 8; v++) red[wid][v] = acc[v];
    __syncthreads();
    if (threadIdx.x < 4) {
        const int b = threadIdx.x;
        const int brow[4] = {0, 1, nu - 2, nu - 1};
        T tx[4] = {0, 0, 0, 0}, ty[4] = {0, 0, 0, 0};
        for (int w = 0; w < nw; w++)
#pragma unroll
            for (int q = 0; q < 4; q++) {
                tx[q] += red[w][2 * q];
                ty[q] += red[w][2 * q + 1];
            }
        T dx = 0, dy = 0;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            dx += coef.c[4 * q + b] * tx[q];
            dy += coef.c[4 * q + b] * ty[q];
        }
        // the rows b are distinct (N_u >= 4): one thread each
        V o = B[(size_t)m * nu + brow[b]];
        B[(size_t)m * nu + brow[b]] = V{o.x + dx, o.y + dy};
    }
}

// ===========================================================================
// Backward P1b: row i, z = (gF_r + i gF_phi) beta^{-p i}, FFT, split into
// the half spectra of gF_r (-> A) and gF_phi (-> C), staged and stored
// mode-major.  R = slots rows per row block, arriving as two bulk copies.
// ===========================================================================
template <typename T, int E, int LG = 0>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 256 : 512) k_bwd_rows(const T* __restrict__ gr, const T* __restrict__ gp,
                                                  const T* __restrict__ wpost, typename CX<T>::t* __restrict__ A,
                                                  typename CX<T>::t* __restrict__ C, int nu, int nphi, int log2n,
                                                  const typename CX<T>::t* __restrict__ tw, int* err,
                                                  const __grid_constant__ CUtensorMap mapA,
                                                  const __grid_constant__ CUtensorMap mapC, int use_map)
{
    const unsigned long long wlim = sg_wait_budget(err);  // read once, early
    if constexpr (LG > 0) {  // the length is a compile-time constant
        nphi = 1 << LG;
        log2n = LG;
    }
    typedef typename CX<T>::t V;
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ __align__(8) uint64_t bar[SG_RING];
    const int N = nphi, NT = N / E, half = N / 2;
    const int slot = threadIdx.x / NT, t = threadIdx.x % NT;
    const int slots = blockDim.x / NT;
    const int R = slots, nblk = (nu + R - 1) / R;
    const int lane = threadIdx.x & 31;
    const bool producer = threadIdx.x < 32;
    const size_t bufE = row_buf_elems<V>(N, slots);
    V* const ring = reinterpret_cast<V*>(align128(smraw));
    const Twd<E, V> twd = make_twd<E>(log2n, t, tw);
    const SgSyncSlot ssync = slot_sync(slot, NT, slots);
    SG_ROWS_BARRIER_INIT();
    auto issue = [&](int rb, int q) {  // thread 0: gF_r rows, then gF_phi rows, into buffer q
        const int rows = min(R, nu - rb * R);
        const uint32_t bytes = (uint32_t)((size_t)rows * N * sizeof(T));
        const uint64_t pol = sg_policy_evict_first();
        V* dst = ring + q * bufE;
        sg_mbar_expect_tx(&bar[q], 2 * bytes);
        SG_IF_OK(rows > 0 && sg_smem_in(smraw, dst, bytes) &&
                     sg_smem_in(smraw, reinterpret_cast<T*>(dst) + (size_t)R * N, bytes),
                 err, 701) {
            sg_bulk_g2s_hint(dst, gr + (size_t)rb * R * N, bytes, &bar[q], pol);
            sg_bulk_g2s_hint(reinterpret_cast<T*>(dst) + (size_t)R * N, gp + (size_t)rb * R * N, bytes, &bar[q], pol);
        }
    };
    sg_grid_dep_launch();
    sg_grid_dep_wait();  // the seeds may come from the previous kernel on the stream
    if (threadIdx.x == 0 && blockIdx.x < nblk) issue(blockIdx.x, 0);
    int it = 0;
    for (int rb = blockIdx.x; rb < nblk; rb += gridDim.x, it++) {
        const int q = it % SG_RING, qn = (it + 1) % SG_RING;
        V* const cur = ring + q * bufE;
        const bool more = rb + (int)gridDim.x < nblk;
        __syncthreads();
        if (producer) {
            if (use_map) sg_bulk_wait_read_prev();
            __syncwarp();
            if (threadIdx.x == 0 && more) {
                sg_fence_proxy_async();
                issue(rb + gridDim.x, qn);
            }
        }
        if (__syncthreads_or(!sg_mbar_wait_bounded(&bar[q], (it / SG_RING) & 1, err, 1, wlim))) {
            if (more) sg_mbar_wait_bounded(&bar[qn], ((it + 1) / SG_RING) & 1, err, 1, wlim);
            if (use_map && producer) sg_bulk_wait_read();
            return;
        }
        const int i = rb * R + slot;
        const bool live = i < nu;
        const T w = wpost[live ? i : 0];
        const T* rr = reinterpret_cast<const T*>(cur) + (size_t)slot * N;
        const T* rp = rr + (size_t)R * N;
        V v[E];
#pragma unroll
        for (int e = 0; e < E; e++) {
            const int n = t + e * NT;
            v[e] = V{rr[n] * w, rp[n] * w};
        }
        V* sm = cur + slot * sg_padded(N);
        __syncthreads();  // the rows overlap other slots' exchange areas: all read before any slot transforms
        fft<E, -1, LG>(v, sm, N, log2n, t, twd, ssync);
        V x0[E / 2], x1[E / 2];
        split_real_pair<E, V, T>(v, sm, N, t, x0, x1, ssync);
        __syncthreads();  // the stages span every slot's area
        V* Sa = cur;
        V* Sc = cur + (size_t)R * half;
        if (live) {
#pragma unroll
            for (int e = 0; e < E / 2; e++) {
                Sa[(t + e * NT) * R + slot] = x0[e];
                Sc[(t + e * NT) * R + slot] = x1[e];
            }
        }
        if (use_map) sg_fence_proxy_async();
        __syncthreads();
        if (!use_map) {
            stage_store(A, Sa, nu, half, rb * R, R);
            stage_store(C, Sc, nu, half, rb * R, R);
        } else if (producer) {
            stage_store_map(&mapA, Sa, half, rb * R, R, lane, err, smraw);
            stage_store_map(&mapC, Sc, half, rb * R, R, lane, err, smraw);
            sg_bulk_commit();
        }
    }
    if (use_map && producer) sg_bulk_wait_read();
}

// ===========================================================================
// Backward P2b: column m: FFT of both zero-padded columns, times conj(Khat),
// summed, inverse FFT, crop, to B.  Shared memory: exchange
// buffer (first N_u entries: landing area of the A column), the C column,
// Khat_r[m] and Khat_phi[m] (m = 0: Khat_r of modes 0 and N_phi/2).  FP32
// with 16 points per thread: the two forward transforms run in lockstep on
// paired FP32 instructions (A in the low lanes, C in the high ones) through
// an exchange area of C2 elements that also holds both landing columns; the
// spectra lie after it.
// ===========================================================================
template <typename T>
__host__ __device__ __forceinline__ size_t bcols_smem_bytes(int nu)
{
    typedef typename CX<T>::t V;
    const int L = 2 * nu, KS = nu + 2;
    if (sizeof(T) == 4 && L >= 16)  // paired exchange area (holding both landing columns), then the spectra
        return sg_align16(sg_padded(L) * sizeof(C2)) + 2 * (size_t)KS * sizeof(V);
    return sg_align16(sg_padded(L) * sizeof(V)) + (size_t)nu * sizeof(V) + 2 * (size_t)KS * sizeof(V);
}

// EDGE (FP32, 16 points per thread, L >= 512): the transposed edge-slope
// update of k_edge_bwd is applied here: the mode's rows of the edge tables
// arrive with the spectra (into the exchange area, which is free until the
// first transform), each thread sums its rows' terms of t_a from the landed
// columns, and the owners of rows 0, 1, N_u-2, N_u-1 add
// sum_a coef[a][b] t_a before their stores.  egr, egp, wpre and ecoef are
// unused otherwise.
template <typename T, int E, int NTB, int LG = 0, bool EDGE = false>
__global__ void SG_COLS_BOUNDS(T, NTB) k_bwd_cols(const typename CX<T>::t* __restrict__ A,
                                                  const typename CX<T>::t* __restrict__ C,
                                                  const typename CX<T>::t* __restrict__ Kr,
                                                  const typename CX<T>::t* __restrict__ Kp,
                                                  typename CX<T>::t* __restrict__ B, int nu, int nphi, int log2L,
                                                  const typename CX<T>::t* __restrict__ tw, int* err,
                                                  const T* __restrict__ egr, const T* __restrict__ egp,
                                                  const T* __restrict__ wpre, EdgeCoef<T> ecoef)
{
    const unsigned long long wlim = sg_wait_budget(err);  // read once, early
    if constexpr (LG > 0) {  // the length is a compile-time constant
        nu = 1 << (LG - 1);
        log2L = LG;
    }
    typedef typename CX<T>::t V;
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ __align__(8) uint64_t bar[2];  // [0]: the A column, [1]: the C column and the spectra
    const int L = 2 * nu, NT = L / E, half = nphi / 2, KS = nu + 2;
    const int t = threadIdx.x;
    const int m = blockIdx.x;
    constexpr bool paired = sizeof(T) == 4 && E == 16;
    V* sm = reinterpret_cast<V*>(smraw);
    V* cs = paired ? sm + nu : reinterpret_cast<V*>(smraw + sg_align16(sg_padded(L) * sizeof(V)));  // nu entries
    V* kr_s = paired ? reinterpret_cast<V*>(smraw + sg_align16(sg_padded(L) * sizeof(C2))) : cs + nu;
    V* kp_s = kr_s + KS;
    if (t == 0) {
        sg_mbar_init(&bar[0], 1);
        sg_mbar_init(&bar[1], 1);
    }
    __syncthreads();
    const uint32_t ab = (uint32_t)(nu * sizeof(V)), kb = (uint32_t)(KS * sizeof(V));
    const uint64_t drop = sg_policy_evict_first();
    const int GS = sg_edge_stride(nu, sizeof(T));
    const uint32_t gb = (uint32_t)(GS * sizeof(T));
    // EDGE: 2 GS entries, read before the first exchange: they land in the
    // exchange area after the two columns (16 N_u + 8 GS bytes fit in its
    // 16 sg_padded(L) for N_u >= 8)
    T* const g_s = reinterpret_cast<T*>(smraw + 2 * (size_t)nu * sizeof(V));
    // LG > 0: A and C arrive as one column of the pair layout (A holds the
    // pairs), on bar[0]
    constexpr bool pairs = LG > 0;
    if (t == 0) {  // the spectra first (written only by the build)
        sg_mbar_expect_tx(&bar[1], (pairs ? 0 : ab) + 2 * kb + (EDGE ? 2 * gb : 0));
        SG_IF_OK(m < half && sg_smem_in(smraw, kr_s, 2 * kb), err, 405) {
            sg_bulk_g2s_hint(kr_s, Kr + (size_t)m * KS, kb, &bar[1], drop);
            sg_bulk_g2s_hint(kp_s, (m == 0 ? Kr + (size_t)half * KS : Kp + (size_t)m * KS), kb, &bar[1], drop);
        }
        if constexpr (EDGE) {  // likewise the edge tables' rows
            SG_IF_OK(m < half && sg_smem_in(smraw, g_s, 2 * gb), err, 406) {
                sg_bulk_g2s_hint(g_s, egr + (size_t)m * GS, gb, &bar[1], drop);
                sg_bulk_g2s_hint(g_s + GS, (m == 0 ? egr + (size_t)half * GS : egp + (size_t)m * GS), gb, &bar[1],
                                 drop);
            }
        }
    }
    sg_grid_dep_launch();
    sg_grid_dep_wait();  // A and C are the previous pass's results
    if (t == 0) {
        if constexpr (pairs) {
            sg_mbar_expect_tx(&bar[0], 2 * ab);
            SG_IF_OK(sg_in((long long)2 * m * nu, 2 * nu, (long long)2 * half * nu) && sg_smem_in(smraw, sm, 2 * ab),
                     err, 401)
            sg_bulk_g2s_hint(sm, A + (size_t)2 * m * nu, 2 * ab, &bar[0], drop);
        } else {
            sg_mbar_expect_tx(&bar[0], ab);
            SG_IF_OK(sg_in((long long)m * nu, nu, (long long)half * nu) && sg_smem_in(smraw, sm, ab) &&
                         sg_smem_in(smraw, cs, ab),
                     err, 402) {
                sg_bulk_g2s_hint(sm, A + (size_t)m * nu, ab, &bar[0], drop);
                sg_bulk_g2s_hint(cs, C + (size_t)m * nu, ab, &bar[1], drop);
            }
        }
    }
    const Twd<E, V> twd = make_twd<E>(log2L, t, tw);
    const uint64_t keep = sg_policy_evict_last();
    if (__syncthreads_or(!sg_mbar_wait_bounded(&bar[0], 0, err, 1, wlim))) {
        sg_mbar_wait_bounded(&bar[1], 0, err, 1, wlim);
        return;
    }
    if constexpr (paired) {
        if (__syncthreads_or(!sg_mbar_wait_bounded(&bar[1], 0, err, 1, wlim))) return;
        C2 w[E];  // (X_a, X_c) of each frequency, paired
        if constexpr (pairs) {
            const float4* q = reinterpret_cast<const float4*>(sm);
#pragma unroll
            for (int e = 0; e < E; e++) {
                const float4 u = e < E / 2 ? q[t + e * NT] : make_float4(0.f, 0.f, 0.f, 0.f);
                w[e] = C2{f2(u.x, u.z), f2(u.y, u.w)};
            }
        } else {
#pragma unroll
            for (int e = 0; e < E; e++)
                w[e] = (e < E / 2) ? c2(sm[t + e * NT], cs[t + e * NT]) : c2(V{0, 0}, V{0, 0});
        }
        __shared__ T red[NTB / 32][8];  // EDGE: per-warp sums of t_a
        if constexpr (EDGE) {
            // this thread's rows' terms of t_a = sum_i wpre[i] (gr[i - a] A_i + i gp[i - a] C_i)
            const T* g0 = g_s;
            const T* g1 = g_s + GS;
            T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
            for (int e = 0; e < E / 2; e++) {
                const int i = t + e * NT;
                const int idx[4] = {i + 1 + nu, i + nu, i + 1, i};
                const T wi = wpre[i];
                const V a = c2_lo(w[e]), c = c2_hi(w[e]);
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const T x0 = wi * g0[idx[q]], x1 = wi * g1[idx[q]];
                    if (m == 0) {  // DC spectrum on the real parts, Nyquist on the imaginary ones
                        acc[2 * q] += x0 * a.x;
                        acc[2 * q + 1] += x1 * a.y;
                    } else {
                        acc[2 * q] += x0 * a.x - x1 * c.y;  // i gp c = gp (-c.y + i c.x)
                        acc[2 * q + 1] += x0 * a.y + x1 * c.x;
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < 8; v++)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc[v] += sg_shfl_xor(acc[v], o);
            if ((t & 31) == 0)
#pragma unroll
                for (int v = 0; v < 8; v++) red[t >> 5][v] = acc[v];
            // read after the transforms' barriers
        }
        // rows >= N_u are zero; the transform's first exchange waits for the landing reads
        sg_fft_pair<-1, LG, true>(w, reinterpret_cast<C2*>(smraw), L, log2L, t, twd.h);
        V y[E];
        if (m == 0) {
            // X_a is the FFT of (DC + i Nyquist); the phi kernel vanishes at
            // modes 0 and N_phi/2, so X_c is not needed
#pragma unroll
            for (int e = 0; e < E; e++) sm[sg_pad(t + e * NT)] = c2_lo(w[e]);
            __syncthreads();
#pragma unroll
            for (int e = 0; e < E; e++) {
                const int k = t + e * NT;
                const V z = c2_lo(w[e]), zc = cconj(sm[sg_pad((L - k) & (L - 1))]);
                const V a = cscale(cadd(z, zc), (T)0.5);
                const V d = csub(z, zc);
                const V b = V{d.y * (T)0.5, -d.x * (T)0.5};
                y[e] = cadd(cmul(a, cconj(khat_r_s(kr_s, k, L, nu))), cmuli(cmul(b, cconj(khat_r_s(kp_s, k, L, nu)))));
            }
        } else {
#pragma unroll
            for (int e = 0; e < E; e++) {
                V a, b;
                khat_at<E>(kr_s, kp_s, t, e, NT, a, b);
                y[e] = cadd(cmul(c2_lo(w[e]), cconj(a)), cmul(c2_hi(w[e]), cconj(b)));
            }
        }
        fft<E, +1, LG>(y, sm, L, log2L, t, twd);  // waits for the mirror reads
        if constexpr (EDGE) {
            // rows 0, 1 are element 0 of threads 0, 1; rows N_u-2, N_u-1 element
            // E/2-1 of threads NT-2, NT-1 (N_u = 8 NT, NT >= 2)
            auto update = [&](int b) {
                T tx[4] = {0, 0, 0, 0}, ty[4] = {0, 0, 0, 0};
                for (int w8 = 0; w8 < (int)(blockDim.x >> 5); w8++)
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        tx[q] += red[w8][2 * q];
                        ty[q] += red[w8][2 * q + 1];
                    }
                V d{0, 0};
#pragma unroll
                for (int q = 0; q < 4; q++) d = V{d.x + ecoef.c[4 * q + b] * tx[q], d.y + ecoef.c[4 * q + b] * ty[q]};
                return d;
            };
            if (t < 2) y[0] = cadd(y[0], update(t));
            if (t >= NT - 2) y[E / 2 - 1] = cadd(y[E / 2 - 1], update(t - NT + 4));
        }
#pragma unroll
        for (int e = 0; e < E / 2; e++)
            SG_IF_OK(sg_in((long long)m * nu + t + e * NT, 1, (long long)half * nu), err, 403)
            sg_st_hint(B + (size_t)m * nu + t + e * NT, y[e], keep);
        return;
    } else {
    V v[E];
#pragma unroll
    for (int e = 0; e < E; e++) v[e] = (e < E / 2) ? sm[t + e * NT] : V{0, 0};
    // Three transforms share one copy of the FFT code: FFT of the A column,
    // FFT of the C column, inverse FFT of the sum as conj(FFT(conj Y)).  The
    // partial sum Y_r = X_a conj(Khat_r) is parked at st[0, L), over the C
    // column (read first, element by element by the same thread) and the
    // dead Khat_r.
    V* st = cs;
#pragma unroll 1
    for (int pass = 0; pass < 3; pass++) {
        fft<E, -1, LG>(v, sm, L, log2L, t, twd);
        if (pass == 0) {
            if (__syncthreads_or(!sg_mbar_wait_bounded(&bar[1], 0, err, 1, wlim))) return;
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
                    v[e] = cadd(cmul(a, cconj(khat_r_s(kr_s, k, L, nu))), cmuli(cmul(b, cconj(khat_r_s(kp_s, k, L, nu)))));
                }
            } else {
#pragma unroll
                for (int e = 0; e < E; e++) v[e] = cmul(v[e], cconj(khat_r_s(kr_s, t + e * NT, L, nu)));
            }
            __syncthreads();  // Khat_r (and the mirror buffer) fully read
#pragma unroll
            for (int e = 0; e < E; e++) {
                const int k = t + e * NT;
                if (e < E / 2) {
                    const V c = cs[k];
                    st[k] = v[e];
                    v[e] = c;
                } else {
                    st[k] = v[e];
                    v[e] = V{0, 0};
                }
            }
        } else if (pass == 1) {
            // mode 0: the phi kernel vanishes at modes 0 and N_phi/2
#pragma unroll
            for (int e = 0; e < E; e++) {
                const int k = t + e * NT;
                const V y = m == 0 ? st[k] : cadd(st[k], cmul(v[e], cconj(khat_p_s(kp_s, k, L, nu))));
                v[e] = cconj(y);
            }
        } else {
#pragma unroll
            for (int e = 0; e < E / 2; e++)
                SG_IF_OK(sg_in((long long)m * nu + t + e * NT, 1, (long long)half * nu), err, 404)
                sg_st_hint(B + (size_t)m * nu + t + e * NT, cconj(v[e]), keep);
        }
    }
    }
}

// ===========================================================================
// Backward P3b: rows (i0, i1): Zhat = S_i0 + i S_i1 with S the Hermitian
// extension of each half spectrum; inverse FFT gives rows i0 (Re), i1 (Im).
// Each slot takes one pair of a row block (R = 2 slots rows); the stage of
// the block's B rows takes the next block's rows once the pair is read.
// ===========================================================================
template <typename V>
__host__ __device__ __forceinline__ size_t rows_bwd_inv_smem_bytes(int N, int slots)
{
    return ((size_t)slots * N + (size_t)slots * sg_padded(N)) * sizeof(V) + 128;
}

template <typename T, int E, int NTB, int LG = 0>
__global__ void __launch_bounds__(NTB, (sizeof(T) == 4 && NTB == 256) ? 2 : 1) k_bwd_rows_inv(const typename CX<T>::t* __restrict__ B,
                                                      const T* __restrict__ wpre, T* __restrict__ gs, int nu,
                                                      int nphi, int log2n, const typename CX<T>::t* __restrict__ tw,
                                                      int* err, const __grid_constant__ CUtensorMap mapB, int use_map)
{
    const unsigned long long wlim = sg_wait_budget(err);  // read once, early
    if constexpr (LG > 0) {  // the length is a compile-time constant
        nphi = 1 << LG;
        log2n = LG;
    }
    typedef typename CX<T>::t V;
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ __align__(8) uint64_t bar;
    const int N = nphi, NT = N / E, half = N / 2;
    const int slot = threadIdx.x / NT, t = threadIdx.x % NT;
    const int slots = blockDim.x / NT;
    const int R = 2 * slots, nblk = (nu + R - 1) / R;
    const int lane = threadIdx.x & 31;
    V* const Sb = reinterpret_cast<V*>(align128(smraw));
    V* const sm = Sb + (size_t)R * half + (size_t)slot * sg_padded(N);
    const Twd<E, V> twd = make_twd<E>(log2n, t, tw);
    const SgSyncSlot ssync = slot_sync(slot, NT, slots);
    if (threadIdx.x == 0) sg_mbar_init(&bar, 1);
    __syncthreads();
    auto issue = [&](int rb) {  // use_map: warp 0; else every thread
        if (use_map) {
            if (lane == 0) sg_mbar_expect_tx(&bar, (uint32_t)((size_t)half * R * sizeof(V)));
            __syncwarp();
            stage_load_map(Sb, &mapB, half, rb * R, R, &bar, lane, err, smraw);
        } else {
            stage_load(Sb, B, nu, half, rb * R, R);
            sg_cp_async_commit();
        }
    };
    sg_grid_dep_launch();
    sg_grid_dep_wait();  // B is the previous pass's result
    if (blockIdx.x < nblk && (!use_map || threadIdx.x < 32)) issue(blockIdx.x);
    int it = 0;
    for (int rb = blockIdx.x; rb < nblk; rb += gridDim.x, it++) {
        const bool more = rb + (int)gridDim.x < nblk;
        if (use_map) {
            if (__syncthreads_or(!sg_mbar_wait_bounded(&bar, it & 1, err, 1, wlim))) return;
        } else {
            asm volatile("cp.async.wait_all;" ::: "memory");
            __syncthreads();
        }
        const V* b0s = Sb + 2 * slot;  // this pair's rows are r = 2 slot, 2 slot + 1
        const V* b1s = b0s + 1;
        V v[E];
#pragma unroll
        for (int e = 0; e < E; e++) {
            const int n = t + e * NT;
            V s0, s1;
            if (e < E / 2) {
                if (n == 0) {
                    s0 = V{b0s[0].x, 0};
                    s1 = V{b1s[0].x, 0};
                } else {
                    ld_pair(b0s + n * R, s0, s1);
                }
            } else {
                if (n == half) {
                    s0 = V{b0s[0].y, 0};
                    s1 = V{b1s[0].y, 0};
                } else {
                    ld_pair(b0s + (N - n) * R, s0, s1);
                    s0 = cconj(s0);
                    s1 = cconj(s1);
                }
            }
            v[e] = cadd(s0, cmuli(s1));
        }
        __syncthreads();  // the stage is read: it takes the next block's rows
        if (more && (!use_map || threadIdx.x < 32)) {
            if (use_map) sg_fence_proxy_async();
            issue(rb + gridDim.x);
        }
        fft<E, +1, LG>(v, sm, N, log2n, t, twd, ssync);
        const int pair = rb * slots + slot;
        if (pair < nu / 2) {
            const int i0 = 2 * pair;
            const T w0 = wpre[i0], w1 = wpre[i0 + 1];
#pragma unroll
            for (int e = 0; e < E; e++) {
                const int n = t + e * NT;
                gs[(size_t)i0 * N + n] = v[e].x * w0;
                gs[(size_t)(i0 + 1) * N + n] = v[e].y * w1;
            }
        }
    }
    if (!use_map) asm volatile("cp.async.wait_all;" ::: "memory");
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
    extern __shared__ __align__(128) unsigned char smraw[];
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
    extern __shared__ __align__(128) unsigned char smraw[];
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
// FP32 row passes with the transform length N = 2^LG fixed at compile time,
// moving the mode-major spectra in whole 32-byte L2 sectors.  A copy of
// 16-byte pieces (one mode of two FP32 complex rows) runs at half the rate
// of 32-byte ones, on the TMA unit and the load-store path alike, so every
// thread or stage row here carries four complex values of one mode.
//
// One block per unit of rows: TPG = GT / (N/16) paired transforms
// (sg_fft_pair: two complex FFTs in lockstep on the f32x2 instructions) of
// GT = 256 threads (512 for 8192 points).  The unit's input lands in the
// block's one shared-memory area by bulk or tensor copies, is read into
// registers, and the area then serves as the transforms' exchange areas.
// Blocks are small enough for three per SM (80 registers, 70 KB), so that
// while one waits for its copies the others compute, as in the column pass.
//
//  k_rows_r2c<LG, BWD>: per transform four real rows in two complex FFTs,
//    split into their half spectra.  Forward (P1): rows i0..i0+3 of sigma,
//    z1 = w_i0 sigma_i0 + i w_i0+1 sigma_i0+1, z2 likewise for i0+2, i0+3;
//    A[m][i0..i0+3] (8 bytes each) leave in one 256-bit store.  Adjoint
//    (P1b): z1 = wpost_i0 (gF_r + i gF_phi)_i0, z2 for i0+1; the (A, C)
//    pairs of both rows leave in one 256-bit store.
//  k_rows_c2r<LG, BWD>: per transform one paired inverse FFT, staged by
//    tensor copies whose box rows are 32 bytes (one mode of the transform's
//    rows), stored with the 32-byte swizzle so that the stage reads are free
//    of bank conflicts.  Forward (P3): rows (i0, i0+1) of the (B, C) pairs,
//    Z = B + i C each; F_r, F_phi = Re, Im Z times wpost.  Adjoint (P3b):
//    rows i0..i0+3 of B, Z = S_i0 + i S_i0+1 and S_i0+2 + i S_i0+3; gsigma
//    = Re, Im times wpre.
//
// The pair layout P keeps two complex values per (mode, row) in 16 bytes:
// P[m nu + i] = {X_i, Y_i}, m < N_phi/2 (forward X = B, Y = C; adjoint
// X = A, Y = C); the single layout S[m nu + i] keeps one (forward A,
// adjoint B).  Mode 0 packs (DC, Nyquist) in both.
// ===========================================================================
// blocks per SM the fixed-length row passes' registers are bounded for
// (3: 80 registers, the shared memory of three 70 KB areas)
#ifndef SG_ROWS_MINB
#define SG_ROWS_MINB 3
#endif
template <int LG>
struct RowUnit {
    static constexpr int N = 1 << LG, NT = N / 16;
    static constexpr int GT = LG <= 12 ? 256 : 512;  // threads per block
    static constexpr int TPG = GT / NT;              // paired transforms per block
    static constexpr int MINB = LG <= 12 ? SG_ROWS_MINB : 1;
    // the area: the transforms' exchange areas (C2 elements), plus the 1 KB alignment slack
    static constexpr size_t SMEM = (size_t)TPG * (N + N / 16 + 1) * 16 + 1024;
};

// The half spectra of the real pairs packed in a paired transform: w holds
// FFT(z1) in the low lanes and FFT(z2) in the high lanes (z = a + i b); on
// return A[e] = (X_a of z1, X_a of z2) and B[e] = (X_b of z1, X_b of z2) at
// m = t + e NT < N/2, mode 0 packed (DC, Nyquist).  sm is the transform's
// exchange area (sg_padded(N) C2 elements), free on entry and on return.
template <typename Sync>
__device__ __forceinline__ void split_real_pair2(const C2 (&w)[16], C2* sm, int N, int t, C2 (&A)[8], C2 (&B)[8],
                                                 const Sync& sync)
{
    const int NT = N / 16;
#pragma unroll
    for (int e = 0; e < 16; e++) sm[sg_pad(t + e * NT)] = w[e];
    sync();
    const F2 h = f2(0.5f, 0.5f);
#pragma unroll
    for (int e = 0; e < 8; e++) {
        const int m = t + e * NT;
        const C2 z = w[e];
        const C2 zm = sm[sg_pad((N - m) & (N - 1))];  // Z[N - m]; conj of it below
        if (m == 0) {
            const C2 zn = sm[sg_pad(N / 2)];
            A[e] = C2{z.x, zn.x};
            B[e] = C2{z.y, zn.y};
        } else {
            A[e] = C2{(z.x + zm.x) * h, (z.y - zm.y) * h};  // (Z + conj Z[N-m]) / 2
            B[e] = C2{(z.y + zm.y) * h, (zm.x - z.x) * h};  // (Z - conj Z[N-m]) / 2i
        }
    }
    sync();  // every mirror read is done: the area is free
}

template <int LG>
__host__ __device__ __forceinline__ size_t rows_unit_smem_bytes()
{
    return RowUnit<LG>::SMEM;
}

// DIRECT (forward only): sigma is memory the GPU reaches only by plain loads
// (pinned host memory), read straight into registers without bulk copies
// One unit of the row R2C pass: rows u R .. u R + R - 1 (the pass kernel
// below runs one per block; the batched kernel takes units from its work
// queue).  smraw: the block's dynamic shared memory (RowUnit<LG>::SMEM
// bytes); bar: an initialised mbarrier whose next phase has parity `phase`;
// wave > 0: unit u + wave has its input rows brought into L2 now (0: none);
// PDL: the pass kernel's programmatic-dependent-launch waits.
// Returns false if the unit's inputs never arrived (the flag is set and the
// unit's outputs are not written); the barrier's phase has then completed
// only if its copies landed after all, which `landed` tells.
template <int LG, bool BWD, bool DIRECT, bool PDL>
__device__ __forceinline__ bool rows_r2c_unit(const float* __restrict__ x0, const float* __restrict__ x1,
                                              const float* __restrict__ wrow, float2* __restrict__ out, int nu,
                                              const float2* __restrict__ tw, int* err, int u, int wave,
                                              unsigned char* smraw, uint64_t& bar, uint32_t phase,
                                              unsigned long long wlim, bool* landed = nullptr)
{
    typedef RowUnit<LG> RU;
    constexpr int N = RU::N, NT = RU::NT, TPG = RU::TPG;
    constexpr int RPT = BWD ? 2 : 4;  // rows per transform
    constexpr int R = RPT * TPG;      // rows per block
    unsigned char* const area = align128(smraw);
    const int tr = threadIdx.x / NT, t = threadIdx.x % NT;  // transform, thread in it
    const int i0 = u * R + tr * RPT;
    const Twd<16, float2> twd = make_twd<16>(LG, t, tw);
    // the weights: forward w_i0..i0+3, adjoint (w_i0, w_i0, w_i1, w_i1); loaded while the rows land
    float wt[4] = {0.f, 0.f, 0.f, 0.f};
    SG_IF_OK(i0 + (BWD ? 2 : 4) <= nu, err, 101) {
#pragma unroll
        for (int r = 0; r < 4; r++) wt[r] = __ldg(&wrow[i0 + (BWD ? r / 2 : r)]);
    }
    if constexpr (PDL) {
        sg_grid_dep_launch();
        sg_grid_dep_wait();  // the inputs may come from the previous kernel on the stream
    }
    if (!DIRECT && threadIdx.x == 0) {
        // forward: rows u R .. u R + R - 1 of sigma; adjoint: the same rows of gF_r, then of gF_phi
        const uint64_t pol = sg_policy_evict_first();
        const uint32_t bytes = (uint32_t)R * N * 4;
        float* dst = reinterpret_cast<float*>(area);
        sg_mbar_expect_tx(&bar, BWD ? 2 * bytes : bytes);
        SG_IF_OK(sg_in((long long)u * R, R, nu) && sg_smem_in(smraw, dst, (BWD ? 2 : 1) * bytes), err, 102) {
            sg_bulk_g2s_hint(dst, x0 + (size_t)u * R * N, bytes, &bar, pol);
            if constexpr (BWD) sg_bulk_g2s_hint(dst + (size_t)R * N, x1 + (size_t)u * R * N, bytes, &bar, pol);
        }
        // a later unit (one wave later in the pass kernel) has its rows
        // brought into L2 now, so that its block does not wait on DRAM
        const int un = u + wave;
        if (wave > 0 && un * R < nu) {
            sg_prefetch_l2(x0 + (size_t)un * R * N, bytes);
            if constexpr (BWD) sg_prefetch_l2(x1 + (size_t)un * R * N, bytes);
        }
    }
    if constexpr (!DIRECT) {
        if (__syncthreads_or(!sg_mbar_wait_bounded(&bar, phase, err, 1, wlim, landed))) return false;  // inputs never arrived
    }
    // the four real rows (p, q, r, s) of this transform: z1 = p + i q, z2 = r + i s
    const float *rp, *rq, *rr, *rs;
    if constexpr (DIRECT) {
#ifdef SG_DEBUG
        const int ir = (i0 + 4 <= nu || sg_dbg_fail(err, 104)) ? i0 : 0;  // a failed check reads row 0 instead
#else
        const int ir = i0;
#endif
        rp = x0 + (size_t)ir * N;
        rq = rp + N;
        rr = rp + 2 * N;
        rs = rp + 3 * N;
    } else {
        const float* in = reinterpret_cast<const float*>(area);
        if constexpr (BWD) {
            rp = in + (size_t)tr * 2 * N;        // gF_r row i0
            rr = rp + N;                          // gF_r row i0 + 1
            rq = in + (size_t)(R + tr * 2) * N;  // gF_phi row i0
            rs = rq + N;                          // gF_phi row i0 + 1
        } else {
            rp = in + (size_t)tr * 4 * N;
            rq = rp + N;
            rr = rp + 2 * N;
            rs = rp + 3 * N;
        }
    }
    const F2 wx = f2(wt[0], wt[2]), wy = f2(wt[1], wt[3]);
    C2 w[16];
#pragma unroll
    for (int e = 0; e < 16; e++) {
        const int n = t + e * NT;
        w[e] = C2{f2(rp[n], rr[n]) * wx, f2(rq[n], rs[n]) * wy};
    }
    __syncthreads();  // every transform has read its rows: the area holds the exchange areas
    C2* const sm = reinterpret_cast<C2*>(area) + (size_t)tr * sg_padded(N);
    const SgSyncBlock bsync;
    sg_fft_pair<-1, LG>(w, sm, N, LG, t, twd.h, bsync);
    C2 xa[8], xb[8];
    split_real_pair2(w, sm, N, t, xa, xb, bsync);
    // forward: A[m][i0..i0+3]; adjoint: {A, C} of rows i0, i0+1 (32 bytes, aligned)
    const uint64_t keep = sg_policy_evict_last();  // the column pass reads the spectra from L2
#pragma unroll
    for (int e = 0; e < 8; e++) {
        const size_t mi = (size_t)(t + e * NT) * nu + i0;
        float* q = reinterpret_cast<float*>(out) + (BWD ? 4 : 2) * mi;
        SG_IF_OK(sg_in((long long)mi, BWD ? 2 : 4, (long long)(N / 2) * nu), err, 103)
        sg_st256_hint(q, make_float4(f2_lo(xa[e].x), f2_lo(xa[e].y), f2_lo(xb[e].x), f2_lo(xb[e].y)),
                      make_float4(f2_hi(xa[e].x), f2_hi(xa[e].y), f2_hi(xb[e].x), f2_hi(xb[e].y)), keep);
    }
    return true;
}

template <int LG, bool BWD, bool DIRECT = false>
__global__ void __launch_bounds__(RowUnit<LG>::GT, RowUnit<LG>::MINB)
    k_rows_r2c(const float* __restrict__ x0, const float* __restrict__ x1, const float* __restrict__ wrow,
               float2* __restrict__ out, int nu, const float2* __restrict__ tw, int* err, int wave)
{
    const unsigned long long wlim = sg_wait_budget(err);  // read once, early
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) sg_mbar_init(&bar, 1);
    __syncthreads();
    // the unit one wave later (wave = blocks resident at once) is prefetched
    rows_r2c_unit<LG, BWD, DIRECT, true>(x0, x1, wrow, out, nu, tw, err, blockIdx.x, wave, smraw, bar, 0, wlim);
}

// One unit of the row C2R pass (rows u R .. u R + R - 1), shared like
// rows_r2c_unit; map: the tensor map in kernel-parameter or global memory.
template <int LG, bool BWD, bool PDL>
__device__ __forceinline__ bool rows_c2r_unit(const CUtensorMap* map, const float* __restrict__ wrow,
                                              float* __restrict__ y0, float* __restrict__ y1, int nu,
                                              const float2* __restrict__ tw, int* err, int u, unsigned char* smraw,
                                              uint64_t& bar, uint32_t phase, unsigned long long wlim,
                                              bool* landed = nullptr)
{
    typedef RowUnit<LG> RU;
    constexpr int N = RU::N, NT = RU::NT, TPG = RU::TPG, half = N / 2;
    constexpr int RPT = BWD ? 4 : 2;  // rows per transform
    constexpr int R = RPT * TPG;      // rows per block
    constexpr int MB = half < 256 ? half : 256, NBOX = half / MB;
    unsigned char* const area = align_smem<1024>(smraw);  // the swizzle repeats every 256 bytes
    const int tr = threadIdx.x / NT, t = threadIdx.x % NT;
    const int i0 = u * R + tr * RPT;
    const Twd<16, float2> twd = make_twd<16>(LG, t, tw);
    // the output rows' weights: forward (w_i0, w_i0, w_i0+1, w_i0+1), adjoint w_i0..i0+3
    float wt[4] = {0.f, 0.f, 0.f, 0.f};
    const bool rows_ok = i0 + (BWD ? 4 : 2) <= nu;
    (void)rows_ok;  // read by the checked build only
    SG_IF_OK(rows_ok, err, 201) {
#pragma unroll
        for (int r = 0; r < 4; r++) wt[r] = __ldg(&wrow[i0 + (BWD ? r : r / 2)]);
    }
    if constexpr (PDL) {
        sg_grid_dep_launch();
        sg_grid_dep_wait();  // the spectra are the previous pass's results
    }
    if (threadIdx.x < 32) {
        // transform j's rows land at j N x 16 bytes, mode n of them at 32 n
        const int lane = threadIdx.x;
        if (lane == 0) sg_mbar_expect_tx(&bar, (uint32_t)(TPG * half * 32));
        __syncwarp();
        const uint64_t drop = sg_policy_evict_first();  // the spectra are consumed here
        for (int j = lane; j < TPG * NBOX; j += 32) {
            const int s = j / NBOX, b = j % NBOX;
            const int x = (BWD ? 1 : 2) * (u * R + s * RPT);  // 8-byte units: x even keeps the 16-byte rule
            SG_IF_OK((x & 1) == 0 && sg_in(x, 4, (BWD ? 1 : 2) * (long long)nu) && sg_in(b * MB, MB, half) &&
                         sg_smem_in(smraw, area + (size_t)s * N * 16 + (size_t)b * MB * 32, MB * 32),
                     err, 202)
            sg_tma_load_2d(area + (size_t)s * N * 16 + (size_t)b * MB * 32, map, x, b * MB, &bar, drop);
        }
    }
    if (__syncthreads_or(!sg_mbar_wait_bounded(&bar, phase, err, 1, wlim, landed))) return false;  // inputs never arrived
    const float4* const S4 = reinterpret_cast<const float4*>(area) + (size_t)tr * N;  // this transform's modes
    // Z of both lanes at frequency n.  Each mode holds two 16-byte units u0,
    // u1 (forward: {B, C} of rows i0, i0+1; adjoint: {S_i0, S_i0+1}, {S_i0+2,
    // S_i0+3}), the halves of modes with bit 2 set swapped by the swizzle.
    // With u = (p.x, p.y, q.x, q.y): Z = p + i q below N/2 and conj p + i
    // conj q above (q of mode 0 vanishes in the forward direction: the
    // azimuthal kernel is odd)
    C2 w[16];
#pragma unroll
    for (int e = 0; e < 16; e++) {
        const int n = t + e * NT;
        const int mo = e < 8 ? n : (n == half ? 0 : N - n);  // n = N/2 reads mode 0 (Nyquist)
        const int sw = (mo >> 2) & 1;
        const float4 u0 = S4[2 * mo + sw], u1 = S4[2 * mo + (sw ^ 1)];
        if (n == 0)
            w[e] = C2{f2(u0.x, u1.x), f2(u0.z, u1.z)};
        else if (n == half)
            w[e] = C2{f2(u0.y, u1.y), f2(u0.w, u1.w)};
        else if (e < 8)
            w[e] = C2{f2(u0.x - u0.w, u1.x - u1.w), f2(u0.y + u0.z, u1.y + u1.z)};
        else
            w[e] = C2{f2(u0.x + u0.w, u1.x + u1.w), f2(u0.z - u0.y, u1.z - u1.y)};
    }
    __syncthreads();  // the exchange areas lie over the other transforms' stages
    sg_fft_pair<+1, LG>(w, reinterpret_cast<C2*>(area) + (size_t)tr * sg_padded(N), N, LG, t, twd.h);
    // the four output rows: forward (F_r, F_phi) of i0, then of i0+1;
    // adjoint gsigma of i0 .. i0+3; values Re, Im of the low, then high lanes
    float* o[4];
    if constexpr (BWD) {
#pragma unroll
        for (int r = 0; r < 4; r++) o[r] = y0 + (size_t)(i0 + r) * N;
    } else {
        o[0] = y0 + (size_t)i0 * N;
        o[1] = y1 + (size_t)i0 * N;
        o[2] = y0 + (size_t)(i0 + 1) * N;
        o[3] = y1 + (size_t)(i0 + 1) * N;
    }
    SG_IF_OK(rows_ok, err, 203) {
#pragma unroll
        for (int e = 0; e < 16; e++) {
            const int n = t + e * NT;
            o[0][n] = f2_lo(w[e].x) * wt[0];
            o[1][n] = f2_lo(w[e].y) * wt[1];
            o[2][n] = f2_hi(w[e].x) * wt[2];
            o[3][n] = f2_hi(w[e].y) * wt[3];
        }
    }
    return true;
}

// map: 2-D tensor map over the input (forward: the pair layout, two 8-byte
// units per row; adjoint: the single layout, one unit per row) with boxes
// of 4 units x min(N/2, 256) modes and the 32-byte swizzle
template <int LG, bool BWD>
__global__ void __launch_bounds__(RowUnit<LG>::GT, RowUnit<LG>::MINB)
    k_rows_c2r(const __grid_constant__ CUtensorMap map, const float* __restrict__ wrow, float* __restrict__ y0,
               float* __restrict__ y1, int nu, const float2* __restrict__ tw, int* err)
{
    const unsigned long long wlim = sg_wait_budget(err);  // read once, early
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) sg_mbar_init(&bar, 1);
    __syncthreads();
    rows_c2r_unit<LG, BWD, true>(&map, wrow, y0, y1, nu, tw, err, blockIdx.x, smraw, bar, 0, wlim);
}

// ===========================================================================
// FP32 pass kernels whose transform length 2^LG is fixed at compile time.
// Each length's instances are compiled in a translation unit of their own
// (fftconv_lg<LG>.cu, which includes this file for its kernels only) and
// reached through fixed_pass_kernels().  A plan whose row length N_phi and
// column length 2 N_u both have instances runs all its passes on them, with
// the column spectra in the pair layout; other plans take the run-time
// instances and separate B, C buffers.  Row blocks are 256 threads up to
// 4096 points (several slots below), one 512-thread transform beyond;
// column blocks are one transform of 2 N_u / 16 threads.
// ===========================================================================
// the pass kernels' signatures (spelled out: naming an instance here would
// refer to kernels that each translation unit does not define)
typedef void (*RowsR2CFn)(const float*, const float*, const float*, float2*, int, const float2*, int*, int);
typedef void (*RowsC2RFn)(CUtensorMap, const float*, float*, float*, int, const float2*, int*);
typedef void (*FwdColsFn)(const float2*, const float2*, const float2*, float2*, float2*, int, int, int,
                          const float2*, int*, const float*, const float*, const float*, EdgeCoef<float>,
                          WedgeArgs<float>);
typedef void (*BwdColsFn)(const float2*, const float2*, const float2*, const float2*, float2*, int, int, int,
                          const float2*, int*, const float*, const float*, const float*, EdgeCoef<float>);

struct FixedPassKernels {
    RowsR2CFn fwd_rows;         // k_rows_r2c, forward
    RowsR2CFn fwd_rows_direct;  // the same reading sigma from host memory the GPU can reach
    RowsR2CFn bwd_rows;         // k_rows_r2c, adjoint
    RowsC2RFn fwd_rows_inv;  // k_rows_c2r, forward
    RowsC2RFn bwd_rows_inv;  // k_rows_c2r, adjoint
    size_t r2c_smem, c2r_smem;
    FwdColsFn fwd_cols;
    FwdColsFn fwd_cols_edge;        // with the edge-slope update
    FwdColsFn fwd_cols_edge_wedge;  // with the edge-slope and origin-wedge updates
    BwdColsFn bwd_cols;
    BwdColsFn bwd_cols_edge;  // with the transposed edge-slope update
    int threads;  // block size of the row instances
    int slots;    // paired transforms per row block (RowUnit::TPG)
};

template <int LG>
FixedPassKernels make_fixed_pass_kernels()
{
    constexpr int NB = (1 << LG) / 16 > 256 ? 512 : 256;
    return FixedPassKernels{k_rows_r2c<LG, false>,
                            k_rows_r2c<LG, false, true>,
                            k_rows_r2c<LG, true>,
                            k_rows_c2r<LG, false>,
                            k_rows_c2r<LG, true>,
                            rows_unit_smem_bytes<LG>(),
                            rows_unit_smem_bytes<LG>(),
                            k_fwd_cols<float, 16, NB, LG>,
                            k_fwd_cols<float, 16, NB, LG, true>,
                            k_fwd_cols<float, 16, NB, LG, true, true>,
                            k_bwd_cols<float, 16, NB, LG>,
                            k_bwd_cols<float, 16, NB, LG, true>,
                            RowUnit<LG>::GT,
                            RowUnit<LG>::TPG};
}

// defined in fftconv_lg<LG>.cu
FixedPassKernels fixed_pass_kernels_lg8();
FixedPassKernels fixed_pass_kernels_lg9();
FixedPassKernels fixed_pass_kernels_lg10();
FixedPassKernels fixed_pass_kernels_lg11();
FixedPassKernels fixed_pass_kernels_lg12();
FixedPassKernels fixed_pass_kernels_lg13();

#ifndef SG_FFTCONV_KERNELS_ONLY
// the instances for transforms of 2^lg points, or null
static const FixedPassKernels* fixed_pass_kernels(int lg)
{
    static const FixedPassKernels table[6] = {fixed_pass_kernels_lg8(),  fixed_pass_kernels_lg9(),
                                              fixed_pass_kernels_lg10(), fixed_pass_kernels_lg11(),
                                              fixed_pass_kernels_lg12(), fixed_pass_kernels_lg13()};
    return lg >= 8 && lg <= 13 ? &table[lg - 8] : nullptr;
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
// shared-memory-heavy kernel per SM).  Done once per kernel, device and
// size: later launches (for example while a stream is being captured) make
// no attribute calls.
struct LaunchCache {
    std::mutex mu;
    std::map<std::tuple<const void*, int, int, size_t>, int> occ;  // (kernel, device, threads, smem) -> blocks/SM
    std::map<std::tuple<const void*, int>, size_t> smem;            // (kernel, device) -> opted-in bytes
};
static LaunchCache& launch_cache()
{
    static LaunchCache c;
    return c;
}
static int current_device()
{
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess) {
        cudaGetLastError();
        d = 0;
    }
    return d;
}

template <typename K>
static cudaError_t set_smem(K kernel, size_t smem, bool carveout = false)
{
    LaunchCache& c = launch_cache();
    const auto key = std::make_tuple((const void*)kernel, current_device());
    std::lock_guard<std::mutex> lock(c.mu);
    auto it = c.smem.find(key);
    if (it != c.smem.end() && it->second >= smem) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (smem > 48 * 1024) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && carveout)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess) c.smem[key] = it != c.smem.end() && it->second > smem ? it->second : smem;
    return e;
}

// NVTX range around the enqueue of one pass (visible in Nsight timelines;
// near-free when no tool is attached)
struct PassRange {
    explicit PassRange(const char* name) { nvtxRangePushA(name); }
    ~PassRange() { nvtxRangePop(); }
};

// Launch with programmatic stream serialization: the kernel may start while
// the previous one on the stream finishes; it waits (sg_grid_dep_wait)
// before it reads that kernel's results.
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t st,
                              Args&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Blocks of a kernel resident on the GPU at once (occupancy x SMs), cached
// per kernel, device and launch shape.
template <typename K>
static int resident_blocks(K kernel, int threads, size_t smem, int sms)
{
    LaunchCache& c = launch_cache();
    const auto key = std::make_tuple((const void*)kernel, current_device(), threads, smem);
    int occ = 0;
    {
        std::lock_guard<std::mutex> lock(c.mu);
        auto it = c.occ.find(key);
        if (it != c.occ.end()) occ = it->second;
    }
    if (occ == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) != cudaSuccess || occ < 1) {
            cudaGetLastError();
            occ = 1;
        }
        std::lock_guard<std::mutex> lock(c.mu);
        c.occ[key] = occ;
    }
    return occ * (sms > 0 ? sms : 1);
}

// Grid of a persistent row pass: as many blocks as fit on the GPU at once
// (each loops over row blocks), at most one per row block.
template <typename K>
static int persistent_grid(K kernel, int threads, size_t smem, int nblk, int sms)
{
    LaunchCache& c = launch_cache();
    const auto key = std::make_tuple((const void*)kernel, current_device(), threads, smem);
    int occ = 0;
    {
        std::lock_guard<std::mutex> lock(c.mu);
        auto it = c.occ.find(key);
        if (it != c.occ.end()) occ = it->second;
    }
    if (occ == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) != cudaSuccess || occ < 1) {
            cudaGetLastError();
            occ = 1;
        }
        std::lock_guard<std::mutex> lock(c.mu);
        c.occ[key] = occ;
    }
    const int g = occ * (sms > 0 ? sms : 1);
    return nblk < g ? nblk : g;
}

// threads a row-pass block should have at least (several slots per block)
static int row_min_threads(size_t elem) { return elem == 4 ? 512 : 64; }

#ifndef SG_FFTCONV_DF  // the tensor maps are made once, in this translation unit
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry points (no
// link-time dependency on the driver library); null if unavailable
static EncodeTiledFn tensor_map_encoder()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
        else
            cudaGetLastError();
    });
    return fn;
}

void make_row_maps(int nu, int nphi, size_t elem, void* const bufs[3], SgRowMaps out[2])
{
    out[0].R = out[1].R = 0;
    EncodeTiledFn enc = tensor_map_encoder();
    if (!enc) return;
    const int S = elem == 4 ? shape_for<float2>(nphi, row_min_threads(elem)).slots
                            : shape_for<double2>(nphi, row_min_threads(elem)).slots;
    const int half = nphi / 2, c = (int)(2 * elem / 8), MB = row_box_modes(half);
    for (int k = 0; k < 2; k++) {
        const int R = k == 0 ? S : 2 * S;
        // inner box of at least 16 bytes and at most 256 elements; 128-byte
        // aligned boxes in shared memory
        if (nphi < 32 || c * R < 2 || c * R > 256 || R > nu || ((size_t)MB * c * R * 8) % 128) continue;
        const cuuint64_t dims[2] = {(cuuint64_t)c * nu, (cuuint64_t)half};
        const cuuint64_t strides[1] = {(cuuint64_t)c * nu * 8};
        const cuuint32_t box[2] = {(cuuint32_t)(c * R), (cuuint32_t)MB};
        const cuuint32_t estr[2] = {1, 1};
        bool ok = true;
        for (int b = 0; b < 3 && ok; b++)
            ok = enc(&out[k].m[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, bufs[b], dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
        if (ok) out[k].R = R;
    }
}

bool make_pair_maps(int nu, int nphi, void* wa, void* wb, CUtensorMap out[2])
{
    EncodeTiledFn enc = tensor_map_encoder();
    if (!enc || nphi < 32) return false;
    const int half = nphi / 2, MB = row_box_modes(half);
    for (int k = 0; k < 2; k++) {
        const int c = k == 0 ? 2 : 1;  // 8-byte units per row: (X, Y) pairs, single values
        const cuuint64_t dims[2] = {(cuuint64_t)c * nu, (cuuint64_t)half};
        const cuuint64_t strides[1] = {(cuuint64_t)c * nu * 8};
        const cuuint32_t box[2] = {4, (cuuint32_t)MB};
        const cuuint32_t estr[2] = {1, 1};
        if (enc(&out[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, k == 0 ? wb : wa, dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    return true;
}
#endif

// the map of buffer b for row blocks of R rows, or null
static const CUtensorMap* row_map(const PlanView& p, int R, int b, int nphi)
{
    if (!p.maps || nphi < 32) return nullptr;
    for (int k = 0; k < 2; k++)
        if (p.maps[k].R == R) return &p.maps[k].m[b];
    return nullptr;
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
static cudaError_t launch_edges(const PlanView& p, bool adjoint, cudaStream_t st)
{
    typedef typename CX<T>::t V;
    PassRange range_(adjoint ? "sg adjoint edge slopes" : "sg forward edge slopes");
    EdgeCoef<T> coef;
    for (int j = 0; j < 16; j++) coef.c[j] = (T)p.ecoef[j];
    // the pair layout: wb holds (B, C) forward and (A, C) in the adjoint, wa the adjoint's B
    const int ps = p.pairs ? 2 : 1;
    V* const X = (V*)p.wb;
    V* const Y = p.pairs ? (V*)p.wb + 1 : (V*)p.wc;
    if (adjoint)
        k_edge_bwd<T><<<p.nphi / 2, 256, 0, st>>>(p.pairs ? X : (const V*)p.wa, Y, p.pairs ? (V*)p.wa : X,
                                                  (const T*)p.egr, (const T*)p.egp, (const T*)p.wpre, coef, p.nu,
                                                  p.nphi, ps);
    else
        k_edge_fwd<T><<<p.nphi / 2, 256, 0, st>>>((const V*)p.wa, X, Y, (const T*)p.egr, (const T*)p.egp,
                                                  (const T*)p.wpre, coef, p.nu, p.nphi, ps);
    return cudaGetLastError();
}

// The fixed-length instances of both transform lengths, when every pass of
// the plan can run on them: FP32, N_phi and 2 N_u of 256 .. 8192 points, the
// pair layout's tensor maps made, N_u a multiple of the row blocks.  The
// passes then keep the column spectra in the pair layout.
template <typename T>
static bool fixed_path(const PlanView& p, const FixedPassKernels*& fr, const FixedPassKernels*& fc)
{
    fr = fc = nullptr;
    if (sizeof(T) != 4 || !p.imaps) return false;
    const FixedPassKernels* a = fixed_pass_kernels(sg_ilog2(p.nphi));
    const FixedPassKernels* b = fixed_pass_kernels(sg_ilog2(2 * p.nu));
    if (!a || !b || p.nu % (4 * a->slots) != 0) return false;
    fr = a;
    fc = b;
    return true;
}

template <typename T>
cudaError_t launch_forward(const PlanView& p0, const T* sigma, T* Fr, T* Fp, cudaStream_t st, cudaEvent_t* ev,
                           bool sigma_direct)
{
    typedef typename CX<T>::t V;
    const FixedPassKernels *fr, *fc;
    PlanView p = p0;
    p.pairs = fixed_path<T>(p0, fr, fc) ? 1 : 0;
    const V* tw = (const V*)p.tw;
    V* A = (V*)p.wa;
    V* B = (V*)p.wb;
    V* C = (V*)p.wc;
    const int ln = sg_ilog2(p.nphi), lL = sg_ilog2(2 * p.nu);
    cudaError_t err;
    if (ev && (err = cudaEventRecord(ev[0], st)) != cudaSuccess) return err;
    // FP32 columns of 16 points per thread with one-sided edges take the
    // wedge's update inside the column pass; the wedge row's spectrum is
    // formed first, ahead of the chained passes
    const bool wedge_fused = sizeof(T) == 4 && 2 * p.nu >= 16 && p.edges && p.wedge;
    if (wedge_fused && (err = launch_wedge_dft<T>(p, st)) != cudaSuccess) return err;
    {
        PassRange range_("sg forward rows");
        if (sizeof(T) == 4 && p.tcm) {
            if ((err = launch_dft_r2c(p, (const float*)sigma, st)) != cudaSuccess) return err;
        } else if (p.pairs) {
            const int nblk = p.nu / (4 * fr->slots);
            auto k = sigma_direct ? fr->fwd_rows_direct : fr->fwd_rows;
            if ((err = set_smem(k, fr->r2c_smem, true)) != cudaSuccess) return err;
            const int wave = resident_blocks(k, fr->threads, fr->r2c_smem, p.sms);
            if ((err = launch_pdl(k, nblk, fr->threads, fr->r2c_smem, st, (const float*)sigma, (const float*)nullptr,
                                  (const float*)p.wpre, (float2*)p.wa, p.nu, (const float2*)p.tw, p.err, wave)) !=
                cudaSuccess)
                return err;
        } else {
            Shape s = shape_for<V>(p.nphi, sizeof(T) == 8 ? 64 : 256);
            const int R = 2 * s.slots, nblk = (p.nu + R - 1) / R;
            const size_t smem = rows_fwd_smem_bytes<V>(p.nphi, s.slots);
            const CUtensorMap* mA = row_map(p, R, 0, p.nphi);
            SG_DISPATCH_E(s.E, {
                auto k = k_fwd_rows<T, EE, 256>;
                if constexpr (sizeof(T) == 4)  // FP64 blocks are at most 256 threads
                    if (s.threads > 256) k = k_fwd_rows<T, EE, 512>;
                if ((err = set_smem(k, smem, true)) != cudaSuccess) return err;
                if ((err = launch_pdl(k, persistent_grid(k, s.threads, smem, nblk, p.sms), s.threads, smem, st,
                                      sigma, (const T*)p.wpre, A, p.nu, p.nphi, ln, tw, p.err,
                                      mA ? *mA : CUtensorMap{}, mA != nullptr, sigma_direct ? 1 : 0)) != cudaSuccess)
                    return err;
            });
        }
    }
    if (ev && (err = cudaEventRecord(ev[1], st)) != cudaSuccess) return err;
    bool edges_done = false;  // the column pass applied the edge-slope update itself
    {
        PassRange range_("sg forward columns");
        const int L = 2 * p.nu, E = L >= 16 ? 16 : L;
        EdgeCoef<T> coef;
        for (int j = 0; j < 16; j++) coef.c[j] = p.edges ? (T)p.ecoef[j] : (T)0;
        const WedgeArgs<T> wdg{(const V*)p.wtmp, (const T*)p.wtab};
        SG_DISPATCH_E(E, {
            const bool fuse = sizeof(T) == 4 && EE == 16 && p.edges;
            const bool fusew = fuse && p.wedge;  // == wedge_fused
            auto k = k_fwd_cols<T, EE, 256>;
            if constexpr (sizeof(T) == 4)  // FP64 columns are at most 256 threads
                if (L / EE > 256) k = k_fwd_cols<T, EE, 512>;
            if constexpr (sizeof(T) == 4 && EE == 16) {
                if (fuse) k = L / EE > 256 ? k_fwd_cols<T, 16, 512, 0, true> : k_fwd_cols<T, 16, 256, 0, true>;
                if (fusew)
                    k = L / EE > 256 ? k_fwd_cols<T, 16, 512, 0, true, true> : k_fwd_cols<T, 16, 256, 0, true, true>;
                if (p.pairs)  // the fixed-length instance writes the (B, C) pairs into wb
                    k = fusew ? fc->fwd_cols_edge_wedge : fuse ? fc->fwd_cols_edge : fc->fwd_cols;
            }
            const size_t smem =
                cols_smem_bytes<T>(p.nu) + (fuse ? 2 * (size_t)sg_edge_stride(p.nu, sizeof(T)) * sizeof(T) : 0);
            if ((err = set_smem(k, smem, true)) != cudaSuccess) return err;
            if ((err = launch_pdl(k, p.nphi / 2, L / EE, smem, st, A, (const V*)p.kr, (const V*)p.kp, B, C, p.nu,
                                  p.nphi, lL, tw, p.err, (const T*)p.egr, (const T*)p.egp, (const T*)p.wpre,
                                  coef, wdg)) != cudaSuccess)
                return err;
            edges_done = fuse;
        });
    }
    if (p.edges && !edges_done && (err = launch_edges<T>(p, false, st)) != cudaSuccess) return err;
    if (p.wedge && !wedge_fused && (err = launch_wedge<T>(p, false, st)) != cudaSuccess) return err;
    if (ev && (err = cudaEventRecord(ev[2], st)) != cudaSuccess) return err;
    {
        PassRange range_("sg forward inverse rows");
        if (sizeof(T) == 4 && p.tcm) {
            if ((err = launch_dft_c2r(p, (float*)Fr, (float*)Fp, st)) != cudaSuccess) return err;
        } else if (p.pairs) {
            const int nblk = p.nu / (2 * fr->slots);
            auto k = fr->fwd_rows_inv;
            if ((err = set_smem(k, fr->c2r_smem, true)) != cudaSuccess) return err;
            if ((err = launch_pdl(k, nblk, fr->threads,
                                  fr->c2r_smem, st, p.imaps[0], (const float*)p.wpost, (float*)Fr, (float*)Fp, p.nu,
                                  (const float2*)p.tw, p.err)) != cudaSuccess)
                return err;
        } else {
            Shape s = shape_for<V>(p.nphi, sizeof(T) == 8 ? 64 : 256);
            const int R = 2 * s.slots, nblk = (p.nu + R - 1) / R;
            const size_t smem = rows_inv_smem_bytes<V>(p.nphi, s.slots);
            const CUtensorMap* mB = row_map(p, R, 1, p.nphi);
            const CUtensorMap* mC = row_map(p, R, 2, p.nphi);
            const bool um = mB && mC;
            SG_DISPATCH_E(s.E, {
                auto k = k_fwd_rows_inv<T, EE, 256>;
                if constexpr (sizeof(T) == 4)  // FP64 blocks are at most 256 threads
                    if (s.threads > 256) k = k_fwd_rows_inv<T, EE, 512>;
                if ((err = set_smem(k, smem, true)) != cudaSuccess) return err;
                if ((err = launch_pdl(k, persistent_grid(k, s.threads, smem, nblk, p.sms), s.threads, smem, st, B,
                                      C, (const T*)p.wpost, Fr, Fp, p.nu, p.nphi, ln, tw, p.err,
                                      um ? *mB : CUtensorMap{}, um ? *mC : CUtensorMap{}, um)) != cudaSuccess)
                    return err;
            });
        }
    }
    if (ev && (err = cudaEventRecord(ev[3], st)) != cudaSuccess) return err;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_backward(const PlanView& p0, const T* gr, const T* gp, T* gs, cudaStream_t st, cudaEvent_t* ev)
{
    typedef typename CX<T>::t V;
    const FixedPassKernels *fr, *fc;
    PlanView p = p0;
    p.pairs = fixed_path<T>(p0, fr, fc) ? 1 : 0;
    const V* tw = (const V*)p.tw;
    V* A = (V*)p.wa;
    V* B = (V*)p.wb;
    V* C = (V*)p.wc;
    const int ln = sg_ilog2(p.nphi), lL = sg_ilog2(2 * p.nu);
    cudaError_t err;
    bool edges_done = false;  // the column pass applied the transposed edge update itself
    if (ev && (err = cudaEventRecord(ev[0], st)) != cudaSuccess) return err;
    {
        PassRange range_("sg adjoint rows");
        if (sizeof(T) == 4 && p.tcm) {
            if ((err = launch_dft_r2c_adjoint(p, (const float*)gr, (const float*)gp, st)) != cudaSuccess) return err;
        } else if (p.pairs) {  // (A, C) pairs into wb
            const int nblk = p.nu / (2 * fr->slots);
            auto k = fr->bwd_rows;
            if ((err = set_smem(k, fr->r2c_smem, true)) != cudaSuccess) return err;
            const int wave = resident_blocks(k, fr->threads, fr->r2c_smem, p.sms);
            if ((err = launch_pdl(k, nblk, fr->threads, fr->r2c_smem, st, (const float*)gr, (const float*)gp,
                                  (const float*)p.wpost, (float2*)p.wb, p.nu, (const float2*)p.tw, p.err, wave)) !=
                cudaSuccess)
                return err;
        } else {
            Shape s = shape_for<V>(p.nphi, row_min_threads(sizeof(T)));
            const int R = s.slots, nblk = (p.nu + R - 1) / R;
            const size_t smem = row_smem_bytes<V>(p.nphi, s.slots);
            const CUtensorMap* mA = row_map(p, R, 0, p.nphi);
            const CUtensorMap* mC = row_map(p, R, 2, p.nphi);
            const bool um = mA && mC;
            SG_DISPATCH_E(s.E, {
                auto k = k_bwd_rows<T, EE>;
                if ((err = set_smem(k, smem, true)) != cudaSuccess) return err;
                if ((err = launch_pdl(k, persistent_grid(k, s.threads, smem, nblk, p.sms), s.threads, smem, st, gr,
                                      gp, (const T*)p.wpost, A, C, p.nu, p.nphi, ln, tw, p.err,
                                      um ? *mA : CUtensorMap{}, um ? *mC : CUtensorMap{}, um)) != cudaSuccess)
                    return err;
            });
        }
    }
    if (ev && (err = cudaEventRecord(ev[1], st)) != cudaSuccess) return err;
    {
        PassRange range_("sg adjoint columns");
        const int L = 2 * p.nu, E = L >= 16 ? 16 : L;
        EdgeCoef<T> coef;
        for (int j = 0; j < 16; j++) coef.c[j] = p.edges ? (T)p.ecoef[j] : (T)0;
        SG_DISPATCH_E(E, {
            // the transposed edge update inside the pass needs whole warps (L >= 512)
            const bool fuse = sizeof(T) == 4 && EE == 16 && p.edges && L >= 512;
            auto k = k_bwd_cols<T, EE, 256>;
            if constexpr (sizeof(T) == 4)  // FP64 columns are at most 256 threads
                if (L / EE > 256) k = k_bwd_cols<T, EE, 512>;
            if constexpr (sizeof(T) == 4 && EE == 16) {
                if (fuse) k = L / EE > 256 ? k_bwd_cols<T, 16, 512, 0, true> : k_bwd_cols<T, 16, 256, 0, true>;
                if (p.pairs) k = fuse ? fc->bwd_cols_edge : fc->bwd_cols;  // reads the (A, C) pairs of wb
            }
            const size_t smem = bcols_smem_bytes<T>(p.nu);  // the edge rows share the exchange area
            if ((err = set_smem(k, smem, true)) != cudaSuccess) return err;
            // the pair layout: the (A, C) pairs in wb, B into wa
            if ((err = launch_pdl(k, p.nphi / 2, L / EE, smem, st, p.pairs ? B : A, C, (const V*)p.kr,
                                  (const V*)p.kp, p.pairs ? A : B, p.nu, p.nphi, lL, tw, p.err, (const T*)p.egr,
                                  (const T*)p.egp, (const T*)p.wpre, coef)) != cudaSuccess)
                return err;
            edges_done = fuse;
        });
    }
    if (p.edges && !edges_done && (err = launch_edges<T>(p, true, st)) != cudaSuccess) return err;
    if (p.wedge && (err = launch_wedge<T>(p, true, st)) != cudaSuccess) return err;
    if (ev && (err = cudaEventRecord(ev[2], st)) != cudaSuccess) return err;
    {
        PassRange range_("sg adjoint inverse rows");
        if (sizeof(T) == 4 && p.tcm) {
            if ((err = launch_dft_c2r_adjoint(p, (float*)gs, st)) != cudaSuccess) return err;
        } else if (p.pairs) {  // B from wa
            const int nblk = p.nu / (4 * fr->slots);
            auto k = fr->bwd_rows_inv;
            if ((err = set_smem(k, fr->c2r_smem, true)) != cudaSuccess) return err;
            if ((err = launch_pdl(k, nblk, fr->threads,
                                  fr->c2r_smem, st, p.imaps[1], (const float*)p.wpre, (float*)gs, (float*)nullptr,
                                  p.nu, (const float2*)p.tw, p.err)) != cudaSuccess)
                return err;
        } else {
            Shape s = shape_for<V>(p.nphi, sizeof(T) == 8 ? 64 : 256);
            const int R = 2 * s.slots, nblk = (p.nu + R - 1) / R;
            const size_t smem = rows_bwd_inv_smem_bytes<V>(p.nphi, s.slots);
            const CUtensorMap* mB = row_map(p, R, 1, p.nphi);
            SG_DISPATCH_E(s.E, {
                auto k = k_bwd_rows_inv<T, EE, 256>;
                if constexpr (sizeof(T) == 4)
                    if (s.threads > 256) k = k_bwd_rows_inv<T, EE, 512>;
                if ((err = set_smem(k, smem, true)) != cudaSuccess) return err;
                if ((err = launch_pdl(k, persistent_grid(k, s.threads, smem, nblk, p.sms), s.threads, smem, st, B,
                                      (const T*)p.wpre, gs, p.nu, p.nphi, ln, tw, p.err, mB ? *mB : CUtensorMap{},
                                      mB != nullptr)) != cudaSuccess)
                    return err;
            });
        }
    }
    if (ev && (err = cudaEventRecord(ev[3], st)) != cudaSuccess) return err;
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

#ifndef SG_FFTCONV_DF  // fftconv_df.cu instantiates the compensated plans' passes
template cudaError_t launch_forward<float>(const PlanView&, const float*, float*, float*, cudaStream_t, cudaEvent_t*,
                                           bool);
template cudaError_t launch_forward<double>(const PlanView&, const double*, double*, double*, cudaStream_t,
                                              cudaEvent_t*, bool);
template cudaError_t launch_backward<float>(const PlanView&, const float*, const float*, float*, cudaStream_t,
                                            cudaEvent_t*);
template cudaError_t launch_backward<double>(const PlanView&, const double*, const double*, double*, cudaStream_t,
                                             cudaEvent_t*);
template cudaError_t launch_spectra<float2>(const PlanView&, const double*, const double*, double2*, float2*,
                                            float2*, cudaStream_t);
template cudaError_t launch_spectra<double2>(const PlanView&, const double*, const double*, double2*, double2*,
                                             double2*, cudaStream_t);
#endif
#endif  // SG_FFTCONV_KERNELS_ONLY

}  // namespace sg
