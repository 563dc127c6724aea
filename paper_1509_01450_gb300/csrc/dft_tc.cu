// dft_tc.cu -- the azimuthal transforms of the forward and adjoint passes
// as dense DFT-matrix products on the tensor cores (build option short_dft,
// FP32 plans with 32 <= N_phi <= 256).
//
// Sec. 2 writes the forces as convolutions that are periodic in phi; the
// row passes take each row's discrete Fourier transform in phi (P1) and,
// after the column pass, the inverse transform back (P3).  For short rows the
// transform is a product with the N_phi x N_phi real DFT matrix:
//
//   P1: y_i = x_i D,  x_i = sigma row i,
//       D[n][0] = 1, D[n][1] = (-1)^n, D[n][2m] = cos(2 pi n m / N),
//       D[n][2m+1] = -sin(2 pi n m / N)  (0 < m < N/2),
//       so that (y_i[2m], y_i[2m+1]) = X_i(m) and (y_i[0], y_i[1]) = (X_i(0),
//       X_i(N/2)): the half spectrum with mode 0 holding (DC, Nyquist), times
//       the row weight w_i, goes to A[m nu + i].
//   P3: F_r,i = b_i E wpost_i, F_phi,i = c_i E wpost_i, with b_i[2m], b_i[2m+1]
//       = Re, Im B_i(m) (mode 0: DC, Nyquist) and c_i from C likewise,
//       E[0][k] = 1, E[1][k] = (-1)^k, E[2m][k] = 2 cos(2 pi m k / N),
//       E[2m+1][k] = -2 sin(2 pi m k / N): the real inverse transform of the
//       Hermitian spectrum whose half is B (or C).
//   The adjoint's row passes are the same two products: P1b takes gF_r and
//   gF_phi through D (times wpost) to the half spectra A and C, P3b the
//   column pass's B through E (times wpre) to gsigma.
//
// The products run as tcgen05 MMAs of kind::tf32 (M = 128 rows per CTA, N =
// NT output columns per CTA, K = 8 per instruction) accumulating in FP32 in
// tensor memory.  Every operand is split in two TF32 parts, v = hi + lo with
// hi = v rounded to TF32 and lo = v - hi (exact in FP32); the product takes
// the three terms hi hi + hi lo + lo hi, which leaves an error of about
// 2^-21 of each operand, so the transform keeps FP32 accuracy.  The matrices
// are built in FP64 on the host and split there; the rows are split by the
// threads as they stage them.
//
// Shared-memory operands are K-major without swizzling: core matrices of 8
// rows x 4 values (128 contiguous bytes), the KC = 32 values of one K chunk
// as 8 core matrices side by side (128 bytes apart), the 8-row groups 1024
// bytes apart.  A CTA keeps its column tile of the matrix resident (bulk
// copies two chunks ahead of the MMAs) and streams the rows through a ring
// of row buffers: eight warps stage chunk after chunk and arrive on the
// buffer's "full" mbarrier, one thread of a ninth warp issues the chunk's
// MMAs and commits them to its "empty" mbarrier, and a buffer is refilled
// only after that commit (every wait bounded).
#include "sg_internal.cuh"
#include "sg_tc.cuh"

#include <math.h>
#include <string.h>

namespace sg {

namespace {

constexpr int TC_M = 128;   // rows per CTA (tensor-memory lanes)
constexpr int TC_STAGE = 256;  // staging threads: two per row, each staging half of a chunk
constexpr int TC_T = TC_STAGE + 32;  // and one more warp, whose first lane issues the MMAs
constexpr int TC_KC = 32;   // K values per staged chunk
constexpr int TC_ABYTES = TC_M * TC_KC * 4;  // one A operand part of one chunk: 16 KB
// Accumulators.  The tensor core's FP32 accumulation loses up to about one
// unit in the last place of the running sum per MMA step, and MMAs into the
// same accumulator wait for one another.  So each product keeps TC_ACC(G)
// main accumulators and as many for the two correction terms (2^-11 of the
// main ones), the K step s of every chunk going to accumulator s mod
// TC_ACC: consecutive MMAs then write different accumulators, each main
// accumulator takes N / (8 TC_ACC) steps, and the epilogue adds them all with
// rounding to nearest.  2 TC_ACC G NT = 512 columns for NT = 64.
__host__ __device__ constexpr int tc_acc(int G) { return G == 1 ? 4 : 2; }
constexpr int TC_MAX_CHUNKS = 8;  // N <= 256

__host__ __device__ constexpr uint32_t tc_pow2(int n)
{
    return n <= 32 ? 32u : n <= 64 ? 64u : n <= 128 ? 128u : n <= 256 ? 256u : 512u;
}

// Offset (in values) of (row r, k) in a K-major core-matrix tile whose rows
// hold TC_KC values: core matrix (r / 8, k / 4) at 32 (8 (r / 8) + k / 4).
__host__ __device__ inline int tc_off(int r, int k) { return ((r >> 3) * (TC_KC / 4) + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3); }

template <int NT>
__host__ __device__ constexpr int tc_mbytes()
{
    return NT * TC_KC * 4;  // one matrix part of one chunk
}

// bytes of one row staging buffer: G row operands, hi and lo parts each
// (NB of them in a ring)
template <int G>
__host__ __device__ constexpr int tc_rowbuf_bytes()
{
    return 2 * G * TC_ABYTES;
}

// the CTA's shared memory: its column tile of the matrix (all N / KC chunks,
// hi and lo), NB row staging buffers, alignment slack
template <int NT, int G, int NB>
size_t tc_smem_bytes(int N)
{
    return (size_t)(N / TC_KC) * 2 * tc_mbytes<NT>() + NB * (size_t)tc_rowbuf_bytes<G>() + 1024;
}

__device__ __forceinline__ float4 tc_hi(float4 v)
{
    return make_float4(__uint_as_float(sg_tf32_bits(__float_as_uint(v.x))),
                       __uint_as_float(sg_tf32_bits(__float_as_uint(v.y))),
                       __uint_as_float(sg_tf32_bits(__float_as_uint(v.z))),
                       __uint_as_float(sg_tf32_bits(__float_as_uint(v.w))));
}
__device__ __forceinline__ float4 tc_sub(float4 a, float4 b)
{
    return make_float4(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y), __fsub_rn(a.z, b.z), __fsub_rn(a.w, b.w));
}

// Stage four values (k .. k + 3 of row r) of one row operand: the TF32 part
// into hi, the remainder into lo.
__device__ __forceinline__ void tc_stage4(float* hi, float* lo, int r, int k, float4 v)
{
    const float4 h = tc_hi(v);
    *reinterpret_cast<float4*>(hi + tc_off(r, k)) = h;
    *reinterpret_cast<float4*>(lo + tc_off(r, k)) = tc_sub(v, h);
}

}  // namespace

// The transform kernel: G products of 128-row tiles with one matrix.
//   DIR 0 (P1, P1b): rows -> half spectra.  Forward G = 1: sigma -> A.
//     Adjoint G = 2: gF_r, gF_phi -> A, C (PAIRS: {A, C} pairs).
//   DIR 1 (P3, P3b): half spectra -> rows.  Forward G = 2: B, C (PAIRS: the
//     {B, C} pairs) -> F_r, F_phi.  Adjoint G = 1: B -> gsigma.
// Outputs are scaled by the row weight w_i.  One CTA per tile: rows
// row_tile 128 .. + 127, output columns col_tile NT .. + NT - 1; 288 threads,
// threads r and r + 128 staging the two halves of each chunk of row
// row_tile 128 + r, whose results sit in tensor-memory lane r, and thread 256
// issuing the MMAs.
template <int NT, int DIR, int G, bool PAIRS, int NB>
__device__ __forceinline__ void dft_tc_tile(const TcArgs& a, int row_tile, int col_tile)
{
    constexpr int RB = tc_rowbuf_bytes<G>();
    constexpr int MB = tc_mbytes<NT>();
    // accumulators: column (j G + g) NT for the main sum j of product g,
    // (ACC + j) G + g for its correction sum j (j < ACC)
    constexpr int ACC = tc_acc(G);
    constexpr uint32_t NCOLS = tc_pow2(2 * ACC * G * NT);
    const int nu = a.nu, N = a.N;
    int* const err = a.err;
    const unsigned long long wlim = sg_wait_budget(err);
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ __align__(8) uint64_t empty[NB];            // per row buffer: its chunk's MMAs have completed
    __shared__ __align__(8) uint64_t full[NB];             // per row buffer: its chunk is staged
    __shared__ __align__(8) uint64_t lbar[TC_MAX_CHUNKS];  // per chunk: its matrix parts have landed
    __shared__ uint32_t tbase_s;
    unsigned char* const area = reinterpret_cast<unsigned char*>(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    const int r = threadIdx.x & (TC_M - 1), h = threadIdx.x / TC_M, warp = threadIdx.x >> 5;
    const int i = row_tile * TC_M + r;
    const bool row_ok = i < nu;
    const int ct = col_tile, nch = N / TC_KC;
    constexpr int QH = TC_KC / 8;  // float4s of one row's half chunk
    // the matrix's stored tiles are LNT = min(N, 64) columns wide; a CTA of
    // NT = 32 columns takes half of one, which is contiguous
    const int LNT = N < 64 ? N : 64;
    const size_t mat_part = (size_t)N * N;
    unsigned char* const rows_area = area + (size_t)nch * 2 * MB;
    if (warp == 0) {
        sg_tc_alloc(&tbase_s, NCOLS);
        sg_tc_relinquish();
    }
    if (threadIdx.x == 0) {
        for (int b = 0; b < NB; b++) {
            sg_mbar_init(&empty[b], 1);
            sg_mbar_init(&full[b], TC_STAGE);
        }
        for (int c = 0; c < nch; c++) sg_mbar_init(&lbar[c], 1);
    }
    sg_tc_fence_before();
    __syncthreads();
    sg_tc_fence_after();
    const uint32_t tbase = tbase_s;
    const uint32_t idesc = sg_tc_idesc_tf32(TC_M, NT);
    const float wi = row_ok ? __ldg(&a.w[i]) : 0.f;
    // the CTA's column tile of the matrix stays resident: chunk c's two parts
    // (hi, lo) arrive by two bulk copies on lbar[c].  The MMA thread copies
    // two chunks ahead of its MMAs, so that the first chunks' copies do not
    // queue behind the whole tile's
    const uint64_t keep = sg_policy_evict_last();  // every CTA of the column tile reads it
    auto copy_matrix = [&](int c) {
        const size_t tile0 = (size_t)(ct * NT / LNT), sub = (size_t)(ct * NT % LNT) * TC_KC;
        float* const dh = reinterpret_cast<float*>(area + (size_t)c * 2 * MB);
        const float* const gh = a.mat + (tile0 * nch + c) * ((size_t)LNT * TC_KC) + sub;
        SG_IF_OK(tile0 * nch + c < (size_t)(N / LNT) * nch, err, 403) {
            sg_mbar_expect_tx(&lbar[c], 2 * MB);
            sg_bulk_g2s_hint(dh, gh, MB, &lbar[c], keep);
            sg_bulk_g2s_hint(dh + MB / 4, gh + mat_part, MB, &lbar[c], keep);
        }
    };
    // this thread's half of chunk c of row i: v[g QH + q] = values
    // KC h / 2 + 4 q .. + 3 of product g
    auto load_rows = [&](int c, float4 (&v)[G * QH]) {
        if constexpr (DIR == 0) {
#pragma unroll
            for (int g = 0; g < G; g++) {
                const float4* src = reinterpret_cast<const float4*>(a.x[g] + (size_t)(row_ok ? i : 0) * N +
                                                                    c * TC_KC + h * (TC_KC / 2));
#pragma unroll
                for (int q = 0; q < QH; q++)
                    v[g * QH + q] = row_ok ? __ldg(src + q) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        } else {
            // modes c KC / 2 + h KC / 4 .. + KC / 4 - 1 of row i, two per float4
            const int m0 = c * (TC_KC / 2) + h * (TC_KC / 4);
#pragma unroll
            for (int q = 0; q < QH; q++) {
#pragma unroll
                for (int g = 0; g < G; g++) v[g * QH + q] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (row_ok) {
                    const size_t e0 = (size_t)(m0 + 2 * q) * nu + i, e1 = e0 + nu;
                    if constexpr (PAIRS && G == 2) {
                        const float4 p0 = __ldg(a.pin + e0), p1 = __ldg(a.pin + e1);
                        v[q] = make_float4(p0.x, p0.y, p1.x, p1.y);
                        v[QH + q] = make_float4(p0.z, p0.w, p1.z, p1.w);
                    } else {
#pragma unroll
                        for (int g = 0; g < G; g++) {
                            const float2 b0 = __ldg(a.in[g] + e0), b1 = __ldg(a.in[g] + e1);
                            v[g * QH + q] = make_float4(b0.x, b0.y, b1.x, b1.y);
                        }
                    }
                }
            }
        }
    };
    // Warp-specialised pipeline: warps 0-7 stage chunk c into row buffer
    // c mod NB (after the MMAs of chunk c - NB freed it: "empty") and arrive
    // on "full"; the last warp's first lane waits for a full buffer and the
    // chunk's matrix, issues its MMAs and commits them to "empty".  No
    // block-wide barrier per chunk; every wait is bounded, and a wait that
    // gave up stops its side, which the other side then sees as a wait that
    // gives up in turn.
    bool fail = false;
    if (threadIdx.x < TC_STAGE) {
        auto stage = [&](int c, float4 (&cur)[G * QH], float4 (&nxt)[G * QH]) -> bool {
            float* const ahi = reinterpret_cast<float*>(rows_area + (size_t)(c % NB) * RB);  // [g][hi, lo]
            if (c + 2 < nch) load_rows(c + 2, nxt);  // chunk c + 1's rows are in flight already
            if (c >= NB && !sg_mbar_wait_bounded(&empty[c % NB], ((c / NB) - 1) & 1, err, 1, wlim)) return false;
#pragma unroll
            for (int g = 0; g < G; g++) {
                float* hi = ahi + (size_t)g * 2 * (TC_ABYTES / 4);
                float* lo = hi + TC_ABYTES / 4;
#pragma unroll
                for (int q = 0; q < QH; q++) tc_stage4(hi, lo, r, h * (TC_KC / 2) + 4 * q, cur[g * QH + q]);
            }
            sg_fence_proxy_async_smem();  // the stores above, for the tensor core's reads
            sg_mbar_arrive(&full[c % NB]);
            return true;
        };
        // three register sets in turn: the rows arrive two chunks after
        // their loads are issued, and no prefetched value is moved
        float4 va[G * QH], vb[G * QH], vc[G * QH];
        load_rows(0, va);
        if (nch > 1) load_rows(1, vb);
        for (int c = 0; c < nch && !fail; c += 3) {
            fail = !stage(c, va, vc);
            if (!fail && c + 1 < nch) fail = !stage(c + 1, vb, va);
            if (!fail && c + 2 < nch) fail = !stage(c + 2, vc, vb);
        }
        // the last chunk's completion covers every MMA issued before it
        const int c = nch - 1;
        if (!fail) fail = !sg_mbar_wait_bounded(&empty[c % NB], (c / NB) & 1, err, 1, wlim);
    } else if (threadIdx.x == TC_STAGE) {
        int issued = 0;   // chunks whose MMAs have been committed
        int landed = -1;  // the last chunk whose matrix copy was waited for
        int copied = nch < 2 ? nch - 1 : 1;  // the last chunk whose matrix copy was issued
        for (int c = 0; c <= copied; c++) copy_matrix(c);
        for (int c = 0; c < nch; c++) {
            if (!sg_mbar_wait_bounded(&full[c % NB], (c / NB) & 1, err, 1, wlim)) {
                fail = true;
                break;
            }
            const bool in_time = sg_mbar_wait_bounded(&lbar[c], 0, err, 1, wlim);
            landed = c;
            if (!in_time) {
                fail = true;
                break;
            }
            sg_tc_fence_after();
            float* const ahi = reinterpret_cast<float*>(rows_area + (size_t)(c % NB) * RB);
            // descriptors of the chunk's first K step; a step of 8 values
            // (256 bytes) adds 16 to the start-address field
            const uint64_t bh0 = sg_tc_smem_desc(sg_smem_u32(area + (size_t)c * 2 * MB), 128, 1024);
            const uint64_t bl0 = bh0 + (MB >> 4);
            const uint64_t ah0 = sg_tc_smem_desc(sg_smem_u32(ahi), 128, 1024);
            // three rounds over the chunk's K steps (K = 8 values, two core
            // matrices, per MMA) and products: the main terms, then each
            // correction term; K step s writes accumulator s mod ACC, so an
            // MMA's predecessor on the same accumulator is ACC G or more issues back
#pragma unroll
            for (int round = 0; round < 3; round++)
#pragma unroll
                for (int s = 0; s < TC_KC / 8; s++)
#pragma unroll
                    for (int g = 0; g < G; g++) {
                        const uint64_t ah = ah0 + (uint64_t)((g * 2 * TC_ABYTES) >> 4) + 16 * s;
                        const int j = s % ACC;
                        const uint32_t first = (c == 0 && s < ACC) ? 0u : 1u;  // 0: the accumulator's first write
                        if (round == 0)
                            sg_tc_mma_tf32(tbase + (uint32_t)((j * G + g) * NT), ah, bh0 + 16 * s, idesc, first);
                        else if (round == 1)
                            sg_tc_mma_tf32(tbase + (uint32_t)(((ACC + j) * G + g) * NT), ah, bl0 + 16 * s, idesc, first);
                        else
                            sg_tc_mma_tf32(tbase + (uint32_t)(((ACC + j) * G + g) * NT), ah + (TC_ABYTES >> 4),
                                           bh0 + 16 * s, idesc, 1u);
                    }
            sg_tc_commit(&empty[c % NB]);
            issued = c + 1;
            if (c + 2 < nch) copy_matrix(copied = c + 2);
        }
        // matrix copies still in flight after a wait that gave up land, and
        // the MMAs issued complete, before the shared and tensor memory are
        // given back
        for (int c = landed + 1; c <= copied; c++) sg_mbar_wait_bounded(&lbar[c], 0, err, 1, wlim);
        if (fail && issued > 0) {
            const int c = issued - 1;
            sg_mbar_wait_bounded(&empty[c % NB], (c / NB) & 1, err, 1, wlim);
        }
    }
    bool ok = !__syncthreads_or(fail);
    if (ok && threadIdx.x < TC_STAGE) {
        sg_tc_fence_after();
        // warps w and w + 4 read the same 32 lanes (rows): the two halves of
        // the CTA take alternate blocks of 32 columns
        const uint32_t lane_base = tbase + ((uint32_t)((warp & 3) * 32) << 16);
#pragma unroll
        for (int cb = h; cb < NT / 32; cb += 2) {
            // each product's sum of accumulators, in FP32 with rounding to
            // nearest: the correction sums first, then the main ones
            float y[G][32];
#pragma unroll
            for (int g = 0; g < G; g++) {
                float t[32];
                sg_tc_ld32(lane_base + (uint32_t)((ACC * G + g) * NT + cb * 32), y[g]);
                sg_tc_wait_ld();
                for (int k = 1; k < 2 * ACC; k++) {
                    const int j = k < ACC ? ACC + k : k - ACC;  // corrections 1 .. ACC-1, then main 0 .. ACC-1
                    sg_tc_ld32(lane_base + (uint32_t)((j * G + g) * NT + cb * 32), t);
                    sg_tc_wait_ld();
#pragma unroll
                    for (int q = 0; q < 32; q++) y[g][q] = __fadd_rn(y[g][q], t[q]);
                }
#pragma unroll
                for (int q = 0; q < 32; q++) y[g][q] = __fmul_rn(y[g][q], wi);
            }
            const int j0 = ct * NT + cb * 32;  // first output column
            if constexpr (DIR == 0) {  // columns j0 .. j0 + 31: modes j0 / 2 .. j0 / 2 + 15
                SG_IF_OK(!row_ok || (j0 / 2 + 16 <= N / 2), err, 401)
                if (row_ok) {
#pragma unroll
                    for (int q = 0; q < 16; q++) {
                        const size_t e = (size_t)(j0 / 2 + q) * nu + i;
                        if constexpr (PAIRS && G == 2)
                            a.pout[e] = make_float4(y[0][2 * q], y[0][2 * q + 1], y[G - 1][2 * q], y[G - 1][2 * q + 1]);
                        else
#pragma unroll
                            for (int g = 0; g < G; g++) a.out[g][e] = make_float2(y[g][2 * q], y[g][2 * q + 1]);
                    }
                }
            } else {
                SG_IF_OK(!row_ok || j0 + 32 <= N, err, 402)
                if (row_ok) {
#pragma unroll
                    for (int g = 0; g < G; g++) {
                        float4* o = reinterpret_cast<float4*>(a.y[g] + (size_t)i * N + j0);
#pragma unroll
                        for (int q = 0; q < 8; q++)
                            o[q] = make_float4(y[g][4 * q], y[g][4 * q + 1], y[g][4 * q + 2], y[g][4 * q + 3]);
                    }
                }
            }
        }
    }
    sg_tc_fence_before();
    __syncthreads();  // every tensor-memory read is done (or none happens)
    if (warp == 0) sg_tc_dealloc(tbase, NCOLS);
}

// One plan: grid (ceil(nu / 128), N / NT).
template <int NT, int DIR, int G, bool PAIRS, int NB>
__global__ void __launch_bounds__(TC_T, 1) k_dft_tc(const TcArgs a)
{
    dft_tc_tile<NT, DIR, G, PAIRS, NB>(a, blockIdx.x, blockIdx.y);
}

// The disks of a batch: grid (row tiles of the largest disk, column tiles of
// the longest rows, disks); a CTA beyond its disk's rows or columns leaves
// before it takes any tensor memory.
template <int NT, int DIR, int G, bool PAIRS, int NB>
__global__ void __launch_bounds__(TC_T, 1) k_dft_tc_batch(const TcArgs* __restrict__ args)
{
    const TcArgs a = args[blockIdx.z];
    if ((int)blockIdx.x * TC_M >= a.nu || (int)blockIdx.y * NT >= a.N) return;
    dft_tc_tile<NT, DIR, G, PAIRS, NB>(a, blockIdx.x, blockIdx.y);
}

// ---- host side ----------------------------------------------------------------

static int tc_nt(int N) { return N < 64 ? N : 64; }

bool dft_tc_supported(int nphi) { return nphi >= 32 && nphi <= 256 && (nphi & (nphi - 1)) == 0; }

size_t dft_tc_matrix_floats(int nphi) { return (size_t)4 * nphi * nphi; }

static float tf32_round(float v)
{
    uint32_t u;
    memcpy(&u, &v, 4);
    u = sg_tf32_bits(u);
    float h;
    memcpy(&h, &u, 4);
    return h;
}

// Both matrices (P1's D, P3's E) for rows of N values, each as [part][column
// tile][K chunk][NT x KC core-matrix tile] with the operand's row index the
// output column and K the input index: out[0 .. 2 N^2) holds D, out[2 N^2 ..
// 4 N^2) holds E.  Entries are formed in FP64 (the angle reduced exactly:
// 2 pi (n m mod N) / N) and split into the TF32 part and the FP32 remainder.
void dft_tc_matrices(int N, float* out)
{
    const int NT = tc_nt(N), nch = N / TC_KC;
    const size_t part = (size_t)N * N;
    for (int dir = 0; dir < 2; dir++) {
        float* hi = out + (size_t)dir * 2 * part;
        float* lo = hi + part;
        for (int j = 0; j < N; j++)       // output column: the operand's row
            for (int k = 0; k < N; k++) {  // input index: K
                // P1: D[k][j]; P3: E[k][j] (k the packed spectrum index, j the point)
                const int n = dir == 0 ? k : j;    // point index
                const int q = dir == 0 ? j : k;    // packed spectrum index
                const int m = q >> 1;
                double val;
                if (q == 0)
                    val = 1.0;
                else if (q == 1)
                    val = (n & 1) ? -1.0 : 1.0;
                else {
                    const double a = 6.283185307179586476925286766559 * (double)(((long long)n * m) % N) / (double)N;
                    val = (q & 1) ? -sin(a) : cos(a);
                    if (dir == 1) val *= 2.0;
                }
                const float h = tf32_round((float)val);
                const float l = (float)(val - (double)h);
                const int t = j / NT, jj = j % NT, c = k / TC_KC, kk = k % TC_KC;
                const size_t at = ((size_t)t * nch + c) * ((size_t)NT * TC_KC) + tc_off(jj, kk);
                hi[at] = h;
                lo[at] = l;
            }
    }
}

template <int NT, int DIR, int G, bool PAIRS, int NB>
static cudaError_t tc_launch(const TcArgs& a, cudaStream_t st)
{
    auto k = k_dft_tc<NT, DIR, G, PAIRS, NB>;
    const size_t smem = tc_smem_bytes<NT, G, NB>(a.N);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((a.nu + TC_M - 1) / TC_M, a.N / NT);
    k<<<grid, TC_T, smem, st>>>(a);
    return cudaGetLastError();
}

// columns per CTA: 64 (32 for rows of 32); row buffers: three for one
// product, two for two, and one for two products of rows of 256, whose
// 128 KB matrix tile leaves room for one only
template <int DIR, int G, bool PAIRS>
static cudaError_t tc_launch_nt(const TcArgs& a, cudaStream_t st)
{
    constexpr int NB = G == 1 ? 3 : 2;
    if (a.N < 64) return tc_launch<32, DIR, G, PAIRS, NB>(a, st);
    if (G == 2 && a.N > 128) return tc_launch<64, DIR, G, PAIRS, 1>(a, st);
    return tc_launch<64, DIR, G, PAIRS, NB>(a, st);
}

static TcArgs tc_args(const PlanView& p, int dir, const float* w)
{
    TcArgs a{};
    a.mat = (const float*)p.tcm + (size_t)dir * 2 * p.nphi * p.nphi;
    a.w = w;
    a.nu = p.nu;
    a.N = p.nphi;
    a.err = p.err;
    return a;
}

// The batched form's row passes of its short_dft disks (rows of 256): one
// launch for all of them; dir 0: P1 (args as launch_dft_r2c's), dir 1: P3
// with the {B, C} pairs.  d_args: n argument sets in device memory.
cudaError_t launch_dft_tc_batch(const TcArgs* d_args, int n, int dir, int max_nu, cudaStream_t st)
{
    constexpr int N = 256;
    const dim3 grid((max_nu + TC_M - 1) / TC_M, N / 64, n);
    cudaError_t e;
    if (dir == 0) {
        auto k = k_dft_tc_batch<64, 0, 1, false, 3>;
        const size_t smem = tc_smem_bytes<64, 1, 3>(N);
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        k<<<grid, TC_T, smem, st>>>(d_args);
    } else {
        auto k = k_dft_tc_batch<64, 1, 2, true, 1>;
        const size_t smem = tc_smem_bytes<64, 2, 1>(N);
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        k<<<grid, TC_T, smem, st>>>(d_args);
    }
    return cudaGetLastError();
}

// P1 on the tensor cores: sigma rows -> A (wa), weighted by wpre.
cudaError_t launch_dft_r2c(const PlanView& p, const float* sigma, cudaStream_t st)
{
    TcArgs a = tc_args(p, 0, (const float*)p.wpre);
    a.x[0] = sigma;
    a.out[0] = (float2*)p.wa;
    return tc_launch_nt<0, 1, false>(a, st);
}

// P3 on the tensor cores: the column pass's B and C (pairs: the {B, C} pairs
// at wb; otherwise B at wb, C at wc) -> F_r, F_phi, weighted by wpost.
cudaError_t launch_dft_c2r(const PlanView& p, float* Fr, float* Fp, cudaStream_t st)
{
    TcArgs a = tc_args(p, 1, (const float*)p.wpost);
    a.pin = (const float4*)p.wb;
    a.in[0] = (const float2*)p.wb;
    a.in[1] = (const float2*)p.wc;
    a.y[0] = Fr;
    a.y[1] = Fp;
    return p.pairs ? tc_launch_nt<1, 2, true>(a, st) : tc_launch_nt<1, 2, false>(a, st);
}

// P1b on the tensor cores: gF_r, gF_phi rows -> A, C weighted by wpost
// (pairs: the {A, C} pairs into wb; otherwise A into wa, C into wc).
cudaError_t launch_dft_r2c_adjoint(const PlanView& p, const float* gr, const float* gp, cudaStream_t st)
{
    TcArgs a = tc_args(p, 0, (const float*)p.wpost);
    a.x[0] = gr;
    a.x[1] = gp;
    a.pout = (float4*)p.wb;
    a.out[0] = (float2*)p.wa;
    a.out[1] = (float2*)p.wc;
    return p.pairs ? tc_launch_nt<0, 2, true>(a, st) : tc_launch_nt<0, 2, false>(a, st);
}

// P3b on the tensor cores: B (pairs: at wa; otherwise at wb) -> gsigma,
// weighted by wpre.
cudaError_t launch_dft_c2r_adjoint(const PlanView& p, float* gs, cudaStream_t st)
{
    TcArgs a = tc_args(p, 1, (const float*)p.wpre);
    a.in[0] = (const float2*)(p.pairs ? p.wa : p.wb);
    a.y[0] = gs;
    return tc_launch_nt<1, 1, false>(a, st);
}

}  // namespace sg
