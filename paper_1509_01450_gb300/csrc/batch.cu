// batch.cu -- the batched forward pass (sg_forces_batched) as one
// persistent launch per pass kind.  Every disk's three passes are cut into
// work items -- row units of the R2C pass, groups of modes of the column
// pass, row units of the C2R pass -- and three kernels, each resident on
// every SM, take the items of their pass for all disks from a queue in
// device memory (an atomic head over a list prepared on the host), largest
// disks first.  The launches follow one another on the stream, which orders
// the passes.  The items run the same unit functions as the single-plan
// pass kernels, so every disk's forces are bit-equal to a single call's,
// and their waits for their input copies are bounded like the passes'
// (a wait that runs out sets the disk's plan flag).
//
// Eligible batches: FP32 plans on the fixed-length path (both transform
// lengths 2^8 .. 2^12, one row block per 256 threads), without the edge or
// wedge updates; others take the per-plan path of api.cu.
#define SG_FFTCONV_KERNELS_ONLY
#include "fftconv.cu"

#include <algorithm>
#include <atomic>
#include <deque>
#include <mutex>
#include <string>
#include <vector>

namespace sg {

// One disk, as the kernel sees it (aligned as its tensor map requires).
struct BatchDisk {
    CUtensorMap map;  // the plan's map over the pair layout (the C2R pass's input)
    const float* sigma;
    float* Fr;
    float* Fp;
    const float* wpre;
    const float* wpost;
    float2* A;  // the R2C pass's half spectra (single layout)
    float2* P;  // the column pass's (B, C) pairs
    const float2* Kr;
    const float2* Kp;
    const float2* tw;
    int* err;
    int nu, nphi, lgr, lgc;  // sizes; log2 N_phi and log2 2 N_u
    int n_rows, n_cols, n_inv;  // items of the R2C, column and C2R passes
    int rows_mult, cols_mult;   // units per row item (both row passes), mode groups per column item (tuned)
};

enum { KIND_ROWS = 0, KIND_COLS = 1, KIND_INV = 2 };

#define SG_BATCH_THREADS 256

// bytes of one mode's column area in the batched column items (128-aligned)
__host__ __device__ inline size_t batch_col_bytes(int nu) { return (cols_smem_bytes<float>(nu) + 127) & ~(size_t)127; }
// modes per column group: 256 threads / (2 N_u / 16) per mode
__host__ __device__ inline int batch_col_slots(int lgc) { return 1 << (12 - lgc); }

template <int LG>
__device__ __forceinline__ bool batch_rows(const BatchDisk& D, int u, unsigned char* smraw, uint64_t& bar,
                                           uint32_t& ph, unsigned long long wlim)
{
    bool landed = true;
    rows_r2c_unit<LG, false, false, false>(D.sigma, nullptr, D.wpre, D.A, D.nu, D.tw, D.err, u, 0, smraw, bar, ph, wlim,
                                           &landed);
    landed = __syncthreads_or(landed);  // the phase completed if any thread saw it complete
    if (landed) ph ^= 1;
    return landed;
}

template <int LG>
__device__ __forceinline__ bool batch_inv(const BatchDisk& D, int u, unsigned char* smraw, uint64_t& bar,
                                          uint32_t& ph, unsigned long long wlim)
{
    bool landed = true;
    rows_c2r_unit<LG, false, false>(&D.map, D.wpost, D.Fr, D.Fp, D.nu, D.tw, D.err, u, smraw, bar, ph, wlim, &landed);
    landed = __syncthreads_or(landed);
    if (landed) ph ^= 1;
    return landed;
}

// Modes g S .. g S + S - 1 of the column pass, S = batch_col_slots(LGC), one
// per N_T = 2 N_u / 16 threads, each on its own part of shared memory.
// Returns false if a barrier's copies never landed.
template <int LGC>
__device__ __forceinline__ bool batch_cols(const BatchDisk& D, int g, unsigned char* smraw, uint64_t* bar,
                                           uint32_t& ph0, uint32_t& ph1, unsigned long long wlim)
{
    constexpr int L = 1 << LGC, nu = L / 2, NT = L / 16, S = 1 << (12 - LGC), KS = nu + 2;
    const int slot = threadIdx.x / NT, t = threadIdx.x % NT;
    const int half = D.nphi / 2;
    const int m = g * S + slot;
    const size_t CB = batch_col_bytes(nu);
    unsigned char* const base = smraw + (size_t)slot * CB;
    float2* const sm = reinterpret_cast<float2*>(base);
    float2* const kr_s = reinterpret_cast<float2*>(base + sg_align16(sg_padded(L) * sizeof(float2)));
    float2* const kp_s = kr_s + KS;
    const uint32_t ab = (uint32_t)(nu * sizeof(float2)), kb = (uint32_t)(KS * sizeof(float2));
    if (threadIdx.x == 0) {
        const uint64_t drop = sg_policy_evict_first();
        sg_mbar_expect_tx(&bar[1], S * 2 * kb);
        sg_mbar_expect_tx(&bar[0], S * ab);
        for (int s = 0; s < S; s++) {
            const int ms = g * S + s;
            unsigned char* const cs = smraw + (size_t)s * CB;
            float2* const ks = reinterpret_cast<float2*>(cs + sg_align16(sg_padded(L) * sizeof(float2)));
            SG_IF_OK(ms < half && sg_smem_in(smraw, ks, 2 * kb), D.err, 801) {
                sg_bulk_g2s_hint(ks, D.Kr + (size_t)ms * KS, kb, &bar[1], drop);
                // mode 0 holds (DC, Nyquist): the Nyquist mode's Khat_r instead of Khat_phi
                sg_bulk_g2s_hint(ks + KS, (ms == 0 ? D.Kr + (size_t)half * KS : D.Kp + (size_t)ms * KS), kb, &bar[1],
                                 drop);
            }
            SG_IF_OK(sg_in((long long)ms * nu, nu, (long long)half * nu) && sg_smem_in(smraw, cs, ab), D.err, 802)
            sg_bulk_g2s_hint(cs, D.A + (size_t)ms * nu, ab, &bar[0], drop);
        }
    }
    const Twd<16, float2> twd = make_twd<16>(LGC, t, D.tw);
    bool landed0 = true, landed1 = true, spectra = false;
    const bool got = !__syncthreads_or(!sg_mbar_wait_bounded(&bar[0], ph0, D.err, 1, wlim, &landed0));
    landed0 = __syncthreads_or(landed0);
    if (landed0) ph0 ^= 1;
    if (got) {
        float2 v[16];
#pragma unroll
        for (int e = 0; e < 16; e++) v[e] = (e < 8) ? sm[t + e * NT] : float2{0.f, 0.f};  // rows >= nu: zero pad
        C2 w[16];
        const auto wait_spectra = [&] {
            spectra = true;
            const bool ok = !__syncthreads_or(!sg_mbar_wait_bounded(&bar[1], ph1, D.err, 1, wlim, &landed1));
            landed1 = __syncthreads_or(landed1);
            if (landed1) ph1 ^= 1;
            return ok;
        };
        if (fwd_cols_math<LGC, true>(v, sm, kr_s, kp_s, reinterpret_cast<C2*>(base), m, t, nu, LGC, twd, wait_spectra,
                                     w)) {
            const uint64_t keep = sg_policy_evict_last();  // the C2R pass reads the pairs from L2
            float4* const P = reinterpret_cast<float4*>(D.P) + (size_t)m * nu;
#pragma unroll
            for (int e = 0; e < 8; e++)  // crop to N_u rows
                SG_IF_OK(sg_in((long long)m * nu + t + e * NT, 1, (long long)half * nu), D.err, 803)
                sg_st_hint(P + t + e * NT, make_float4(f2_lo(w[e].x), f2_lo(w[e].y), f2_hi(w[e].x), f2_hi(w[e].y)),
                           keep);
        }
    }
    if (!spectra) {  // the columns never arrived: still collect the spectra copies
        sg_mbar_wait_bounded(&bar[1], ph1, D.err, 1, wlim, &landed1);
        landed1 = __syncthreads_or(landed1);
        if (landed1) ph1 ^= 1;
    }
    return landed0 && landed1;
}

// One pass kind over all disks: items[i] = (disk, index), taken in order
// through the queue head *head (zeroed before the launch).  A block whose
// copies never landed stops (its barriers cannot be reused); the others
// take the remaining items.
template <int KIND, int MINB>
__global__ void __launch_bounds__(SG_BATCH_THREADS, MINB)
    k_batch_pass(const BatchDisk* __restrict__ disks, const int2* __restrict__ items, int nitems, int* head)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_item;
    if (threadIdx.x == 0) {
        sg_mbar_init(&bar[0], 1);
        if (KIND == KIND_COLS) sg_mbar_init(&bar[1], 1);
    }
    __syncthreads();
    uint32_t ph0 = 0, ph1 = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(head, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const int2 item = items[it];
        const BatchDisk& D = disks[item.x];
        const unsigned long long wlim = sg_wait_budget(D.err);
        bool alive = true;
        if constexpr (KIND == KIND_COLS) {
            for (int k = 0; k < D.cols_mult && alive; k++) {
                const int g = item.y * D.cols_mult + k;
                switch (D.lgc) {
                    case 8: alive = batch_cols<8>(D, g, smraw, bar, ph0, ph1, wlim); break;
                    case 9: alive = batch_cols<9>(D, g, smraw, bar, ph0, ph1, wlim); break;
                    case 10: alive = batch_cols<10>(D, g, smraw, bar, ph0, ph1, wlim); break;
                    case 11: alive = batch_cols<11>(D, g, smraw, bar, ph0, ph1, wlim); break;
                    default: alive = batch_cols<12>(D, g, smraw, bar, ph0, ph1, wlim); break;
                }
                __syncthreads();  // shared memory reused by the next group
            }
        } else {
            for (int k = 0; k < D.rows_mult && alive; k++) {
                const int u = item.y * D.rows_mult + k;
                if constexpr (KIND == KIND_ROWS) {
                    switch (D.lgr) {
                        case 8: alive = batch_rows<8>(D, u, smraw, bar[0], ph0, wlim); break;
                        case 9: alive = batch_rows<9>(D, u, smraw, bar[0], ph0, wlim); break;
                        case 10: alive = batch_rows<10>(D, u, smraw, bar[0], ph0, wlim); break;
                        case 11: alive = batch_rows<11>(D, u, smraw, bar[0], ph0, wlim); break;
                        default: alive = batch_rows<12>(D, u, smraw, bar[0], ph0, wlim); break;
                    }
                } else {
                    switch (D.lgr) {
                        case 8: alive = batch_inv<8>(D, u, smraw, bar[0], ph0, wlim); break;
                        case 9: alive = batch_inv<9>(D, u, smraw, bar[0], ph0, wlim); break;
                        case 10: alive = batch_inv<10>(D, u, smraw, bar[0], ph0, wlim); break;
                        case 11: alive = batch_inv<11>(D, u, smraw, bar[0], ph0, wlim); break;
                        default: alive = batch_inv<12>(D, u, smraw, bar[0], ph0, wlim); break;
                    }
                }
                __syncthreads();  // shared memory reused by the next unit
            }
        }
        if (!alive) break;
    }
}

// ---------------------------------------------------------------------------
// Host side: the prepared work lists and the tuned schedules.
// ---------------------------------------------------------------------------
static size_t rows_smem_max()
{
    size_t b = 0;
    b = std::max(b, rows_unit_smem_bytes<8>());
    b = std::max(b, rows_unit_smem_bytes<9>());
    b = std::max(b, rows_unit_smem_bytes<10>());
    b = std::max(b, rows_unit_smem_bytes<11>());
    b = std::max(b, rows_unit_smem_bytes<12>());
    return b;
}
static size_t cols_smem_max()
{
    size_t b = 0;
    for (int lgc = 8; lgc <= 12; lgc++) b = std::max(b, (size_t)batch_col_slots(lgc) * batch_col_bytes(1 << (lgc - 1)));
    return b;
}

// paired row transforms per 256-thread block for rows of 2^lg points
static int row_slots(int lg) { return SG_BATCH_THREADS / ((1 << lg) / 16); }

bool batch_eligible(const sg_plan* p)
{
    if (p->dtype != SG_F32 || !p->built || p->edges || p->wedge || !p->have_imaps) return false;
    const int lgr = sg_ilog2(p->nphi), lgc = sg_ilog2(2 * p->nu);
    if (lgr < 8 || lgr > 12 || lgc < 8 || lgc > 12) return false;
    return p->nu % (4 * row_slots(lgr)) == 0;
}

typedef void (*BatchKernel)(const BatchDisk*, const int2*, int, int*);

// The schedule: the disk order (largest first, or as given), the blocks per
// SM of each pass kind, and per size class (log2 N_phi, log2 2 N_u) the row
// units per row item (both row passes) and the mode groups per column item.
struct BatchTuning {
    int natural = 0;
    int minb[3] = {3, 3, 3};  // blocks per SM of each pass kind's kernel (2 or 3)
    unsigned char rows_mult[5][5], cols_mult[5][5];
    BatchTuning()
    {
        for (int a = 0; a < 5; a++)
            for (int b = 0; b < 5; b++) rows_mult[a][b] = cols_mult[a][b] = 1;
    }
};

struct BatchList {
    std::vector<const void*> key;  // (plan, sigma, F_r, F_phi) per item: the list it was prepared for
    int device = -1;
    int ndisks = 0;
    int nitems[3] = {0, 0, 0}, grid[3] = {0, 0, 0};  // per pass kind
    size_t smem[3] = {0, 0, 0};
    BatchKernel kernel[3] = {nullptr, nullptr, nullptr};
    BatchDisk* d_disks = nullptr;
    int2* d_items = nullptr;  // the three item lists, one after the other
    int* d_ctrl = nullptr;    // the three queue heads
    unsigned char* d_work = nullptr;  // each item's half spectra and pairs (12 bytes per cell)
    // items whose plan takes the row passes on the tensor cores (short_dft,
    // rows of 256): their P1 arguments, then their P3 arguments, one batched
    // launch each; the persistent kernels take only their column items
    TcArgs* d_tc = nullptr;
    int ntc = 0, tc_max_nu = 0;
};

static std::mutex g_batch_mu;
static std::deque<BatchList> g_lists;  // most recently prepared first
static const size_t SG_BATCH_LISTS = 4;
static std::vector<std::pair<std::string, BatchTuning>> g_tunings;  // by batch signature

static void free_list(BatchList& b)
{
    sg_free(b.d_disks);
    sg_free(b.d_items);
    sg_free(b.d_ctrl);
    sg_free(b.d_work);
    sg_free(b.d_tc);
    b.d_tc = nullptr;
    b.d_disks = nullptr;
    b.d_items = nullptr;
    b.d_ctrl = nullptr;
    b.d_work = nullptr;
}

static std::vector<const void*> list_key(const sg_batch_item* items, int n)
{
    std::vector<const void*> k((size_t)4 * n);
    for (int b = 0; b < n; b++) {
        k[4 * b] = items[b].plan;
        k[4 * b + 1] = items[b].sigma;
        k[4 * b + 2] = items[b].F_r;
        k[4 * b + 3] = items[b].F_phi;
    }
    return k;
}

// "sms=<n>;<N_u>x<N_phi>*<count>;..." over the sorted sizes: what a schedule is tuned for
static std::string batch_signature(const sg_batch_item* items, int n, int sms)
{
    std::vector<std::pair<int, int>> sz;
    // a plan with tensor-core rows (short_dft) counts as its own size class ("t")
    for (int b = 0; b < n; b++)
        sz.push_back({items[b].plan->nu, 2 * items[b].plan->nphi + (items[b].plan->short_dft ? 1 : 0)});
    std::sort(sz.begin(), sz.end());
    std::string s = "sms=" + std::to_string(sms) + ";";
    for (size_t i = 0; i < sz.size();) {
        size_t j = i;
        while (j < sz.size() && sz[j] == sz[i]) j++;
        s += std::to_string(sz[i].first) + "x" + std::to_string(sz[i].second / 2) + (sz[i].second & 1 ? "t" : "") +
             "*" + std::to_string(j - i) + ";";
        i = j;
    }
    return s;
}

static const BatchTuning* find_tuning(const std::string& sig)
{
    for (auto& t : g_tunings)
        if (t.first == sig) return &t.second;
    return nullptr;
}

static void set_tuning(const std::string& sig, const BatchTuning& t)
{
    for (auto& e : g_tunings)
        if (e.first == sig) {
            e.second = t;
            return;
        }
    g_tunings.push_back({sig, t});
}

// each pass kind compiled for three blocks per SM (80 registers) and for two
// (128 registers, no spills); the schedule picks one per kind
static const BatchKernel k_batch[3][2] = {{k_batch_pass<KIND_ROWS, 2>, k_batch_pass<KIND_ROWS, 3>},
                                          {k_batch_pass<KIND_COLS, 2>, k_batch_pass<KIND_COLS, 3>},
                                          {k_batch_pass<KIND_INV, 2>, k_batch_pass<KIND_INV, 3>}};

// every block of the pass resident at once: blocks per SM x SMs
static sg_status batch_grid(int device, BatchKernel k, size_t smem, int* grid)
{
    int sms = 0, per = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return SG_ERR_CUDA;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, SG_BATCH_THREADS, smem) != cudaSuccess || per < 1) {
        cudaGetLastError();
        return SG_ERR_CUDA;
    }
    *grid = sms * per;
    return SG_OK;
}

// Builds the device work list for the items with the given schedule (host
// work and synchronous copies: not while the stream is being captured).
static sg_status make_list(const sg_batch_item* items, int n, const BatchTuning& tu, cudaStream_t st, BatchList* out)
{
    BatchList b;
    b.key = list_key(items, n);
    b.device = items[0].plan->device;
    b.smem[KIND_ROWS] = b.smem[KIND_INV] = rows_smem_max();
    b.smem[KIND_COLS] = cols_smem_max();
    sg_status s = SG_OK;
    for (int k = 0; k < 3 && !s; k++) {
        b.kernel[k] = k_batch[k][tu.minb[k] == 2 ? 0 : 1];
        s = batch_grid(b.device, b.kernel[k], b.smem[k], &b.grid[k]);
    }
    if (s) return s;
    // each item has a workspace of its own (items may share a plan): the
    // half spectra A (4 bytes per cell) and the (B, C) pairs P (8 bytes per
    // cell), 256-byte aligned
    std::vector<size_t> off_a(n), off_p(n);
    size_t work = 0;
    for (int i = 0; i < n; i++) {
        const size_t cells = (size_t)items[i].plan->nu * items[i].plan->nphi;
        off_a[i] = work;
        work += (4 * cells + 255) & ~(size_t)255;
        off_p[i] = work;
        work += (8 * cells + 255) & ~(size_t)255;
    }
    if (sg_malloc((void**)&b.d_work, work) != cudaSuccess) return SG_ERR_ALLOC;
    std::vector<BatchDisk> D(n);
    std::vector<int> n_rows(n), n_cols(n), n_inv(n);
    std::vector<TcArgs> tc1, tc3;  // short_dft disks: P1, P3 arguments
    for (int i = 0; i < n; i++) {
        const sg_plan* p = items[i].plan;
        BatchDisk& d = D[i];
        memset(&d, 0, sizeof(d));
        d.A = (float2*)(b.d_work + off_a[i]);
        d.P = (float2*)(b.d_work + off_p[i]);
        CUtensorMap maps[2];
        if (!make_pair_maps(p->nu, p->nphi, d.A, d.P, maps)) {
            free_list(b);
            return SG_ERR_CUDA;
        }
        d.map = maps[0];
        d.sigma = (const float*)items[i].sigma;
        d.Fr = (float*)items[i].F_r;
        d.Fp = (float*)items[i].F_phi;
        d.wpre = (const float*)p->wpre;
        d.wpost = (const float*)p->wpost;
        d.Kr = (const float2*)p->kr;
        d.Kp = (const float2*)p->kp;
        d.tw = (const float2*)p->tw;
        d.err = p->derr;
        d.nu = p->nu;
        d.nphi = p->nphi;
        d.lgr = sg_ilog2(p->nphi);
        d.lgc = sg_ilog2(2 * p->nu);
        const int slots = row_slots(d.lgr);
        d.rows_mult = tu.rows_mult[d.lgr - 8][d.lgc - 8];
        d.cols_mult = tu.cols_mult[d.lgr - 8][d.lgc - 8];
        const int r2c_units = p->nu / (4 * slots), c2r_units = p->nu / (2 * slots);
        const int groups = (p->nphi / 2) / batch_col_slots(d.lgc);
        // a multiple that does not divide the unit count falls back to 1
        if (r2c_units % d.rows_mult || c2r_units % d.rows_mult) d.rows_mult = 1;
        if (groups % d.cols_mult) d.cols_mult = 1;
        n_rows[i] = r2c_units / d.rows_mult;
        n_inv[i] = c2r_units / d.rows_mult;
        n_cols[i] = groups / d.cols_mult;
        if (p->short_dft) {  // rows of 256 on the tensor cores, beside the persistent kernels
            if (p->nphi != 256) {  // eligible short_dft plans have rows of exactly 256
                free_list(b);
                return SG_ERR_UNSUPPORTED;
            }
            n_rows[i] = n_inv[i] = 0;
            TcArgs t{};
            t.nu = p->nu;
            t.N = p->nphi;
            t.err = p->derr;
            t.mat = (const float*)p->tcm;
            t.w = (const float*)p->wpre;
            t.x[0] = d.sigma;
            t.out[0] = d.A;
            tc1.push_back(t);
            t = TcArgs{};
            t.nu = p->nu;
            t.N = p->nphi;
            t.err = p->derr;
            t.mat = (const float*)p->tcm + 2 * (size_t)p->nphi * p->nphi;
            t.w = (const float*)p->wpost;
            t.pin = (const float4*)d.P;
            t.y[0] = d.Fr;
            t.y[1] = d.Fp;
            tc3.push_back(t);
            b.tc_max_nu = std::max(b.tc_max_nu, p->nu);
        }
    }
    // each pass's items, the disks' in order of decreasing work (largest
    // first, so that the small ones fill the last wave) unless natural
    std::vector<int> order(n);
    for (int i = 0; i < n; i++) order[i] = i;
    if (!tu.natural)
        std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
            return (long)D[a].nu * D[a].nphi > (long)D[c].nu * D[c].nphi;
        });
    std::vector<int2> q;
    const std::vector<int>* counts[3] = {&n_rows, &n_cols, &n_inv};
    for (int k = 0; k < 3; k++) {
        const size_t start = q.size();
        for (int d : order)
            for (int j = 0; j < (*counts[k])[d]; j++) q.push_back(make_int2(d, j));
        b.nitems[k] = (int)(q.size() - start);
    }
    b.ndisks = n;
    b.ntc = (int)tc1.size();
    if (b.ntc) {
        tc1.reserve(2 * tc3.size());
        for (const TcArgs& t : tc3) tc1.push_back(t);
        if (sg_malloc((void**)&b.d_tc, sizeof(TcArgs) * tc1.size()) != cudaSuccess) {
            free_list(b);
            return SG_ERR_ALLOC;
        }
        if (cudaMemcpyAsync(b.d_tc, tc1.data(), sizeof(TcArgs) * tc1.size(), cudaMemcpyHostToDevice, st) !=
            cudaSuccess) {
            free_list(b);
            return SG_ERR_CUDA;
        }
    }
    if ((s = (sg_malloc((void**)&b.d_disks, sizeof(BatchDisk) * n) == cudaSuccess &&
                      sg_malloc((void**)&b.d_items, sizeof(int2) * q.size()) == cudaSuccess &&
                      sg_malloc((void**)&b.d_ctrl, sizeof(int) * 4) == cudaSuccess)
                     ? SG_OK
                     : SG_ERR_ALLOC)) {
        free_list(b);
        return s;
    }
    if (cudaMemcpyAsync(b.d_disks, D.data(), sizeof(BatchDisk) * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(b.d_items, q.data(), sizeof(int2) * q.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        free_list(b);
        return SG_ERR_CUDA;
    }
    *out = b;
    return SG_OK;
}

// the three queue heads zeroed, then one launch per pass kind (a row kind
// with no items is not launched); the short_dft disks' P1 before the column
// kernel and their P3 after it, one batched launch each
static sg_status launch_list(const BatchList& b, cudaStream_t st)
{
    if (cudaMemsetAsync(b.d_ctrl, 0, sizeof(int) * 4, st) != cudaSuccess) return SG_ERR_CUDA;
    if (b.ntc && launch_dft_tc_batch(b.d_tc, b.ntc, 0, b.tc_max_nu, st) != cudaSuccess) return SG_ERR_CUDA;
    const int2* items = b.d_items;
    for (int k = 0; k < 3; k++) {
        if (b.nitems[k] > 0 || k == KIND_COLS)
            b.kernel[k]<<<b.grid[k], SG_BATCH_THREADS, b.smem[k], st>>>(b.d_disks, items, b.nitems[k], b.d_ctrl + k);
        items += b.nitems[k];
    }
    if (b.ntc && launch_dft_tc_batch(b.d_tc + b.ntc, b.ntc, 1, b.tc_max_nu, st) != cudaSuccess) return SG_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

// Prepares (or finds) the list for these items; the caller holds g_batch_mu.
static sg_status find_or_make(const sg_batch_item* items, int n, cudaStream_t st, bool may_build, BatchList** out)
{
    const std::vector<const void*> key = list_key(items, n);
    for (auto it = g_lists.begin(); it != g_lists.end(); ++it)
        if (it->key == key) {
            *out = &*it;
            return SG_OK;
        }
    if (!may_build) return SG_ERR_UNSUPPORTED;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, items[0].plan->device);
    const BatchTuning* tu = find_tuning(batch_signature(items, n, sms));
    BatchList b;
    sg_status s = make_list(items, n, tu ? *tu : BatchTuning(), st, &b);
    if (s) return s;
    while (g_lists.size() >= SG_BATCH_LISTS) {
        free_list(g_lists.back());
        g_lists.pop_back();
    }
    g_lists.push_front(b);
    *out = &g_lists.front();
    return SG_OK;
}

static bool capturing(cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

// every plan eligible, all on one device
static bool batch_qualifies(const sg_batch_item* items, int n)
{
    for (int b = 0; b < n; b++)
        if (!batch_eligible(items[b].plan) || items[b].plan->device != items[0].plan->device) return false;
    return true;
}

// sg_forces_batched's persistent path: SG_ERR_UNSUPPORTED if the items do
// not qualify, or their list was not prepared and the stream is being
// captured (the caller then takes the per-plan path).
sg_status batch_forward(const sg_batch_item* items, int n, cudaStream_t st)
{
    if (!batch_qualifies(items, n)) return SG_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_batch_mu);
    BatchList* b = nullptr;
    sg_status s = find_or_make(items, n, st, !capturing(st), &b);
    if (s) return s;
    return launch_list(*b, st);
}

sg_status batch_prepare(const sg_batch_item* items, int n, cudaStream_t st)
{
    if (!batch_qualifies(items, n)) return SG_ERR_UNSUPPORTED;
    if (capturing(st)) return SG_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_batch_mu);
    BatchList* b = nullptr;
    return find_or_make(items, n, st, true, &b);
}

// ---- the tuner -------------------------------------------------------------
static sg_status time_schedule(const sg_batch_item* items, int n, const BatchTuning& tu, cudaStream_t st, float* ms)
{
    BatchList b;
    sg_status s = make_list(items, n, tu, st, &b);
    if (s) return s;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float best = 1e30f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) s = SG_ERR_CUDA;
    for (int rep = 0; rep < 7 && !s; rep++) {  // the first run warms up; the best of the others counts
        if (cudaEventRecord(e0, st) != cudaSuccess || (s = launch_list(b, st)) ||
            cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            s = s ? s : SG_ERR_CUDA;
            break;
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (rep > 0) best = std::min(best, t);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    free_list(b);
    *ms = best;
    return s;
}

static std::string format_tuning(const std::string& sig, const BatchTuning& t)
{
    std::string s = "sg-batch-schedule v2 " + sig + " natural=" + std::to_string(t.natural) + " minb=" +
                    std::to_string(t.minb[0]) + "," + std::to_string(t.minb[1]) + "," + std::to_string(t.minb[2]);
    for (int a = 0; a < 5; a++)
        for (int b = 0; b < 5; b++)
            if (t.rows_mult[a][b] != 1 || t.cols_mult[a][b] != 1)
                s += " " + std::to_string(a + 8) + "x" + std::to_string(b + 8) + "=" + std::to_string(t.rows_mult[a][b]) +
                     "," + std::to_string(t.cols_mult[a][b]);
    return s;
}

static bool parse_tuning(const std::string& line, const std::string& sig, BatchTuning* t)
{
    const std::string head = "sg-batch-schedule v2 " + sig + " ";
    if (line.compare(0, head.size(), head) != 0) return false;
    BatchTuning r;
    size_t pos = head.size();
    while (pos < line.size()) {
        size_t end = line.find(' ', pos);
        if (end == std::string::npos) end = line.size();
        const std::string tok = line.substr(pos, end - pos);
        pos = end + 1;
        int a, b, rm, cm;
        int c3;
        if (sscanf(tok.c_str(), "natural=%d", &a) == 1) {
            r.natural = a != 0;
        } else if (sscanf(tok.c_str(), "minb=%d,%d,%d", &a, &b, &c3) == 3) {
            const int v[3] = {a, b, c3};
            for (int k = 0; k < 3; k++) {
                if (v[k] != 2 && v[k] != 3) return false;
                r.minb[k] = v[k];
            }
        } else if (sscanf(tok.c_str(), "%dx%d=%d,%d", &a, &b, &rm, &cm) == 4) {
            if (a < 8 || a > 12 || b < 8 || b > 12 || rm < 1 || rm > 8 || cm < 1 || cm > 8) return false;
            r.rows_mult[a - 8][b - 8] = (unsigned char)rm;
            r.cols_mult[a - 8][b - 8] = (unsigned char)cm;
        } else if (!tok.empty()) {
            return false;
        }
    }
    *t = r;
    return true;
}

sg_status batch_tune(const sg_batch_item* items, int n, const char* path, cudaStream_t st, float ms_out[2])
{
    if (!batch_qualifies(items, n)) return SG_ERR_UNSUPPORTED;
    if (capturing(st)) return SG_ERR_ARG;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, items[0].plan->device) != cudaSuccess)
        return SG_ERR_CUDA;
    const std::string sig = batch_signature(items, n, sms);
    BatchTuning best;
    bool have = false;
    if (path) {  // a schedule tuned before for this signature
        if (FILE* f = fopen(path, "r")) {
            char buf[4096];
            while (fgets(buf, sizeof buf, f)) {
                std::string line(buf);
                while (!line.empty() && (line.back() == '\n' || line.back() == '\r')) line.pop_back();
                if (parse_tuning(line, sig, &best)) have = true;  // the last entry wins
            }
            fclose(f);
        }
    }
    float t_default = 0.f, t_best = 0.f;
    sg_status s = time_schedule(items, n, BatchTuning(), st, &t_default);
    if (s) return s;
    if (!have) {
        // the disk order and each kind's occupancy first, then each size
        // class's item sizes, largest classes first
        t_best = t_default;
        auto consider = [&](const BatchTuning& c) -> sg_status {
            float t;
            sg_status e = time_schedule(items, n, c, st, &t);
            if (!e && t < t_best) {
                t_best = t;
                best = c;
            }
            return e;
        };
        {
            BatchTuning c = best;
            c.natural = 1;
            if ((s = consider(c))) return s;
        }
        for (int k = 0; k < 3; k++) {
            BatchTuning c = best;
            c.minb[k] = 2;
            if ((s = consider(c))) return s;
        }
        std::vector<std::pair<long, std::pair<int, int>>> classes;
        for (int b = 0; b < n; b++) {
            const sg_plan* p = items[b].plan;
            const std::pair<int, int> c{sg_ilog2(p->nphi) - 8, sg_ilog2(2 * p->nu) - 8};
            bool found = false;
            for (auto& e : classes)
                if (e.second == c) {
                    e.first += (long)p->nu * p->nphi;
                    found = true;
                }
            if (!found) classes.push_back({(long)p->nu * p->nphi, c});
        }
        std::sort(classes.begin(), classes.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
        const int mults[3][2] = {{2, 1}, {1, 2}, {2, 2}};
        for (auto& e : classes) {
            const BatchTuning base = best;
            for (auto& mm : mults) {
                BatchTuning c = base;
                c.rows_mult[e.second.first][e.second.second] = (unsigned char)mm[0];
                c.cols_mult[e.second.first][e.second.second] = (unsigned char)mm[1];
                if ((s = consider(c))) return s;
            }
        }
        if (path) {
            if (FILE* f = fopen(path, "a")) {
                fprintf(f, "%s\n", format_tuning(sig, best).c_str());
                fclose(f);
            } else {
                return SG_ERR_IO;
            }
        }
    } else if ((s = time_schedule(items, n, best, st, &t_best))) {
        return s;
    }
    std::lock_guard<std::mutex> lock(g_batch_mu);
    set_tuning(sig, best);
    // the prepared list for these items now follows the tuned schedule
    const std::vector<const void*> key = list_key(items, n);
    for (auto it = g_lists.begin(); it != g_lists.end(); ++it)
        if (it->key == key) {
            free_list(*it);
            g_lists.erase(it);
            break;
        }
    BatchList* b = nullptr;
    if ((s = find_or_make(items, n, st, true, &b))) return s;
    if (ms_out) {
        ms_out[0] = t_default;
        ms_out[1] = t_best;
    }
    return SG_OK;
}

// a plan being destroyed: the lists that refer to it go with it (a later
// plan at the same address must not find them)
void batch_forget_plan(const sg_plan* p)
{
    std::lock_guard<std::mutex> lock(g_batch_mu);
    for (auto it = g_lists.begin(); it != g_lists.end();) {
        bool uses = false;
        for (size_t k = 0; k < it->key.size(); k += 4) uses |= it->key[k] == p;
        if (uses) {
            free_list(*it);
            it = g_lists.erase(it);
        } else {
            ++it;
        }
    }
}

}  // namespace sg
