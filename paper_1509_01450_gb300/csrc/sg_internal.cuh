// sg_internal.cuh -- plan object and launcher declarations shared by the
// translation units of libsgdisk.so.
#pragma once
#include "../../include/sg.h"
#include "sg_common.cuh"

// 2-D tensor maps over the three mode-major half-spectrum buffers (wa, wb,
// wc), for the row passes' tensor copies of R rows x up to 256 modes; R = 0
// when there are none (the passes then use cp.async and plain stores).
struct SgRowMaps {
    CUtensorMap m[3];
    int R;
};

// The plan behind the opaque sg_plan handle.
struct sg_plan {
    int nu, nphi;
    sg_dtype dtype;
    double u_min, du, G;
    int weight_p;
    int built;
    int loaded;      // spectra read from a plan file: the FP64 build tables are absent
    double rtol;     // quadrature tolerance of the build
    int device;      // device the plan's memory lives on
    int sms;         // its multiprocessor count
    size_t elem;     // bytes of one real in the working dtype
    // working-dtype device buffers
    void* tw;        // twiddle table, SG_NMAX complex
    void* wa;        // half spectra, mode-major X[m nu + i], nu * nphi/2 complex
    void* wb;        // same; wb and wc are one allocation (wc = wb + nu nphi/2 values), which
    void* wc;        // the fixed-length FP32 passes use as one buffer of (B, C) or (A, C) pairs
    void* kr;        // Khat_r, (nphi/2 + 1) x (nu + 2) complex
    void* kp;        // Khat_phi, same shape
    void* wpre;      // beta^{p (i - i_ref)}, nu reals
    void* wpost;     // beta^{-p (i - i_ref)}
    int* derr;       // device: int flags of the passes' bounded waits, then (at +8 bytes)
                     // the first-wait budget in ns (unsigned long long)
    // FP64 device buffers
    void* tw64;      // twiddle table, SG_NMAX double complex
    double* cells;   // 6 x (2 nu + 1) x nphi raw cell kernels (kept after build)
    double* keff;    // 2 x (2 nu - 1) x nphi folded kernels K^eff
    // host-API staging (allocated on first sg_forces_host)
    // SG_F32X2: the double-float working fields of sigma, F_r, F_phi (or of
    // the adjoint's gF_r, gF_phi, gsigma) and of the wedge row's density and
    // gradient (2 N_phi); the API's FP64 fields are converted into and out of them
    void* xf;
    void* xw;
    void* h_sigma;
    void* h_fr;
    void* h_fp;
    size_t bytes;    // device bytes held
    SgRowMaps maps[2];     // for R = slots and 2 slots rows per row block
    SgRowMaps na_maps[2];  // the same over the allocation-free scratch
    int have_na_maps;
    // tensor maps of the fixed-length FP32 inverse row passes (make_pair_maps):
    // [0] over wb in the pair layout, [1] over wa; have_imaps = 0 if none
    CUtensorMap imaps[2];
    int have_imaps;
    CUtensorMap na_imaps[2];  // the same over the allocation-free scratch
    int have_na_imaps;
    cudaStream_t bstream;         // this plan's items of a batch run here, concurrently with other plans'
    cudaEvent_t bfork, bjoin;     // fork from / join back to the batch caller's stream
    cudaEvent_t ev[4];  // pass timing (sg_forces_timed), created on first use
    int have_ev;
    int report[4];      // last build: flag bits, failed offsets, one failed (k, q)
    // one-sided radial slopes at the first and last rows (radial_edges = 1)
    int edges;
    void* egr;          // working dtype, [nphi/2 + 1][sg_edge_stride]: G beta^k / N_phi times the
    void* egp;          // phi-DFT of K^{r,r}[k, .] (cosine sum) and of K^{phi,r}[k, .] (sine sum)
    double ecoef[16];   // [a][b]: slope change of row a in {-1, 0, nu-1, nu} per weighted
                        // sigma of row b in {0, 1, nu-2, nu-1}
    // the origin wedge below the first row (sg_build_opts.wedge = 1)
    int wedge;
    void* wtab;         // working dtype, [4][nphi/2 + 1][nu]: Wr, Wphi, Vr, Vphi spectra (wedge.cu)
    void* wtmp;         // [nphi/2] complex values of the working dtype (16 B each allocated): the adjoint's per-mode sums
    // the row passes as dense DFT-matrix products on the tensor cores
    // (sg_build_opts.short_dft = 1; FP32, 32 <= nphi <= 256)
    int short_dft;
    void* tcm;          // FP32 [4 nphi^2]: the split matrices of dft_tc_matrices
};

namespace sg {

// Plain view of a plan passed to the launchers.
struct PlanView {
    int nu, nphi;
    int sms;
    const void* tw;
    const void* tw64;
    void *wa, *wb, *wc;
    const void* kr;
    const void* kp;
    const void* wpre;
    const void* wpost;
    int* err;
    const SgRowMaps* maps;  // [2] over wa, wb, wc, or null
    const CUtensorMap* imaps;  // [2] of make_pair_maps over wb (pairs) and wa, or null
    int pairs;              // set by the launchers: the column spectra are in the pair layout
                            // (forward: wb holds (B, C); adjoint: wb holds (A, C), wa holds B)
    int edges;              // one-sided radial edge slopes: egr, egp, ecoef below
    const void* egr;
    const void* egp;
    const double* ecoef;
    int wedge;              // the origin wedge: wtab, wtmp, and per call sigw / gsigw
    const void* wtab;
    void* wtmp;
    const void* sigw;       // forward: the wedge densities (N_phi, working dtype), set per call
    void* gsigw;            // adjoint: their gradient, set per call
    const void* tcm;        // FP32 plans with short_dft: the tensor-core DFT matrices; null otherwise
};

inline PlanView view(const sg_plan* p)
{
    PlanView v;
    v.nu = p->nu;
    v.nphi = p->nphi;
    v.sms = p->sms;
    v.tw = p->tw;
    v.tw64 = p->tw64;
    v.wa = p->wa;
    v.wb = p->wb;
    v.wc = p->wc;
    v.kr = p->kr;
    v.kp = p->kp;
    v.wpre = p->wpre;
    v.wpost = p->wpost;
    v.err = p->derr;
    v.maps = p->maps;
    v.imaps = p->have_imaps ? p->imaps : nullptr;
    v.pairs = 0;
    v.edges = p->edges;
    v.egr = p->egr;
    v.egp = p->egp;
    v.ecoef = p->ecoef;
    v.wedge = p->wedge;
    v.wtab = p->wtab;
    v.wtmp = p->wtmp;
    v.sigw = nullptr;
    v.gsigw = nullptr;
    v.tcm = p->short_dft ? p->tcm : nullptr;
    return v;
}

// ev: optional 4 events recorded before P1, after P1, after P2, after P3
template <typename T>
// sigma_direct: sigma is memory that the GPU reaches only by plain loads
// (mapped pinned host memory); the row pass then reads it without bulk copies
cudaError_t launch_forward(const PlanView& p, const T* sigma, T* Fr, T* Fp, cudaStream_t st,
                           cudaEvent_t* ev = nullptr, bool sigma_direct = false);
// ev: optional 4 events recorded before P1b, after P1b, after P2b (and the
// edge or wedge update), after P3b
template <typename T>
cudaError_t launch_backward(const PlanView& p, const T* gr, const T* gp, T* gs, cudaStream_t st,
                            cudaEvent_t* ev = nullptr);
// wedge.cu: the origin wedge's update between the column and inverse-row
// passes (forward: p.sigw; adjoint: writes p.gsigw)
template <typename T>
cudaError_t launch_wedge(const PlanView& p, bool adjoint, cudaStream_t st);
// the wedge row's phi-spectrum per mode into p.wtmp (for the fused update)
template <typename T>
cudaError_t launch_wedge_dft(const PlanView& p, cudaStream_t st);
// Tensor maps of the row passes over the buffers bufs[3] (the layout of wa,
// wb, wc); out[k].R = 0 where a map cannot be made.
void make_row_maps(int nu, int nphi, size_t elem, void* const bufs[3], SgRowMaps out[2]);
// Tensor maps of the fixed-length FP32 inverse row passes: out[0] over wb as
// the pair layout (two 8-byte units per row), out[1] over wa (one unit per
// row); boxes of 4 units x min(N_phi/2, 256) modes with the 32-byte swizzle.
// False if they cannot be made (the passes then use the run-time instances).
bool make_pair_maps(int nu, int nphi, void* wa, void* wb, CUtensorMap out[2]);
// noalloc.cu: the allocation-free entry point's set-up at plan build and load
sg_status noalloc_prepare(sg_plan* p, cudaStream_t stream);
// fftconv_df.cu: FP64 fields into and out of double-float working fields
cudaError_t launch_to_df(const double* in, dfloat* out, size_t n, int sms, cudaStream_t st);
cudaError_t launch_from_df(const dfloat* in, double* out, size_t n, int sms, cudaStream_t st);
// batch.cu: sg_forces_batched's persistent path and its preparation
sg_status batch_forward(const sg_batch_item* items, int n, cudaStream_t st);
sg_status batch_prepare(const sg_batch_item* items, int n, cudaStream_t st);
sg_status batch_tune(const sg_batch_item* items, int n, const char* path, cudaStream_t st, float ms_out[2]);
void batch_forget_plan(const sg_plan* p);
bool batch_eligible(const sg_plan* p);
// dft_tc.cu: the row passes (forward and adjoint) as tensor-core DFT-matrix products.
// Arguments of its transform kernel (the four row passes take different
// subsets).  Row fields are row-major, N values per row; spectra are
// mode-major, element (m, i) at m nu + i, mode 0 holding (DC, Nyquist).
struct TcArgs {
    const float* x[2];    // rows -> spectra: the input row fields (one or two)
    const float4* pin;    // spectra -> rows, pair layout: {X, Y} (16 bytes per element)
    const float2* in[2];  // spectra -> rows otherwise: the single-layout spectra
    const float* mat;     // the direction's matrix: [part (hi, lo)][column tile][K chunk][64 x 32 core-matrix tile]
    const float* w;       // the row weights (nu values), applied to the outputs
    float4* pout;         // rows -> spectra, two products, pair layout: the output pairs
    float2* out[2];       // rows -> spectra otherwise: the single-layout output spectra
    float* y[2];          // spectra -> rows: the output row fields
    int nu, N;
    int* err;
};
bool dft_tc_supported(int nphi);
size_t dft_tc_matrix_floats(int nphi);
void dft_tc_matrices(int nphi, float* out);  // host: D then E, each [hi, lo][tile][chunk][NT x 32]
cudaError_t launch_dft_r2c(const PlanView& p, const float* sigma, cudaStream_t st);
cudaError_t launch_dft_c2r(const PlanView& p, float* Fr, float* Fp, cudaStream_t st);
cudaError_t launch_dft_r2c_adjoint(const PlanView& p, const float* gr, const float* gp, cudaStream_t st);
cudaError_t launch_dft_c2r_adjoint(const PlanView& p, float* gs, cudaStream_t st);
cudaError_t launch_dft_tc_batch(const TcArgs* d_args, int n, int dir, int max_nu, cudaStream_t st);
// every device allocation of the library, through the sg_test_fail_alloc
// hook, and its release (sg_test_live_allocations counts the difference)
cudaError_t sg_malloc(void** ptr, size_t bytes);
void sg_free(void* ptr);
template <typename VO>
cudaError_t launch_spectra(const PlanView& p, const double* nsr, const double* nsp, double2* W, VO* Kr, VO* Kp,
                           cudaStream_t st);

// kbuild.cu
// pot: the potential's cells (SG_KERNEL_POTENTIAL) instead of the forces'
cudaError_t launch_cells(int nu, int nphi, double du, double rtol, double* cells, int* flag, cudaStream_t st,
                         int pot = 0);
// row stride (elements) of the edge tables: the 2 nu + 1 offsets rounded up
// to 16 bytes, so that one mode's row moves by one bulk copy
__host__ __device__ inline int sg_edge_stride(int nu, int elem)
{
    const int per = 16 / elem;
    return (2 * nu + 1 + per - 1) / per * per;
}
// the phi-spectra of the radial slope kernels for the one-sided edge slopes
template <typename T>
cudaError_t launch_edge_spectra(int nu, int nphi, double du, double G, const double* cells, const void* tw64, T* gr,
                                T* gp, cudaStream_t st);
// the trapezoidal variant of the cell integrals over a table launch_cells made
cudaError_t launch_cells_tpz(int nu, int nphi, double du, int ntpz, double rtol, double* cells, int* flag,
                             cudaStream_t st);
// the particle kinds' tables (sg_kernel_kind 1-3; for 2 with the exact own cell)
cudaError_t launch_point_cells(int nu, int nphi, double du, int kind, double soften, double rtol, double* cells,
                               int* flag, cudaStream_t st);
// the origin wedge's cells ([6][nu][nphi] FP64 scratch) and its four spectra
// tables (wedge.cu reads them); flag bit 4 marks a cell that ran out of budget
template <typename T>
cudaError_t launch_wedge_tables(int nu, int nphi, double du, double G, double rtol, int pot, double* wcells,
                                const void* tw64, T* tab, int* flag, cudaStream_t st);
// the folded Cartesian kernels (SG_KERNEL_CARTESIAN) straight into keff and
// the spectra's inputs; the cell table is zeroed
cudaError_t launch_cart_fold(int nu, int nphi, double h, double G, double* cells, double* keff, double* nsr,
                             double* nsp, cudaStream_t st);
cudaError_t launch_fold(int nu, int nphi, double du, double G, int p, const double* cells, double* keff,
                        double* nsr, double* nsp, cudaStream_t st);
void gauss_legendre(int n, double* x, double* w);

}  // namespace sg
