// api.cu -- the extern "C" entry points of libsgdisk.so (declared in
// include/sg.h): plan lifecycle, the one-time kernel build, and dispatch of
// the forward / adjoint passes.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "sg_internal.cuh"

using namespace sg;

#define SG_TRY(call)                           \
    do {                                       \
        cudaError_t e_ = (call);               \
        if (e_ != cudaSuccess) return SG_ERR_CUDA; \
    } while (0)

static bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// sg_test_fail_alloc: allocations still to succeed (-1: all)
static std::atomic<int> g_alloc_budget{-1};
static std::atomic<int> g_live_allocs{0};  // sg_malloc'd and not yet sg_free'd
static std::atomic<int> g_bounds_site{0};

namespace sg {
cudaError_t sg_malloc(void** ptr, size_t bytes)
{
    int n = g_alloc_budget.load();
    while (n >= 0) {
        if (n == 0) {
            *ptr = nullptr;
            return cudaErrorMemoryAllocation;
        }
        if (g_alloc_budget.compare_exchange_weak(n, n - 1)) break;
    }
    const cudaError_t e = cudaMalloc(ptr, bytes);
    if (e == cudaSuccess) g_live_allocs++;
    return e;
}
void sg_free(void* ptr)
{
    if (ptr && cudaFree(ptr) == cudaSuccess) g_live_allocs--;
}
}  // namespace sg

int sg_test_live_allocations(void) { return g_live_allocs.load(); }

int sg_test_fail_alloc(int after) { return g_alloc_budget.exchange(after < 0 ? -1 : after); }

int sg_checked_build(void)
{
#ifdef SG_DEBUG
    return 1;
#else
    return 0;
#endif
}

int sg_last_bounds_site(void) { return g_bounds_site.load(); }

static sg_status dev_alloc(sg_plan* p, void** ptr, size_t bytes)
{
    if (sg_malloc(ptr, bytes) != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return SG_ERR_ALLOC;
    }
    p->bytes += bytes;
    return SG_OK;
}

static void free_plan(sg_plan* p)
{
    if (p->have_ev)
        for (int i = 0; i < 4; i++) cudaEventDestroy(p->ev[i]);
    if (p->bjoin) cudaEventDestroy(p->bjoin);
    if (p->bfork) cudaEventDestroy(p->bfork);
    if (p->bstream) cudaStreamDestroy(p->bstream);
    // wc lies inside wb's allocation
    void* bufs[] = {p->tw, p->wa, p->wb, p->kr, p->kp, p->wpre, p->wpost, p->tw64, p->cells, p->keff,
                    p->h_sigma, p->h_fr, p->h_fp, p->derr, p->egr, p->egp, p->wtab, p->wtmp, p->xf, p->xw,
                    p->tcm};
    for (void* b : bufs)
        sg_free(b);
    free(p);
}

// exp(-2 pi i j / SG_NMAX) in double.  Every angle is reduced to a in
// [0, pi/4] by exact octant identities, so cos and sin are evaluated only
// where libm is accurate to about half an ulp.
static void twiddles(std::vector<double>& re, std::vector<double>& im)
{
    const int N = SG_NMAX, E8 = SG_NMAX / 8;
    re.resize(N);
    im.resize(N);
    for (int j = 0; j < N; j++) {
        const int o = j / E8, r = j - o * E8;
        double cc, ss;  // cos and sin of 2 pi j / N
        if ((o & 1) == 0) {  // theta = o pi/4 + a
            const double a = 2.0 * M_PI * r / N, c = cos(a), s = sin(a);
            switch (o) {
                case 0: cc = c; ss = s; break;
                case 2: cc = -s; ss = c; break;
                case 4: cc = -c; ss = -s; break;
                default: cc = s; ss = -c; break;  // o == 6
            }
        } else {  // theta = (o + 1) pi/4 - a
            const double a = 2.0 * M_PI * (E8 - r) / N, c = cos(a), s = sin(a);
            switch (o) {
                case 1: cc = s; ss = c; break;
                case 3: cc = -c; ss = s; break;
                case 5: cc = -s; ss = -c; break;
                default: cc = c; ss = -s; break;  // o == 7
            }
        }
        re[j] = cc;
        im[j] = -ss;
    }
}

extern "C" {

const char* sg_status_string(sg_status s)
{
    switch (s) {
        case SG_OK: return "ok";
        case SG_ERR_ARG: return "invalid argument";
        case SG_ERR_ALLOC: return "allocation failed";
        case SG_ERR_CUDA: return "CUDA error";
        case SG_ERR_UNSUPPORTED: return "unsupported size";
        case SG_ERR_NOT_BUILT: return "kernels not built (call sg_kernels_build)";
        case SG_ERR_TIMEOUT: return "quadrature or device wait did not converge";
        case SG_ERR_IO: return "plan file could not be written or read, or is not a plan file of this library";
        case SG_ERR_BOUNDS: return "an index check of a pass failed (checked build); results invalid";
    }
    return "unknown status";
}

sg_status sg_plan_create(sg_plan** out, int nu, int nphi, double u_min, double du, double G, sg_dtype dtype)
{
    if (!out) return SG_ERR_ARG;
    if (!(du > 0.0) || !isfinite(du) || !isfinite(u_min) || !isfinite(G)) return SG_ERR_ARG;
    if (dtype != SG_F32 && dtype != SG_F64 && dtype != SG_F32X2) return SG_ERR_ARG;
    if (!is_pow2(nu) || !is_pow2(nphi)) return SG_ERR_UNSUPPORTED;
    const int numax = dtype == SG_F32 ? 4096 : 2048;
    const int nphimax = dtype == SG_F32 ? 8192 : 4096;
    if (nu < 4 || nu > numax || nphi < 4 || nphi > nphimax) return SG_ERR_UNSUPPORTED;

    sg_plan* p = (sg_plan*)calloc(1, sizeof(sg_plan));
    if (!p) return SG_ERR_ALLOC;
    p->nu = nu;
    p->nphi = nphi;
    p->dtype = dtype;
    p->u_min = u_min;
    p->du = du;
    p->G = G;
    p->weight_p = 2;
    p->elem = dtype == SG_F32 ? sizeof(float) : sizeof(double);  // a double-float takes 8 bytes too
    const size_t cx = 2 * p->elem;
    if (cudaGetDevice(&p->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
        free(p);
        return SG_ERR_CUDA;
    }

    const size_t nhalf = (size_t)nu * (nphi / 2);
    const size_t nk = (size_t)(nphi / 2 + 1) * (nu + 2);
    sg_status st;
    if ((st = dev_alloc(p, &p->tw, SG_NMAX * cx)) || (st = dev_alloc(p, &p->tw64, SG_NMAX * sizeof(double2))) ||
        (st = dev_alloc(p, &p->wa, nhalf * cx)) || (st = dev_alloc(p, &p->wb, 2 * nhalf * cx)) ||
        (st = dev_alloc(p, &p->kr, nk * cx)) ||
        (st = dev_alloc(p, &p->kp, nk * cx)) || (st = dev_alloc(p, &p->wpre, nu * p->elem)) ||
        (st = dev_alloc(p, &p->wpost, nu * p->elem)) || (st = dev_alloc(p, (void**)&p->derr, 16)) ||
        (st = dev_alloc(p, (void**)&p->cells, (size_t)6 * (2 * nu + 1) * nphi * sizeof(double))) ||
        (st = dev_alloc(p, (void**)&p->keff, (size_t)2 * (2 * nu - 1) * nphi * sizeof(double))) ||
        (dtype == SG_F32X2 && ((st = dev_alloc(p, &p->xf, (size_t)3 * nu * nphi * sizeof(dfloat))) ||
                               (st = dev_alloc(p, &p->xw, (size_t)2 * nphi * sizeof(dfloat)))))) {
        free_plan(p);
        return st;
    }
    const unsigned long long flag_block[2] = {0ull, SG_WAIT_NS};  // flags, first-wait budget (ns)
    if (cudaMemcpy(p->derr, flag_block, 16, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->bstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->bfork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->bjoin, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        free_plan(p);
        return SG_ERR_CUDA;
    }
    p->wc = (unsigned char*)p->wb + nhalf * cx;
    {
        void* const bufs[3] = {p->wa, p->wb, p->wc};
        make_row_maps(nu, nphi, p->elem, bufs, p->maps);
        p->have_imaps = dtype == SG_F32 && make_pair_maps(nu, nphi, p->wa, p->wb, p->imaps) ? 1 : 0;
    }
    std::vector<double> re, im;
    twiddles(re, im);
    std::vector<double> t64(2 * SG_NMAX);
    for (int j = 0; j < SG_NMAX; j++) {
        t64[2 * j] = re[j];
        t64[2 * j + 1] = im[j];
    }
    if (cudaMemcpy(p->tw64, t64.data(), SG_NMAX * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess) {
        free_plan(p);
        return SG_ERR_CUDA;
    }
    cudaError_t ce;
    if (dtype == SG_F32) {
        std::vector<float> t32(2 * SG_NMAX);
        for (int j = 0; j < 2 * SG_NMAX; j++) t32[j] = (float)t64[j];
        ce = cudaMemcpy(p->tw, t32.data(), SG_NMAX * sizeof(float2), cudaMemcpyHostToDevice);
    } else if (dtype == SG_F32X2) {
        std::vector<dfloat> tdf(2 * SG_NMAX);
        for (int j = 0; j < 2 * SG_NMAX; j++) tdf[j] = dfloat(t64[j]);
        ce = cudaMemcpy(p->tw, tdf.data(), SG_NMAX * sizeof(dfloat2), cudaMemcpyHostToDevice);
    } else {
        ce = cudaMemcpy(p->tw, t64.data(), SG_NMAX * sizeof(double2), cudaMemcpyHostToDevice);
    }
    if (ce != cudaSuccess) {
        free_plan(p);
        return SG_ERR_CUDA;
    }
    *out = p;
    return SG_OK;
}

sg_status sg_dft_tc_matrices(int N_phi, float* out)
{
    if (!out) return SG_ERR_ARG;
    if (!dft_tc_supported(N_phi)) return SG_ERR_UNSUPPORTED;
    dft_tc_matrices(N_phi, out);
    return SG_OK;
}

sg_status sg_plan_destroy(sg_plan* p)
{
    if (!p) return SG_ERR_ARG;
    batch_forget_plan(p);
    free_plan(p);
    return SG_OK;
}

sg_status sg_plan_info(const sg_plan* p, int dims[4])
{
    if (!p || !dims) return SG_ERR_ARG;
    dims[0] = p->nu;
    dims[1] = p->nphi;
    dims[2] = (int)p->dtype;
    dims[3] = p->built;
    return SG_OK;
}

size_t sg_plan_device_bytes(const sg_plan* p) { return p ? p->bytes : 0; }

sg_status sg_plan_set_wait_limit(sg_plan* p, double seconds)
{
    if (!p || !(seconds >= 0.0) || !(seconds <= 60.0)) return SG_ERR_ARG;
    const unsigned long long ns = (unsigned long long)(seconds * 1e9);
    SG_TRY(cudaMemcpy(reinterpret_cast<unsigned char*>(p->derr) + 8, &ns, sizeof(ns), cudaMemcpyHostToDevice));
    return SG_OK;
}

// Plan file: a fixed header, then K̂_r, K̂_phi and the two weight rows in the
// working dtype, exactly as they sit on the device.
struct PlanFileHeader {
    char magic[8];  // "SGPLAN01"
    int32_t version, nu, nphi, dtype, weight_p, reserved[3];
    double u_min, du, G, rtol;
    uint64_t spectrum_bytes, weight_bytes;
};
static const char kPlanMagic[8] = {'S', 'G', 'P', 'L', 'A', 'N', '0', '1'};

static size_t spectrum_bytes(const sg_plan* p) { return (size_t)(p->nphi / 2 + 1) * (p->nu + 2) * 2 * p->elem; }

sg_status sg_plan_save(const sg_plan* p, const char* path, cudaStream_t stream)
{
    if (!p || !path) return SG_ERR_ARG;
    if (!p->built) return SG_ERR_NOT_BUILT;
    if (p->edges || p->wedge) return SG_ERR_UNSUPPORTED;  // the file holds no edge or wedge tables
    const size_t kb = spectrum_bytes(p), wb = (size_t)p->nu * p->elem;
    std::vector<unsigned char> buf(2 * kb + 2 * wb);
    SG_TRY(cudaMemcpyAsync(buf.data(), p->kr, kb, cudaMemcpyDeviceToHost, stream));
    SG_TRY(cudaMemcpyAsync(buf.data() + kb, p->kp, kb, cudaMemcpyDeviceToHost, stream));
    SG_TRY(cudaMemcpyAsync(buf.data() + 2 * kb, p->wpre, wb, cudaMemcpyDeviceToHost, stream));
    SG_TRY(cudaMemcpyAsync(buf.data() + 2 * kb + wb, p->wpost, wb, cudaMemcpyDeviceToHost, stream));
    SG_TRY(cudaStreamSynchronize(stream));
    PlanFileHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, kPlanMagic, 8);
    h.version = 1;
    h.nu = p->nu;
    h.nphi = p->nphi;
    h.dtype = (int32_t)p->dtype;
    h.weight_p = p->weight_p;
    h.u_min = p->u_min;
    h.du = p->du;
    h.G = p->G;
    h.rtol = p->rtol;
    h.spectrum_bytes = kb;
    h.weight_bytes = wb;
    FILE* f = fopen(path, "wb");
    if (!f) return SG_ERR_IO;
    const bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(buf.data(), 1, buf.size(), f) == buf.size();
    if (fclose(f) != 0 || !ok) return SG_ERR_IO;
    return SG_OK;
}

sg_status sg_plan_load(sg_plan** out, const char* path, cudaStream_t stream)
{
    if (!out || !path) return SG_ERR_ARG;
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) return SG_ERR_IO;
    PlanFileHeader h;
    if (fread(&h, sizeof(h), 1, f) != 1 || memcmp(h.magic, kPlanMagic, 8) != 0 || h.version != 1 ||
        (h.dtype != SG_F32 && h.dtype != SG_F64 && h.dtype != SG_F32X2)) {
        fclose(f);
        return SG_ERR_IO;
    }
    sg_plan* p = nullptr;
    sg_status st = sg_plan_create(&p, h.nu, h.nphi, h.u_min, h.du, h.G, (sg_dtype)h.dtype);
    if (st) {
        fclose(f);
        return st;
    }
    const size_t kb = spectrum_bytes(p), wb = (size_t)p->nu * p->elem;
    std::vector<unsigned char> buf(2 * kb + 2 * wb);
    const bool ok = h.spectrum_bytes == kb && h.weight_bytes == wb && fread(buf.data(), 1, buf.size(), f) == buf.size() &&
                    fgetc(f) == EOF;
    fclose(f);
    if (!ok) {
        sg_plan_destroy(p);
        return SG_ERR_IO;
    }
    if (cudaMemcpyAsync(p->kr, buf.data(), kb, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
        cudaMemcpyAsync(p->kp, buf.data() + kb, kb, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
        cudaMemcpyAsync(p->wpre, buf.data() + 2 * kb, wb, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
        cudaMemcpyAsync(p->wpost, buf.data() + 2 * kb + wb, wb, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess) {
        cudaGetLastError();
        sg_plan_destroy(p);
        return SG_ERR_CUDA;
    }
    p->weight_p = h.weight_p;
    p->rtol = h.rtol;
    p->loaded = 1;
    p->built = 1;
    if ((st = noalloc_prepare(p, stream)) != SG_OK) {
        sg_plan_destroy(p);
        return st;
    }
    *out = p;
    return SG_OK;
}

sg_status sg_kernels_build(sg_plan* p, const sg_build_opts* opts, cudaStream_t stream)
{
    if (!p) return SG_ERR_ARG;
    double rtol = 1e-14, soften = 0.0;
    int wp = 0, kind = SG_KERNEL_SIM, ntpz = 0, edges = 0, wedge = 0, short_dft = 0;
    if (opts) {
        if (opts->rtol > 0.0) rtol = opts->rtol;
        wp = opts->weight_p;
        if (wp < -8 || wp > 8) return SG_ERR_ARG;
        kind = opts->kind;
        if (kind < SG_KERNEL_SIM || kind > SG_KERNEL_CARTESIAN) return SG_ERR_ARG;
        soften = opts->soften;
        if (kind == SG_KERNEL_SOFTENED && !(soften > 0.0 && soften < 1e3)) return SG_ERR_ARG;
        ntpz = opts->n_tpz;
        if (ntpz < 0 || ntpz > 1024 || (ntpz > 0 && kind != SG_KERNEL_SIM)) return SG_ERR_ARG;
        edges = opts->radial_edges;
        if (edges != 0 && edges != 1) return SG_ERR_ARG;
        if (kind == SG_KERNEL_CARTESIAN && (wp != 0 || edges != 0)) return SG_ERR_ARG;
        wedge = opts->wedge;
        if (wedge != 0 && wedge != 1) return SG_ERR_ARG;
        // the wedge takes the place of the inner ghost row: one-sided edge
        // slopes, and the kinds whose cells are integrals over the source
        if (wedge && (!edges || (kind != SG_KERNEL_SIM && kind != SG_KERNEL_POTENTIAL))) return SG_ERR_ARG;
        short_dft = opts->short_dft;
        if (short_dft != 0 && short_dft != 1) return SG_ERR_ARG;
        if (short_dft && (p->dtype != SG_F32 || !dft_tc_supported(p->nphi))) return SG_ERR_UNSUPPORTED;
    }
    // beta^{p (i - i_ref)} must stay in range for both dtypes
    if (fabs((double)wp * p->du * p->nu) > 60.0) return SG_ERR_UNSUPPORTED;
    p->built = 0;  // until every table below is rewritten
    p->weight_p = wp;
    p->rtol = rtol;
    const int nu = p->nu, nphi = p->nphi, L = 2 * nu;

    // row weights
    {
        std::vector<double> pre(nu), post(nu);
        const int iref = nu / 2;
        for (int i = 0; i < nu; i++) {
            pre[i] = exp(wp * (i - iref) * p->du);
            post[i] = exp(-wp * (i - iref) * p->du);
            // the potential carries the target radius: Phi_i = G r_i sum sigma K^P
            if (kind == SG_KERNEL_POTENTIAL) post[i] *= 0.5 * exp(p->u_min + i * p->du) * (1.0 + exp(p->du));
        }
        if (p->dtype == SG_F32X2) {
            std::vector<dfloat> a(nu), b(nu);
            for (int i = 0; i < nu; i++) {
                a[i] = dfloat(pre[i]);
                b[i] = dfloat(post[i]);
            }
            SG_TRY(cudaMemcpyAsync(p->wpre, a.data(), nu * sizeof(dfloat), cudaMemcpyHostToDevice, stream));
            SG_TRY(cudaMemcpyAsync(p->wpost, b.data(), nu * sizeof(dfloat), cudaMemcpyHostToDevice, stream));
            SG_TRY(cudaStreamSynchronize(stream));
        } else if (p->dtype == SG_F32) {
            std::vector<float> a(nu), b(nu);
            for (int i = 0; i < nu; i++) {
                a[i] = (float)pre[i];
                b[i] = (float)post[i];
            }
            SG_TRY(cudaMemcpyAsync(p->wpre, a.data(), nu * sizeof(float), cudaMemcpyHostToDevice, stream));
            SG_TRY(cudaMemcpyAsync(p->wpost, b.data(), nu * sizeof(float), cudaMemcpyHostToDevice, stream));
            SG_TRY(cudaStreamSynchronize(stream));
        } else {
            SG_TRY(cudaMemcpyAsync(p->wpre, pre.data(), nu * sizeof(double), cudaMemcpyHostToDevice, stream));
            SG_TRY(cudaMemcpyAsync(p->wpost, post.data(), nu * sizeof(double), cudaMemcpyHostToDevice, stream));
            SG_TRY(cudaStreamSynchronize(stream));
        }
    }
    // one-sided edge slopes: s_a = sum_b c[a][b] sigma_b for the slope change
    // r_a (delta^onesided - delta^ghost) of the rows a = -1, 0, N-1, N
    // (bb = beta - 1/beta, beta - 1, 1 - 1/beta), divided by the weights of
    // the rows b = 0, 1, N-2, N-1 that the passes hold sigma with
    p->edges = 0;
    if (edges) {
        const double bb = 2.0 * sinh(p->du), bm = expm1(p->du), bi = -expm1(-p->du);
        const double c[16] = {-1.0 / bb, 0.0, 0.0, 0.0,                 // a = -1: ghost slope removed
                              -1.0 / bm, 1.0 / bm - 1.0 / bb, 0.0, 0.0,  // a = 0
                              0.0, 0.0, 1.0 / bb - 1.0 / bi, 1.0 / bi,   // a = N-1
                              0.0, 0.0, 0.0, 1.0 / bb};                 // a = N: ghost slope removed
        const int brow[4] = {0, 1, nu - 2, nu - 1};
        for (int a = 0; a < 4; a++)
            for (int b = 0; b < 4; b++) p->ecoef[4 * a + b] = c[4 * a + b] * exp(-wp * (brow[b] - nu / 2) * p->du);
        const size_t n = (size_t)(nphi / 2 + 1) * sg_edge_stride(nu, (int)p->elem) * p->elem;
        sg_status st = SG_OK;
        if ((!p->egr && (st = dev_alloc(p, &p->egr, n))) || (!p->egp && (st = dev_alloc(p, &p->egp, n)))) return st;
    }
    p->short_dft = 0;
    if (short_dft) {
        // the split DFT matrices of both forward row passes (host FP64, rounded)
        std::vector<float> m(dft_tc_matrix_floats(nphi));
        dft_tc_matrices(nphi, m.data());
        sg_status st = SG_OK;
        if (!p->tcm && (st = dev_alloc(p, &p->tcm, m.size() * sizeof(float)))) return st;
        SG_TRY(cudaMemcpyAsync(p->tcm, m.data(), m.size() * sizeof(float), cudaMemcpyHostToDevice, stream));
        SG_TRY(cudaStreamSynchronize(stream));
    }
    p->wedge = 0;
    if (wedge) {
        const size_t n = (size_t)4 * (nphi / 2 + 1) * nu * p->elem;
        sg_status st = SG_OK;
        if ((!p->wtab && (st = dev_alloc(p, &p->wtab, n))) ||
            (!p->wtmp && (st = dev_alloc(p, &p->wtmp, (size_t)(nphi / 2) * sizeof(double2)))))
            return st;
    }
    int* flag = nullptr;
    double *nsr = nullptr, *nsp = nullptr, *wcells = nullptr;
    double2* W = nullptr;
    sg_status ret = SG_OK;
    if (sg_malloc((void**)&flag, 4 * sizeof(int)) != cudaSuccess ||
        sg_malloc((void**)&nsr, (size_t)L * nphi * sizeof(double)) != cudaSuccess ||
        sg_malloc((void**)&nsp, (size_t)L * nphi * sizeof(double)) != cudaSuccess ||
        sg_malloc((void**)&W, (size_t)(nphi / 2 + 1) * L * sizeof(double2)) != cudaSuccess ||
        (wedge && sg_malloc((void**)&wcells, (size_t)6 * nu * nphi * sizeof(double)) != cudaSuccess)) {
        cudaGetLastError();
        ret = SG_ERR_ALLOC;
        goto done;
    }
    if (cudaMemsetAsync(flag, 0, 4 * sizeof(int), stream) != cudaSuccess) {
        ret = SG_ERR_CUDA;
        goto done;
    }
    if (kind == SG_KERNEL_CARTESIAN) {
        if (launch_cart_fold(nu, nphi, p->du, p->G, p->cells, p->keff, nsr, nsp, stream) != cudaSuccess) {
            ret = SG_ERR_CUDA;
            goto done;
        }
    } else if ((kind == SG_KERNEL_SIM || kind == SG_KERNEL_POTENTIAL
                    ? launch_cells(nu, nphi, p->du, rtol, p->cells, flag, stream, kind == SG_KERNEL_POTENTIAL)
                    : launch_point_cells(nu, nphi, p->du, kind, soften, rtol, p->cells, flag, stream)) !=
                   cudaSuccess ||
               (kind == SG_KERNEL_SIM && ntpz > 0 &&
                launch_cells_tpz(nu, nphi, p->du, ntpz, rtol, p->cells, flag, stream) != cudaSuccess) ||
               launch_fold(nu, nphi, p->du, p->G, wp, p->cells, p->keff, nsr, nsp, stream) != cudaSuccess ||
        (edges && (p->dtype == SG_F32
                       ? launch_edge_spectra<float>(nu, nphi, p->du, p->G, p->cells, p->tw64, (float*)p->egr,
                                                    (float*)p->egp, stream)
                   : p->dtype == SG_F32X2
                       ? launch_edge_spectra<dfloat>(nu, nphi, p->du, p->G, p->cells, p->tw64, (dfloat*)p->egr,
                                                     (dfloat*)p->egp, stream)
                       : launch_edge_spectra<double>(nu, nphi, p->du, p->G, p->cells, p->tw64, (double*)p->egr,
                                                     (double*)p->egp, stream)) != cudaSuccess)) {
        ret = SG_ERR_CUDA;
        goto done;
    }
    if (wedge && (p->dtype == SG_F32
                      ? launch_wedge_tables<float>(nu, nphi, p->du, p->G, rtol, kind == SG_KERNEL_POTENTIAL, wcells,
                                                   p->tw64, (float*)p->wtab, flag, stream)
                  : p->dtype == SG_F32X2
                      ? launch_wedge_tables<dfloat>(nu, nphi, p->du, p->G, rtol, kind == SG_KERNEL_POTENTIAL, wcells,
                                                    p->tw64, (dfloat*)p->wtab, flag, stream)
                      : launch_wedge_tables<double>(nu, nphi, p->du, p->G, rtol, kind == SG_KERNEL_POTENTIAL, wcells,
                                                    p->tw64, (double*)p->wtab, flag, stream)) != cudaSuccess) {
        ret = SG_ERR_CUDA;
        goto done;
    }
    {
        PlanView v = view(p);
        cudaError_t e = p->dtype == SG_F32
                            ? launch_spectra<float2>(v, nsr, nsp, W, (float2*)p->kr, (float2*)p->kp, stream)
                        : p->dtype == SG_F32X2
                            ? launch_spectra<dfloat2>(v, nsr, nsp, W, (dfloat2*)p->kr, (dfloat2*)p->kp, stream)
                            : launch_spectra<double2>(v, nsr, nsp, W, (double2*)p->kr, (double2*)p->kp, stream);
        if (e != cudaSuccess) {
            ret = SG_ERR_CUDA;
            goto done;
        }
    }
    {
        if (cudaMemcpyAsync(p->report, flag, 4 * sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess) {
            ret = SG_ERR_CUDA;
            goto done;
        }
        p->built = 1;
        p->edges = edges;
        p->wedge = wedge;
        p->short_dft = short_dft;
        if (p->report[0]) ret = SG_ERR_TIMEOUT;
    }
    if (ret == SG_OK && (ret = noalloc_prepare(p, stream)) != SG_OK) p->built = 0;
done:
    sg_free(wcells);
    sg_free(flag);
    sg_free(nsr);
    sg_free(nsp);
    sg_free(W);
    return ret;
}

static sg_status check_fields(const sg_plan* p, const void* a, const void* b, const void* c)
{
    if (!p) return SG_ERR_ARG;
    if (!p->built) return SG_ERR_NOT_BUILT;
    const void* ptrs[3] = {a, b, c};
    for (const void* q : ptrs)
        if (!q || ((uintptr_t)q & 15)) return SG_ERR_ARG;
    if (p->wedge) return SG_ERR_UNSUPPORTED;  // the wedge densities come through sg_forces_wedge
    return SG_OK;
}

// The passes on the plan's working type.  The compensated plans (SG_F32X2)
// take and give FP64 fields: their inputs are split into double-float
// working fields first and the results rounded back to FP64 after.
static cudaError_t run_forward(sg_plan* p, PlanView v, const void* sigma, void* Fr, void* Fp, cudaStream_t st,
                               cudaEvent_t* ev = nullptr, bool direct = false)
{
    if (p->dtype == SG_F32)
        return launch_forward<float>(v, (const float*)sigma, (float*)Fr, (float*)Fp, st, ev, direct);
    if (p->dtype == SG_F64)
        return launch_forward<double>(v, (const double*)sigma, (double*)Fr, (double*)Fp, st, ev, direct);
    const size_t n = (size_t)p->nu * p->nphi;
    dfloat* const xs = (dfloat*)p->xf;
    dfloat* const xr = xs + n;
    dfloat* const xp = xs + 2 * n;
    cudaError_t e;
    if ((e = launch_to_df((const double*)sigma, xs, n, p->sms, st)) != cudaSuccess) return e;
    if (v.sigw) {
        if ((e = launch_to_df((const double*)v.sigw, (dfloat*)p->xw, p->nphi, p->sms, st)) != cudaSuccess) return e;
        v.sigw = p->xw;
    }
    if ((e = launch_forward<dfloat>(v, xs, xr, xp, st, ev, false)) != cudaSuccess) return e;
    if ((e = launch_from_df(xr, (double*)Fr, n, p->sms, st)) != cudaSuccess) return e;
    return launch_from_df(xp, (double*)Fp, n, p->sms, st);
}

static cudaError_t run_backward(sg_plan* p, PlanView v, const void* gr, const void* gp, void* gs, cudaStream_t st,
                                cudaEvent_t* ev = nullptr)
{
    if (p->dtype == SG_F32) return launch_backward<float>(v, (const float*)gr, (const float*)gp, (float*)gs, st, ev);
    if (p->dtype == SG_F64)
        return launch_backward<double>(v, (const double*)gr, (const double*)gp, (double*)gs, st, ev);
    const size_t n = (size_t)p->nu * p->nphi;
    dfloat* const xr = (dfloat*)p->xf;
    dfloat* const xp = xr + n;
    dfloat* const xs = xr + 2 * n;
    cudaError_t e;
    if ((e = launch_to_df((const double*)gr, xr, n, p->sms, st)) != cudaSuccess) return e;
    if ((e = launch_to_df((const double*)gp, xp, n, p->sms, st)) != cudaSuccess) return e;
    double* const gsw = (double*)v.gsigw;
    if (gsw) v.gsigw = (dfloat*)p->xw + p->nphi;
    if ((e = launch_backward<dfloat>(v, xr, xp, xs, st, ev)) != cudaSuccess) return e;
    if (gsw && (e = launch_from_df((const dfloat*)v.gsigw, gsw, p->nphi, p->sms, st)) != cudaSuccess) return e;
    return launch_from_df(xs, (double*)gs, n, p->sms, st);
}

sg_status sg_forces_wedge(sg_plan* p, const void* sigma, const void* sigma_w, void* Fr, void* Fp, cudaStream_t stream)
{
    if (!p) return SG_ERR_ARG;
    if (!p->built) return SG_ERR_NOT_BUILT;
    if (!p->wedge) return SG_ERR_ARG;
    const void* ptrs[3] = {sigma, Fr, Fp};
    for (const void* q : ptrs)
        if (!q || ((uintptr_t)q & 15)) return SG_ERR_ARG;
    if (!sigma_w || ((uintptr_t)sigma_w % p->elem)) return SG_ERR_ARG;
    if (sigma == Fr || sigma == Fp || Fr == Fp || sigma_w == Fr || sigma_w == Fp) return SG_ERR_ARG;
    PlanView v = view(p);
    v.sigw = sigma_w;
    cudaError_t e = run_forward(p, v, sigma, Fr, Fp, stream);
    return e == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

sg_status sg_forces_wedge_backward(sg_plan* p, const void* gr, const void* gp, void* gs, void* gs_w,
                                   cudaStream_t stream)
{
    if (!p) return SG_ERR_ARG;
    if (!p->built) return SG_ERR_NOT_BUILT;
    if (!p->wedge) return SG_ERR_ARG;
    const void* ptrs[3] = {gr, gp, gs};
    for (const void* q : ptrs)
        if (!q || ((uintptr_t)q & 15)) return SG_ERR_ARG;
    if (!gs_w || ((uintptr_t)gs_w % p->elem)) return SG_ERR_ARG;
    if (gs == gr || gs == gp || gs_w == gr || gs_w == gp || gs_w == gs) return SG_ERR_ARG;
    PlanView v = view(p);
    v.gsigw = gs_w;
    cudaError_t e = run_backward(p, v, gr, gp, gs, stream);
    return e == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

sg_status sg_forces(sg_plan* p, const void* sigma, void* Fr, void* Fp, cudaStream_t stream)
{
    sg_status st = check_fields(p, sigma, Fr, Fp);
    if (st) return st;
    if (sigma == Fr || sigma == Fp || Fr == Fp) return SG_ERR_ARG;
    PlanView v = view(p);
    cudaError_t e = run_forward(p, v, sigma, Fr, Fp, stream);
    return e == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

// the plan's four timing events, created on first use
static sg_status timing_events(sg_plan* p)
{
    if (!p->have_ev) {
        for (int i = 0; i < 4; i++)
            if (cudaEventCreate(&p->ev[i]) != cudaSuccess) {
                for (int j = 0; j < i; j++) cudaEventDestroy(p->ev[j]);
                return SG_ERR_CUDA;
            }
        p->have_ev = 1;
    }
    return SG_OK;
}

// the three pass durations and the span from the recorded events
static sg_status event_times(sg_plan* p, float ms[4])
{
    SG_TRY(cudaEventSynchronize(p->ev[3]));
    for (int i = 0; i < 3; i++) SG_TRY(cudaEventElapsedTime(&ms[i], p->ev[i], p->ev[i + 1]));
    SG_TRY(cudaEventElapsedTime(&ms[3], p->ev[0], p->ev[3]));
    return SG_OK;
}

sg_status sg_forces_timed(sg_plan* p, const void* sigma, void* Fr, void* Fp, cudaStream_t stream, float ms[4])
{
    sg_status st = check_fields(p, sigma, Fr, Fp);
    if (st) return st;
    if (!ms || sigma == Fr || sigma == Fp || Fr == Fp) return SG_ERR_ARG;
    if ((st = timing_events(p))) return st;
    PlanView v = view(p);
    cudaError_t e = run_forward(p, v, sigma, Fr, Fp, stream, p->ev);
    if (e != cudaSuccess) return SG_ERR_CUDA;
    return event_times(p, ms);
}

sg_status sg_forces_backward_timed(sg_plan* p, const void* gr, const void* gp, void* gs, cudaStream_t stream,
                                   float ms[4])
{
    sg_status st = check_fields(p, gr, gp, gs);
    if (st) return st;
    if (!ms || gs == gr || gs == gp) return SG_ERR_ARG;
    if ((st = timing_events(p))) return st;
    PlanView v = view(p);
    cudaError_t e = run_backward(p, v, gr, gp, gs, stream, p->ev);
    if (e != cudaSuccess) return SG_ERR_CUDA;
    return event_times(p, ms);
}

sg_status sg_forces_backward(sg_plan* p, const void* gr, const void* gp, void* gs, cudaStream_t stream)
{
    sg_status st = check_fields(p, gr, gp, gs);
    if (st) return st;
    if (gs == gr || gs == gp) return SG_ERR_ARG;
    PlanView v = view(p);
    cudaError_t e = run_backward(p, v, gr, gp, gs, stream);
    return e == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

// Device address of a host buffer that the GPU of the plan can read and
// write directly (pinned and mapped, e.g. cudaHostAlloc or torch pin_memory),
// or null for pageable memory.
static void* mapped_host(const void* h, int device)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    (void)device;
    return a.devicePointer;
}

sg_status sg_forces_host(sg_plan* p, const void* sigma_h, void* Fr_h, void* Fp_h, cudaStream_t stream)
{
    if (!p || !sigma_h || !Fr_h || !Fp_h) return SG_ERR_ARG;
    if (!p->built) return SG_ERR_NOT_BUILT;
    if (p->wedge) return SG_ERR_UNSUPPORTED;
    const size_t bytes = (size_t)p->nu * p->nphi * p->elem;
    // Pinned, mapped buffers: the row pass reads sigma and the inverse-row
    // pass writes F_r, F_phi over the host link directly (no staging copies).
    void* ds = mapped_host(sigma_h, p->device);
    void* dr = ds ? mapped_host(Fr_h, p->device) : nullptr;
    void* dp = dr ? mapped_host(Fp_h, p->device) : nullptr;
    // (the compensated plans convert their fields on the device: staged)
    if (dp && p->dtype != SG_F32X2 && !(((uintptr_t)ds | (uintptr_t)dr | (uintptr_t)dp) & 15) && ds != dr &&
        ds != dp && dr != dp) {
        PlanView v = view(p);
        cudaError_t e = run_forward(p, v, ds, dr, dp, stream, nullptr, true);
        if (e != cudaSuccess) return SG_ERR_CUDA;
        return sg_plan_check(p, stream);  // synchronises; reports a device-side timeout
    }
    sg_status st;
    // each staging buffer on its first use (a call that could not allocate
    // them all leaves the others for the next call)
    if ((!p->h_sigma && (st = dev_alloc(p, &p->h_sigma, bytes))) || (!p->h_fr && (st = dev_alloc(p, &p->h_fr, bytes))) ||
        (!p->h_fp && (st = dev_alloc(p, &p->h_fp, bytes))))
        return st;
    SG_TRY(cudaMemcpyAsync(p->h_sigma, sigma_h, bytes, cudaMemcpyHostToDevice, stream));
    if ((st = sg_forces(p, p->h_sigma, p->h_fr, p->h_fp, stream))) return st;
    SG_TRY(cudaMemcpyAsync(Fr_h, p->h_fr, bytes, cudaMemcpyDeviceToHost, stream));
    SG_TRY(cudaMemcpyAsync(Fp_h, p->h_fp, bytes, cudaMemcpyDeviceToHost, stream));
    return sg_plan_check(p, stream);  // synchronises; reports a device-side timeout
}

static sg_status check_batch(const sg_batch_item* items, int n)
{
    if (n <= 0 || !items) return SG_ERR_ARG;
    for (int b = 0; b < n; b++) {
        if (!items[b].plan) return SG_ERR_ARG;
        sg_status st = check_fields(items[b].plan, items[b].sigma, items[b].F_r, items[b].F_phi);
        if (st) return st;
        if (items[b].plan->dtype != items[0].plan->dtype) return SG_ERR_ARG;
    }
    return SG_OK;
}

sg_status sg_batch_prepare(const sg_batch_item* items, int n, cudaStream_t stream)
{
    sg_status st = check_batch(items, n);
    return st ? st : batch_prepare(items, n, stream);
}

sg_status sg_batch_tune(const sg_batch_item* items, int n, const char* cache_path, cudaStream_t stream, float ms[2])
{
    sg_status st = check_batch(items, n);
    return st ? st : batch_tune(items, n, cache_path, stream, ms);
}

sg_status sg_forces_batched(const sg_batch_item* items, int n, cudaStream_t stream)
{
    if (n < 0 || (n > 0 && !items)) return SG_ERR_ARG;
    if (n == 0) return SG_OK;
    sg_status st0 = check_batch(items, n);
    if (st0) return st0;
    // one persistent launch when every item qualifies
    st0 = batch_forward(items, n, stream);
    if (st0 != SG_ERR_UNSUPPORTED) return st0;
    // Items of one plan share its workspace and run in item order; items of
    // different plans are independent.  With several plans, each plan's items
    // go to the plan's own stream, forked from `stream` and joined back to it
    // by events (in a captured graph: parallel branches), so that the small
    // launches of different sizes share the GPU.
    std::vector<sg_plan*> plans;
    for (int b = 0; b < n; b++)
        if (std::find(plans.begin(), plans.end(), items[b].plan) == plans.end()) plans.push_back(items[b].plan);
    if (plans.size() <= 1) {
        for (int b = 0; b < n; b++) {
            sg_status st = sg_forces(items[b].plan, items[b].sigma, items[b].F_r, items[b].F_phi, stream);
            if (st) return st;
        }
        return SG_OK;
    }
    SG_TRY(cudaEventRecord(plans[0]->bfork, stream));
    for (sg_plan* p : plans) {
        SG_TRY(cudaStreamWaitEvent(p->bstream, plans[0]->bfork, 0));
        for (int b = 0; b < n; b++) {
            if (items[b].plan != p) continue;
            sg_status st = sg_forces(p, items[b].sigma, items[b].F_r, items[b].F_phi, p->bstream);
            if (st) return st;
        }
        SG_TRY(cudaEventRecord(p->bjoin, p->bstream));
        SG_TRY(cudaStreamWaitEvent(stream, p->bjoin, 0));
    }
    return SG_OK;
}

sg_status sg_plan_check(sg_plan* p, cudaStream_t stream)
{
    if (!p) return SG_ERR_ARG;
    int h[2] = {0, 0};  // flags, site of the first failed index check
    SG_TRY(cudaMemcpyAsync(h, p->derr, 2 * sizeof(int), cudaMemcpyDeviceToHost, stream));
    SG_TRY(cudaStreamSynchronize(stream));
    if (h[0]) {
        SG_TRY(cudaMemsetAsync(p->derr, 0, 2 * sizeof(int), stream));
        SG_TRY(cudaStreamSynchronize(stream));
        if (h[0] & SG_FLAG_BOUNDS) {
            g_bounds_site.store(h[1]);
            return SG_ERR_BOUNDS;
        }
        return SG_ERR_TIMEOUT;
    }
    return SG_OK;
}

sg_status sg_plan_build_report(const sg_plan* p, int report[4])
{
    if (!p || !report) return SG_ERR_ARG;
    for (int i = 0; i < 4; i++) report[i] = p->report[i];
    return SG_OK;
}

sg_status sg_plan_kernels(sg_plan* p, double* Kr_h, double* Kp_h, cudaStream_t stream)
{
    if (!p || !Kr_h || !Kp_h) return SG_ERR_ARG;
    if (!p->built) return SG_ERR_NOT_BUILT;
    if (p->loaded) return SG_ERR_UNSUPPORTED;  // plan files carry the spectra only
    const size_t n = (size_t)(2 * p->nu - 1) * p->nphi;
    SG_TRY(cudaMemcpyAsync(Kr_h, p->keff, n * sizeof(double), cudaMemcpyDeviceToHost, stream));
    SG_TRY(cudaMemcpyAsync(Kp_h, p->keff + n, n * sizeof(double), cudaMemcpyDeviceToHost, stream));
    SG_TRY(cudaStreamSynchronize(stream));
    return SG_OK;
}

sg_status sg_plan_cells(sg_plan* p, double* cells_h, cudaStream_t stream)
{
    if (!p || !cells_h) return SG_ERR_ARG;
    if (!p->built) return SG_ERR_NOT_BUILT;
    if (p->loaded) return SG_ERR_UNSUPPORTED;
    const size_t n = (size_t)6 * (2 * p->nu + 1) * p->nphi;
    SG_TRY(cudaMemcpyAsync(cells_h, p->cells, n * sizeof(double), cudaMemcpyDeviceToHost, stream));
    SG_TRY(cudaStreamSynchronize(stream));
    return SG_OK;
}

}  // extern "C"
