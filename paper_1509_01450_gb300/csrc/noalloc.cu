// noalloc.cu -- sg_forces_noalloc: the forward pass with its scratch in a
// fixed, statically reserved device array instead of the plan's workspace.
//
// Who needs this: code that must not call cudaMalloc at the moment it
// computes forces -- for example a host application whose device memory is
// handed out by another framework's allocator, a real-time loop where an
// allocation (and the implicit synchronisation it can cause) is not
// allowed, or a pool-limited process that has already committed its memory.
// Such a caller still creates and builds a plan beforehand (that allocates);
// this call then allocates nothing.
//
// The scratch is SG_NOALLOC_BYTES of __device__ memory that every GPU which
// loads this file's module reserves until the process exits.  All calls on
// a device share it, so calls whose work overlaps on the GPU (two streams,
// or two threads) race on it and must be serialised by the caller.  Building
// or loading a plan (sg_kernels_build, sg_plan_load) looks up the array's
// device address (cudaGetSymbolAddress) with the plan's device current and
// runs one forward pass through it, which loads this module and the pass
// kernels' modules; under lazy module loading a module is loaded, and may
// allocate, at its first use, and that first use is then the build's.  No
// part of the scratch needs to start at zero: the row pass writes every
// element the column pass reads, and the column pass writes every element
// the inverse row pass reads.
#include <mutex>

#include "sg_internal.cuh"

using namespace sg;

// 24 MiB: three half-spectrum buffers of N_u x N_phi/2 complex values, i.e.
// 12 bytes per grid cell in FP32 (up to 2^21 cells, e.g. 1024 x 2048) or 24
// bytes per cell in FP64 (up to 2^20 cells).
#define SG_NOALLOC_BYTES (24u << 20)
#define SG_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char sg_noalloc_scratch[SG_NOALLOC_BYTES];

static void* g_scratch[SG_NOALLOC_MAX_DEVICES];
static std::mutex g_scratch_mutex;

// Device address of the scratch on the current device (looked up once per
// device; host code cannot use the symbol's host-side name as an address).
// Under lazy module loading the first lookup also loads this file's module
// and with it the array.
static sg_status scratch_address(void** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SG_ERR_CUDA;
    if (dev < 0 || dev >= SG_NOALLOC_MAX_DEVICES) return SG_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, sg_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SG_ERR_CUDA;
        }
        g_scratch[dev] = p;
    }
    *out = g_scratch[dev];
    return SG_OK;
}

// one half-spectrum buffer of the plan, and whether three fit the scratch
static size_t half_bytes(const sg_plan* p) { return (size_t)p->nu * (p->nphi / 2) * 2 * p->elem; }
// the compensated plans convert their fields through working buffers of their own: not served here
static bool fits(const sg_plan* p) { return p->dtype != SG_F32X2 && 3 * half_bytes(p) <= SG_NOALLOC_BYTES; }

// the forward passes over the scratch (arguments checked by the caller)
static sg_status noalloc_forward(sg_plan* p, const void* sigma, void* F_r, void* F_phi, cudaStream_t stream)
{
    const size_t half = half_bytes(p);
    void* scratch = nullptr;
    sg_status st = scratch_address(&scratch);
    if (st) return st;
    PlanView v = view(p);
    v.wa = scratch;
    v.wb = (unsigned char*)scratch + half;
    v.wc = (unsigned char*)scratch + 2 * half;
    {
        // tensor maps of the row passes over the scratch (host-side encoding only)
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (!p->have_na_maps) {
            void* const bufs[3] = {v.wa, v.wb, v.wc};
            make_row_maps(p->nu, p->nphi, p->elem, bufs, p->na_maps);
            p->have_na_imaps = p->dtype == SG_F32 && make_pair_maps(p->nu, p->nphi, v.wa, v.wb, p->na_imaps) ? 1 : 0;
            p->have_na_maps = 1;
        }
    }
    v.maps = p->na_maps;
    v.imaps = p->have_na_imaps ? p->na_imaps : nullptr;
    cudaError_t e = p->dtype == SG_F32
                        ? launch_forward<float>(v, (const float*)sigma, (float*)F_r, (float*)F_phi, stream)
                        : launch_forward<double>(v, (const double*)sigma, (double*)F_r, (double*)F_phi, stream);
    return e == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

namespace sg {
// Called by the plan build and load, which allocate anyway: resolve the
// scratch address on the plan's device and run one forward pass through
// the scratch on a zero density, so that every module of the path is loaded
// (under lazy module loading a module loads, and may allocate, at its first
// use) and every launch attribute set; sg_forces_noalloc then loads and
// allocates nothing.  Plans the entry point refuses are skipped.
sg_status noalloc_prepare(sg_plan* p, cudaStream_t stream)
{
    if (p->wedge || !fits(p)) return SG_OK;
    const size_t field = (size_t)p->nu * p->nphi * p->elem;
    unsigned char* buf = nullptr;
    if (sg_malloc((void**)&buf, 3 * field) != cudaSuccess) {
        cudaGetLastError();
        return SG_ERR_ALLOC;
    }
    sg_status st = SG_OK;
    if (cudaMemsetAsync(buf, 0, field, stream) != cudaSuccess)
        st = SG_ERR_CUDA;
    else
        st = noalloc_forward(p, buf, buf + field, buf + 2 * field, stream);
    if (cudaStreamSynchronize(stream) != cudaSuccess && st == SG_OK) st = SG_ERR_CUDA;
    sg_free(buf);
    return st;
}
}  // namespace sg

extern "C" sg_status sg_forces_noalloc(sg_plan* p, const void* sigma, void* F_r, void* F_phi, cudaStream_t stream)
{
    if (!p) return SG_ERR_ARG;
    if (!p->built) return SG_ERR_NOT_BUILT;
    if (p->wedge) return SG_ERR_UNSUPPORTED;  // the wedge densities come through sg_forces_wedge
    const void* ptrs[3] = {sigma, F_r, F_phi};
    for (const void* q : ptrs)
        if (!q || ((uintptr_t)q & 15)) return SG_ERR_ARG;
    if (sigma == F_r || sigma == F_phi || F_r == F_phi) return SG_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SG_ERR_CUDA;
    if (dev != p->device) return SG_ERR_ARG;  // the plan's spectra live on p->device
    if (!fits(p)) return SG_ERR_UNSUPPORTED;
    return noalloc_forward(p, sigma, F_r, F_phi, stream);
}
