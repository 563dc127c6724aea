/*
 * sg.h -- C ABI of the GB300 thin-disk self-gravity library (libsgdisk.so).
 *
 * Computes the in-plane gravitational forces F_r, F_phi of an infinitesimally
 * thin disk on a log-polar grid, following Wang, Yen & Taam, "Self-
 * gravitational force calculation of second order accuracy for
 * infinitesimally thin gaseous disks in polar coordinates":
 *
 *   grid (Sec. 3.2.1): row i has faces e^{u_min} beta^i, e^{u_min} beta^{i+1}
 *     (beta = e^{du}) and centre r_i = e^{u_min} beta^i (1 + beta) / 2;
 *     column j has centre phi_j = (j + 1/2) 2 pi / N_phi.
 *   forces (Eq. 23-24, 26-29, A7-A10): the second-order sums with the
 *     piecewise-linear density of Eq. 25 (central slopes; the density is zero
 *     outside the grid) and the exact cell-integrated kernels of Eq. 30-32 and
 *     A11-A13, whose singular self-cell values follow Sec. 4 / Eq. 33.
 *     The slope terms fold into one kernel per component, so that
 *       F_r[i,j]   = G sum_{m,l} sigma[m,l] Kr  [i-m, (j-l) mod N_phi]
 *       F_phi[i,j] = G sum_{m,l} sigma[m,l] Kphi[i-m, (j-l) mod N_phi],
 *     a convolution that is zero-padded in u = ln r and periodic in phi
 *     (Eq. 27-29 in convolution form, evaluated by FFT as in Sec. 2).
 *
 * Layout of every field (sigma, F_r, F_phi and their gradients): row-major
 * [N_u][N_phi], phi fastest, in the plan's dtype (float for SG_F32, double
 * for SG_F64 and SG_F32X2), 16-byte aligned, caller-owned device memory (or
 * host memory for the *_host entry points).
 *
 * Execution: every call that takes a stream enqueues asynchronous work on it
 * and returns without synchronising, except where stated.  sg_forces and
 * sg_forces_backward allocate nothing and may be captured in a CUDA graph;
 * so may sg_forces_batched once its list of items is prepared (it allocates
 * and synchronises only when it builds a list).  A plan must not be used by
 * two streams at once.
 *
 * Errors: no exception crosses this boundary; every call returns an
 * sg_status.  A CUDA launch error is reported as SG_ERR_CUDA; errors of
 * already enqueued work surface at the caller's next synchronisation.
 */
#ifndef SG_H
#define SG_H

#include <stddef.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SG_OK = 0,
    SG_ERR_ARG = 1,         /* null pointer, bad size, misaligned buffer, mismatched plan */
    SG_ERR_ALLOC = 2,       /* device or host allocation failed */
    SG_ERR_CUDA = 3,        /* a CUDA call or launch failed */
    SG_ERR_UNSUPPORTED = 4, /* sizes outside the supported set (see sg_plan_create) */
    SG_ERR_NOT_BUILT = 5,   /* forces requested before sg_kernels_build */
    SG_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up */
    SG_ERR_IO = 7,          /* a plan file could not be written or read, or is not one */
    SG_ERR_BOUNDS = 8       /* checked builds only (sg_checked_build): a pass's index check
                               failed and the access was skipped (sg_last_bounds_site) */
} sg_status;

/* Working precision of a plan.  SG_F32X2, the compensated FP32 plans: the
   fields are FP64 in memory (as for SG_F64), the passes carry each value as
   the unevaluated sum of two FP32 numbers (double-float arithmetic from
   error-free transformations, about 48 significant bits) on the FP32 pipes,
   and the kernel spectra are stored the same way.  Sizes as for SG_F64. */
typedef enum { SG_F32 = 0, SG_F64 = 1, SG_F32X2 = 2 } sg_dtype;

typedef struct sg_plan sg_plan;

/* Which force kernels the plan convolves with (Sec. 3.2 and 5.3).  All
   of them feed the same fold, spectra and passes; only the table of the six
   per-offset kernels differs.  Source cell (i', j') of target (i, j), offset
   (k, q) = (i - i', j - j'); M = sigma A' is the source cell's mass with
   A' = r_i' (r_i'+1/2 - r_i'-1/2) dphi its exact area. */
typedef enum {
    SG_KERNEL_SIM = 0,           /* second order: the exact cell integrals of
                                    Eq. 30-32 and A11-A13 with the central
                                    slopes of Eq. 28-29, self cell by the
                                    singular integral of Sec. 4 */
    SG_KERNEL_PARTICLE = 1,      /* the particle method: the mass M at the
                                    source centre (Eq. 35), no slopes, nothing
                                    from the target's own cell */
    SG_KERNEL_PARTICLE_PLUS = 2, /* the modified particle method (Eq. 36-37):
                                    the particle kernel plus the target cell's
                                    own exact terms sigma K^{.,0}_{0,0} +
                                    r_i delta^r K^{.,r}_{0,0} + delta^phi
                                    K^{.,phi}_{0,0} */
    SG_KERNEL_SOFTENED = 3,      /* the particle kernel with a softening length
                                    eps = soften * r_i added in quadrature to
                                    the distance (the BM08 comparison method of
                                    Sec. 5.3), own cell included */
    SG_KERNEL_POTENTIAL = 4,     /* the gravitational potential instead of the
                                    forces (the paper's Sec. 6 notes that the
                                    method carries over): the same cells and
                                    slopes with the integrand -eta / F, so
                                    Phi_i = G r_i sum sigma K^P; sg_forces then
                                    writes Phi into F_r and zeros into F_phi
                                    (up to the rounding of the inverse
                                    transform), and the adjoint is that map's
                                    transpose.  Build FP32 plans with
                                    weight_p = 1: Phi carries r_i and the
                                    kernel grows like r'/r toward outer
                                    sources, which p = 1 evens out */
    SG_KERNEL_CARTESIAN = 5      /* the Cartesian second-order scheme of
                                    Sec. 3.1.1 (Eq. 6-15, closed forms of
                                    App. A) on square cells of side du: the
                                    plan's rows are x (N_x = N_u, zero-padded
                                    by the passes), its columns y with
                                    N_phi = 2 N_y, the last N_y of them the
                                    padding that makes the periodic direction
                                    a linear convolution.  sigma must be zero
                                    in columns N_y .. N_phi - 1; F there is
                                    not a force.  F_r is F^x, F_phi is F^y;
                                    central slopes with sigma zero outside
                                    the grid, as for SG_KERNEL_SIM; u_min is
                                    unused.  weight_p and radial_edges must
                                    be 0; sg_plan_cells returns zeros (the
                                    kernels are folded from their closed
                                    forms directly) */
} sg_kernel_kind;

/* Options of the one-time kernel preparation (Sec. 2: the kernels depend
   only on the grid, so they are built once and kept).  Pass NULL for the defaults; a zero-filled struct
   gives them too. */
typedef struct {
    double rtol;   /* relative tolerance of the cell quadrature; default 1e-14 */
    int weight_p;  /* weighting exponent p of sigma e^{p u} (the kernels carry
                      beta^{p k}, the result e^{-p u}); algebraically neutral;
                      default 0 */
    int kind;      /* sg_kernel_kind; default SG_KERNEL_SIM (0) */
    double soften; /* SG_KERNEL_SOFTENED: eps / r_i, > 0; ignored otherwise */
    int n_tpz;     /* SG_KERNEL_SIM: 0 (default) for the exact cell integrals;
                      N in [1, 1024] for the trapezoidal rule of Eq. 41-43
                      with N trapezoids per cell in phi (exact in r) for
                      K^{r,0}, K^{r,r}, K^{r,phi} and K^{phi,phi}, the own
                      cell still exact (Sec. 4; the paper's SIM uses 19);
                      ignored by the particle kinds */
    int radial_edges; /* 0 (default): sigma is zero outside the grid and the
                      central radial slopes of Eq. 25 apply wherever the
                      stencil touches it, ghost rows 0 and N_u + 1 included
                      (a pure convolution); 1: no ghost rows, and the slopes
                      of the first and last rows are one-sided, (sigma_2 -
                      sigma_1) / (r_2 - r_1) and (sigma_N - sigma_{N-1}) /
                      (r_N - r_{N-1}).  With 1 a rank-4 correction per phi
                      mode runs after the column pass (and its transpose in
                      the adjoint), and the forces keep second order up to
                      the radial edges when sigma does not vanish there */
    int wedge;     /* 0 (default); 1: the origin wedge of Sec. 3.2.1, the cells
                      [0, r_in] x [phi_{j-1/2}, phi_{j+1/2}] below the first
                      row (r_in = e^{u_min}), enter through the third terms of
                      Eq. 27-29: single sums over N_phi wedge densities given
                      per call to sg_forces_wedge.  The wedge's density is its
                      value at r_in / 2, its radial slope one-sided toward
                      the first row, its azimuthal slope central.  Needs
                      radial_edges = 1 (the wedge replaces the inner ghost
                      row) and SG_KERNEL_SIM or SG_KERNEL_POTENTIAL */
    int short_dft; /* 0 (default): every azimuthal transform by FFT.  1: the
                      azimuthal (row) transforms of the forward call (sigma ->
                      half spectra, the column pass's spectra -> F_r, F_phi)
                      and of the adjoint (gF_r, gF_phi -> half spectra, the
                      column pass's spectrum -> gsigma) as products with the
                      N_phi x N_phi real DFT matrix on the tensor cores
                      (tcgen05, kind::tf32): every operand split into a TF32
                      part and an FP32 remainder, three products per pair
                      (hi hi + hi lo + lo hi), FP32 accumulation, so the
                      result keeps FP32 accuracy.  Only SG_F32 plans with
                      32 <= N_phi <= 256 (else SG_ERR_UNSUPPORTED).  The
                      option is not kept by sg_plan_save.  In sg_forces_batched
                      such plans with N_phi = 256 keep the persistent path:
                      their row passes run as two batched tensor-core launches
                      (before and after the column kernel), their column items
                      in the persistent column kernel */
} sg_build_opts;

/*
 * Create a plan for an N_u x N_phi grid.
 *   N_u, N_phi : powers of two; 4 <= N_u <= 4096 and 4 <= N_phi <= 8192
 *                for SG_F32, 4 <= N_u <= 2048 and 4 <= N_phi <= 4096 for
 *                SG_F64 (one transform must fit one block's registers and
 *                shared memory); anything else returns SG_ERR_UNSUPPORTED.
 *   u_min      : ln of the inner face radius (Sec. 3.2.1, M_in).
 *   du         : log-radial step, beta = e^{du} > 1.
 *   G          : gravitational constant (the paper uses G = 1).
 *   dtype      : working precision of the forward/backward passes and of
 *                the stored kernel spectra.  The kernels are always built in
 *                FP64.
 * Allocates the plan's device memory (spectra, workspace, twiddle tables) on
 * the current device; the plan owns it until sg_plan_destroy.  *out is set
 * only on SG_OK.
 */
sg_status sg_plan_create(sg_plan** out, int N_u, int N_phi, double u_min, double du, double G, sg_dtype dtype);

/*
 * Build the cell-integrated kernels (Eq. 30-32, A11-A13; self cell per
 * Sec. 4), fold the slope terms, apply G beta^{p k} and transform to spectra
 * (FP64, stored in the plan's dtype).  opts may be NULL.  opts->kind
 * selects the particle-method kernels of sg_kernel_kind instead; they go
 * through the same fold (their slope cells are zero away from the own
 * cell).  Runs on stream and blocks the host until it completes; must be
 * called once before sg_forces (again to rebuild with other options).
 * Returns SG_ERR_TIMEOUT (the plan is still usable) if a cell integral
 * could not reach the tolerance within the quadrature's budget, and
 * SG_ERR_ARG for an unknown kind, soften <= 0 with SG_KERNEL_SOFTENED,
 * n_tpz outside [0, 1024] (or n_tpz > 0 with another kind than
 * SG_KERNEL_SIM), radial_edges not 0 or 1, |weight_p| > 8, weight_p or
 * radial_edges not 0 with SG_KERNEL_CARTESIAN, or wedge not 0 or 1 (1 without
 * radial_edges = 1, or with a kind other than SG_KERNEL_SIM and
 * SG_KERNEL_POTENTIAL).  wedge = 1 also allocates the plan's wedge tables,
 * 4 (N_phi/2 + 1) N_u values of the working dtype, and for the build an FP64
 * scratch of 6 N_u N_phi values.
 * Allocates and frees FP64 scratch for the spectra; radial_edges = 1 also
 * allocates the plan's edge tables, 2 (N_phi/2 + 1)(2 N_u + 1) values of
 * the working dtype.  Any other error than SG_ERR_TIMEOUT (SG_ERR_ALLOC,
 * SG_ERR_CUDA, also from the set-up of sg_forces_noalloc at the end) leaves
 * the plan unbuilt: SG_ERR_NOT_BUILT until a build succeeds.
 */
sg_status sg_kernels_build(sg_plan* plan, const sg_build_opts* opts, cudaStream_t stream);

/*
 * Forward pass: F_r, F_phi from sigma (device pointers, layout above).
 * F_r and F_phi are overwritten.  sigma may not alias F_r or F_phi.
 * SG_ERR_NOT_BUILT before sg_kernels_build.  The column pass waits for its
 * asynchronous input copies with a time limit (about a second); if that
 * ever runs out the outputs are invalid and the plan's error flag is set
 * (sg_plan_check).
 */
sg_status sg_forces(sg_plan* plan, const void* sigma, void* F_r, void* F_phi, cudaStream_t stream);

/*
 * Adjoint: gsigma = A^T (gF_r, gF_phi) where A is the linear map of
 * sg_forces, i.e. gsigma[m,l] = G sum_{i,j} gF_r[i,j] Kr[i-m, j-l]
 *                                      + gF_phi[i,j] Kphi[i-m, j-l].
 * gsigma is overwritten (not accumulated).
 */
sg_status sg_forces_backward(sg_plan* plan, const void* gF_r, const void* gF_phi, void* gsigma,
                             cudaStream_t stream);

/*
 * Forces with the origin wedge (a plan built with wedge = 1): as sg_forces,
 * plus the wedge's single sums (the third terms of Eq. 27-29 and A8-A10)
 * over sigma_w, the N_phi wedge densities (device, working dtype, contiguous,
 * aligned to the element size; the caller keeps ownership).  The update runs
 * inside the forward column pass (FP32, N_u >= 8) or between the column
 * and inverse-row passes.  sg_forces, sg_forces_timed, sg_forces_backward,
 * sg_forces_host, sg_forces_batched and sg_forces_noalloc return
 * SG_ERR_UNSUPPORTED on such a plan.  SG_ERR_ARG if the plan has no wedge,
 * for null, misaligned or aliased buffers.
 */
sg_status sg_forces_wedge(sg_plan* plan, const void* sigma, const void* sigma_w, void* F_r, void* F_phi,
                          cudaStream_t stream);

/*
 * The adjoint of sg_forces_wedge: gsigma (N_u x N_phi) and gsigma_w (N_phi)
 * from gF_r, gF_phi.  Same rules as sg_forces_backward.
 */
sg_status sg_forces_wedge_backward(sg_plan* plan, const void* gF_r, const void* gF_phi, void* gsigma,
                                   void* gsigma_w, cudaStream_t stream);

/*
 * Same as sg_forces with HOST buffers, then synchronises the stream and
 * returns what sg_plan_check returns.  When all three buffers are pinned and
 * mapped into the device's address space (cudaHostAlloc, cudaHostRegister
 * with mapping, torch pin_memory), the row pass reads sigma and the
 * inverse-row pass writes F_r and F_phi over the host link directly, with
 * no staging copies.  Otherwise sigma is copied to plan-owned device staging
 * buffers (allocated on first use), the forward pass runs there, and F_r,
 * F_phi are copied back, all on stream.
 */
sg_status sg_forces_host(sg_plan* plan, const void* sigma_h, void* F_r_h, void* F_phi_h, cudaStream_t stream);

/*
 * sg_forces with per-pass timing: records CUDA events (owned by the plan,
 * created on first use) on stream before the row pass, between the passes
 * and after the inverse row pass, synchronises the stream and writes the
 * three pass durations in milliseconds to ms[0..2] (rows, columns, inverse
 * rows) and the whole span to ms[3].  For measurement; same results as
 * sg_forces.
 */
sg_status sg_forces_timed(sg_plan* plan, const void* sigma, void* F_r, void* F_phi, cudaStream_t stream,
                          float ms[4]);

/*
 * sg_forces_backward with per-pass timing, as sg_forces_timed: ms[0..2] are
 * the adjoint's row, column and inverse-row passes (any edge or wedge
 * update counted with the columns), ms[3] the whole span.  Synchronises the
 * stream.  Same results and errors as sg_forces_backward.
 */
sg_status sg_forces_backward_timed(sg_plan* plan, const void* gF_r, const void* gF_phi, void* gsigma,
                                   cudaStream_t stream, float ms[4]);

/*
 * sg_forces for callers that cannot allocate device memory when they compute
 * forces (their memory belongs to another framework's allocator, or their
 * loop may not allocate or synchronise): the scratch that sg_forces takes
 * from the plan comes instead from a fixed 24 MiB array that the library
 * reserves on each device where it is used, until the process exits.  The
 * paper has no counterpart; this is a deployment variant of sg_forces with
 * the same arguments and results.
 *   - Allocates nothing, and loads no module.  The plan must be built or
 *     loaded (that allocated earlier): sg_kernels_build and sg_plan_load look
 *     up the array's device address on the plan's device and run one forward
 *     pass through it, which loads the array's module and the pass kernels'
 *     (under lazy module loading a module loads, and may allocate, at its
 *     first use).
 *   - Supported up to 3 N_u (N_phi/2) complex values of scratch: N_u N_phi <=
 *     2^21 cells in SG_F32, 2^20 in SG_F64; larger plans, and SG_F32X2
 *     plans (whose conversions use working fields of the plan), get
 *     SG_ERR_UNSUPPORTED.  The plan's device must be the current device
 *     (SG_ERR_ARG otherwise).
 *   - All calls on a device share the array: calls whose work overlaps on
 *     the GPU (other streams, other threads) race and must be serialised.
 *     Nothing in it needs to start at zero.
 */
sg_status sg_forces_noalloc(sg_plan* plan, const void* sigma, void* F_r, void* F_phi, cudaStream_t stream);

/* One disk of a batch: its plan (built) and its device fields. */
typedef struct {
    sg_plan* plan;
    const void* sigma;
    void* F_r;
    void* F_phi;
} sg_batch_item;

/*
 * Forward pass for n disks of possibly different sizes, all of one dtype.
 * items is a host array; every item is validated before any work is
 * enqueued.  The paper prepares each disk's kernels once and evaluates the
 * forces every step (Sec. 2); this is that step for many disks at once.
 *   - One persistent launch when every plan is SG_F32 with both transform
 *     lengths in 2^8 .. 2^12 (N_phi 256 .. 4096, N_u 128 .. 2048) and
 *     neither radial_edges nor wedge: a kernel resident on every SM takes
 *     work items -- row units of a disk's R2C pass, mode groups of its
 *     column pass, row units of its C2R pass -- from a queue in device
 *     memory, each disk's column items after all its row items and its C2R
 *     items after all its column items (per-disk counters, waits bounded
 *     like the passes' copy waits: a wait that runs out sets the plan's
 *     flag, see sg_plan_check).  Each disk's forces are bit-equal to
 *     sg_forces on the same plan.  The work list is built on the host the
 *     first time a list of items (plans and buffers, in order) is seen, or
 *     by sg_batch_prepare / sg_batch_tune; its schedule is the one
 *     sg_batch_tune chose for this set of sizes, if any.
 *   - Otherwise, and for a list first seen while the stream is being
 *     captured: items that share a plan share its workspace and run in
 *     item order; the items of different plans run on the plans' own
 *     streams, forked from `stream` and joined back to it by events.
 * Capturable in a CUDA graph (prepare the list first).  A plan may appear
 * in only one batch or call in flight at a time, and two calls with the
 * same list must not overlap.  Allocates only when it builds a work list.
 */
sg_status sg_forces_batched(const sg_batch_item* items, int n, cudaStream_t stream);

/*
 * Builds the persistent path's work list for these items (synchronises
 * stream) so that later sg_forces_batched calls with the same items, also
 * captured ones, take it.  Allocates the list's device memory, held until
 * one of the plans is destroyed: each item's own intermediate spectra (12
 * bytes per cell; items may share a plan), a descriptor of 256 bytes per
 * item and 8 bytes per work item.  The library keeps the 4 lists prepared
 * last (a call with a new list of items builds one: host work and a
 * synchronising copy).  SG_ERR_UNSUPPORTED if the items do not qualify
 * for the persistent path; SG_ERR_ARG while stream is being captured.
 */
sg_status sg_batch_prepare(const sg_batch_item* items, int n, cudaStream_t stream);

/*
 * Tunes the persistent path's schedule for this set of disk sizes: the lag
 * between an item and its dependencies in the queue, the disk order, and
 * per size class (N_u, N_phi) the row units per row item and the mode
 * groups per column item.  Each candidate runs the batch (the items' F_r,
 * F_phi are overwritten) and the fastest is kept.  cache_path (or NULL): a
 * text file of schedules, one line per set of sizes and SM count; a
 * schedule found there is taken without tuning, a new one is appended.
 * Then prepares the items' list with the schedule (as sg_batch_prepare).
 * ms[0], ms[1] (ms may be NULL): the batch's time with the default and with
 * the chosen schedule.  Synchronises stream.  SG_ERR_UNSUPPORTED as
 * sg_batch_prepare; SG_ERR_IO if the file cannot be appended to.
 */
sg_status sg_batch_tune(const sg_batch_item* items, int n, const char* cache_path, cudaStream_t stream, float ms[2]);

sg_status sg_plan_destroy(sg_plan* plan);

const char* sg_status_string(sg_status s);

/* ---- plan introspection (host-side; no GPU work) ---------------------- */

/* Fills dims[0..3] = N_u, N_phi, dtype, built (0/1). */
sg_status sg_plan_info(const sg_plan* plan, int dims[4]);

/*
 * Copies the plan's folded FP64 kernels to host memory (for checking the
 * kernel builder): Kr, Kphi each [(2 N_u - 1) * N_phi] doubles, row k + N_u
 * - 1 for k in [-(N_u-1), N_u-1], column q in [0, N_phi); these are
 * K^eff (without G and without the beta^{pk} weight).  Synchronises stream.
 */
sg_status sg_plan_kernels(sg_plan* plan, double* Kr_h, double* Kphi_h, cudaStream_t stream);

/*
 * Copies the six raw FP64 cell kernels [6][(2 N_u + 1) * N_phi] (k in
 * [-N_u, N_u], q in [0, N_phi); order K^{r,0}, K^{r,r}, K^{r,phi},
 * K^{phi,0}, K^{phi,r}, K^{phi,phi}) to host memory.  Synchronises stream.
 * For the particle kinds, K^{r,0} and K^{phi,0} hold the point kernels
 * M K^{.,p} / sigma and the other four are zero, except the own cell's
 * exact values at (0, 0) for SG_KERNEL_PARTICLE_PLUS.
 */
sg_status sg_plan_cells(sg_plan* plan, double* cells_h, cudaStream_t stream);

/*
 * Convergence report of the last sg_kernels_build: report[0] = bit 1 if some
 * cell integrals stopped at the quadrature budget, bit 2 if the self-cell
 * rule did not reach its tolerance, bit 4 if some wedge integrals stopped at
 * the budget; report[1] = number of such offsets; report[2], report[3] =
 * (k, q) of one of them (for a wedge cell: (target row, q)).  All zero after
 * a clean build.
 */
sg_status sg_plan_build_report(const sg_plan* plan, int report[4]);

/*
 * Device-side status of the work enqueued so far with this plan: reads (and
 * clears) the plan's error flags after synchronising stream.  SG_ERR_TIMEOUT
 * means a pass gave up waiting for its asynchronous input copies (its
 * results are invalid); SG_ERR_BOUNDS (checked builds only) that an index
 * check of a pass failed (its results are invalid; the failing check's site
 * number is kept for sg_last_bounds_site); SG_OK otherwise.
 */
sg_status sg_plan_check(sg_plan* plan, cudaStream_t stream);

/*
 * Budget of the device-side waits of the passes for their asynchronous input
 * copies, in seconds (default 1; at most 60).  A pass whose copies do not
 * arrive within it sets the plan's error flag (sg_plan_check returns
 * SG_ERR_TIMEOUT), waits up to one more second for the copies still in
 * flight, and leaves its outputs unwritten.  0 makes every pass give up at
 * once: a test of that error path.  Synchronous; not for use while work of
 * the plan is in flight.
 */
sg_status sg_plan_set_wait_limit(sg_plan* plan, double seconds);

/*
 * Checkpoint of a built plan (the paper prepares its kernels once and keeps
 * them in memory, Sec. 2): sg_plan_save writes the kernel spectra and the
 * weight rows in the working dtype, with the plan's sizes, grid, G,
 * weighting exponent and build tolerance, to a file (synchronises stream).
 * sg_plan_load creates a built plan from such a file (on the current
 * device; synchronises stream), which computes the same forces bit for bit
 * without rebuilding.  A loaded plan holds no FP64 build tables:
 * sg_plan_kernels and sg_plan_cells return SG_ERR_UNSUPPORTED for it.
 * SG_ERR_IO: the file cannot be written or read, is truncated or too long,
 * or is not a plan file of this library.  A plan built with radial_edges = 1
 * is not saved (SG_ERR_UNSUPPORTED).
 */
sg_status sg_plan_save(const sg_plan* plan, const char* path, cudaStream_t stream);
sg_status sg_plan_load(sg_plan** out, const char* path, cudaStream_t stream);

/*
 * The tensor-core DFT matrices of short_dft plans with N_phi points per row,
 * computed on the host (no device needed): out receives 4 N_phi^2 floats,
 * first the forward matrix D (y = x D: y[0] = X(0), y[1] = X(N/2), y[2m],
 * y[2m+1] = Re, Im X(m) of X(m) = sum_n x_n e^{-2 pi i n m / N}), then the
 * inverse matrix E (F = b E for the packed half spectrum b of a real row:
 * E[0][k] = 1, E[1][k] = (-1)^k, E[2m][k] = 2 cos, E[2m+1][k] = -2 sin of
 * 2 pi m k / N).  Each matrix is stored as its TF32 part, then its FP32
 * remainder, each as [N / NT column tiles][N / 32 K chunks][NT x 32 values]
 * with NT = min(N, 64), a tile's entry (output column j, input index k) at
 * 32 (8 (j / 8) + k / 4) + 4 (j % 8) + k % 4 (core matrices of 8 x 4 values,
 * K-major).  SG_ERR_UNSUPPORTED unless 32 <= N_phi <= 256 is a power of two.
 */
sg_status sg_dft_tc_matrices(int N_phi, float* out);

/* Bytes of device memory the plan holds. */
size_t sg_plan_device_bytes(const sg_plan* plan);

/*
 * Checked builds.  The library compiled with -DSG_DEBUG (the build script's
 * `checked` variant, libsgdisk_checked.so) tests, before every global copy,
 * store and tensor-copy coordinate of its pass kernels, that the access
 * stays inside its buffer and inside the block's shared memory; a failed
 * test skips the access and flags the plan (sg_plan_check returns
 * SG_ERR_BOUNDS).  sg_checked_build returns 1 for such a library, 0 for the
 * ordinary one; sg_last_bounds_site the site number of the last failure
 * sg_plan_check reported in this process (0: none).
 */
int sg_checked_build(void);
int sg_last_bounds_site(void);

/*
 * Testing hook for the SG_ERR_ALLOC paths: after the next `after` device
 * allocations of this library succeed, every further one fails as if the
 * device were out of memory, until the hook is called again; after < 0
 * (the initial state) lets every allocation go to the device.  Returns the
 * number of allocations that were still to succeed before the call (or -1),
 * so that after(N) ... after(-1) counts the allocations made in between.
 * Process-wide.  Every call that allocates releases what it took when a
 * later allocation fails: sg_plan_create and sg_plan_load return no plan,
 * sg_kernels_build leaves the plan unbuilt, sg_forces_host returns before
 * any copy (its staging buffers are taken on a later call).
 */
int sg_test_fail_alloc(int after);
/* Device allocations of this library not yet released (process-wide). */
int sg_test_live_allocations(void);

#ifdef __cplusplus
}
#endif
#endif /* SG_H */
