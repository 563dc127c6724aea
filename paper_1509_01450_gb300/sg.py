"""Thin Python binding of libsgdisk.so (include/sg.h).

Argument marshalling only: every step of the force computation runs in the
library's CUDA kernels.  PyTorch provides device memory and the current
stream.  If the library has not been built the calls raise; there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SG_LIBRARY_VARIANT=checked loads the index-checked build (libsgdisk_checked.so,
# python -m paper_1509_01450_gb300.build --checked) instead of the ordinary one
_VARIANT = os.environ.get("SG_LIBRARY_VARIANT", "")
if _VARIANT not in ("", "checked"):
    raise RuntimeError(f"SG_LIBRARY_VARIANT={_VARIANT!r}: expected 'checked' or nothing")
LIB_PATH = os.path.join(_HERE, "libsgdisk_checked.so" if _VARIANT == "checked" else "libsgdisk.so")

(SG_OK, SG_ERR_ARG, SG_ERR_ALLOC, SG_ERR_CUDA, SG_ERR_UNSUPPORTED, SG_ERR_NOT_BUILT, SG_ERR_TIMEOUT, SG_ERR_IO,
 SG_ERR_BOUNDS) = range(9)
SG_F32, SG_F64, SG_F32X2 = 0, 1, 2
# plan precisions by name: FP32, FP64, and the compensated FP32 plans
# (double-float passes on the FP32 pipes; fields FP64 like SG_F64)
PRECISIONS = {"float32": SG_F32, "f32": SG_F32, "torch.float32": SG_F32, "float64": SG_F64, "f64": SG_F64,
              "torch.float64": SG_F64, "float32x2": SG_F32X2, "f32x2": SG_F32X2, "compensated": SG_F32X2}

EXPORTS = ("sg_plan_create", "sg_kernels_build", "sg_forces", "sg_forces_backward", "sg_forces_host", "sg_forces_timed",
           "sg_forces_backward_timed",
           "sg_forces_batched", "sg_batch_prepare", "sg_batch_tune", "sg_plan_destroy", "sg_status_string", "sg_plan_info",
           "sg_plan_kernels", "sg_plan_cells", "sg_plan_device_bytes", "sg_plan_build_report", "sg_forces_noalloc", "sg_plan_check",
           "sg_plan_set_wait_limit", "sg_plan_save", "sg_plan_load", "sg_forces_wedge", "sg_forces_wedge_backward",
           "sg_checked_build", "sg_last_bounds_site", "sg_test_fail_alloc", "sg_test_live_allocations",
           "sg_dft_tc_matrices")


class SgError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


# sg_kernel_kind: which force kernels a plan is built with (Sec. 3.2, 5.3)
SG_KERNEL_SIM = 0            # second order: exact cell integrals, central slopes, singular own cell
SG_KERNEL_PARTICLE = 1       # point mass at each source centre (Eq. 35)
SG_KERNEL_PARTICLE_PLUS = 2  # point masses plus the own cell's exact terms (Eq. 36-37)
SG_KERNEL_SOFTENED = 3       # point masses with softening eps = soften r_i (BM08 comparison)
SG_KERNEL_POTENTIAL = 4      # the potential Phi (into F_r; F_phi zero) with the same construction
SG_KERNEL_CARTESIAN = 5      # the Cartesian scheme on N_x x (2 N_y) with the y-padding zero
KERNEL_KINDS = {"sim": SG_KERNEL_SIM, "particle": SG_KERNEL_PARTICLE, "particle+": SG_KERNEL_PARTICLE_PLUS,
                "softened": SG_KERNEL_SOFTENED, "potential": SG_KERNEL_POTENTIAL, "cartesian": SG_KERNEL_CARTESIAN}


class BuildOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("weight_p", ctypes.c_int), ("kind", ctypes.c_int),
                ("soften", ctypes.c_double), ("n_tpz", ctypes.c_int), ("radial_edges", ctypes.c_int),
                ("wedge", ctypes.c_int), ("short_dft", ctypes.c_int)]


class BatchItem(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("sigma", ctypes.c_void_p), ("F_r", ctypes.c_void_p),
                ("F_phi", ctypes.c_void_p)]


_lib = None


def lib():
    """Load libsgdisk.so (raises if it is missing: no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run `python -m paper_1509_01450_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.sg_plan_create.argtypes = [ctypes.POINTER(vp), ip, ip, dp, dp, dp, ip]
        L.sg_kernels_build.argtypes = [vp, ctypes.POINTER(BuildOpts), vp]
        L.sg_forces.argtypes = [vp, vp, vp, vp, vp]
        L.sg_forces_backward.argtypes = [vp, vp, vp, vp, vp]
        L.sg_forces_host.argtypes = [vp, vp, vp, vp, vp]
        L.sg_forces_timed.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_float)]
        L.sg_forces_backward_timed.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_float)]
        L.sg_forces_noalloc.argtypes = [vp, vp, vp, vp, vp]
        L.sg_forces_wedge.argtypes = [vp, vp, vp, vp, vp, vp]
        L.sg_forces_wedge_backward.argtypes = [vp, vp, vp, vp, vp, vp]
        L.sg_forces_batched.argtypes = [ctypes.POINTER(BatchItem), ip, vp]
        L.sg_batch_prepare.argtypes = [ctypes.POINTER(BatchItem), ip, vp]
        L.sg_batch_tune.argtypes = [ctypes.POINTER(BatchItem), ip, ctypes.c_char_p, vp, ctypes.POINTER(ctypes.c_float)]
        L.sg_plan_destroy.argtypes = [vp]
        L.sg_status_string.argtypes = [ip]
        L.sg_status_string.restype = ctypes.c_char_p
        L.sg_plan_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
        L.sg_plan_kernels.argtypes = [vp, ctypes.POINTER(dp), ctypes.POINTER(dp), vp]
        L.sg_plan_cells.argtypes = [vp, ctypes.POINTER(dp), vp]
        L.sg_plan_build_report.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
        L.sg_plan_check.argtypes = [vp, vp]
        L.sg_plan_set_wait_limit.argtypes = [vp, dp]
        L.sg_plan_save.argtypes = [vp, ctypes.c_char_p, vp]
        L.sg_plan_load.argtypes = [ctypes.POINTER(vp), ctypes.c_char_p, vp]
        L.sg_checked_build.argtypes = []
        L.sg_last_bounds_site.argtypes = []
        L.sg_test_fail_alloc.argtypes = [ip]
        L.sg_test_live_allocations.argtypes = []
        L.sg_dft_tc_matrices.argtypes = [ip, ctypes.POINTER(ctypes.c_float)]
        L.sg_plan_device_bytes.argtypes = [vp]
        L.sg_plan_device_bytes.restype = ctypes.c_size_t
        for name in EXPORTS:
            if name not in ("sg_status_string", "sg_plan_device_bytes"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().sg_status_string(int(status)).decode()


def _check(status: int, what: str):
    if status != SG_OK:
        raise SgError(status, what)


def _stream(stream):
    import torch

    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """A log-polar grid with its prepared kernel spectra (sg_plan)."""

    def __init__(self, nu: int, nphi: int, u_min: float, du: float, G: float = 1.0, dtype="float32"):
        import torch

        if str(dtype) not in PRECISIONS:
            raise ValueError(f"dtype {dtype!r}: expected one of {sorted(PRECISIONS)}")
        self.code = PRECISIONS[str(dtype)]
        # the fields' torch dtype (FP64 for the compensated plans too)
        self.dtype = torch.float32 if self.code == SG_F32 else torch.float64
        self.nu, self.nphi, self.u_min, self.du, self.G = int(nu), int(nphi), float(u_min), float(du), float(G)
        h = ctypes.c_void_p()
        _check(lib().sg_plan_create(ctypes.byref(h), self.nu, self.nphi, self.u_min, self.du, self.G, self.code),
               "sg_plan_create")
        self.handle = h

    # -- one-time preparation ------------------------------------------------
    def build(self, rtol: float = 1e-14, weight_p: int = 0, kind="sim", soften: float = 0.0, n_tpz: int = 0,
              radial_edges: int = 0, wedge: int = 0, short_dft: int = 0, stream=None):
        """Build the kernels.  kind: "sim" (default; n_tpz > 0 for the
        trapezoidal rule of Eq. 41-43 with n_tpz trapezoids), "particle",
        "particle+" or "softened" (with soften = eps / r_i), "potential"
        (Phi into F_r; weight_p = 1 for FP32), "cartesian" (square cells of
        side du; N_phi = 2 N_y with sigma zero in the last N_y columns), or
        an SG_KERNEL_* code.
        radial_edges = 1: one-sided radial slopes at the first and last rows
        instead of ghost rows.  wedge = 1 (with radial_edges = 1): the origin
        wedge below the first row, whose densities forces_wedge takes.
        short_dft = 1 (FP32, 32 <= N_phi <= 256): the row transforms of the
        forward and adjoint calls as split-TF32 DFT-matrix products on the
        tensor cores."""
        code = KERNEL_KINDS[kind] if isinstance(kind, str) else int(kind)
        opts = BuildOpts(rtol, weight_p, code, soften, n_tpz, radial_edges, wedge, short_dft)
        _check(lib().sg_kernels_build(self.handle, ctypes.byref(opts), _stream(stream)), "sg_kernels_build")
        return self

    # -- forward / adjoint ---------------------------------------------------
    def _new(self):
        import torch

        return torch.empty((self.nu, self.nphi), dtype=self.dtype, device="cuda")

    def forces(self, sigma, F_r=None, F_phi=None, stream=None):
        F_r = self._new() if F_r is None else F_r
        F_phi = self._new() if F_phi is None else F_phi
        for t in (sigma, F_r, F_phi):
            self._check_field(t)
        _check(lib().sg_forces(self.handle, _ptr(sigma), _ptr(F_r), _ptr(F_phi), _stream(stream)), "sg_forces")
        return F_r, F_phi

    def forces_wedge(self, sigma, sigma_w, F_r=None, F_phi=None, stream=None):
        """sg_forces_wedge: the forces with the origin wedge's densities
        sigma_w (N_phi values on the device)."""
        F_r = self._new() if F_r is None else F_r
        F_phi = self._new() if F_phi is None else F_phi
        for t in (sigma, F_r, F_phi):
            self._check_field(t)
        self._check_wedge_row(sigma_w)
        _check(lib().sg_forces_wedge(self.handle, _ptr(sigma), _ptr(sigma_w), _ptr(F_r), _ptr(F_phi),
                                     _stream(stream)), "sg_forces_wedge")
        return F_r, F_phi

    def backward_wedge(self, gF_r, gF_phi, gsigma=None, gsigma_w=None, stream=None):
        """sg_forces_wedge_backward: (gsigma, gsigma_w)."""
        import torch

        gsigma = self._new() if gsigma is None else gsigma
        if gsigma_w is None:
            gsigma_w = torch.empty(self.nphi, dtype=self.dtype, device="cuda")
        for t in (gF_r, gF_phi, gsigma):
            self._check_field(t)
        self._check_wedge_row(gsigma_w)
        _check(lib().sg_forces_wedge_backward(self.handle, _ptr(gF_r), _ptr(gF_phi), _ptr(gsigma), _ptr(gsigma_w),
                                              _stream(stream)), "sg_forces_wedge_backward")
        return gsigma, gsigma_w

    def _check_wedge_row(self, t):
        if tuple(t.shape) != (self.nphi,) or t.dtype != self.dtype or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"expected a contiguous CUDA {self.dtype} tensor of shape ({self.nphi},)")

    def forces_noalloc(self, sigma, F_r, F_phi, stream=None):
        """sg_forces using the library's fixed scratch array: no device
        allocation in the call (for callers that may not allocate then).
        Calls that overlap on the GPU share that scratch and must not run
        concurrently."""
        for t in (sigma, F_r, F_phi):
            self._check_field(t)
        _check(lib().sg_forces_noalloc(self.handle, _ptr(sigma), _ptr(F_r), _ptr(F_phi), _stream(stream)),
               "sg_forces_noalloc")
        return F_r, F_phi

    def forces_timed(self, sigma, F_r, F_phi, stream=None):
        """sg_forces with per-pass CUDA-event timing; returns (rows, cols,
        inverse rows, span) in ms (synchronises the stream)."""
        for t in (sigma, F_r, F_phi):
            self._check_field(t)
        ms = (ctypes.c_float * 4)()
        _check(lib().sg_forces_timed(self.handle, _ptr(sigma), _ptr(F_r), _ptr(F_phi), _stream(stream), ms),
               "sg_forces_timed")
        return tuple(ms)

    def backward_timed(self, gF_r, gF_phi, gsigma, stream=None):
        """sg_forces_backward with per-pass CUDA-event timing; returns (rows,
        cols, inverse rows, span) in ms (synchronises the stream)."""
        self._check_field(gF_r)
        self._check_field(gF_phi)
        self._check_field(gsigma)
        ms = (ctypes.c_float * 4)()
        _check(lib().sg_forces_backward_timed(self.handle, _ptr(gF_r), _ptr(gF_phi), _ptr(gsigma), _stream(stream),
                                              ms), "sg_forces_backward_timed")
        return tuple(ms)

    def backward(self, gF_r, gF_phi, gsigma=None, stream=None):
        gsigma = self._new() if gsigma is None else gsigma
        for t in (gF_r, gF_phi, gsigma):
            self._check_field(t)
        _check(lib().sg_forces_backward(self.handle, _ptr(gF_r), _ptr(gF_phi), _ptr(gsigma), _stream(stream)),
               "sg_forces_backward")
        return gsigma

    def forces_host(self, sigma_h, F_r_h, F_phi_h, stream=None):
        """Host buffers (pinned torch CPU tensors); copies are inside the call."""
        for t in (sigma_h, F_r_h, F_phi_h):
            assert t.device.type == "cpu" and t.is_contiguous() and t.dtype == self.dtype
        _check(lib().sg_forces_host(self.handle, _ptr(sigma_h), _ptr(F_r_h), _ptr(F_phi_h), _stream(stream)),
               "sg_forces_host")
        return F_r_h, F_phi_h

    def _check_field(self, t):
        if t.dtype != self.dtype or tuple(t.shape) != (self.nu, self.nphi) or not t.is_contiguous() or not t.is_cuda:
            raise ValueError(f"field must be a contiguous CUDA {self.dtype} tensor of shape ({self.nu}, {self.nphi})")

    # -- introspection ---------------------------------------------------------
    def info(self):
        d = (ctypes.c_int * 4)()
        _check(lib().sg_plan_info(self.handle, d), "sg_plan_info")
        return tuple(d)

    def set_wait_limit(self, seconds: float):
        """Budget of the passes' device-side waits for their input copies
        (default 1 s); 0 makes every pass give up at once (tests that path)."""
        _check(lib().sg_plan_set_wait_limit(self.handle, float(seconds)), "sg_plan_set_wait_limit")

    def save(self, path: str, stream=None):
        """Write the built plan's spectra and parameters to a file."""
        _check(lib().sg_plan_save(self.handle, os.fsencode(path), _stream(stream)), "sg_plan_save")

    @classmethod
    def load(cls, path: str, stream=None):
        """A built plan from a file written by save (no rebuild)."""
        import torch

        h = ctypes.c_void_p()
        _check(lib().sg_plan_load(ctypes.byref(h), os.fsencode(path), _stream(stream)), "sg_plan_load")
        self = cls.__new__(cls)
        self.handle = h
        d = (ctypes.c_int * 4)()
        _check(lib().sg_plan_info(h, d), "sg_plan_info")
        self.nu, self.nphi = int(d[0]), int(d[1])
        self.code = int(d[2])
        self.dtype = torch.float32 if d[2] == SG_F32 else torch.float64
        self.u_min = self.du = self.G = None  # kept in the file and the plan, not needed here
        return self

    def check(self, stream=None):
        """Raise if a pass of the enqueued work reported a device-side
        timeout, or (checked builds) a failed index check (synchronises the
        stream)."""
        _check(lib().sg_plan_check(self.handle, _stream(stream)), "sg_plan_check")

    def build_report(self):
        """(flag bits, failed offsets, k, q) of the last build (all 0 if clean)."""
        d = (ctypes.c_int * 4)()
        _check(lib().sg_plan_build_report(self.handle, d), "sg_plan_build_report")
        return tuple(d)

    def kernels(self, stream=None):
        """Folded FP64 kernels K^eff (Kr, Kphi), each [2 Nu - 1, Nphi]."""
        n = (2 * self.nu - 1) * self.nphi
        kr = np.zeros(n)
        kp = np.zeros(n)
        dpp = ctypes.POINTER(ctypes.c_double)
        _check(lib().sg_plan_kernels(self.handle, kr.ctypes.data_as(dpp), kp.ctypes.data_as(dpp), _stream(stream)),
               "sg_plan_kernels")
        return kr.reshape(2 * self.nu - 1, self.nphi), kp.reshape(2 * self.nu - 1, self.nphi)

    def cells(self, stream=None):
        """Raw FP64 cell kernels [6, 2 Nu + 1, Nphi]."""
        out = np.zeros(6 * (2 * self.nu + 1) * self.nphi)
        _check(lib().sg_plan_cells(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   _stream(stream)), "sg_plan_cells")
        return out.reshape(6, 2 * self.nu + 1, self.nphi)

    def device_bytes(self) -> int:
        return int(lib().sg_plan_device_bytes(self.handle))

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().sg_plan_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dft_tc_matrices(nphi: int):
    """sg_dft_tc_matrices: the split tensor-core DFT matrices of short_dft
    plans (host only), as a float32 numpy array of 4 nphi^2 values."""
    import numpy as np

    out = np.zeros(4 * nphi * nphi, dtype=np.float32)
    _check(lib().sg_dft_tc_matrices(int(nphi), out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
           "sg_dft_tc_matrices")
    return out


def _batch_array(items):
    arr = (BatchItem * len(items))()
    for n, (p, s, fr, fp) in enumerate(items):
        for t in (s, fr, fp):
            p._check_field(t)
        arr[n] = BatchItem(p.handle.value, s.data_ptr(), fr.data_ptr(), fp.data_ptr())
    return arr


def forces_batched(items, stream=None):
    """items: list of (plan, sigma, F_r, F_phi) with device tensors."""
    _check(lib().sg_forces_batched(_batch_array(items), len(items), _stream(stream)), "sg_forces_batched")


def batch_prepare(items, stream=None):
    """Build the persistent path's work list for these items (synchronises)."""
    _check(lib().sg_batch_prepare(_batch_array(items), len(items), _stream(stream)), "sg_batch_prepare")


def batch_tune(items, cache_path=None, stream=None):
    """Tune the persistent path's schedule for these sizes (or read it from
    cache_path); returns (default ms, tuned ms).  Overwrites the items' F."""
    ms = (ctypes.c_float * 2)()
    path = os.fsencode(cache_path) if cache_path else None
    _check(lib().sg_batch_tune(_batch_array(items), len(items), path, _stream(stream), ms), "sg_batch_tune")
    return float(ms[0]), float(ms[1])


def _autograd_fn():
    import torch

    class SelfGravity(torch.autograd.Function):
        """(F_r, F_phi) = A sigma; backward gives A^T (gF_r, gF_phi) through
        the library's adjoint passes."""

        @staticmethod
        def forward(ctx, sigma, plan):
            ctx.plan = plan
            return plan.forces(sigma.contiguous())

        @staticmethod
        def backward(ctx, gF_r, gF_phi):
            plan = ctx.plan
            gr = gF_r.contiguous() if gF_r is not None else torch.zeros((plan.nu, plan.nphi), dtype=plan.dtype,
                                                                         device="cuda")
            gp = gF_phi.contiguous() if gF_phi is not None else torch.zeros_like(gr)
            return plan.backward(gr, gp), None

    return SelfGravity


_SG = None


def self_gravity(sigma, plan):
    """Differentiable forces: returns (F_r, F_phi)."""
    global _SG
    if _SG is None:
        _SG = _autograd_fn()
    return _SG.apply(sigma, plan)
