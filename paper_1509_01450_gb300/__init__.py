"""GB300-native second-order self-gravity for infinitesimally thin disks on a
log-polar grid (Wang, Yen & Taam, arXiv:1509.01450).

The compute path is libsgdisk.so (CUDA for sm_103a, C ABI in include/sg.h);
``sg`` is its ctypes binding.
"""
from .sg import Plan, SgError, batch_prepare, batch_tune, forces_batched, lib, self_gravity, status_string  # noqa: F401
