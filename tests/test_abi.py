"""The C-ABI library loads and exports every entry point that include/sg.h
declares; host-side argument checks (no device work) behave as documented."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1509_01450_gb300 import build

    build.build()
    from paper_1509_01450_gb300 import sg

    return sg.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sg_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("sg_plan_create", "sg_kernels_build", "sg_forces", "sg_forces_backward", "sg_forces_batched",
                 "sg_plan_destroy", "sg_status_string"):
        assert want in names


def test_every_declared_symbol_is_exported(L):
    from paper_1509_01450_gb300 import sg

    for name in declared_functions():
        assert hasattr(L, name), name
    assert set(declared_functions()) <= set(sg.EXPORTS)


def test_status_strings(L):
    from paper_1509_01450_gb300 import sg

    for code in range(9):
        assert isinstance(sg.status_string(code), str) and sg.status_string(code)
    assert "not built" in sg.status_string(sg.SG_ERR_NOT_BUILT)


@pytest.mark.parametrize("nu,nphi,dtype,want", [
    (3, 16, 0, 4), (16, 12, 0, 4), (2, 16, 0, 4), (16, 2, 0, 4), (8192, 16, 0, 4), (4096, 16, 1, 4),
    (16, 16384, 0, 4), (16, 8192, 1, 4), (16, 16, 7, 1),
])
def test_plan_create_rejects_bad_sizes_before_touching_the_device(L, nu, nphi, dtype, want):
    h = ctypes.c_void_p()
    assert L.sg_plan_create(ctypes.byref(h), nu, nphi, 0.0, 0.1, 1.0, dtype) == want
    assert h.value is None


def test_bad_scalars_and_nulls(L):
    h = ctypes.c_void_p()
    assert L.sg_plan_create(ctypes.byref(h), 16, 16, 0.0, 0.0, 1.0, 0) == 1  # du <= 0
    assert L.sg_plan_create(ctypes.byref(h), 16, 16, 0.0, float("nan"), 1.0, 0) == 1
    assert L.sg_plan_create(None, 16, 16, 0.0, 0.1, 1.0, 0) == 1
    assert L.sg_forces(None, None, None, None, None) == 1
    assert L.sg_forces_backward(None, None, None, None, None) == 1
    assert L.sg_kernels_build(None, None, None) == 1
    assert L.sg_plan_destroy(None) == 1
    assert L.sg_forces_batched(None, -1, None) == 1
    assert L.sg_forces_batched(None, 0, None) == 0  # empty batch is a no-op


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures against the C compiler's layout of
    sg_build_opts and sg_batch_item (gcc on include/sg.h)."""
    import shutil
    import subprocess

    from paper_1509_01450_gb300 import sg

    gcc = shutil.which("gcc")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if gcc is None or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime_api.h")):
        pytest.skip("gcc or the CUDA headers are not available")
    fields = [f for f, _ in sg.BuildOpts._fields_]
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include "sg.h"', "int main(void) {",
             '  printf("%zu\\n", sizeof(sg_build_opts));']
    lines += [f'  printf("%zu\\n", offsetof(sg_build_opts, {f}));' for f in fields]
    lines += ['  printf("%zu\\n", sizeof(sg_batch_item));']
    lines += [f'  printf("%zu\\n", offsetof(sg_batch_item, {f}));' for f, _ in sg.BatchItem._fields_]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c99", "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, str(src), "-o", str(exe)],
                   check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(sg.BuildOpts)] + [getattr(sg.BuildOpts, f).offset for f in fields]
    want += [ctypes.sizeof(sg.BatchItem)] + [getattr(sg.BatchItem, f).offset for f, _ in sg.BatchItem._fields_]
    assert got == want
