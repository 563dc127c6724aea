"""The index-checked build (-DSG_DEBUG, libsgdisk_checked.so) on every pass
kernel family: run in a child process, every plan's flags stay clear (no
index check fails: sg_plan_check would report SG_ERR_BOUNDS and the child
would exit non-zero), and its results agree with the ordinary library's.
The checks only guard accesses, so the two agree to rounding (the compiler
may schedule the checked kernels' arithmetic differently)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_runs_clean_and_agrees(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_01450_gb300 import build, sg

    build.build()
    assert sg.lib().sg_checked_build() == 0
    path = str(tmp_path / "checked.npz")
    env = dict(os.environ, SG_LIBRARY_VARIANT="checked")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_cases.py"), path], env=env,
                       capture_output=True, text=True, timeout=1200)
    assert p.returncode == 0, p.stdout[-3000:] + p.stderr[-3000:]
    got = np.load(path)
    from tests import checked_cases

    ref = checked_cases.run_all()
    assert set(got.files) == set(ref)
    for k, a in ref.items():
        b = got[k]
        tol = 1e-5 if "fp64" not in k else 1e-12
        den = np.linalg.norm(a)
        assert np.linalg.norm(b - a) <= tol * den, k
