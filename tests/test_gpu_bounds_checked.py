"""The bounds-checked debug build (TRTR_BOUNDS_CHECK=1, libtrtr_checked.so).

Its kernels check every plane index, two-node store, bulk row copy and TMA load coordinate
against the ghosted layout, record what is out of bounds and skip it (nothing traps), and the
next synchronising call returns TRTR_EBOUNDS.  Two checks here:
  * the recording path: a probe kernel hands the checks four bad arguments and accesses
    nothing with them; the checked build reports the four, the default build none;
  * the GPU parity suites run again in a child process on the checked build, where a conftest
    fixture also asserts after every test that nothing was recorded.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2312_10316_gb300 import trtr as T  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUITES = ["tests/test_gpu_parity.py", "tests/test_gpu_step2.py", "tests/test_gpu_paper.py", "tests/test_gpu_batch.py",
          "tests/test_gpu_adjoint.py", "tests/test_gpu_bounds_checked.py"]


def test_recording_path_without_a_bad_access():
    nx, ny = 40, 24
    p = T.Params(nx=nx, ny=ny, dx=0.1, dt=0.02, precision=T.TRTR_F32)
    with T.Solver(p) as s:
        s.set_fields(np.zeros((ny, nx)), np.zeros((ny, nx)), np.full((ny, nx), 0.05))
        s.init_equilibrium(np.ones((ny, nx)))
        st = T.trtr_check_bounds_path(s.ctx)
        if T.BOUNDS_CHECKED:
            assert st == T.TRTR_EBOUNDS
            assert f"4 out-of-bounds accesses; the first of kind 1 at ({nx + 2}, 0)" in T.trtr_last_error(s.ctx)
        else:
            assert st == T.TRTR_OK
        # the record was cleared as it was reported: the context runs on
        s.step(3)
        assert np.abs(s.moments() - 1.0).max() <= 1e-6
        assert T.trtr_bounds_report() == (0, 0, 0, 0)


@pytest.mark.skipif(T.BOUNDS_CHECKED, reason="already running on the checked build")
def test_parity_suites_on_the_bounds_checked_build():
    from paper_2312_10316_gb300.build import build_library

    build_library(checked=True)
    env = dict(os.environ, TRTR_BOUNDS_CHECK="1")
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
           "-k", "not fullsize", *SUITES]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = r.stdout[-4000:] + r.stderr[-2000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout and " failed" not in r.stdout, tail
