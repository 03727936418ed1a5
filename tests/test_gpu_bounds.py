"""The bounds-checking build (liblbmpf_debug.so, compiled with
LBM_CHECK_BOUNDS: every population and field index a kernel computes is
checked against its buffer, a failing access is skipped and recorded, and
lbm_sync returns LBM_EBOUNDS) runs every kernel family on grids that
exercise its edge paths without a single failed check, and computes the same
states as the release library bit for bit -- the checks change no arithmetic.
The adjoint's scalar gradients come from float atomics (their order varies
from run to run), so those compare within 1e-6 relative."""
import os
import subprocess
import sys

import numpy as np
import pytest

import _bounds_cases as BC

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def debug_results(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("bounds") / "debug.npz")
    env = dict(os.environ, LBM_PF_DEBUG="1", PYTHONPATH=os.pathsep.join([ROOT, HERE]))
    res = subprocess.run([sys.executable, os.path.join(HERE, "_bounds_cases.py"), out],
                         env=env, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stdout[-4000:] + res.stderr[-4000:]
    return dict(np.load(out))


def test_debug_library_selected_by_environment(debug_results):
    from paper_2003_06342_b300 import _binding as B
    assert not B.DEBUG and B.LIB_PATH.endswith("liblbmpf.so")


@pytest.mark.parametrize("case", BC.STEP_CASES, ids=[c[0] for c in BC.STEP_CASES])
def test_step_kernels_checked_and_bit_identical(debug_results, case):
    name, make, storage, kernel, steps = case
    rel = BC.run_step_case(make, storage, kernel, steps)
    assert np.array_equal(rel, debug_results[name]), name


@pytest.mark.parametrize("case", BC.CAC_CASES, ids=[c[0] for c in BC.CAC_CASES])
def test_phase_field_kernel_checked_and_bit_identical(debug_results, case):
    name, n, storage, speed, period, steps = case
    rel = BC.run_cac_case(n, storage, speed, period, steps)
    assert np.array_equal(rel, debug_results[name]), name


@pytest.mark.parametrize("biased", [False, True], ids=["central", "biased"])
def test_adjoint_kernels_checked(debug_results, biased):
    rel = BC.run_adjoint_case(biased)
    dbg = debug_results["adjoint_biased" if biased else "adjoint"]
    assert np.all(np.isfinite(dbg))
    assert np.allclose(rel, dbg, rtol=1e-6, atol=1e-12 * np.abs(rel).max())


def test_noalloc_sums_ragged_both_builds(debug_results):
    """The allocation-free sums on a ragged size in both builds.  Its kernel
    has no handle and so no status word: its only indexed loads sit behind the
    guard c < n, and this case checks that a ragged last block gives the same
    FP64 sums (fixed summation order) in both builds."""
    rel = BC.run_noalloc_case()
    assert np.array_equal(rel, debug_results["noalloc"])
