"""The bounded waits of the TMA-staged step kernels, made to run out on
purpose and without a stalled copy: lbm_set_first_wait_limit(0) lets the
first mbarrier wait of every block poll zero times, so each block gives up
at once, waits (with the full limit) for the bulk copies it has issued,
records the timeout and returns.  lbm_sync must then report LBM_ETIMEOUT,
the context must stay usable, and with the default limit restored the same
handle must step exactly like the tiled kernel again."""
import pytest
import torch

import workloads as W
from paper_2003_06342_b300 import _binding as B

from _parity import gpu_solver

pytestmark = pytest.mark.gpu


def _film2d():
    return W.film_boiling_2d(128, 96, rho_ratio=10.0, y0=32.0, amplitude=2.0, phi_wall=(1.0, 0.0))


def _film3d():
    return W.film_boiling_3d(64, 24, 70, modes=1, z0=20.0, phi_wall=(1.0, 0.0))


@pytest.mark.parametrize("make", [_film2d, _film3d], ids=["2d", "3d"])
def test_expired_wait_reports_timeout_and_context_survives(make):
    w = make()
    s = gpu_solver(w)
    s.set_kernel("tma")
    assert s.kernel() == "tma"
    B.check(B.lib.lbm_set_first_wait_limit(0), "lbm_set_first_wait_limit")
    try:
        s.step(2)
        with pytest.raises(B.LBMError) as e:
            s.sync()
        assert e.value.code == B.LBM_ETIMEOUT
    finally:
        B.check(B.lib.lbm_set_first_wait_limit(-1), "lbm_set_first_wait_limit")
    torch.cuda.synchronize()                  # the context is still usable
    # the status was reported and cleared; a fresh start runs clean and
    # matches the tiled kernel bit for bit
    s.init(w.phi0, w.T0, p0=w.p0)
    s.step(5)
    s.sync()
    t = gpu_solver(w)
    t.set_kernel("tiled")
    t.step(5)
    assert torch.equal(s.get_state(), t.get_state())
