"""The periodic state check (lbm_set_health_check): a healthy run passes, a
NaN planted in the initial temperature or a bound that the bulk phases
violate is reported by lbm_sync as LBM_ENONFINITE, the check's launches are
counted, and with the check off the same NaN run syncs cleanly (the failure
then only shows in the FP64 sums)."""
import numpy as np
import pytest

import workloads as W
from paper_2003_06342_b300._binding import LBMError, LBM_ENONFINITE

from _parity import gpu_solver

pytestmark = pytest.mark.gpu


def _film(nx=96, ny=48):
    return W.film_boiling_2d(nx, ny, rho_ratio=10.0, y0=16.0, amplitude=2.0, phi_wall=(1.0, 0.0))


def _nan_film():
    w = _film()
    T0 = w.T0.copy()
    T0[10, 20] = float("nan")
    w.T0 = T0
    return w


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_healthy_run_passes(storage):
    s = gpu_solver(_film(), storage=storage).set_health_check(5, 0.6)
    s.step(20)
    assert s.last_launches() == 20 + 4
    s.sync()


def test_healthy_3d_and_phase_field_runs_pass():
    w = W.film_boiling_3d(40, 16, 24, modes=1, z0=8.0, phi_wall=(1.0, 0.0))
    s = gpu_solver(w).set_health_check(2, 0.6)
    s.step(6)
    s.sync()
    from paper_2003_06342_b300 import Solver
    v = W.vortex_disk(n=41)
    c = Solver(v.n, v.periodic, v.params)
    c.set_velocity(v.extra["u"], v.extra["period"]).init(v.phi0, v.T0)
    c.set_health_check(1, 0.6).step(5)
    c.sync()


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_nan_is_reported(storage):
    s = gpu_solver(_nan_film(), storage=storage).set_health_check(1, 0.6)
    s.step(3)
    with pytest.raises(LBMError) as e:
        s.sync()
    assert e.value.code == LBM_ENONFINITE
    s.sync()                                   # reported once, context usable


def test_nan_is_not_reported_with_the_check_off():
    s = gpu_solver(_nan_film())
    s.step(3)
    s.sync()
    with pytest.raises(LBMError) as e:
        s.reduce()
    assert e.value.code == LBM_ENONFINITE


def test_bound_violated_by_the_bulk_phases_is_reported():
    """Bulk liquid and vapour sit at phi = 0 and 1, so |phi - 1/2| = 1/2
    exceeds a bound of 0.3 in the first checked step; 3D as well."""
    s = gpu_solver(_film()).set_health_check(4, 0.3)
    s.step(3)
    s.sync()                                   # not yet checked
    s.step(1)
    with pytest.raises(LBMError) as e:
        s.sync()
    assert e.value.code == LBM_ENONFINITE
    w = W.film_boiling_3d(40, 16, 24, modes=1, z0=8.0, phi_wall=(1.0, 0.0))
    s3 = gpu_solver(w, storage="fp16").set_health_check(1, 0.3)
    s3.step(1)
    with pytest.raises(LBMError):
        s3.sync()
