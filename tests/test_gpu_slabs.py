"""Slab domain decomposition on one GPU (the emulated multi-domain run of the
paper's multi-GPU scheme): N slabs, each a Solver on its own grid with ghost
columns, exchanging column blocks through lbm_pack_columns /
lbm_unpack_columns after every step.  After 50 steps every owned column's
stored state (populations, phi^{n-1}, lagged source) equals the undivided
run's bit for bit."""
import pytest
import torch

import workloads as W
from paper_2003_06342_b300.slabs import LocalSlabs, SolverSlab, halo_width, partition

from _parity import gpu_solver

pytestmark = pytest.mark.gpu


def _film(nx, ny, **extra):
    w = W.film_boiling_2d(nx, ny, rho_ratio=10.0, y0=ny / 3.0, amplitude=2.0, phi_wall=(1.0, 0.0))
    w.params.update(**extra)
    return w


CASES = [
    ("2d_fp32_2slabs", lambda: _film(96, 70), "fp32", 2),
    ("2d_fp32_4slabs", lambda: _film(96, 70), "fp32", 4),
    ("2d_fp16_3slabs_ragged", lambda: _film(100, 45), "fp16", 3),
    ("2d_bf16_biased_3slabs", lambda: _film(90, 40, grad_scheme="biased2"), "bf16", 3),
    ("2d_mrt_2slabs", lambda: _film(80, 40, collision="mrt", mrt_rates=(1.4, 1.4, 1.2),
                                    mrt_rates_g=(1.3, 1.2, 1.1, 1.25)), "fp32", 2),
    ("2d_droplet_periodic_4slabs", lambda: W.droplet_2d(64, 12.0, T_offset=0.05), "fp32", 4),
    ("3d_fp32_2slabs", lambda: W.film_boiling_3d(64, 20, 30, modes=1, z0=10.0, phi_wall=(1.0, 0.0)), "fp32", 2),
    ("3d_fp16_3slabs", lambda: W.film_boiling_3d(48, 12, 26, modes=1, z0=8.0, phi_wall=(1.0, 0.0)), "fp16", 3),
    ("3d_mrt_biased_2slabs", lambda: _film3d_opts(collision="mrt", mrt_rates=(1.4, 1.4, 1.2),
                                                  mrt_rates_g=(1.3, 0.0, 0.0, 1.25), grad_scheme="biased2"),
     "fp32", 2),
]


def _film3d_opts(**extra):
    w = W.film_boiling_3d(64, 16, 24, modes=1, z0=8.0, phi_wall=(1.0, 0.0))
    w.params.update(**extra)
    return w


@pytest.mark.parametrize("name,make,storage,nslabs", CASES, ids=[c[0] for c in CASES])
def test_slabs_bit_identical_to_undivided(name, make, storage, nslabs):
    w = make()
    steps = 50
    h = halo_width(w.params)
    slabs = [SolverSlab(w.n, w.periodic, w.params, lo, hi, h, storage=storage).init(w.phi0, w.T0, p0=w.p0)
             for lo, hi in partition(w.n[0], nslabs, h)]
    run = LocalSlabs(slabs).start().step(steps)
    ref = gpu_solver(w, storage=storage)
    ref.step(steps)
    for s in run.slabs:
        got = s.pack(h, s.width)
        want = ref.pack_columns(s.lo, s.width)
        torch.cuda.synchronize()
        assert torch.equal(got, want), (name, s.lo, s.hi)
    F, Fr = run.fields(), ref.fields()
    assert torch.equal(F["phi"], Fr["phi"]) and torch.equal(F["T"], Fr["T"])


def test_pack_unpack_roundtrip_and_errors():
    w = _film(40, 20)
    s = gpu_solver(w)
    s.step(3)
    a = s.pack_columns(5, 7)
    assert a.numel() == s.columns_bytes(7)
    t = gpu_solver(w)
    t.unpack_columns(5, 7, a)
    assert torch.equal(t.pack_columns(5, 7), a)
    from paper_2003_06342_b300 import _binding as B
    with pytest.raises(B.LBMError):
        s.pack_columns(35, 7)             # beyond nx
