"""The two-relaxation-time collision option (LBM_COLLISION_TRT) on the GPU
against the FP64 oracle's TRT step (oracle.model with collision = "trt"):
parity within 1e-5 on 2D and 3D geometries, the TMA-staged kernels equal
to the tiled ones bit for bit, and the exact Poiseuille profile that the
magic value 3/16 gives with half-way bounce-back walls."""
import numpy as np
import pytest
import torch

import workloads as W

from _parity import gpu_fields, gpu_solver, max_errors, oracle_fields

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _trt(w, magic=(0.25, 0.25, 0.25)):
    w.params.update(collision="trt", trt_magic=magic)
    return w


def _film(nx, ny, **kw):
    return W.film_boiling_2d(nx, ny, rho_ratio=10.0, y0=ny / 3.0, amplitude=2.0, phi_wall=(1.0, 0.0), **kw)


CASES = [
    ("film_ragged", lambda: _trt(_film(100, 70)), 40),
    ("droplet_periodic", lambda: _trt(W.droplet_2d(48, 12.0, T_offset=0.05), (3.0 / 16.0, 0.25, 1.0 / 6.0)), 40),
    ("stefan_x_walls", lambda: _trt(W.stefan_1d(nx=90, ny=2), (0.25, 0.1, 0.3)), 80),
    ("film_3d", lambda: _trt(W.film_boiling_3d(37, 10, 21, modes=2, z0=7.0, phi_wall=(1.0, 0.0))), 15),
]


@pytest.mark.parametrize("name,make,steps", CASES, ids=[c[0] for c in CASES])
def test_trt_parity_with_oracle(name, make, steps):
    w = make()
    ref = oracle_fields(w, steps)
    s = gpu_solver(w)
    s.step(steps)
    err = max_errors(gpu_fields(s), ref)
    print(name, err)
    assert all(v < TOL for v in err.values()), err


def test_trt_differs_from_bgk():
    w = _film(64, 40)
    a = gpu_solver(w)
    b = gpu_solver(_trt(_film(64, 40)))
    a.step(20)
    b.step(20)
    assert np.abs(gpu_fields(a)["phi"] - gpu_fields(b)["phi"]).max() > 1e-7


TMA_CASES = [
    ("2d_fp32", lambda: _trt(_film(128, 96)), "fp32", 20),
    ("2d_fp16", lambda: _trt(_film(128, 96)), "fp16", 20),
    ("3d_fp32", lambda: _trt(W.film_boiling_3d(64, 24, 70, modes=2, z0=20.0, phi_wall=(1.0, 0.0))), "fp32", 8),
    ("3d_ragged", lambda: _trt(W.film_boiling_3d(44, 13, 37, modes=1, z0=12.0, phi_wall=(1.0, 0.0))), "fp32", 8),
    ("3d_bf16", lambda: _trt(W.film_boiling_3d(64, 16, 40, modes=2, z0=12.0, phi_wall=(1.0, 0.0))), "bf16", 8),
]


@pytest.mark.parametrize("name,make,storage,steps", TMA_CASES, ids=[c[0] for c in TMA_CASES])
def test_trt_tma_matches_tiled_bit_for_bit(name, make, storage, steps):
    w = make()
    a = gpu_solver(w, storage=storage)
    b = gpu_solver(w, storage=storage)
    a.set_kernel("tma")
    b.set_kernel("tiled")
    a.step(steps)
    b.step(steps)
    sa, sb = a.get_state(), b.get_state()
    torch.cuda.synchronize()
    assert torch.equal(sa, sb), name


def _poiseuille_error(collision, nu=0.5, H=8, G=1e-5, steps=1500):
    params = W.base_params(rho_l=1.0, rho_g=1.0, nu_l=nu, nu_g=nu, alpha_l=0.05, alpha_g=0.05, sigma=0.0,
                           gravity=(0.0, 0.0, 0.0), body_force=(G, 0.0, 0.0), source_on=0,
                           phi_wall=(0.0, 0.0), T_wall=(1.0, 1.0), collision=collision,
                           trt_magic=(3.0 / 16.0, 0.25, 0.25))
    from paper_2003_06342_b300 import Solver
    s = Solver((2, H), (True, False), params)
    s.init(np.zeros((H, 2)), np.ones((H, 2)))
    s.step(steps)
    u = s.fields()["u"][0].double().cpu().numpy()[:, 0]
    y = np.arange(H)
    exact = G / (2 * nu) * (y + 0.5) * (H - 0.5 - y)
    return float(np.abs(u - exact).max() / exact.max())


def test_trt_magic_3_16_poiseuille_on_gpu():
    err_trt, err_bgk = _poiseuille_error("trt"), _poiseuille_error("bgk")
    print("poiseuille rel err TRT", err_trt, "BGK", err_bgk)
    assert err_trt < 1e-4
    assert err_bgk > 1e-2
