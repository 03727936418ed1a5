"""The multiple-relaxation-time collision of the flow and phase-field sets
(LBM_COLLISION_MRT; D2Q9, and D3Q19 / D3Q7 in 3D) on the GPU against the
FP64 oracle's MRT step (oracle.model with collision = "mrt"): parity within
1e-5 on walled, periodic and ragged 2D and 3D grids, with g on BGK or on its
own MRT rates and with the biased gradient; the 16-bit storages within their
own bound; the TMA-staged kernels equal to the tiled ones bit for bit; equal
rates equal to the BGK kernel; phi mass conserved with the source off; the
exact Poiseuille profile at the magic rate s_q = 8 (2 - s_nu)/(8 - s_nu) in
2D and 3D; and the unsupported cases."""
import numpy as np
import pytest
import torch

import workloads as W

from _parity import gpu_fields, gpu_solver, max_errors, oracle_fields

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _mrt(w, rates=(1.4, 1.3, 1.2), rates_g=(0.0, 0.0, 0.0, 0.0)):
    w.params.update(collision="mrt", mrt_rates=rates, mrt_rates_g=rates_g)
    return w


G_RATES = (1.2, 1.5, 1.1, 1.7)


def _film(nx, ny, **kw):
    return W.film_boiling_2d(nx, ny, rho_ratio=10.0, y0=ny / 3.0, amplitude=2.0, phi_wall=(1.0, 0.0), **kw)


def _film3d(nx, ny, nz, periodic_z=False, grad_scheme=None):
    w = W.film_boiling_3d(nx, ny, nz, modes=2, z0=nz / 3.0, phi_wall=(1.0, 0.0))
    if periodic_z:
        w.periodic = (True, True, True)
    if grad_scheme:
        w.params.update(grad_scheme=grad_scheme)
    return w


CASES = [
    ("film_ragged", lambda: _mrt(_film(100, 70)), 40),
    ("droplet_periodic", lambda: _mrt(W.droplet_2d(48, 12.0, T_offset=0.05), (1.1, 1.6, 1.8)), 40),
    ("stefan_x_walls", lambda: _mrt(W.stefan_1d(nx=90, ny=2), (1.0, 1.2, 1.5)), 80),
    ("film_biased", lambda: _mrt(_film(70, 45, grad_scheme="biased2")), 30),
    # the phase-field set on MRT too (a rate of 0 is the BGK rate)
    ("film_ragged_g", lambda: _mrt(_film(100, 70), rates_g=G_RATES), 40),
    ("droplet_periodic_g", lambda: _mrt(W.droplet_2d(48, 12.0, T_offset=0.05), (1.1, 1.6, 1.8),
                                        (0.0, 1.3, 1.6, 0.0)), 40),
    ("film_biased_g", lambda: _mrt(_film(70, 45, grad_scheme="biased2"), rates_g=G_RATES), 30),
    # 3D: D3Q19 flow set, D3Q7 phase-field set (g: s_e and s_p; s_eps, s_q unused)
    ("film3d_ragged", lambda: _mrt(_film3d(37, 10, 21)), 15),
    ("film3d_ragged_g", lambda: _mrt(_film3d(37, 10, 21), (1.1, 1.6, 1.8), G_RATES), 15),
    ("film3d_periodic_g", lambda: _mrt(_film3d(24, 16, 20, periodic_z=True), rates_g=(1.5, 0.0, 0.0, 1.2)), 15),
    ("film3d_biased_g", lambda: _mrt(_film3d(33, 12, 19, grad_scheme="biased2"), rates_g=G_RATES), 12),
]


@pytest.mark.parametrize("name,make,steps", CASES, ids=[c[0] for c in CASES])
def test_mrt_parity_with_oracle(name, make, steps):
    w = make()
    ref = oracle_fields(w, steps)
    s = gpu_solver(w)
    s.step(steps)
    err = max_errors(gpu_fields(s), ref)
    print(name, err)
    assert all(v < TOL for v in err.values()), err


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_mrt_16bit_storage_near_oracle(storage):
    # the same bound the BGK step meets with 16-bit storage on this film
    w = _mrt(_film(64, 48), rates_g=G_RATES)
    ref = oracle_fields(w, 20)
    err = max_errors(gpu_fields(_stepped(gpu_solver(w, storage=storage), 20)), ref)
    bgk = _film(64, 48)
    ref_b = oracle_fields(bgk, 20)
    err_b = max_errors(gpu_fields(_stepped(gpu_solver(bgk, storage=storage), 20)), ref_b)
    print(storage, "mrt", err, "bgk", err_b)
    assert all(err[k] < 4.0 * err_b[k] + 1e-5 for k in err), (err, err_b)


def _stepped(s, n):
    s.step(n)
    return s


def test_mrt_differs_from_bgk_and_equal_rates_match_bgk():
    w = _film(64, 40)
    a = gpu_solver(w)
    b = gpu_solver(_mrt(_film(64, 40)))
    a.step(20)
    b.step(20)
    fa, fb = gpu_fields(a), gpu_fields(b)
    assert np.abs(fa["phi"] - fb["phi"]).max() > 1e-7
    # every rate at the BGK rate: equal to the BGK kernel within FP32 rounding
    om = 1.0 / (3.0 * 0.1 + 0.5)
    wl = W.droplet_2d(40, 10.0, T_offset=0.04)
    wl.params.update(nu_l=0.1, nu_g=0.1)
    c = gpu_solver(wl)
    wm = W.droplet_2d(40, 10.0, T_offset=0.04)
    wm.params.update(nu_l=0.1, nu_g=0.1, collision="mrt", mrt_rates=(om, om, om))
    d = gpu_solver(wm)
    c.step(30)
    d.step(30)
    err = max_errors(gpu_fields(c), gpu_fields(d))
    assert all(v < 1e-6 for v in err.values()), err


TMA_CASES = [("2d_fp32", "fp32", (0.0,) * 4), ("2d_fp16", "fp16", (0.0,) * 4), ("2d_bf16", "bf16", (0.0,) * 4),
             ("2d_fp32_g", "fp32", G_RATES), ("2d_fp16_g", "fp16", G_RATES), ("2d_bf16_g", "bf16", G_RATES)]


@pytest.mark.parametrize("name,storage,rates_g", TMA_CASES, ids=[c[0] for c in TMA_CASES])
def test_mrt_tma_matches_tiled_bit_for_bit(name, storage, rates_g):
    w = _mrt(_film(128, 96), rates_g=rates_g)
    a = gpu_solver(w, storage=storage)
    b = gpu_solver(w, storage=storage)
    a.set_kernel("tma")
    b.set_kernel("tiled")
    a.step(20)
    b.step(20)
    sa, sb = a.get_state(), b.get_state()
    torch.cuda.synchronize()
    assert torch.equal(sa, sb), name


def _poiseuille_error(rates, nu=0.5, H=8, G=1e-5, steps=1500):
    params = W.base_params(rho_l=1.0, rho_g=1.0, nu_l=nu, nu_g=nu, alpha_l=0.05, alpha_g=0.05, sigma=0.0,
                           gravity=(0.0, 0.0, 0.0), body_force=(G, 0.0, 0.0), source_on=0,
                           phi_wall=(0.0, 0.0), T_wall=(1.0, 1.0), collision="mrt", mrt_rates=rates)
    from paper_2003_06342_b300 import Solver
    s = Solver((2, H), (True, False), params)
    s.init(np.zeros((H, 2)), np.ones((H, 2)))
    s.step(steps)
    u = s.fields()["u"][0].double().cpu().numpy()[:, 0]
    y = np.arange(H)
    exact = G / (2 * nu) * (y + 0.5) * (H - 0.5 - y)
    return float(np.abs(u - exact).max() / exact.max())


def test_mrt_magic_rate_poiseuille_on_gpu():
    s_nu = 1.0 / (0.5 * 3.0 + 0.5)
    s_q = 8.0 * (2.0 - s_nu) / (8.0 - s_nu)
    err_magic, err_off = _poiseuille_error((1.1, 1.3, s_q)), _poiseuille_error((1.1, 1.3, 1.9))
    print("poiseuille rel err MRT magic", err_magic, "off", err_off)
    assert err_magic < 1e-4
    assert err_off > 1e-3


def test_mrt_unsupported_cases():
    from paper_2003_06342_b300 import Solver
    wc = W.cac_params()
    wc.update(collision="mrt", mrt_rates=(1.4, 1.3, 1.2))
    with pytest.raises(RuntimeError):
        Solver((32, 32), (True, True), wc)
    w = _mrt(_film(32, 24), rates=(1.4, 2.0, 1.2))
    with pytest.raises(RuntimeError):
        Solver(w.n, w.periodic, w.params)
    w3 = _mrt(_film3d(16, 8, 12), rates_g=(1.2, 0.0, 0.0, 2.5))
    with pytest.raises(RuntimeError):
        Solver(w3.n, w3.periodic, w3.params)


def _mass_drift(w, steps):
    s = gpu_solver(w)
    m0, _ = s.reduce()
    s.step(steps)
    m1, _ = s.reduce()
    return m0, abs(m1 - m0)


def _assert_mass_kept(w_mrt, w_bgk, steps):
    # the MRT correction leaves phi's moment alone, so its drift is FP32
    # rounding of the same size as the BGK kernel's on the same input: at most
    # a few times that, or a few ulps of the sum per step
    m0, d_mrt = _mass_drift(w_mrt, steps)
    _, d_bgk = _mass_drift(w_bgk, steps)
    floor = 4.0 * 6e-8 * m0 * np.sqrt(steps)
    print("phi mass drift MRT", d_mrt, "BGK", d_bgk, "floor", floor)
    assert d_mrt <= 4.0 * d_bgk + floor, (d_mrt, d_bgk, floor)


def test_mrt_g_conserves_phi_mass_with_the_source_off():
    def make(mrt):
        w = W.droplet_2d(64, 16.0, T_offset=0.05)
        if mrt:
            _mrt(w, rates_g=G_RATES)
        w.params.update(source_on=0)
        return w
    _assert_mass_kept(make(True), make(False), 200)


# ---- 3D

TMA3_CASES = [("3d_fp32", "fp32", (0.0,) * 4, None), ("3d_fp16", "fp16", (0.0,) * 4, None),
              ("3d_bf16", "bf16", (0.0,) * 4, None), ("3d_fp32_g", "fp32", G_RATES, None),
              ("3d_fp16_g", "fp16", G_RATES, None), ("3d_bf16_g", "bf16", G_RATES, None),
              ("3d_fp32_biased_g", "fp32", G_RATES, "biased2"), ("3d_fp16_biased_g", "fp16", G_RATES, "biased2")]


@pytest.mark.parametrize("name,storage,rates_g,grad", TMA3_CASES, ids=[c[0] for c in TMA3_CASES])
def test_mrt3d_tma_matches_tiled_bit_for_bit(name, storage, rates_g, grad):
    # 64 x 24 x 70: whole 32 x 4 tiles in x and y (the biased TMA path needs
    # them), a ragged last z block
    w = _mrt(_film3d(64, 24, 70, grad_scheme=grad), rates_g=rates_g)
    a = gpu_solver(w, storage=storage)
    b = gpu_solver(w, storage=storage)
    a.set_kernel("tma")
    b.set_kernel("tiled")
    a.step(8)
    b.step(8)
    sa, sb = a.get_state(), b.get_state()
    torch.cuda.synchronize()
    assert torch.equal(sa, sb), name


def test_mrt3d_parity_on_the_tma_kernel():
    w = _mrt(_film3d(64, 24, 30), (1.1, 1.6, 1.8), G_RATES)
    ref = oracle_fields(w, 10)
    s = gpu_solver(w)
    s.set_kernel("tma")
    s.step(10)
    err = max_errors(gpu_fields(s), ref)
    print("tma", err)
    assert all(v < TOL for v in err.values()), err


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_mrt3d_16bit_storage_near_oracle(storage):
    w = _mrt(_film3d(32, 12, 24), rates_g=G_RATES)
    ref = oracle_fields(w, 10)
    err = max_errors(gpu_fields(_stepped(gpu_solver(w, storage=storage), 10)), ref)
    bgk = _film3d(32, 12, 24)
    ref_b = oracle_fields(bgk, 10)
    err_b = max_errors(gpu_fields(_stepped(gpu_solver(bgk, storage=storage), 10)), ref_b)
    print(storage, "mrt", err, "bgk", err_b)
    assert all(err[k] < 4.0 * err_b[k] + 1e-5 for k in err), (err, err_b)


def test_mrt3d_equal_rates_match_bgk():
    om = 1.0 / (3.0 * 0.1 + 0.5)
    wl = _film3d(32, 12, 24)
    wl.params.update(nu_l=0.1, nu_g=0.1)
    wm = _film3d(32, 12, 24)
    wm.params.update(nu_l=0.1, nu_g=0.1, collision="mrt", mrt_rates=(om, om, om))
    c, d = gpu_solver(wl), gpu_solver(wm)
    c.step(15)
    d.step(15)
    err = max_errors(gpu_fields(c), gpu_fields(d))
    assert all(v < 1e-6 for v in err.values()), err
    e = gpu_solver(_mrt(_film3d(32, 12, 24), (1.1, 1.6, 1.8), G_RATES))
    e.step(15)
    assert np.abs(gpu_fields(e)["phi"] - gpu_fields(c)["phi"]).max() > 1e-7


def test_mrt3d_g_conserves_phi_mass_with_the_source_off():
    def make(mrt):
        w = _film3d(24, 16, 20, periodic_z=True)
        if mrt:
            _mrt(w, (1.3, 1.1, 1.6), G_RATES)
        w.params.update(source_on=0)
        return w
    _assert_mass_kept(make(True), make(False), 100)


def _poiseuille3d_error(rates, nu=0.5, H=8, G=1e-5, steps=1500):
    params = W.base_params(rho_l=1.0, rho_g=1.0, nu_l=nu, nu_g=nu, alpha_l=0.05, alpha_g=0.05, sigma=0.0,
                           gravity=(0.0, 0.0, 0.0), body_force=(G, 0.0, 0.0), source_on=0,
                           phi_wall=(0.0, 0.0), T_wall=(1.0, 1.0), collision="mrt", mrt_rates=rates)
    from paper_2003_06342_b300 import Solver
    s = Solver((4, 4, H), (True, True, False), params)
    s.init(np.zeros((H, 4, 4)), np.ones((H, 4, 4)))
    s.step(steps)
    u = s.fields()["u"][0].double().cpu().numpy()[:, 0, 0]
    z = np.arange(H)
    exact = G / (2 * nu) * (z + 0.5) * (H - 0.5 - z)
    return float(np.abs(u - exact).max() / exact.max())


def test_mrt3d_magic_rate_poiseuille_on_gpu():
    s_nu = 1.0 / (0.5 * 3.0 + 0.5)
    s_q = 8.0 * (2.0 - s_nu) / (8.0 - s_nu)
    err_magic, err_off = _poiseuille3d_error((1.1, 1.3, s_q)), _poiseuille3d_error((1.1, 1.3, 1.9))
    print("3d poiseuille rel err MRT magic", err_magic, "off", err_off)
    assert err_magic < 1e-4
    assert err_off > 1e-3
