"""The oracle's coupled step against the paper's validation cases (Sec. 4):
1D Stefan problem (closed form with the root of Eq. SolStefan_TranscendEq),
layered Poiseuille flow (Eq. AnalyticalSol_Poiseuille-1), Laplace law
(Eq. LaplaceLaw) and stationarity of the kernel profile (Eq. Kernel-Function)
under the conservative Allen-Cahn scheme.  Sizes are reduced so the CPU suite
stays within minutes; tolerances cover discretisation and diffuse-interface
error, and each fails on a dropped term or a wrong sign (checked by hand
when the bounds were set: a flipped counter term, buoyancy, latent heat or
forcing sign moves these quantities by far more than the bound)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import closed_forms as CF
from oracle import model as M


def _run(w, steps):
    P, G = M.Params.from_dict(w.params), M.Grid(w.n, w.periodic)
    st = M.init_state(w.phi0, w.T0, P, G, p0=w.p0)
    st = M.run(st, P, G, steps)
    return M.fields(st, P, G)


def _interface_position(phi_row, x):
    j = int(np.argmax(phi_row > 0.5))
    return x[j - 1] + (0.5 - phi_row[j - 1]) / (phi_row[j] - phi_row[j - 1])


@pytest.mark.slow
@pytest.mark.parametrize("alpha_l,alpha_g,theta_I,xtol,ttol", [
    (0.14, 0.14, 0.0, 0.3, 0.01),
    (0.14, 0.014, 0.05, 1.0, 0.025),
])
def test_stefan_problem(alpha_l, alpha_g, theta_I, xtol, ttol):
    steps = 2500
    w = W.stefan_1d(nx=96, ny=1, alpha_l=alpha_l, alpha_g=alpha_g, theta_I=theta_I)
    F = _run(w, steps)
    x = np.arange(96) + 0.5              # distance from the left (half-way) wall
    xi = CF.stefan_xi(alpha_l, alpha_g, -0.3, 0.3, theta_I)
    xI = _interface_position(F["phi"][0].numpy(), x)
    assert abs(xI - CF.stefan_interface(steps, xi, alpha_l)) < xtol
    theta = F["T"][0].numpy() - 1.0
    exact = CF.stefan_theta(x, steps, xi, alpha_l, alpha_g, -0.3, 0.3, theta_I)
    assert np.abs(theta - exact)[:60].max() < ttol
    assert np.abs(F["u"][0]).max() < 1e-12            # no flow in this case


@pytest.mark.slow
@pytest.mark.parametrize("nu_A,nu_B,rho_A,rho_B", [(0.1, 0.3, 1.0, 1.0), (0.07, 0.07, 1.0, 2.0)])
def test_layered_poiseuille(nu_A, nu_B, rho_A, rho_B):
    ny = 24
    w = W.layered_poiseuille(ny=ny, nx=2, nu_A=nu_A, nu_B=nu_B, rho_A=rho_A, rho_B=rho_B)
    F = _run(w, 5000)
    ux = F["u"][0][:, 0].numpy()
    y = np.arange(ny) + 0.5 - ny / 2.0
    e = w.extra
    exact = CF.layered_poiseuille(y, e["h"], e["G"], e["eta_A"], e["eta_B"])
    assert np.linalg.norm(ux - exact) / np.linalg.norm(exact) < 0.03
    assert np.abs(F["u"][1]).max() < 1e-3 * np.abs(exact).max()


@pytest.mark.slow
def test_laplace_law():
    sigma, R, n = 0.02, 10.0, 48
    w = W.static_drop_2d(n=n, radius=R, sigma=sigma)
    F = _run(w, 2000)
    p = F["p"].numpy()
    dp = p[n // 2, n // 2] - p[0, 0]
    assert abs(dp / CF.laplace_pressure_jump(sigma, R) - 1.0) < 0.05
    assert max(np.abs(u).max() for u in F["u"]) < 1e-4


def test_kernel_profile_is_stationary():
    n, Wd = 48, 4.0
    params = W.base_params(rho_l=1.0, rho_g=1.0, nu_l=0.1, nu_g=0.1, sigma=0.0, W=Wd, M_phi=0.08,
                           gravity=(0.0, 0.0, 0.0), source_on=0)
    y = np.arange(n) + 0.5
    prof = 0.5 * (1 + np.tanh(2 * (y - 12) / Wd)) - 0.5 * (1 + np.tanh(2 * (y - 36) / Wd))
    phi0 = np.broadcast_to(prof[:, None], (n, 3)).copy()
    w = W.Workload("slab", (3, n), (True, True), params, phi0, np.ones_like(phi0))
    F = _run(w, 800)
    assert np.abs(F["phi"].numpy() - phi0).max() < 1e-2
