"""16-bit population storage against the FP64 oracle (error stated per
field), and the GPU path against the paper's closed-form validation cases at
the paper's sizes (Sec. 4): Stefan problem on 512 cells for 2e5 steps,
layered Poiseuille flow on a 100-cell channel, Laplace law for three radii."""
import numpy as np
import pytest

import workloads as W
from oracle import closed_forms as CF

from _parity import gpu_fields, gpu_solver, max_errors, oracle_fields

pytestmark = pytest.mark.gpu

# max-abs error bounds of 16-bit storage after STORAGE_STEPS steps of the
# 128 x 96 film-boiling case, per field (measured values are printed)
STORAGE_STEPS = 200
STORAGE_BOUNDS = {
    "fp16": {"phi": 5e-3, "T": 5e-3, "u": 5e-4, "p": 5e-3},
    "bf16": {"phi": 5e-2, "T": 5e-2, "u": 5e-3, "p": 5e-2},
}


def _film():
    return W.film_boiling_2d(128, 96, rho_ratio=10.0, y0=30.0, amplitude=2.0, phi_wall=(1.0, 0.0))


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_16bit_storage_error_2d(storage):
    w = _film()
    ref = oracle_fields(w, STORAGE_STEPS)
    s = gpu_solver(w, storage=storage)
    s.step(STORAGE_STEPS)
    got = gpu_fields(s)
    err = max_errors(got, ref)
    print(f"{storage} 2d errors after {STORAGE_STEPS} steps:", err)
    for k, bound in STORAGE_BOUNDS[storage].items():
        assert np.isfinite(err[k]) and err[k] < bound, (storage, k, err)


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_16bit_storage_error_3d(storage):
    w = W.film_boiling_3d(40, 24, 30, modes=2, z0=10.0, phi_wall=(1.0, 0.0))
    ref = oracle_fields(w, 30)
    s = gpu_solver(w, storage=storage)
    s.step(30)
    err = max_errors(gpu_fields(s), ref)
    print(f"{storage} 3d errors after 30 steps:", err)
    for k, bound in STORAGE_BOUNDS[storage].items():
        assert np.isfinite(err[k]) and err[k] < bound, (storage, k, err)


@pytest.mark.parametrize("alpha_l,alpha_g,theta_I", [(0.14, 0.14, 0.0), (0.14, 0.014, 0.05)])
def test_stefan_paper_size(alpha_l, alpha_g, theta_I):
    """Sec. 4.2 at the paper's resolution: 512 x 32 cells (here 512 x 2, the
    problem is 1D), W = 3, M = 0.08, t_f = 2e5 steps."""
    steps = 200_000
    w = W.stefan_1d(nx=512, ny=2, alpha_l=alpha_l, alpha_g=alpha_g, theta_I=theta_I)
    s = gpu_solver(w)
    s.step(steps)
    F = gpu_fields(s)
    x = np.arange(512) + 0.5
    phi = F["phi"][0]
    j = int(np.argmax(phi > 0.5))
    xI = x[j - 1] + (0.5 - phi[j - 1]) / (phi[j] - phi[j - 1])
    xi = CF.stefan_xi(alpha_l, alpha_g, -0.3, 0.3, theta_I)
    exact_xI = CF.stefan_interface(steps, xi, alpha_l)
    theta = F["T"][0] - 1.0
    exact = CF.stefan_theta(x, steps, xi, alpha_l, alpha_g, -0.3, 0.3, theta_I)
    print("stefan", alpha_l, alpha_g, theta_I, "xI", xI, "exact", exact_xI,
          "theta max err", np.abs(theta - exact)[:400].max())
    assert abs(xI - exact_xI) < 1.0 + 0.01 * exact_xI
    assert np.abs(theta - exact)[:400].max() < 0.02


@pytest.mark.parametrize("nu_A,nu_B,rho_A,rho_B", [(0.1, 0.3, 1.0, 1.0), (0.07, 0.35, 1.0, 1.0),
                                                   (0.07, 0.07, 1.0, 2.0)])
def test_layered_poiseuille_100_cells(nu_A, nu_B, rho_A, rho_B):
    ny = 100
    w = W.layered_poiseuille(ny=ny, nx=4, nu_A=nu_A, nu_B=nu_B, rho_A=rho_A, rho_B=rho_B)
    s = gpu_solver(w)
    s.step(150_000)
    F = gpu_fields(s)
    ux = F["u"][0][:, 0]
    y = np.arange(ny) + 0.5 - ny / 2.0
    e = w.extra
    exact = CF.layered_poiseuille(y, e["h"], e["G"], e["eta_A"], e["eta_B"])
    rel = np.linalg.norm(ux - exact) / np.linalg.norm(exact)
    print("poiseuille", nu_A, nu_B, rho_A, rho_B, "rel L2", rel)
    assert rel < 0.02


def test_laplace_law_slope():
    n, sigma = 128, 0.02
    dps, inv_R = [], []
    for R in (16.0, 24.0, 32.0):
        w = W.static_drop_2d(n=n, radius=R, sigma=sigma)
        s = gpu_solver(w)
        s.step(20_000)
        p = gpu_fields(s)["p"]
        dps.append(p[n // 2, n // 2] - p[0, 0])
        inv_R.append(1.0 / R)
    slope = np.polyfit(inv_R, dps, 1)[0]
    print("laplace dp", dps, "slope", slope, "sigma", sigma)
    assert abs(slope / sigma - 1.0) < 0.05
    for dp, ir in zip(dps, inv_R):
        assert abs(dp / (sigma * ir) - 1.0) < 0.08
