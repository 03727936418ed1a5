"""The CUDA discrete adjoint against the FP64 oracle's reverse-mode
gradients (torch autograd through oracle.model.step), for dJ/dL, dJ/dM_phi,
dJ/dsigma and the field dJ/dT_0; J = 1/2 sum (phi^N - phi_target)^2.
Relative tolerance 1e-4 on the scalars (the bound stated for the adjoint) and
on the T_0 gradient field (max-abs difference over max-abs value)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import adjoint as A
from oracle import model as M

pytestmark = pytest.mark.gpu
TOL = 1e-4

CASES = [
    ("droplet_periodic", lambda: W.droplet_2d(24, 6.0, T_offset=0.04, T_noise=0.01, corr_len=4.0), 10, 4),
    ("film_walls", lambda: W.film_boiling_2d(20, 18, rho_ratio=5.0, y0=7.0, amplitude=1.5,
                                             phi_wall=(1.0, 0.0), theta_I=0.05), 8, 3),
]


@pytest.mark.parametrize("name,make,steps,K", CASES, ids=[c[0] for c in CASES])
def test_gpu_adjoint_matches_oracle(name, make, steps, K):
    from paper_2003_06342_b300.adjoint import gradients
    w = make()
    target = w.phi0.copy()
    G = M.Grid(w.n, w.periodic)
    J_ref, g_ref = A.gradients(w.phi0, w.T0, w.params, G, steps, target, p0=w.p0)
    J, g = gradients(w.n, w.periodic, w.params, w.phi0, w.T0, target, steps, K=K, p0=w.p0)
    print(name, "J", J, J_ref, {k: (g[k], g_ref[k]) for k in ("L", "M_phi", "sigma")})
    assert abs(J - J_ref) <= 1e-4 * abs(J_ref)
    for k in ("L", "M_phi", "sigma"):
        assert abs(g[k] - g_ref[k]) <= TOL * abs(g_ref[k]) + 1e-12, (k, g[k], g_ref[k])
    dT = g["T0"].double().cpu().numpy()
    dT_ref = g_ref["T0"].numpy()
    err = np.abs(dT - dT_ref).max() / np.abs(dT_ref).max()
    print(name, "T0 gradient rel err", err)
    assert err <= TOL


def test_checkpoint_interval_does_not_change_gradients():
    from paper_2003_06342_b300.adjoint import gradients
    w = W.droplet_2d(24, 6.0, T_offset=0.04, T_noise=0.01, corr_len=4.0)
    a = gradients(w.n, w.periodic, w.params, w.phi0, w.T0, w.phi0, 9, K=9)
    b = gradients(w.n, w.periodic, w.params, w.phi0, w.T0, w.phi0, 9, K=2)
    # the per-field adjoint is deterministic; the FP64 parameter sums are
    # accumulated with atomics, so only their last bits may differ
    assert abs(a[0] - b[0]) <= 1e-12 * abs(a[0])
    for k in ("L", "M_phi", "sigma"):
        assert abs(a[1][k] - b[1][k]) <= 1e-12 * abs(a[1][k])
    assert torch.equal(a[1]["T0"], b[1]["T0"])


def test_autograd_function():
    from paper_2003_06342_b300.adjoint import FinalPhiMisfit, gradients
    w = W.droplet_2d(24, 6.0, T_offset=0.04, T_noise=0.01, corr_len=4.0)
    T0 = torch.tensor(w.T0, dtype=torch.float32, device="cuda", requires_grad=True)
    L = torch.tensor(w.params["L"], dtype=torch.float64, requires_grad=True)
    Mp = torch.tensor(w.params["M_phi"], dtype=torch.float64, requires_grad=True)
    sg = torch.tensor(w.params["sigma"], dtype=torch.float64, requires_grad=True)
    J = FinalPhiMisfit.apply(T0, L, Mp, sg, w.n, w.periodic, w.params, w.phi0, w.phi0, 5, 2)
    J.backward()
    J2, g = gradients(w.n, w.periodic, w.params, w.phi0, w.T0, w.phi0, 5, K=2)
    assert abs(float(J) - J2) <= 1e-12 * abs(J2)
    assert abs(float(L.grad) - g["L"]) <= 1e-12 * abs(g["L"])
    assert torch.allclose(T0.grad, g["T0"])


def test_gpu_adjoint_matches_central_differences():
    """The CUDA adjoint's gradients against central differences of J taken
    on the FP64 oracle's forward map (step 1e-5 relative for the scalars; for
    T_0 the directional derivative along a seeded Gaussian field)."""
    from paper_2003_06342_b300.adjoint import gradients
    w = W.droplet_2d(24, 6.0, T_offset=0.04, T_noise=0.01, corr_len=4.0)
    target = np.roll(w.phi0, 1, axis=1)
    steps = 10
    G = M.Grid(w.n, w.periodic)
    J, g = gradients(w.n, w.periodic, w.params, w.phi0, w.T0, target, steps, K=4, p0=w.p0)
    for k in ("L", "M_phi", "sigma"):
        h = 1e-5 * abs(w.params[k])
        fd = A.central_difference(w.phi0, w.T0, w.params, G, steps, target, k, h, p0=w.p0)
        print(k, g[k], fd)
        assert abs(g[k] - fd) <= TOL * abs(fd), (k, g[k], fd)
    d = np.random.Generator(np.random.PCG64(11)).standard_normal(w.T0.shape)
    fd = A.central_difference(w.phi0, w.T0, w.params, G, steps, target, "T0", 1e-4, direction=d,
                              p0=w.p0)
    ad = float((g["T0"].double().cpu().numpy() * d).sum())
    print("T0 direction", ad, fd)
    assert abs(ad - fd) <= TOL * abs(fd)


def test_segment_calls_match_single_steps():
    """lbm_step_record keeps exactly the states that stepping and reading the
    state one step at a time gives, and lbm_adjoint_steps over a segment
    equals the same number of lbm_adjoint_step calls."""
    import ctypes
    from paper_2003_06342_b300 import Solver
    from paper_2003_06342_b300 import _binding as Bd
    w = W.droplet_2d(40, 9.0, T_offset=0.04, T_noise=0.01, corr_len=4.0)
    n = 5
    a = Solver(w.n, w.periodic, w.params).init(w.phi0, w.T0)
    b = Solver(w.n, w.periodic, w.params).init(w.phi0, w.T0)
    nb = a.state_bytes()
    rec = torch.zeros((n, nb), dtype=torch.uint8, device="cuda")
    vp = lambda t: ctypes.c_void_p(t.data_ptr())
    Bd.check(Bd.lib.lbm_step_record(a._h, n, vp(rec), rec.stride(0)), "lbm_step_record")
    for k in range(n):
        b.step(1)
        assert torch.equal(rec[k], b.get_state())
    assert a.steps_done() == n
    assert torch.equal(a.get_state(), b.get_state())     # the handle holds the last state
    # 16-bit storage records the same way, and so does the copying path
    # (an unaligned stride)
    for storage, pad in (("fp16", 0), ("fp32", 4)):
        c = Solver(w.n, w.periodic, w.params, storage=storage).init(w.phi0, w.T0)
        d = Solver(w.n, w.periodic, w.params, storage=storage).init(w.phi0, w.T0)
        nbc = c.state_bytes()
        rc = torch.zeros((n, nbc + pad), dtype=torch.uint8, device="cuda")
        Bd.check(Bd.lib.lbm_step_record(c._h, n, vp(rc), rc.stride(0)), "lbm_step_record")
        for k in range(n):
            d.step(1)
            assert torch.equal(rc[k, :nbc], d.get_state()), (storage, pad, k)
        assert torch.equal(c.get_state(), d.get_state()) and c.steps_done() == n
    # reverse over the recorded states both ways
    ab, sb = ctypes.c_size_t(), ctypes.c_size_t()
    Bd.check(Bd.lib.lbm_adjoint_bytes(a._h, ctypes.byref(ab), ctypes.byref(sb)), "bytes")
    seed = torch.randn(ab.value // 4, device="cuda")
    scr = torch.zeros(sb.value // 4, device="cuda")
    l1, l2 = seed.clone(), torch.zeros_like(seed)
    d1 = torch.zeros(3, dtype=torch.float64, device="cuda")
    for k in reversed(range(n)):
        Bd.check(Bd.lib.lbm_adjoint_step(a._h, vp(rec[k]), vp(l1), vp(l2), vp(scr), vp(d1)), "step")
        l1, l2 = l2, l1
    m1, m2 = seed.clone(), torch.zeros_like(seed)
    d2 = torch.zeros(3, dtype=torch.float64, device="cuda")
    Bd.check(Bd.lib.lbm_adjoint_steps(a._h, vp(rec), rec.stride(0), n, vp(m1), vp(m2), vp(scr), vp(d2)),
             "steps")
    res = m2 if n % 2 else m1
    torch.cuda.synchronize()
    assert torch.equal(res, l1)
    assert torch.allclose(d1, d2, rtol=1e-12, atol=0.0)


# Grids that span several tiles of the reverse kernel (32 x 4 cells) in both
# directions, step counts that the checkpoint interval does not divide, and
# targets that differ from the initial phase field.
MULTI_TILE_CASES = [
    ("film_walls_96x40", lambda: W.film_boiling_2d(96, 40, rho_ratio=5.0, y0=13.0, amplitude=1.5,
                                                   phi_wall=(1.0, 0.0), theta_I=0.05),
     30, 7, lambda phi: np.roll(phi, 3, axis=1)),
    ("droplet_periodic_80", lambda: W.droplet_2d(80, 14.0, T_offset=0.04, T_noise=0.01, corr_len=6.0),
     30, 8, lambda phi: np.roll(phi, (2, 3), axis=(0, 1))),
]


def _compare(g, g_ref, J, J_ref, tol=TOL, J_tol=1e-4):
    print("J", J, J_ref, {k: (g[k], g_ref[k]) for k in ("L", "M_phi", "sigma")})
    for k in ("L", "M_phi", "sigma"):
        assert abs(g[k] - g_ref[k]) <= tol * abs(g_ref[k]) + 1e-12, (k, g[k], g_ref[k])
    dT = g["T0"].double().cpu().numpy()
    dT_ref = g_ref["T0"].numpy()
    err = np.abs(dT - dT_ref).max() / np.abs(dT_ref).max()
    assert err <= tol, err
    assert abs(J - J_ref) <= J_tol * abs(J_ref), (J, J_ref)
    return err


@pytest.mark.parametrize("name,make,steps,K,target", MULTI_TILE_CASES, ids=[c[0] for c in MULTI_TILE_CASES])
def test_gpu_adjoint_multi_tile_matches_oracle(name, make, steps, K, target):
    from paper_2003_06342_b300.adjoint import gradients
    w = make()
    tgt = target(w.phi0)
    G = M.Grid(w.n, w.periodic)
    J_ref, g_ref = A.gradients(w.phi0, w.T0, w.params, G, steps, tgt, p0=w.p0, segment=10)
    J, g = gradients(w.n, w.periodic, w.params, w.phi0, w.T0, tgt, steps, K=K, p0=w.p0)
    err = _compare(g, g_ref, J, J_ref)
    print(name, {k: (g[k], g_ref[k]) for k in ("L", "M_phi", "sigma")}, "T0 rel err", err)


def test_gpu_adjoint_multi_tile_matches_central_differences():
    """The 96 x 40 walled film: the CUDA gradients against central
    differences of J on the FP64 oracle's forward map."""
    from paper_2003_06342_b300.adjoint import gradients
    name, make, steps, K, target = MULTI_TILE_CASES[0]
    w = make()
    tgt = target(w.phi0)
    G = M.Grid(w.n, w.periodic)
    J, g = gradients(w.n, w.periodic, w.params, w.phi0, w.T0, tgt, steps, K=K, p0=w.p0)
    for k in ("L", "M_phi", "sigma"):
        h = 1e-5 * abs(w.params[k])
        fd = A.central_difference(w.phi0, w.T0, w.params, G, steps, tgt, k, h, p0=w.p0)
        assert abs(g[k] - fd) <= TOL * abs(fd), (k, g[k], fd)
    d = np.random.Generator(np.random.PCG64(12)).standard_normal(w.T0.shape)
    fd = A.central_difference(w.phi0, w.T0, w.params, G, steps, tgt, "T0", 1e-4, direction=d, p0=w.p0)
    ad = float((g["T0"].double().cpu().numpy() * d).sum())
    assert abs(ad - fd) <= TOL * abs(fd), (ad, fd)


def test_gpu_adjoint_reduced_droplet_job():
    """The evaporating-droplet gradient job at reduced size: 128^2 periodic
    box, radius 10, 200 steps, checkpoint every 20, against a target
    displaced by two cells.  GPU gradients within 1e-4 relative of the
    oracle's reverse mode.  (With the large job's target, a run with L x 1.05,
    M_phi x 0.95 and sigma x 1.1, the misfit at this size is only ~1e-3 per
    interface cell, so the FP32 forward trajectory alone, ~1e-6 from the FP64
    one, moves J and its gradients by several 1e-4.)"""
    from paper_2003_06342_b300.adjoint import gradients
    w = W.droplet_2d(128, 10.0, seed=3, corr_len=4.0)
    steps = 200
    G = M.Grid(w.n, w.periodic)
    tgt = np.roll(w.phi0, 2, axis=1)
    J_ref, g_ref = A.gradients(w.phi0, w.T0, w.params, G, steps, tgt, segment=20)
    J, g = gradients(w.n, w.periodic, w.params, w.phi0, w.T0, tgt, steps, K=20)
    err = _compare(g, g_ref, J, J_ref)
    print("droplet 128", {k: (g[k], g_ref[k]) for k in ("L", "M_phi", "sigma")}, "T0 rel err", err)


BIASED_CASES = [
    ("film_walls_biased", lambda: W.film_boiling_2d(96, 40, rho_ratio=5.0, y0=13.0, amplitude=1.5,
                                                    phi_wall=(1.0, 0.0), theta_I=0.05, grad_scheme="biased2"),
     20, 6, lambda phi: np.roll(phi, 3, axis=1)),
    ("droplet_periodic_biased", lambda: W.droplet_2d(48, 10.0, T_offset=0.04, T_noise=0.01, corr_len=5.0,
                                                     grad_scheme="biased2"),
     20, 7, lambda phi: np.roll(phi, (1, 2), axis=(0, 1))),
]


@pytest.mark.parametrize("name,make,steps,K,target", BIASED_CASES, ids=[c[0] for c in BIASED_CASES])
def test_gpu_adjoint_biased_gradient_matches_oracle(name, make, steps, K, target):
    """The adjoint with the second-order biased gradient (two-ring window in
    kernel A, near and far contributions in kernel B, the biased gradient in
    the initialisation) against the oracle's reverse mode."""
    from paper_2003_06342_b300.adjoint import gradients
    w = make()
    tgt = target(w.phi0)
    G = M.Grid(w.n, w.periodic)
    J_ref, g_ref = A.gradients(w.phi0, w.T0, w.params, G, steps, tgt, p0=w.p0, segment=10)
    J, g = gradients(w.n, w.periodic, w.params, w.phi0, w.T0, tgt, steps, K=K, p0=w.p0)
    err = _compare(g, g_ref, J, J_ref)
    print(name, {k: (g[k], g_ref[k]) for k in ("L", "M_phi", "sigma")}, "T0 rel err", err)
