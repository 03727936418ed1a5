"""Pins of the oracle's step against identities the method must satisfy:
moment consistency of the initial state (App. C variable change), the
moments of the source terms (Eqs. Forcing, SourceTerm_AllenCahn), the
equivalence of the two phase-field collisions (App. C.2), conservation of
phase-field mass with the source off (Eq. Moment_Phi, sum F^g = 0) and the
streaming map against a brute-force loop."""
import itertools

import numpy as np
import pytest
import torch

import workloads as W
from oracle import lattice as Lt
from oracle import model as M


def _grid(w):
    return M.Grid(w.n, w.periodic)


def _small_film_2d():
    return W.film_boiling_2d(24, 20, rho_ratio=10.0, y0=7.0, amplitude=1.5)


def _small_film_3d():
    return W.film_boiling_3d(10, 8, 12, rho_ratio=5.0, modes=2, z0=5.0)


@pytest.mark.parametrize("make", [_small_film_2d, _small_film_3d], ids=["2d", "3d"])
def test_init_moments_return_initial_fields(make):
    w = make()
    G, P = _grid(w), M.Params.from_dict(w.params)
    rng = np.random.default_rng(5)
    u0 = [torch.tensor(rng.uniform(-1e-3, 1e-3, w.phi0.shape)) for _ in range(w.dim)]
    st = M.init_state(w.phi0, w.T0, P, G, u0=u0, p0=w.p0)
    F = M.fields(st, P, G)
    assert torch.allclose(F["phi"], torch.tensor(w.phi0), atol=1e-14, rtol=0)
    assert torch.allclose(F["T"], torch.tensor(w.T0), atol=1e-14, rtol=0)
    assert torch.allclose(F["p"], torch.tensor(w.p0), atol=1e-15, rtol=0)
    for a in range(w.dim):
        assert torch.allclose(F["u"][a], u0[a], atol=1e-16, rtol=0)


@pytest.mark.parametrize("make", [_small_film_2d, _small_film_3d], ids=["2d", "3d"])
def test_source_term_moments(make):
    """sum_i F^g_i = 0, sum_i P^g_i = q, sum_i F^f_i = cs^2 u.grad(rho),
    sum_i F^f_i c_i = cs^2 F_tot, sum_i S^s_i = -(L/Cp) D."""
    w = make()
    G, P = _grid(w), M.Params.from_dict(w.params)
    st = M.init_state(w.phi0, w.T0, P, G, p0=w.p0)
    st = M.run(st, P, G, 3)
    Mo = M.moments(st, P, G)
    q = M.production_rate(Mo["phi"], Mo["T"], P)
    assert q.abs().max() > 1e-6
    E = M.equilibria_and_sources(Mo["phi"], st["phi_prev"], Mo["u"], Mo["p"], Mo["T"], q, Mo, P, G)
    Lf, Lg, _ = Lt.lattices_for(w.dim)
    g_eq, g_F, g_P, _, _ = E["g"]
    assert sum(g_F).abs().max() < 1e-15
    assert torch.allclose(sum(g_P), q, atol=1e-16)
    assert torch.allclose(sum(g_eq), Mo["phi"], atol=1e-14)
    f_eq, f_S, _ = E["f"]
    cs2 = float(Lf.cs2)
    kappa = 1.0 - P.rho_g / P.rho_l
    u_grad_rho = sum(Mo["u"][a] * Mo["grad_rho"][a] for a in range(w.dim))
    expect = cs2 * u_grad_rho + Mo["rho"] * cs2 * q * kappa
    assert torch.allclose(sum(f_S), expect, atol=1e-15)
    assert torch.allclose(sum(f_eq), Mo["p"], atol=1e-15)
    for a in range(w.dim):
        first = sum(f_S[i] * float(Lf.e[i][a]) for i in range(Lf.Q))
        assert torch.allclose(first, cs2 * Mo["F_tot"][a], atol=1e-15)
    s_eq, s_S, _ = E["s"]
    D = (Mo["phi"] - st["phi_prev"]) + sum(Mo["u"][a] * Mo["grad"][a] for a in range(w.dim)) \
        + Mo["phi"] * q * kappa
    assert torch.allclose(sum(s_S), -(P.L / P.Cp) * D, atol=1e-15)
    assert torch.allclose(sum(s_eq), Mo["T"], atol=1e-14)


@pytest.mark.parametrize("make", [_small_film_2d, _small_film_3d], ids=["2d", "3d"])
def test_cac_forms_equivalent(make):
    """App. C.2: the source form and the modified-equilibrium form of the
    phase-field collision give the same post-collision populations."""
    w = make()
    G = _grid(w)
    P1 = M.Params.from_dict(w.params)
    P2 = M.Params.from_dict(w.params)
    P2.g_form = "cac_eq"
    s1 = M.init_state(w.phi0, w.T0, P1, G, p0=w.p0)
    s2 = {k: v.clone() for k, v in s1.items()}
    for _ in range(20):
        s1 = M.step(s1, P1, G)
        s2 = M.step(s2, P2, G)
    for k in ("f", "g", "s", "phi_prev", "q_prev"):
        assert (s1[k] - s2[k]).abs().max() < 1e-13, k


@pytest.mark.parametrize("dim", [2, 3])
def test_mass_conserved_without_source(dim):
    if dim == 2:
        w = W.droplet_2d(32, 8.0, source_on=0)
    else:
        w = W.film_boiling_3d(8, 8, 10, rho_ratio=3.0, modes=1, z0=5.0, source_on=0)
        w.periodic = (True, True, True)
        w.params["gravity"] = (0.0, 0.0, 0.0)
    G, P = _grid(w), M.Params.from_dict(w.params)
    st = M.init_state(w.phi0, w.T0, P, G)
    m0, _ = M.reductions(st, P, G)
    st = M.run(st, P, G, 60)
    m1, _ = M.reductions(st, P, G)
    assert abs(m1 - m0) < 1e-12 * w.cells
    # and the field did evolve
    assert (M.fields(st, P, G)["phi"] - torch.tensor(w.phi0)).abs().max() > 1e-6


def test_mass_changes_with_source():
    """With the source on and a superheated vapour around a liquid drop, the
    vapour fraction sum(phi) grows (evaporation, Eq. ProductionRate)."""
    w = W.droplet_2d(32, 8.0, T_offset=0.05, T_noise=0.0)
    G, P = _grid(w), M.Params.from_dict(w.params)
    st = M.init_state(w.phi0, w.T0, P, G)
    m0, _ = M.reductions(st, P, G)
    st = M.run(st, P, G, 40)
    m1, _ = M.reductions(st, P, G)
    assert m1 > m0 + 1e-4


def _brute_stream_map(lat, n, periodic):
    """Pure-Python loop version of the pull map, for tiny grids."""
    dim = len(n)
    N = int(np.prod(n))
    src = np.zeros((lat.Q, N), dtype=np.int64)
    kind = np.zeros((lat.Q, N), dtype=np.int8)
    for i in range(lat.Q):
        for coords in itertools.product(*[range(m) for m in n]):   # coords = (x, y[, z])
            lin = 0
            for a in reversed(range(dim)):
                lin = lin * n[a] + coords[a]
            s = [coords[a] - int(lat.e[i][a]) for a in range(dim)]
            k = 0
            for a in range(dim):
                if s[a] < 0 or s[a] >= n[a]:
                    if periodic[a]:
                        k = max(k, 1)
                        s[a] %= n[a]
                    else:
                        k = 2 if s[a] < 0 else 3
            if k >= 2:
                src[i, lin], kind[i, lin] = lin, k
            else:
                sl = 0
                for a in reversed(range(dim)):
                    sl = sl * n[a] + s[a]
                src[i, lin], kind[i, lin] = sl, k
    return src, kind


@pytest.mark.parametrize("lat,n,periodic", [
    (Lt.D2Q9, (5, 4), (True, False)),
    (Lt.D2Q9, (4, 3), (False, True)),
    (Lt.D2Q9, (3, 3), (True, True)),
    (Lt.D3Q19, (3, 4, 3), (True, True, False)),
    (Lt.D3Q7, (3, 2, 4), (True, True, False)),
])
def test_stream_map_brute_force(lat, n, periodic):
    src, kind = M.stream_map(lat, M.Grid(n, periodic))
    bsrc, bkind = _brute_stream_map(lat, n, periodic)
    assert np.array_equal(src, bsrc)
    assert np.array_equal(kind, bkind)


def test_stream_is_permutation_and_bounce_conserves_f():
    G = M.Grid((7, 5), (True, False))
    P = M.Params(rho_l=1, rho_g=1, nu_l=.1, nu_g=.1, alpha_l=.1, alpha_g=.1, sigma=0, W=4,
                 M_phi=.1, phi_wall=(0.0, 0.0), T_wall=(0.0, 0.0))
    post = torch.rand((9, 5, 7), dtype=torch.float64, generator=torch.Generator().manual_seed(0))
    out = M.stream(post, Lt.D2Q9, G, "f", P)
    # half-way bounce-back moves every value exactly once
    assert torch.equal(torch.sort(out.reshape(-1)).values, torch.sort(post.reshape(-1)).values)
    # anti bounce-back with zero wall values flips the sign of bounced values
    out_g = M.stream(post, Lt.D2Q9, G, "g", P)
    src, kind = M.stream_map(Lt.D2Q9, G)
    bounced = torch.from_numpy(kind >= 2).reshape(9, 5, 7)
    assert torch.equal(out_g[bounced], -out[bounced])
    assert torch.equal(out_g[~bounced], out[~bounced])


# ---------------------------------------------------------------- mass and enthalpy bookkeeping

def test_energy_sum_hand_value_two_phase_box():
    """reductions() on a box that is vapour (phi = 1) in its left half and
    liquid (phi = 0) in its right half at a uniform temperature: the
    initialisation returns phi and T exactly, so the enthalpy sum is
    N_g rho_g (Cp T + L) + N_l rho_l Cp T and the mass sum N_g."""
    nx, ny, T0 = 12, 10, 1.05
    params = W.base_params(rho_l=10.0, rho_g=1.0, Cp=2.0, L=0.7, T_sat=1.0, gravity=(0.0, 0.0, 0.0))
    phi0 = np.zeros((ny, nx))
    phi0[:, : nx // 2] = 1.0
    w = W.Workload("box", (nx, ny), (True, True), params, phi0, np.full_like(phi0, T0))
    G, P = _grid(w), M.Params.from_dict(w.params)
    mass, energy = M.reductions(M.init_state(w.phi0, w.T0, P, G), P, G)
    ng = nx // 2 * ny
    nl = nx * ny - ng
    assert mass == pytest.approx(ng, rel=1e-14)
    hand = ng * 1.0 * (2.0 * T0 + 0.7) + nl * 10.0 * 2.0 * T0
    assert energy == pytest.approx(hand, rel=1e-14)


def _omega_g(P, dim=2):
    cs2 = 1.0 / 3.0 if dim == 2 else 0.25
    return 1.0 / (P.M_phi / cs2 + 0.5)


def test_phase_mass_balance_with_source():
    """Periodic box with phase change: summing Eq. LBE for g over directions
    and cells (sum Gamma_i = 1, sum F^g_i = 0, sum P^g_i = q) and the lagged
    moment phi = sum g + q^{n-1}/2 gives, step by step,
    sum phi^{n+1} - sum phi^n = sum q^n + (1 - omega_g)/2 (sum q^n - sum q^{n-1})."""
    w = W.droplet_2d(32, 8.0, T_offset=0.06, T_noise=0.01, corr_len=4.0)
    G, P = _grid(w), M.Params.from_dict(w.params)
    om = _omega_g(P)
    st = M.init_state(w.phi0, w.T0, P, G)
    m_prev = M.reductions(st, P, G)[0]
    q_prev = float(st["q_prev"].sum())
    moved = 0.0
    for _ in range(25):
        st = M.step(st, P, G)
        q = float(st["q_prev"].sum())
        m = M.reductions(st, P, G)[0]
        expect = q + 0.5 * (1.0 - om) * (q - q_prev)
        assert m - m_prev == pytest.approx(expect, rel=1e-9, abs=1e-12)
        moved += abs(m - m_prev)
        m_prev, q_prev = m, q
    assert moved > 1e-3          # the source did act


def test_enthalpy_invariant_with_phase_change():
    """Equal densities, no surface tension and no gravity: the flow stays at
    rest, and summing the temperature scheme (Eq. LBE for s with the source
    of Eq. Def_SourceTerms_Temp, moment Eq. Moment_Temp) over a periodic box
    leaves sum [Cp T^n + L (phi^n + phi^{n-1})/2] unchanged while phase
    change moves phi; the energy sum of reductions() is then
    rho (H_0 + L/2 (sum phi^n - sum phi^{n-1}))."""
    w = W.droplet_2d(32, 8.0, T_offset=0.08, T_noise=0.01, corr_len=4.0,
                     rho_l=1.0, rho_g=1.0, sigma=0.0, Cp=1.5, L=0.8)
    G, P = _grid(w), M.Params.from_dict(w.params)
    st = M.init_state(w.phi0, w.T0, P, G)
    H0 = float((P.Cp * torch.as_tensor(w.T0) + P.L * torch.as_tensor(w.phi0)).sum())
    m0 = M.reductions(st, P, G)[0]
    for _ in range(30):
        st = M.step(st, P, G)
        F = M.fields(st, P, G)
        assert max(float(u.abs().max()) for u in F["u"]) == 0.0
        phi, phi_prev = F["phi"], st["phi_prev"]
        H = float((P.Cp * F["T"] + 0.5 * P.L * (phi + phi_prev)).sum())
        assert H == pytest.approx(H0, rel=1e-13)
        mass, energy = M.reductions(st, P, G)
        assert energy == pytest.approx(1.0 * (H0 + 0.5 * P.L * (float(phi.sum()) - float(phi_prev.sum()))),
                                       rel=1e-13)
    assert abs(mass - m0) > 1e-3          # phase change happened


def test_flat_interface_profile_is_stationary_over_1e4_steps():
    """Two flat interfaces of width W = 4 at rest (phase field alone, Sec.
    4.1 setting): within 1000 steps the profile settles on the scheme's
    discrete equilibrium (within 6e-3 of the continuous kernel
    1/2 [1 + tanh(2 d / W)] of Eq. Geq_Allen-Cahn's derivation) and then stays
    put: over the next 9000 steps it moves by less than 1e-5, and sum phi is
    conserved."""
    from oracle import cac as C
    n, Wd = 48, 4.0
    params = W.base_params(rho_l=1.0, rho_g=1.0, nu_l=0.1, nu_g=0.1, sigma=0.0, W=Wd, M_phi=0.08,
                           gravity=(0.0, 0.0, 0.0), source_on=0)
    y = np.arange(n) + 0.5
    prof = 0.5 * (1 + np.tanh(2 * (y - 12) / Wd)) - 0.5 * (1 + np.tanh(2 * (y - 36) / Wd))
    phi0 = np.broadcast_to(prof[:, None], (n, 3)).copy()
    G, P = M.Grid((3, n), (True, True)), M.Params.from_dict(params)
    u = [np.zeros_like(phi0), np.zeros_like(phi0)]
    g = C.run(C.init_state(phi0, u, P, G), u, P, G, 1000)
    a = C.phase_field(g).numpy()
    g = C.run(g, u, P, G, 9000)
    b = C.phase_field(g).numpy()
    assert np.abs(a - phi0).max() < 6e-3
    assert np.abs(b - a).max() < 1e-5
    assert abs(b.sum() - phi0.sum()) < 1e-10
