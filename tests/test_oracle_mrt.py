"""Pins of the oracle's multiple-relaxation-time collision of the flow set
(collision = "mrt", D2Q9), each against something other than the MRT code:

* with every rate equal to the BGK rate it is the BGK step of Eq. LBE;
* with s_e = s_eps = the BGK rate and s_q the TRT antisymmetric rate of a
  magic parameter Lambda it is the TRT step (a different code path);
* with s_q = 8 (2 - s_nu)/(8 - s_nu) (Lambda = 3/16) the steady Poiseuille
  profile between half-way bounce-back walls is the exact parabola, also
  with s_e and s_eps away from the BGK rate, while BGK is off by percents."""
import numpy as np

import workloads as W
from oracle import model as M


def _droplet_fields(**over):
    w = W.droplet_2d(24, 6.0, T_offset=0.04, T_noise=0.01, corr_len=4.0)
    base = dict(w.params, nu_l=0.1, nu_g=0.1, alpha_l=0.05, alpha_g=0.05)
    base.update(over)
    P, G = M.Params.from_dict(base), M.Grid(w.n, w.periodic)
    return M.fields(M.run(M.init_state(w.phi0, w.T0, P, G), P, G, 12), P, G)


def _close(a, b, tol=1e-13):
    return all(float((a[k] - b[k]).abs().max()) < tol for k in ("phi", "T", "p"))


def test_mrt_with_equal_rates_is_bgk():
    om = 1.0 / (0.1 * 3.0 + 0.5)
    bgk = _droplet_fields(collision="bgk")
    mrt = _droplet_fields(collision="mrt", mrt_rates=(om, om, om))
    assert _close(bgk, mrt)
    other = _droplet_fields(collision="mrt", mrt_rates=(1.1, 1.3, 1.2))
    assert float((other["phi"] - bgk["phi"]).abs().max()) > 1e-9


def test_mrt_reduces_to_trt():
    cs2 = 1.0 / 3.0
    tau_f, tau_g, tau_s = 0.1 / cs2, 0.08 / cs2, 0.05 / cs2
    lam = 0.3
    om = 1.0 / (tau_f + 0.5)
    s_q = 1.0 / (lam / tau_f + 0.5)
    trt = _droplet_fields(collision="trt", M_phi=0.08, trt_magic=(lam, tau_g * tau_g, tau_s * tau_s))
    mrt = _droplet_fields(collision="mrt", M_phi=0.08, mrt_rates=(om, om, s_q))
    assert _close(trt, mrt)


def _poiseuille(collision, rates, nu=0.5, H=8, G=1e-5, steps=1500):
    params = W.base_params(rho_l=1.0, rho_g=1.0, nu_l=nu, nu_g=nu, alpha_l=0.05, alpha_g=0.05,
                           sigma=0.0, gravity=(0.0, 0.0, 0.0), body_force=(G, 0.0, 0.0), source_on=0,
                           phi_wall=(0.0, 0.0), T_wall=(1.0, 1.0), collision=collision, mrt_rates=rates)
    P, Gd = M.Params.from_dict(params), M.Grid((2, H), (True, False))
    st = M.run(M.init_state(np.zeros((H, 2)), np.ones((H, 2)), P, Gd), P, Gd, steps)
    u = M.fields(st, P, Gd)["u"][0][:, 0].numpy()
    y = np.arange(H)
    exact = G / (2 * nu) * (y + 0.5) * (H - 0.5 - y)
    return float(np.abs(u - exact).max() / exact.max())


def test_mrt_magic_rate_gives_the_exact_poiseuille_profile():
    s_nu = 1.0 / (0.5 * 3.0 + 0.5)
    s_q = 8.0 * (2.0 - s_nu) / (8.0 - s_nu)
    assert _poiseuille("mrt", (1.1, 1.3, s_q)) < 1e-10
    assert _poiseuille("mrt", (1.1, 1.3, 1.9)) > 1e-3
    assert _poiseuille("bgk", (1.0, 1.0, 1.0)) > 1e-2


# ---- the phase-field set (mrt_rates_g = s_e, s_eps, s_q, s_p; 0: the BGK rate)

def test_mrt_g_default_rates_are_bgk_and_other_rates_differ():
    om = 1.0 / (0.1 * 3.0 + 0.5)
    bgk = _droplet_fields(collision="bgk")
    mrt = _droplet_fields(collision="mrt", mrt_rates=(om, om, om))
    om_g = 1.0 / (bgk_tau_g() + 0.5)
    explicit = _droplet_fields(collision="mrt", mrt_rates=(om, om, om), mrt_rates_g=(om_g, om_g, om_g, om_g))
    assert _close(bgk, mrt) and _close(bgk, explicit)
    other = _droplet_fields(collision="mrt", mrt_rates=(om, om, om), mrt_rates_g=(1.2, 1.5, 1.1, 1.7))
    assert float((other["phi"] - bgk["phi"]).abs().max()) > 1e-9


def bgk_tau_g(M_phi=None):
    w = W.droplet_2d(24, 6.0)
    return (M_phi if M_phi is not None else w.params["M_phi"]) * 3.0


def test_mrt_g_reduces_to_trt_g_with_the_source_off():
    # TRT of g: odd moments at the mobility rate, even ones at w+ = 1/(Lambda/tau_g + 1/2);
    # the same collision as MRT of g with s_q = BGK rate and s_e = s_eps = s_p = w+,
    # once phi's own moment of d vanishes (source off)
    cs2 = 1.0 / 3.0
    tau_f, tau_g, tau_s = 0.1 / cs2, 0.08 / cs2, 0.05 / cs2
    lam = 0.3
    wp = 1.0 / (lam / tau_g + 0.5)
    om_f = 1.0 / (tau_f + 0.5)
    trt = _droplet_fields(collision="trt", M_phi=0.08, source_on=0,
                          trt_magic=(tau_f * tau_f, lam, tau_s * tau_s))
    mrt = _droplet_fields(collision="mrt", M_phi=0.08, source_on=0, mrt_rates=(om_f, om_f, om_f),
                          mrt_rates_g=(wp, wp, 0.0, wp))
    assert _close(trt, mrt)


def test_mrt_g_conserves_phi_mass_with_the_source_off():
    w = W.droplet_2d(24, 6.0, T_offset=0.04, T_noise=0.01, corr_len=4.0)
    params = dict(w.params, nu_l=0.1, nu_g=0.1, alpha_l=0.05, alpha_g=0.05, source_on=0,
                  collision="mrt", mrt_rates=(1.3, 1.1, 1.6), mrt_rates_g=(1.2, 1.6, 1.05, 1.8))
    P, G = M.Params.from_dict(params), M.Grid(w.n, w.periodic)
    st = M.init_state(w.phi0, w.T0, P, G)
    m0 = float(M.fields(st, P, G)["phi"].sum())
    st = M.run(st, P, G, 40)
    m1 = float(M.fields(st, P, G)["phi"].sum())
    assert abs(m1 - m0) < 1e-11 * abs(m0)


def test_mrt_keeps_the_tanh_interface_stationary():
    # a flat two-interface slab at rest is the CAC equilibrium (Sec. 3.2):
    # with every MRT rate away from the BGK one the profile stays in place
    # within the bound the BGK step meets
    n, Wd = 48, 4.0
    params = W.base_params(rho_l=1.0, rho_g=1.0, nu_l=0.1, nu_g=0.1, sigma=0.0, W=Wd, M_phi=0.08,
                           gravity=(0.0, 0.0, 0.0), source_on=0, collision="mrt",
                           mrt_rates=(1.3, 1.1, 1.6), mrt_rates_g=(1.2, 1.5, 1.1, 1.7))
    y = np.arange(n) + 0.5
    prof = 0.5 * (1 + np.tanh(2 * (y - 12) / Wd)) - 0.5 * (1 + np.tanh(2 * (y - 36) / Wd))
    phi0 = np.broadcast_to(prof[:, None], (n, 3)).copy()
    P, G = M.Params.from_dict(params), M.Grid((3, n), (True, True))
    st = M.run(M.init_state(phi0, np.ones_like(phi0), P, G), P, G, 800)
    drift = float(np.abs(M.fields(st, P, G)["phi"].numpy() - phi0).max())
    assert drift < 1e-2, drift


# ---- 3D: D3Q19 for the flow set, D3Q7 for the phase field (same readings)

def _film3d_fields(steps=6, **over):
    w = W.film_boiling_3d(8, 6, 12, rho_ratio=3.0, modes=1, z0=5.0, phi_wall=(1.0, 0.0))
    base = dict(w.params, nu_l=0.1, nu_g=0.1, alpha_l=0.05, alpha_g=0.05)
    base.update(over)
    P, G = M.Params.from_dict(base), M.Grid(w.n, w.periodic)
    return M.fields(M.run(M.init_state(w.phi0, w.T0, P, G, p0=w.p0), P, G, steps), P, G)


def test_mrt3d_basis_is_orthogonal():
    from oracle import lattice as Lt
    for lat, norms in ((Lt.D3Q19, [19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24, 4, 4, 4, 8, 8, 8]),
                       (Lt.D3Q7, [7, 2, 2, 2, 42, 12, 4])):
        B = M.mrt_basis(lat)
        G = (B @ B.T).numpy()
        assert np.array_equal(G, np.diag(norms).astype(float)), lat.name


def test_mrt3d_with_equal_rates_is_bgk():
    om = 1.0 / (0.1 * 3.0 + 0.5)
    bgk = _film3d_fields(collision="bgk")
    mrt = _film3d_fields(collision="mrt", mrt_rates=(om, om, om))
    assert _close(bgk, mrt)
    other = _film3d_fields(collision="mrt", mrt_rates=(1.1, 1.3, 1.2), mrt_rates_g=(1.2, 0.0, 0.0, 1.4))
    assert float((other["phi"] - bgk["phi"]).abs().max()) > 1e-9


def test_mrt3d_reduces_to_trt():
    # flow: even moments at the viscosity rate, odd ones at s_q; phase field
    # (source off): odd moments at the mobility rate, e and the stress moments at w+
    tau_f, tau_g3, tau_s = 0.1 * 3.0, 0.08 * 4.0, 0.05 * 3.0
    lam_f, lam_g = 0.3, 0.2
    om_f = 1.0 / (tau_f + 0.5)
    s_q = 1.0 / (lam_f / tau_f + 0.5)
    wp_g = 1.0 / (lam_g / tau_g3 + 0.5)
    trt = _film3d_fields(collision="trt", M_phi=0.08, source_on=0, trt_magic=(lam_f, lam_g, tau_s * tau_s))
    mrt = _film3d_fields(collision="mrt", M_phi=0.08, source_on=0, mrt_rates=(om_f, om_f, s_q),
                         mrt_rates_g=(wp_g, 0.0, 0.0, wp_g))
    assert _close(trt, mrt)


def test_mrt3d_conserves_phi_mass_with_the_source_off():
    w = W.film_boiling_3d(8, 6, 12, rho_ratio=3.0, modes=1, z0=5.0, phi_wall=(1.0, 0.0))
    params = dict(w.params, nu_l=0.1, nu_g=0.1, source_on=0, collision="mrt",
                  mrt_rates=(1.3, 1.1, 1.6), mrt_rates_g=(1.2, 0.0, 0.0, 1.7))
    P, G = M.Params.from_dict(params), M.Grid(w.n, (True, True, True))
    st = M.init_state(w.phi0, w.T0, P, G, p0=w.p0)
    m0 = float(M.fields(st, P, G)["phi"].sum())
    st = M.run(st, P, G, 20)
    m1 = float(M.fields(st, P, G)["phi"].sum())
    assert abs(m1 - m0) < 1e-11 * abs(m0)


def test_mrt3d_magic_rate_gives_the_exact_poiseuille_profile():
    nu, H, Gf, steps = 0.5, 8, 1e-5, 1500
    s_nu = 1.0 / (nu * 3.0 + 0.5)
    s_q = 8.0 * (2.0 - s_nu) / (8.0 - s_nu)

    def err(collision, rates):
        params = W.base_params(rho_l=1.0, rho_g=1.0, nu_l=nu, nu_g=nu, alpha_l=0.05, alpha_g=0.05,
                               sigma=0.0, gravity=(0.0, 0.0, 0.0), body_force=(Gf, 0.0, 0.0), source_on=0,
                               phi_wall=(0.0, 0.0), T_wall=(1.0, 1.0), collision=collision, mrt_rates=rates)
        P, Gd = M.Params.from_dict(params), M.Grid((2, 2, H), (True, True, False))
        zeros = np.zeros((H, 2, 2))
        st = M.run(M.init_state(zeros, np.ones_like(zeros), P, Gd), P, Gd, steps)
        u = M.fields(st, P, Gd)["u"][0][:, 0, 0].numpy()
        z = np.arange(H)
        exact = Gf / (2 * nu) * (z + 0.5) * (H - 0.5 - z)
        return float(np.abs(u - exact).max() / exact.max())

    assert err("mrt", (1.1, 1.3, s_q)) < 1e-10
    assert err("mrt", (1.1, 1.3, 1.9)) > 1e-3
