"""Pins of the oracle's two-relaxation-time collision (oracle.model,
collision = "trt"), each against something other than the oracle itself:

* with Lambda = tau^2 for every set (uniform properties) the two rates are
  equal and TRT is the BGK step of Eq. LBE to round-off;
* with Lambda_f = 3/16 and half-way bounce-back walls the steady Poiseuille
  profile is the exact parabola u = G/(2 nu) (y + 1/2)(H - 1/2 - y) (the
  known exactness of that magic value), while BGK at the same tau is off by
  percents;
* the decay of a long sine mode of T (heat set) and of phi (phase field, with
  the interface term switched off by a huge W) follows exp(-D k^2 n) with
  D = alpha or M_phi for two different Lambda: the antisymmetric rate carries
  the diffusivity, and the symmetric one does not change it."""
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import model as M


def _uniform_params(**over):
    p = W.base_params(rho_l=1.0, rho_g=1.0, nu_l=0.1, nu_g=0.1, alpha_l=0.05, alpha_g=0.05,
                      gravity=(0.0, 0.0, 0.0))
    p.update(over)
    return p


def test_trt_with_equal_rates_is_bgk():
    w = W.droplet_2d(24, 6.0, T_offset=0.04, T_noise=0.01, corr_len=4.0)
    base = dict(w.params, nu_l=0.1, nu_g=0.1, alpha_l=0.05, alpha_g=0.05)
    cs2 = 1.0 / 3.0
    tf, tg, ts = 0.1 / cs2, base["M_phi"] / cs2, 0.05 / cs2
    G = M.Grid(w.n, w.periodic)
    out = {}
    for coll in ("bgk", "trt"):
        P = M.Params.from_dict(dict(base, collision=coll, trt_magic=(tf * tf, tg * tg, ts * ts)))
        st = M.run(M.init_state(w.phi0, w.T0, P, G), P, G, 12)
        out[coll] = M.fields(st, P, G)
    for k in ("phi", "T", "p"):
        assert float((out["bgk"][k] - out["trt"][k]).abs().max()) < 1e-13, k
    # and with another Lambda the step differs (the option is live)
    P = M.Params.from_dict(dict(base, collision="trt", trt_magic=(0.25, 0.25, 0.25)))
    st = M.run(M.init_state(w.phi0, w.T0, P, G), P, G, 12)
    assert float((M.fields(st, P, G)["phi"] - out["bgk"]["phi"]).abs().max()) > 1e-9


def _poiseuille(collision, magic, nu=0.5, H=8, G=1e-5, steps=1500):
    params = _uniform_params(nu_l=nu, nu_g=nu, sigma=0.0, body_force=(G, 0.0, 0.0), source_on=0,
                             phi_wall=(0.0, 0.0), T_wall=(1.0, 1.0), collision=collision,
                             trt_magic=(magic, 0.25, 0.25))
    P, Gd = M.Params.from_dict(params), M.Grid((2, H), (True, False))
    st = M.run(M.init_state(np.zeros((H, 2)), np.ones((H, 2)), P, Gd), P, Gd, steps)
    u = M.fields(st, P, Gd)["u"][0][:, 0].numpy()
    y = np.arange(H)
    exact = G / (2 * nu) * (y + 0.5) * (H - 0.5 - y)
    return float(np.abs(u - exact).max() / exact.max())


def test_trt_magic_3_16_gives_the_exact_poiseuille_profile():
    assert _poiseuille("trt", 3.0 / 16.0) < 1e-10
    assert _poiseuille("bgk", 0.0) > 1e-2


def _sine_decay(field, magic, n=400, nx=64):
    k = 2.0 * math.pi / nx
    x = np.arange(nx) + 0.5
    amp = 1e-3
    over = dict(collision="trt", sigma=0.0, source_on=0)
    if field == "T":
        over.update(trt_magic=(0.25, 0.25, magic))
        phi0 = np.zeros((1, nx))
        T0 = (1.0 + amp * np.sin(k * x))[None, :]
        D = 0.05
    else:
        over.update(trt_magic=(0.25, magic, 0.25), W=1e9, M_phi=0.05)
        phi0 = (0.5 + amp * np.sin(k * x))[None, :]
        T0 = np.ones((1, nx))
        D = 0.05
    P, G = M.Params.from_dict(_uniform_params(**over)), M.Grid((nx, 1), (True, True))
    st = M.run(M.init_state(phi0, T0, P, G), P, G, n)
    f = M.fields(st, P, G)[field][0].numpy()
    a = 2.0 / nx * float(np.sum((f - f.mean()) * np.sin(k * x)))
    return a / amp, math.exp(-D * k * k * n)


@pytest.mark.parametrize("field", ["T", "phi"])
@pytest.mark.parametrize("magic", [1.0 / 6.0, 0.25])
def test_trt_keeps_the_diffusivity_on_the_antisymmetric_rate(field, magic):
    got, exact = _sine_decay(field, magic)
    assert abs(got - exact) < 0.01 * exact, (got, exact)
