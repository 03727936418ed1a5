"""The oracle's reverse-mode gradients (torch autograd through the FP64 step)
against central finite differences of the same forward map, for the latent
heat, the mobility, the surface tension and a seeded direction in T_0."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import adjoint as A
from oracle import model as M


def _case():
    w = W.droplet_2d(16, 4.5, T_offset=0.04, T_noise=0.01, corr_len=3.0)
    G = M.Grid(w.n, w.periodic)
    return w, G, w.phi0.copy()


@pytest.mark.slow
def test_oracle_adjoint_matches_central_differences():
    w, G, target = _case()
    steps = 6
    J, g = A.gradients(w.phi0, w.T0, w.params, G, steps, target)
    assert J > 0
    for name, rel_h in (("L", 1e-5), ("M_phi", 1e-5), ("sigma", 1e-5)):
        h = rel_h * abs(w.params[name])
        fd = A.central_difference(w.phi0, w.T0, w.params, G, steps, target, name, h)
        assert abs(g[name] - fd) <= 1e-6 * abs(fd) + 1e-12, (name, g[name], fd)
    rng = np.random.default_rng(7)
    direction = rng.standard_normal(w.T0.shape)
    fd = A.central_difference(w.phi0, w.T0, w.params, G, steps, target, "T0", 1e-5, direction)
    ad = float((g["T0"] * torch.as_tensor(direction)).sum())
    assert abs(ad - fd) <= 1e-6 * abs(fd) + 1e-12, (ad, fd)
