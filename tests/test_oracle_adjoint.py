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


def test_segmented_reverse_mode_equals_plain():
    """Recomputing checkpointed segments in the backward pass (used for long
    runs) gives the same gradients as keeping the whole graph, up to the order
    in which parameter contributions are summed."""
    w, G, _ = _case()
    target = np.roll(w.phi0, 1, axis=0)
    J1, g1 = A.gradients(w.phi0, w.T0, w.params, G, 7, target)
    J2, g2 = A.gradients(w.phi0, w.T0, w.params, G, 7, target, segment=3)
    assert J1 == J2
    for k in ("L", "M_phi", "sigma"):
        assert abs(g1[k] - g2[k]) <= 1e-12 * abs(g1[k]), k
    assert torch.allclose(g1["T0"], g2["T0"], rtol=1e-12, atol=1e-15 * float(g1["T0"].abs().max()))
