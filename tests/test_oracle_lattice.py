"""Pins of the oracle's lattice tables, Gamma and stencils against exact
identities (Sec. 3 lattices, Eq. FunctionGamma, Eqs. Grad and Laplacian)."""
import itertools
from fractions import Fraction

import numpy as np
import pytest
import torch

from oracle import lattice as Lt
from oracle import model as M

LATS = [Lt.D2Q9, Lt.D3Q7, Lt.D3Q19]


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_weight_moments_exact(lat):
    D = lat.D
    assert sum(lat.w) == 1
    for a in range(D):
        assert sum(lat.w[i] * int(lat.e[i][a]) for i in range(lat.Q)) == 0
        for b in range(D):
            m2 = sum(lat.w[i] * int(lat.e[i][a]) * int(lat.e[i][b]) for i in range(lat.Q))
            assert m2 == (lat.cs2 if a == b else 0)
            for c in range(D):
                m3 = sum(lat.w[i] * int(lat.e[i][a] * lat.e[i][b] * lat.e[i][c]) for i in range(lat.Q))
                assert m3 == 0


@pytest.mark.parametrize("lat", [Lt.D2Q9, Lt.D3Q19], ids=lambda l: l.name)
def test_fourth_order_isotropy(lat):
    D = lat.D
    for a, b, c, d in itertools.product(range(D), repeat=4):
        m4 = sum(lat.w[i] * int(lat.e[i][a] * lat.e[i][b] * lat.e[i][c] * lat.e[i][d])
                 for i in range(lat.Q))
        expect = lat.cs2 ** 2 * ((a == b) * (c == d) + (a == c) * (b == d) + (a == d) * (b == c))
        assert m4 == expect


def test_paper_constants():
    assert Lt.D3Q7.cs2 == Fraction(1, 4)           # "e^2 = 1/4" for D3Q7
    assert Lt.D2Q9.cs2 == Lt.D3Q19.cs2 == Fraction(1, 3)
    assert Lt.D2Q9.Q == 9 and Lt.D3Q7.Q == 7 and Lt.D3Q19.Q == 19
    # D2Q9 ordering printed in Sec. 3
    assert [tuple(v) for v in Lt.D2Q9.e] == [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1),
                                             (1, 1), (-1, 1), (-1, -1), (1, -1)]


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_opposite(lat):
    opp = lat.opposite
    for i in range(lat.Q):
        assert np.array_equal(lat.e[opp[i]], -lat.e[i])
        assert lat.w[opp[i]] == lat.w[i]


@pytest.mark.parametrize("lat", [Lt.D2Q9, Lt.D3Q19], ids=lambda l: l.name)
def test_gamma_moments(lat):
    rng = np.random.default_rng(0)
    u = [torch.tensor(rng.uniform(-0.05, 0.05, 16)) for _ in range(lat.D)]
    G = M.gamma(lat, u)
    cs2 = float(lat.cs2)
    total = sum(G)
    assert torch.allclose(total, torch.ones(16, dtype=torch.float64), atol=1e-15)
    for a in range(lat.D):
        first = sum(G[i] * float(lat.e[i][a]) for i in range(lat.Q))
        assert torch.allclose(first, u[a], atol=1e-15)
        for b in range(lat.D):
            second = sum(G[i] * float(lat.e[i][a] * lat.e[i][b]) for i in range(lat.Q))
            expect = u[a] * u[b] + (cs2 if a == b else 0.0)
            assert torch.allclose(second, expect, atol=1e-15)


def test_gamma_d3q7_first_moments():
    rng = np.random.default_rng(1)
    u = [torch.tensor(rng.uniform(-0.05, 0.05, 8)) for _ in range(3)]
    G = M.gamma(Lt.D3Q7, u)
    assert torch.allclose(sum(G), torch.ones(8, dtype=torch.float64), atol=1e-15)
    for a in range(3):
        assert torch.allclose(sum(G[i] * float(Lt.D3Q7.e[i][a]) for i in range(7)), u[a], atol=1e-15)


def _params(**kw):
    base = dict(rho_l=1.0, rho_g=1.0, nu_l=0.1, nu_g=0.1, alpha_l=0.1, alpha_g=0.1,
                sigma=0.0, W=4.0, M_phi=0.1)
    base.update(kw)
    return M.Params(**base)


@pytest.mark.parametrize("n,periodic", [((12, 10), (True, False)), ((8, 7, 9), (True, True, False))])
def test_stencils_exact_on_quadratics(n, periodic):
    """Central directional differences are exact on quadratics: the gradient
    of a quadratic and the Laplacian of a quadratic, at cells whose stencil
    stays inside the box."""
    G = M.Grid(n, periodic)
    coords = np.meshgrid(*[np.arange(m, dtype=np.float64) for m in reversed(n)], indexing="ij")
    pos = [coords[G.dim - 1 - a] for a in range(G.dim)]  # pos[a] = coordinate on axis a
    c1 = [0.3, -0.7, 0.11][:G.dim]
    c2 = [0.05, 0.02, -0.03][:G.dim]
    phi = sum(c1[a] * pos[a] + c2[a] * pos[a] ** 2 for a in range(G.dim)) + 0.2 * pos[0] * pos[1]
    grad, lap = M.gradient_laplacian(torch.tensor(phi), G, _params())
    inner = tuple(slice(1, -1) for _ in range(G.dim))
    for a in range(G.dim):
        exact = c1[a] + 2 * c2[a] * pos[a] + 0.2 * (pos[1] if a == 0 else pos[0] if a == 1 else 0.0)
        assert np.abs(grad[a].numpy()[inner] - exact[inner]).max() < 1e-12
    assert np.abs(lap.numpy()[inner] - 2 * sum(c2)).max() < 1e-12


def test_stencil_second_order_convergence_periodic():
    errs = []
    for N in (16, 32, 64):
        G = M.Grid((N, N), (True, True))
        y, x = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
        k = 2 * np.pi / N
        phi = np.sin(k * x) * np.cos(k * y)
        grad, lap = M.gradient_laplacian(torch.tensor(phi), G, _params())
        e_lap = np.abs(lap.numpy() - (-2 * k * k * phi)).max() / (2 * k * k)
        e_gx = np.abs(grad[0].numpy() - k * np.cos(k * x) * np.cos(k * y)).max() / k
        errs.append((e_lap, e_gx))
    for (a1, b1), (a2, b2) in zip(errs, errs[1:]):
        assert 3.5 < a1 / a2 < 4.5 and 3.5 < b1 / b2 < 4.5


def test_wall_ghost_is_dirichlet_value():
    G = M.Grid((6, 5), (True, False))
    phi = torch.full((5, 6), 0.25, dtype=torch.float64)
    P = _params(phi_wall=(1.0, 0.0))
    grad, lap = M.gradient_laplacian(phi, G, P)
    # bottom row sees ghost 1.0 below, top row sees ghost 0.0 above
    # d/dy at bottom = 3 * sum_i w_i e_iy (phi(+)-phi(-))/2 with only the y-neighbour
    # differences non-zero: (1/9 + 2/36) * 3 * (0.25 - 1.0)/2 * (-1) * ... check sign only
    assert (grad[1][0] < 0).all() and (grad[1][-1] < 0).all()
    assert torch.allclose(grad[0], torch.zeros_like(grad[0]))
    # Laplacian at the bottom row: each of the three downward links (weights
    # 1/9, 1/36, 1/36) sees the ghost once as phi(x+e_i) and once, for its
    # opposite direction, as phi(x-e_i): 3 * 2 * (1/9 + 2/36) * (1.0 - 0.25)
    assert torch.allclose(lap[0], torch.full((6,), 3 * 2 * (1 / 9 + 2 / 36) * 0.75, dtype=torch.float64))
