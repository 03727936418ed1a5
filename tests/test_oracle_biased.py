"""Pins of the oracle's second-order biased gradient (grad_scheme "biased2",
Sec. 3.4: e_i . grad(phi) = [-phi(x + 2 e_i) + 4 phi(x + e_i) - 3 phi(x)] / 2
inside Eq. Grad), against values worked out by hand:

* one-sided second-order differences are exact on quadratics, and
  3 sum_i w_i e_i e_i = I, so the gradient of a quadratic is exact;
* on phi = x^3 the biased difference along +e_x gives 3x^2 - 2 and along
  -e_x gives -3x^2 + 2 (the central one 3x^2 + 1 both ways), so the biased
  gradient is (3x^2 - 2, 0) at every interior cell while the central one is
  (3x^2 + 1, 0) -- a sign or coefficient slip in the biased stencil, or a
  fallback to the central one, fails;
* the Laplacian is the central one in both schemes;
* the option is live in a full step."""
import numpy as np
import torch

import workloads as W
from oracle import model as M


def _grid_field(f, nx=24, ny=20):
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    X, Y = np.meshgrid(x, y)
    return torch.tensor(f(X, Y)), X, Y


def _params(scheme):
    return M.Params.from_dict(dict(W.base_params(), grad_scheme=scheme))


def _interior(a, nx=24, ny=20):
    return a[2:ny - 2, 2:nx - 2]


def test_biased_gradient_exact_on_quadratics():
    phi, X, Y = _grid_field(lambda X, Y: 0.3 * X**2 - 0.2 * X * Y + 0.1 * Y**2 + 0.5 * X - 0.7 * Y)
    G = M.Grid((24, 20), (True, True))
    (gx, gy), _ = M.gradient_laplacian(phi, G, _params("biased2"))
    assert np.abs(_interior(gx.numpy() - (0.6 * X - 0.2 * Y + 0.5))).max() < 1e-10
    assert np.abs(_interior(gy.numpy() - (-0.2 * X + 0.2 * Y - 0.7))).max() < 1e-10


def test_biased_and_central_gradients_of_a_cubic():
    phi, X, Y = _grid_field(lambda X, Y: X**3)
    G = M.Grid((24, 20), (True, True))
    (bx, by), lap_b = M.gradient_laplacian(phi, G, _params("biased2"))
    (cx, cy), lap_c = M.gradient_laplacian(phi, G, _params("central"))
    assert np.abs(_interior(bx.numpy() - (3 * X**2 - 2))).max() < 1e-9
    assert np.abs(_interior(by.numpy())).max() < 1e-9
    assert np.abs(_interior(cx.numpy() - (3 * X**2 + 1))).max() < 1e-9
    # the Laplacian of x^3 is 6x with either scheme (central second difference)
    assert np.abs(_interior(lap_b.numpy() - 6 * X)).max() < 1e-9
    assert torch.equal(lap_b, lap_c)


def test_biased_gradient_in_3d_on_a_cubic():
    nx, ny, nz = 12, 10, 9
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    phi = torch.tensor(z**3)
    G = M.Grid((nx, ny, nz), (True, True, True))
    (gx, gy, gz), _ = M.gradient_laplacian(phi, G, _params("biased2"))
    inner = (slice(2, nz - 2), slice(2, ny - 2), slice(2, nx - 2))
    assert np.abs((gz.numpy() - (3 * z**2 - 2))[inner]).max() < 1e-9
    assert np.abs(gx.numpy()[inner]).max() < 1e-9 and np.abs(gy.numpy()[inner]).max() < 1e-9


def test_biased_scheme_changes_the_step():
    w = W.droplet_2d(24, 6.0, T_offset=0.04)
    G = M.Grid(w.n, w.periodic)
    out = {}
    for scheme in ("central", "biased2"):
        P = M.Params.from_dict(dict(w.params, grad_scheme=scheme))
        out[scheme] = M.fields(M.run(M.init_state(w.phi0, w.T0, P, G), P, G, 5), P, G)["phi"]
    d = float((out["central"] - out["biased2"]).abs().max())
    assert 1e-9 < d < 1e-2
