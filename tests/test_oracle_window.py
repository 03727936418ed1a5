"""The locality argument of the full-size sampled parity tests
(test_gpu_fullsize.py): the oracle stepped on the window of radius 2k + 3
around a cell gives that cell's fields after k steps exactly as the oracle
stepped on the whole grid, for interior cells, cells next to either wall and
cells on periodic edges, in 2D and 3D."""
import numpy as np

import workloads as W
from oracle import model as M

from test_gpu_fullsize import _oracle_at, _samples


def _compare(w, steps, band, count):
    P, G = M.Params.from_dict(w.params), M.Grid(w.n, w.periodic)
    full = M.fields(M.run(M.init_state(w.phi0, w.T0, P, G, p0=w.p0), P, G, steps), P, G)
    cells = _samples(w.n, w.periodic, band, np.random.default_rng(1), count=count)
    for c in cells:
        ref = _oracle_at(w, c, steps)
        at = tuple(reversed(c))
        for k in ("phi", "T", "p"):
            assert ref[k] == float(full[k][at]), (c, k)
        for a in range(len(w.n)):
            assert ref["u"][a] == float(full["u"][a][at]), (c, a)


def test_window_equals_whole_grid_2d():
    w = W.film_boiling_2d(96, 64, modes=8, seed=1, y0=20.0, paper=True, phi_wall=(1.0, 0.0))
    _compare(w, 3, (10, 30), 10)


def test_window_equals_whole_grid_3d():
    w = W.film_boiling_3d(40, 24, 30, modes=2, seed=2, z0=10.0, paper=True, phi_wall=(1.0, 0.0))
    _compare(w, 2, (5, 15), 4)
