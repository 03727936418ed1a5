"""Parity at the full benchmark sizes, in the launch configuration bench.py
times (2048 x 4096 2D film on the tiled kernel; 256 x 256 x 512 and
512 x 512 x 768 3D films on the TMA-staged kernel), on sampled cells.

The oracle cannot step 8 M or 34 M cells in a test, but a cell's update over
k steps depends only on the initial fields within a few cells of it (the push
moves a value one cell per step and the phi stencils reach one more cell, so
the fields at x after k steps depend on the initial fields within 2k + 2
cells).  For each sampled cell the oracle therefore steps the window of
radius r = 2k + 3 around it, cut from the same initial fields: periodic axes
wrap, a window that meets a wall keeps that wall, and the window's own edges
(wrapped or cut) are more than 2k + 2 cells from the sample.  With the
biased gradient the phi stencil reaches two cells, so the window radius is
3k + 3.  The sampled cells include the interface band, cells next to both
walls, periodic edges and tile borders.  The MRT and biased-gradient
variants the bench times on the 2D grid are checked the same way."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import model as M

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _samples(n, periodic, band, rng, count=24):
    """Cell coordinates (x, y[, z]): random cells in the interface band along
    the wall axis, cells next to each wall, periodic edges, tile borders."""
    dim = len(n)
    wall = [a for a in range(dim) if not periodic[a]][0]
    out = []
    for _ in range(count):
        c = [int(rng.integers(0, n[a])) for a in range(dim)]
        c[wall] = int(rng.integers(band[0], band[1]))
        out.append(c)
    for wv in (0, 1, n[wall] - 2, n[wall] - 1):
        c = [int(rng.integers(0, n[a])) for a in range(dim)]
        c[wall] = wv
        out.append(c)
    for a in range(dim):
        if periodic[a]:
            for v in (0, n[a] - 1, 31 if a == 0 else 7, 32 if a == 0 else 8):
                c = [int(rng.integers(0, n[b])) for b in range(dim)]
                c[a] = v
                c[wall] = int(rng.integers(band[0], band[1]))
                out.append(c)
    return out


def _window(w, cell, r):
    """Window of the initial fields around `cell`, its grid and the cell's
    position in it."""
    idx, per, pos = [], [], []
    for a, (c, n) in enumerate(zip(cell, w.n)):
        m = 2 * r + 1
        if w.periodic[a]:
            idx.append([(c - r + k) % n for k in range(m)])
            per.append(True)
            pos.append(r)
        else:
            lo = min(max(c - r, 0), n - m)
            idx.append(list(range(lo, lo + m)))
            per.append(False)
            pos.append(c - lo)
    ix = np.ix_(*reversed(idx))                    # arrays are [z][y]x
    cut = lambda f: np.ascontiguousarray(f[ix]) if f is not None else None
    return cut(w.phi0), cut(w.T0), cut(w.p0), tuple(2 * r + 1 for _ in w.n), tuple(per), tuple(pos)


def _oracle_at(w, cell, steps, reach=2):
    """reach: cells a step's value depends on in each direction (the push
    plus the phi stencil: 2 for the central gradient, 3 for the biased one)."""
    r = reach * steps + 3
    phi0, T0, p0, n, per, pos = _window(w, cell, r)
    P, G = M.Params.from_dict(w.params), M.Grid(n, per)
    st = M.run(M.init_state(phi0, T0, P, G, p0=p0), P, G, steps)
    F = M.fields(st, P, G)
    at = tuple(reversed(pos))
    return dict(phi=float(F["phi"][at]), T=float(F["T"][at]), p=float(F["p"][at]),
                u=[float(F["u"][a][at]) for a in range(len(n))])


def _gpu_at(F, cells):
    dim = len(cells[0])
    idx = [torch.tensor([c[a] for c in cells], device=F["phi"].device) for a in reversed(range(dim))]
    pick = lambda t: t[tuple(idx)].double().cpu().numpy()
    return dict(phi=pick(F["phi"]), T=pick(F["T"]), p=pick(F["p"]), u=[pick(F["u"][a]) for a in range(dim)])


def _check(w, kernel, steps, storage="fp32", tol=TOL, seed=0, reach=2):
    from paper_2003_06342_b300 import Solver
    s = Solver(w.n, w.periodic, w.params, storage=storage)
    s.set_kernel(kernel)
    s.init(w.phi0, w.T0, p0=w.p0)
    s.step(steps)
    assert s.kernel() == kernel
    dim = len(w.n)
    wall = [a for a in range(dim) if not w.periodic[a]][0]
    # the interface band: where phi0 crosses 1/2 along the wall axis
    prof = w.phi0.mean(axis=tuple(range(dim - 1)))
    mid = int(np.argmin(np.abs(prof - 0.5)))
    cells = _samples(w.n, w.periodic, (max(mid - 12, 0), min(mid + 12, w.n[wall])), np.random.default_rng(seed))
    got = _gpu_at(s.fields(), cells)
    worst = {k: 0.0 for k in ("phi", "T", "p", "u")}
    for j, cell in enumerate(cells):
        ref = _oracle_at(w, cell, steps, reach)
        for k in ("phi", "T", "p"):
            worst[k] = max(worst[k], abs(got[k][j] - ref[k]))
        worst["u"] = max(worst["u"], max(abs(got["u"][a][j] - ref["u"][a]) for a in range(dim)))
    print(w.name, kernel, storage, steps, len(cells), "cells", worst)
    assert all(v < tol for v in worst.values()), worst


def test_2d_2048x4096_tiled_fp32_sampled():
    _check(W.c2_film_boiling(), "tiled", 3)


def test_2d_2048x4096_tiled_fp32_sampled_20_steps():
    _check(W.c2_film_boiling(), "tiled", 20, seed=1)


def test_2d_2048x4096_tiled_fp16_sampled():
    _check(W.c2_film_boiling(), "tiled", 3, storage="fp16", tol=5e-3)


def _with(w, **extra):
    w.params.update(**extra)
    return w


def test_2d_2048x4096_tiled_mrt_fp32_sampled():
    """The MRT collision of both sets on the full grid (the bench's MRT
    variant), FP32 and FP16 storage."""
    mrt = dict(collision="mrt", mrt_rates=(1.4, 1.4, 1.2))
    _check(_with(W.c2_film_boiling(), **mrt), "tiled", 3, seed=4)
    _check(_with(W.c2_film_boiling(), **mrt), "tiled", 3, storage="fp16", tol=5e-3, seed=5)


def test_2d_2048x4096_tiled_biased_sampled():
    """The biased gradient on the full grid (its two-ring window: a step
    reaches three cells), FP32 and FP16 storage."""
    _check(_with(W.c2_film_boiling(), grad_scheme="biased2"), "tiled", 3, seed=6, reach=3)
    _check(_with(W.c2_film_boiling(), grad_scheme="biased2"), "tiled", 3, storage="fp16", tol=5e-3, seed=7,
           reach=3)


def test_3d_256x256x512_tma_fp32_sampled():
    _check(W.c3_film_boiling_3d(), "tma", 2)


def test_3d_256x256x512_mrt_and_biased_sampled():
    """The 3D MRT collision (TMA kernel, FP32 and FP16) and the biased
    gradient (the kernels AUTO takes: tiled for FP32, TMA for FP16)."""
    mrt = dict(collision="mrt", mrt_rates=(1.4, 1.4, 1.2), mrt_rates_g=(1.3, 0.0, 0.0, 1.25))
    _check(_with(W.c3_film_boiling_3d(), **mrt), "tma", 2, seed=8)
    _check(_with(W.c3_film_boiling_3d(), **mrt), "tma", 2, storage="fp16", tol=5e-3, seed=9)
    _check(_with(W.c3_film_boiling_3d(), grad_scheme="biased2"), "tiled", 2, seed=10, reach=3)
    _check(_with(W.c3_film_boiling_3d(), grad_scheme="biased2"), "tma", 2, storage="fp16", tol=5e-3, seed=11,
           reach=3)


def test_3d_256x256x512_tma_fp16_sampled():
    _check(W.c3_film_boiling_3d(), "tma", 2, storage="fp16", tol=5e-3, seed=2)


def test_3d_512x512x768_tma_fp16_sampled():
    """The largest film (201 M cells, 36 GB of FP16 populations), in the
    configuration the bench times it: TMA kernel, FP16 storage."""
    w = W.c5_film_boiling_3d_large()
    _check(w, "tma", 2, storage="fp16", tol=5e-3, seed=3)
    del w
    torch.cuda.empty_cache()


def _cac_sampled(n, periodic, params, phi0, u, period, steps, storage, tol, seed):
    """The phase field alone at full size: sampled cells against the oracle
    of oracle.cac on windows of radius 2k + 3 cut (every axis periodic) from
    the initial field and the imposed velocity."""
    from oracle import cac as C
    from paper_2003_06342_b300 import Solver
    s = Solver(n, periodic, params, storage=storage)
    s.set_velocity(u, period)
    s.init(phi0, np.ones_like(phi0))
    s.step(steps)
    got = s.fields()["phi"]
    rng = np.random.default_rng(seed)
    dim = len(n)
    # cells of the interface band (0.05 < phi < 0.95), random cells, corners
    # and tile borders
    band = np.argwhere((phi0 > 0.05) & (phi0 < 0.95))
    pick = band[rng.choice(len(band), size=min(24, len(band)), replace=False)]
    cells = [[int(v) for v in reversed(b)] for b in pick]
    cells += [[int(rng.integers(0, n[a])) for a in range(dim)] for _ in range(8)]
    cells += [[0] * dim, [n[a] - 1 for a in range(dim)], [31] + [7] * (dim - 1), [32] + [8] * (dim - 1)]
    r = 2 * steps + 3
    worst = 0.0
    for cell in cells:
        idx = [[(c - r + k) % m for k in range(2 * r + 1)] for c, m in zip(cell, n)]
        ix = np.ix_(*reversed(idx))
        win = tuple(2 * r + 1 for _ in n)
        P, G = M.Params.from_dict(params), M.Grid(win, (True,) * dim)
        uw = [np.ascontiguousarray(ua[ix]) for ua in u]
        g = C.run(C.init_state(np.ascontiguousarray(phi0[ix]), uw, P, G, period), uw, P, G, steps, period)
        ref = float(C.phase_field(g).numpy()[(r,) * dim])
        val = float(got[tuple(reversed(cell))].item())
        worst = max(worst, abs(val - ref))
    print("phase field", n, storage, steps, len(cells), "cells", worst)
    assert worst < tol, worst


def test_phase_field_2d_4096_sampled():
    """The 4096^2 vortex of the bench's phase-field variant, FP32 and FP16."""
    w = W.vortex_disk(n=4096)
    for storage, tol, seed in (("fp32", TOL, 12), ("fp16", 5e-3, 13)):
        _cac_sampled(w.n, w.periodic, w.params, w.phi0, w.extra["u"], w.extra["period"], 3, storage, tol, seed)


def test_phase_field_3d_1024x1024x32_sampled():
    """The thin periodic 3D vortex of the bench's 3D phase-field variant."""
    wv = W.vortex_disk(n=1024)
    nz = 32
    phi = np.repeat(wv.phi0[None], nz, axis=0)
    u = [np.repeat(uu[None], nz, axis=0) for uu in wv.extra["u"]] + [np.zeros_like(phi)]
    for storage, tol, seed in (("fp32", TOL, 14), ("fp16", 5e-3, 15)):
        _cac_sampled((1024, 1024, nz), (True, True, True), wv.params, phi, u, wv.extra["period"], 3, storage, tol,
                     seed)
