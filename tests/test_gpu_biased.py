"""The second-order biased gradient option (LBM_GRAD_BIASED2, Sec. 3.4) on
the GPU against the FP64 oracle with grad_scheme "biased2": parity within
1e-5 on geometries that take every ghost path (walls on y and on x with two
ghost layers, periodic boxes, a one-cell periodic axis that wraps twice,
ragged tiles, 3D with walls on z and a periodic axis shorter than the rings),
combined with TRT, and with 16-bit storage.  In 3D the TMA-staged kernel
takes the biased gradient on grids without ragged tiles (AUTO selects it
there for 16-bit storage) and matches the tiled kernel bit for bit."""
import numpy as np
import pytest

import workloads as W
from paper_2003_06342_b300._binding import LBMError, LBM_EUNSUPPORTED

from _parity import gpu_fields, gpu_solver, max_errors, oracle_fields

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _b(w, **extra):
    w.params.update(grad_scheme="biased2", **extra)
    return w


def _film(nx, ny, **kw):
    return W.film_boiling_2d(nx, ny, rho_ratio=10.0, y0=ny / 3.0, amplitude=2.0, phi_wall=(1.0, 0.0), **kw)


CASES = [
    ("film_ragged_walls_y", lambda: _b(_film(100, 70)), 40),
    ("droplet_periodic", lambda: _b(W.droplet_2d(48, 12.0, T_offset=0.05)), 40),
    ("stefan_walls_x", lambda: _b(W.stefan_1d(nx=90, ny=2)), 80),
    ("one_cell_axis", lambda: _b(W.stefan_1d(nx=40, ny=1)), 40),
    ("film_trt", lambda: _b(_film(67, 45), collision="trt", trt_magic=(3.0 / 16.0, 0.25, 0.25)), 30),
    # wide enough for tiles whose two rings lie inside the grid (the fast
    # path of the 64-wide tiles), with ragged last tiles
    ("film_interior_tiles", lambda: _b(_film(200, 45)), 20),
    # 3D: walls on z, ragged x / y tiles, several z blocks of 32 layers
    ("film_3d_ragged", lambda: _b(W.film_boiling_3d(37, 10, 41, modes=2, z0=12.0, phi_wall=(1.0, 0.0))), 12),
    # a periodic axis of three cells, shorter than the two rings
    ("film_3d_thin_y", lambda: _b(W.film_boiling_3d(40, 3, 20, modes=1, z0=7.0, phi_wall=(1.0, 0.0))), 12),
    ("film_3d_trt", lambda: _b(W.film_boiling_3d(33, 9, 17, modes=1, z0=6.0, phi_wall=(1.0, 0.0)),
                               collision="trt", trt_magic=(3.0 / 16.0, 0.25, 0.25)), 10),
]


def test_biased_parity_with_oracle_on_the_3d_tma_kernel():
    w = _b(W.film_boiling_3d(64, 8, 30, modes=1, z0=10.0, phi_wall=(1.0, 0.0)))
    ref = oracle_fields(w, 10)
    s = gpu_solver(w)
    s.set_kernel("tma")
    s.step(10)
    err = max_errors(gpu_fields(s), ref)
    assert all(v < TOL for v in err.values()), err


@pytest.mark.parametrize("name,make,steps", CASES, ids=[c[0] for c in CASES])
def test_biased_parity_with_oracle(name, make, steps):
    w = make()
    ref = oracle_fields(w, steps)
    s = gpu_solver(w)
    s.step(steps)
    err = max_errors(gpu_fields(s), ref)
    print(name, err)
    assert all(v < TOL for v in err.values()), err


def test_biased_fields_at_init_use_the_biased_gradient():
    w = _b(_film(64, 40))
    F = gpu_fields(gpu_solver(w))
    ref = oracle_fields(w, 0)
    err = max_errors(F, ref)
    assert all(v < 1e-6 for v in err.values()), err


def test_biased_fp16_close_to_fp32_and_tma_refused():
    w = _b(_film(96, 64))
    a = gpu_solver(w)
    b = gpu_solver(w, storage="fp16")
    a.step(30)
    b.step(30)
    fa, fb = gpu_fields(a), gpu_fields(b)
    assert np.abs(fa["phi"] - fb["phi"]).max() < 5e-3
    with pytest.raises(LBMError) as e:
        a.set_kernel("tma")
    assert e.value.code == LBM_EUNSUPPORTED


TMA_CASES = [
    ("fp32", lambda: _b(W.film_boiling_3d(64, 16, 40, modes=1, z0=12.0, phi_wall=(1.0, 0.0))), "fp32", 12),
    # several z blocks of 64 layers (16-bit storage)
    ("fp16_z_blocks", lambda: _b(W.film_boiling_3d(64, 24, 70, modes=2, z0=20.0, phi_wall=(1.0, 0.0))), "fp16", 10),
    ("bf16_trt", lambda: _b(W.film_boiling_3d(64, 8, 33, modes=1, z0=10.0, phi_wall=(1.0, 0.0)),
                            collision="trt", trt_magic=(3.0 / 16.0, 0.25, 0.25)), "bf16", 8),
    # periodic in every axis (no wall in z)
    ("fp32_periodic", lambda: _b(W.droplet_3d(32, 6.0) if hasattr(W, "droplet_3d") else
                                  W.film_boiling_3d(32, 8, 24, modes=1, z0=8.0, phi_wall=(1.0, 0.0))), "fp32", 8),
]


@pytest.mark.parametrize("name,make,storage,steps", TMA_CASES, ids=[c[0] for c in TMA_CASES])
def test_biased_3d_tma_matches_tiled_bit_for_bit(name, make, storage, steps):
    w = make()
    a = gpu_solver(w, storage=storage)
    b = gpu_solver(w, storage=storage)
    # AUTO: the TMA kernel for 16-bit storage, the tiled one for FP32
    assert a.kernel() == ("tiled" if storage == "fp32" else "tma")
    a.set_kernel("tma")
    b.set_kernel("tiled")
    a.step(steps)
    b.step(steps)
    import torch
    assert torch.equal(a.get_state(), b.get_state()), name
    a.sync()


def test_biased_3d_ragged_grid_stays_tiled():
    w = _b(W.film_boiling_3d(44, 13, 20, modes=1, z0=7.0, phi_wall=(1.0, 0.0)))
    s = gpu_solver(w, storage="fp16")
    assert s.kernel() == "tiled"              # ragged tiles: AUTO picks the tiled kernel
    s.step(5)
    assert np.isfinite(gpu_fields(s)["phi"]).all()
    with pytest.raises(LBMError) as e:
        s.set_kernel("tma")
    assert e.value.code == LBM_EUNSUPPORTED
