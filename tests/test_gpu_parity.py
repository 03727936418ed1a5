"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerance: 1e-5 max-abs on phi, T and u (and p), the bound stated for the
FP32 path; index work (the streaming map) must match bit for bit.  Grids are
chosen to span several 32x8 tiles with ragged edges, each wall orientation,
fully periodic boxes, and the degenerate one-cell-wide axis."""
import json
import os

import numpy as np
import pytest
import torch

import workloads as W
from oracle import lattice as Lt
from oracle import model as M

from _parity import gpu_fields, gpu_solver, max_errors, oracle_fields

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _film(nx, ny, **kw):
    kw.setdefault("phi_wall", (1.0, 0.0))
    return W.film_boiling_2d(nx, ny, rho_ratio=10.0, y0=ny / 3.0, amplitude=2.0, **kw)


STREAM_CASES = [
    ("2d_wall_y", lambda: _film(37, 19)),
    ("2d_wall_x", lambda: W.stefan_1d(nx=45, ny=3)),
    ("2d_periodic", lambda: W.droplet_2d(33, 8.0)),
    ("2d_one_cell_axis", lambda: W.stefan_1d(nx=40, ny=1)),
    ("3d_wall_z", lambda: W.film_boiling_3d(35, 9, 11, modes=1, z0=4.0)),
]


@pytest.mark.parametrize("name,make", STREAM_CASES, ids=[c[0] for c in STREAM_CASES])
def test_stream_map_bit_exact(name, make):
    w = make()
    s = gpu_solver(w)
    G = M.Grid(w.n, w.periodic)
    Lf, Lg, _ = Lt.lattices_for(w.dim)
    for which, lat in ((0, Lf), (1, Lg)):
        src, kind = s.stream_map(which)
        osrc, okind = M.stream_map(lat, G)
        assert np.array_equal(src.cpu().numpy().astype(np.int64), osrc), (name, which)
        assert np.array_equal(kind.cpu().numpy(), okind), (name, which)


INIT_CASES = [("2d", lambda: _film(41, 23)), ("3d", lambda: W.film_boiling_3d(19, 10, 13, modes=1, z0=5.0))]


@pytest.mark.parametrize("name,make", INIT_CASES, ids=[c[0] for c in INIT_CASES])
def test_init_returns_fields(name, make):
    w = make()
    s = gpu_solver(w)
    F = gpu_fields(s)
    assert np.abs(F["phi"] - w.phi0).max() < 1e-6
    assert np.abs(F["T"] - w.T0).max() < 1e-6
    assert np.abs(F["p"] - w.p0).max() < 1e-6
    assert max(np.abs(u).max() for u in F["u"]) < 1e-7


PARITY_CASES = [
    ("film_ragged", lambda: _film(100, 70), 60),
    ("film_printed_top_wall", lambda: _film(67, 45, phi_wall=(1.0, 1.0)), 30),
    ("droplet_periodic", lambda: W.droplet_2d(48, 12.0, T_offset=0.05), 60),
    ("stefan_x_walls", lambda: W.stefan_1d(nx=90, ny=2), 100),
    ("poiseuille_body_force", lambda: W.layered_poiseuille(ny=30, nx=5), 100),
    ("laplace_drop", lambda: W.static_drop_2d(n=40, radius=9.0, sigma=0.02), 60),
    ("film_3d", lambda: W.film_boiling_3d(37, 10, 21, modes=2, z0=7.0, phi_wall=(1.0, 0.0)), 30),
    ("film_3d_tiny_z", lambda: W.film_boiling_3d(9, 9, 5, modes=1, z0=2.0, phi_wall=(1.0, 0.0)), 10),
]


@pytest.mark.parametrize("name,make,steps", PARITY_CASES, ids=[c[0] for c in PARITY_CASES])
def test_parity_with_oracle(name, make, steps):
    w = make()
    ref = oracle_fields(w, steps)
    s = gpu_solver(w)
    s.step(steps)
    got = gpu_fields(s)
    err = max_errors(got, ref)
    assert all(v < TOL for v in err.values()), (name, err)


def test_parity_c1_1000_steps():
    """The 128 x 256 film-boiling case for 1000 steps: phi, T, u and p within
    1e-5 of the FP64 oracle.

    For context the test prints what plain FP32 arithmetic costs on this
    trajectory: the oracle's own step run in float32 drifts from float64 by
    the amounts in tests/golden/c1_fp32_floor.json (written from the oracle
    alone; 1.9e-5 in phi, 8.4e-5 in T).  The kernels multiply by each lattice
    weight as a two-float product (the rounded float32 weights do not sum to
    one, a bias that accumulates step after step) and advance T as a
    deviation from T_sat, which keeps them inside the bound."""
    floor = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "c1_fp32_floor.json")))
    w = W.c1_parity()
    ref = oracle_fields(w, w.steps)
    s = gpu_solver(w)
    s.step(w.steps)
    got = gpu_fields(s)
    err = max_errors(got, ref)
    print("c1 1000-step errors", err, "plain-fp32 oracle", floor)
    assert all(v < TOL for v in err.values()), err


def test_reductions_match_oracle():
    w = _film(64, 48)
    ref = oracle_fields(w, 25, state=True)
    s = gpu_solver(w)
    s.step(25)
    mass, energy = s.reduce()
    m_ref, e_ref = ref["reductions"]
    assert abs(mass - m_ref) < 1e-5 * w.cells
    assert abs(energy - e_ref) < 1e-5 * w.cells * 10


def test_state_roundtrip_bit_exact():
    w = _film(50, 30)
    a = gpu_solver(w)
    a.step(7)
    snap = a.get_state()
    a.step(11)
    Fa = gpu_fields(a)
    b = gpu_solver(w)
    b.set_state(snap)
    b.step(11)
    Fb = gpu_fields(b)
    for k in ("phi", "T", "p"):
        assert np.array_equal(Fa[k], Fb[k])
    host = a.get_state(torch.empty(a.state_bytes(), dtype=torch.uint8))
    assert host.numel() == a.state_bytes()


def test_host_paths_match_device_paths():
    w = _film(40, 24)
    a = gpu_solver(w)
    b = gpu_solver(w)
    b.init_host(w.phi0, w.T0, p0=w.p0)
    a.step(5)
    b.step(5)
    Fa = gpu_fields(a)
    Hb = b.fields_host()
    for k in ("phi", "T", "p"):
        assert np.array_equal(Fa[k], Hb[k])
    # float32 host buffers (pinned tensors): the same bits in and out
    c = gpu_solver(w)
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).pin_memory()
    c.init_host(pin(w.phi0), pin(w.T0), p0=pin(w.p0), dtype=np.float32)
    c.step(5)
    out = {k: torch.empty(c.shape, dtype=torch.float32).pin_memory() for k in ("phi", "T", "ux", "uy", "p")}
    Hc = c.fields_host(out=out)
    for k in ("phi", "T", "p"):
        assert np.array_equal(Fa[k], Hc[k].double().numpy())


def test_mass_conservation_source_off_gpu():
    w = W.droplet_2d(96, 20.0, source_on=0)
    s = gpu_solver(w)
    m0, _ = s.reduce()
    s.step(300)
    m1, _ = s.reduce()
    assert abs(m1 - m0) / m0 < 1e-5


def _trt(w):
    w.params.update(collision="trt", trt_magic=(3.0 / 16.0, 0.25, 0.25))
    return w


TMA_CASES = [
    ("film_walls_fp32", lambda: _film(128, 96), "fp32", 40),
    ("film_walls_ragged_y", lambda: _film(96, 83), "fp32", 25),
    ("droplet_periodic_fp32", lambda: W.droplet_2d(96, 20.0, T_offset=0.05), "fp32", 40),
    ("film_walls_fp16", lambda: _film(128, 96), "fp16", 40),
    ("film_walls_bf16", lambda: _film(128, 96), "bf16", 20),
    # 16-bit widths with interior 64-cell tiles of the tiled kernel, and TRT
    ("film_walls_fp16_wide", lambda: _film(320, 72), "fp16", 30),
    ("droplet_periodic_fp16", lambda: W.droplet_2d(256, 40.0, T_offset=0.05), "fp16", 30),
    ("film_trt_fp16_wide", lambda: _trt(_film(256, 64)), "fp16", 20),
    # 3D: periodic x, y (edge tiles wrap), walls in z, several z blocks of 32
    # layers, and a grid whose last tiles are ragged in x and y
    ("film3d_fp32", lambda: W.film_boiling_3d(64, 24, 70, modes=2, z0=20.0, phi_wall=(1.0, 0.0)), "fp32", 12),
    ("film3d_ragged", lambda: W.film_boiling_3d(44, 13, 37, modes=1, z0=12.0, phi_wall=(1.0, 0.0)), "fp32", 10),
    ("film3d_fp16", lambda: W.film_boiling_3d(64, 24, 70, modes=2, z0=20.0, phi_wall=(1.0, 0.0)), "fp16", 12),
    ("film3d_bf16", lambda: W.film_boiling_3d(64, 16, 40, modes=2, z0=12.0, phi_wall=(1.0, 0.0)), "bf16", 8),
]


@pytest.mark.parametrize("name,make,storage,steps", TMA_CASES, ids=[c[0] for c in TMA_CASES])
def test_tma_kernel_matches_tiled_kernel_bit_for_bit(name, make, storage, steps):
    """The persistent TMA-staged kernel and the tiled kernel run the same
    per-cell update on the same values, so their states agree exactly."""
    w = make()
    a = gpu_solver(w, storage=storage)
    b = gpu_solver(w, storage=storage)
    a.set_kernel("tma")
    b.set_kernel("tiled")
    a.step(steps)
    b.step(steps)
    assert a.kernel() == "tma" and b.kernel() == "tiled"
    sa, sb = a.get_state(), b.get_state()
    torch.cuda.synchronize()
    assert torch.equal(sa, sb), name
    a.sync()


def test_tma_kernel_parity_with_oracle():
    w = _film(128, 64)
    ref = oracle_fields(w, 50)
    s = gpu_solver(w)
    s.set_kernel("tma")
    s.step(50)
    assert s.kernel() == "tma"
    err = max_errors(gpu_fields(s), ref)
    assert all(v < TOL for v in err.values()), err


def test_tma3d_kernel_parity_with_oracle():
    w = W.film_boiling_3d(40, 16, 36, modes=1, z0=10.0, phi_wall=(1.0, 0.0))
    ref = oracle_fields(w, 12)
    s = gpu_solver(w)
    s.set_kernel("tma")
    s.step(12)
    assert s.kernel() == "tma"
    err = max_errors(gpu_fields(s), ref)
    assert all(v < TOL for v in err.values()), err


def test_nonfinite_state_is_reported():
    """A NaN planted in the initial temperature reaches the fields and the
    FP64 reduction reports it as LBM_ENONFINITE instead of a number."""
    from paper_2003_06342_b300._binding import LBMError, LBM_ENONFINITE
    w = _film(64, 32)
    T0 = w.T0.copy()
    T0[10, 20] = float("nan")
    w.T0 = T0
    s = gpu_solver(w)
    s.step(3)
    with pytest.raises(LBMError) as e:
        s.reduce()
    assert e.value.code == LBM_ENONFINITE
    s.sync()                                  # the context stays usable
