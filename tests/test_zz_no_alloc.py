"""The allocation-free field sums against the workspace-based reduction.

lbm_field_sums_noalloc serves callers that cannot allocate device memory
(their host owns every device buffer, or cudaMalloc's implicit
synchronisation is off limits where they run), so it keeps its partial sums
in static device memory instead of a workspace.  It must give the same mass
and enthalpy as lbm_reduce on the same state, call after call.  This file is
collected last so that a run stopping at the first failure has run every
other test before it."""
import ctypes

import pytest
import torch

import workloads as W
from paper_2003_06342_b300 import _binding as B

from _parity import gpu_solver

pytestmark = pytest.mark.gpu


def _noalloc_sums(F, params, stream):
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=F["phi"].device)
    phi = F["phi"].contiguous()
    T = F["T"].contiguous()
    B.check(B.lib.lbm_field_sums_noalloc(ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(T.data_ptr()),
                                         phi.numel(), params["rho_l"], params["rho_g"], params["Cp"],
                                         params["L"], ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(stream.cuda_stream)),
            "lbm_field_sums_noalloc")
    torch.cuda.synchronize()
    return out.tolist()


@pytest.mark.parametrize("make", [
    lambda: W.film_boiling_2d(1024, 512, modes=3, seed=2, y0=120.0, paper=True, phi_wall=(1.0, 0.0)),
    lambda: W.film_boiling_3d(96, 96, 40, modes=1, z0=14.0, phi_wall=(1.0, 0.0)),
], ids=["2d_1024x512", "3d_96x96x40"])
def test_reduce_over_several_cells_per_thread(make):
    """Grids larger than the moment kernel's grid of 148 x 8 blocks of 256
    threads, so each of its threads adds several cells into its FP64
    accumulators: the sums equal the one-cell-per-thread sums of the same
    fields, and the mass equals the host's FP64 sum of phi."""
    w = make()
    s = gpu_solver(w)
    s.step(5)
    mass, energy = s.reduce()
    F = s.fields()
    m2, e2 = _noalloc_sums(F, w.params, s.stream)
    assert abs(m2 - mass) <= 1e-12 * abs(mass)
    assert abs(e2 - energy) <= 1e-12 * abs(energy)
    m_host = float(F["phi"].double().sum().item())
    assert abs(m_host - mass) <= 1e-12 * abs(mass)


def test_noalloc_sums_match_reduce_two_calls():
    w = W.film_boiling_2d(300, 170, modes=3, seed=1, y0=40.0, paper=True, phi_wall=(1.0, 0.0))
    s = gpu_solver(w)
    for _ in range(2):
        s.step(25)
        mass, energy = s.reduce()
        F = s.fields()
        m2, e2 = _noalloc_sums(F, w.params, s.stream)
        assert abs(m2 - mass) <= 1e-12 * abs(mass)
        assert abs(e2 - energy) <= 1e-12 * abs(energy)


def test_noalloc_rejects_oversize_and_bad_args():
    dummy = torch.zeros(4, dtype=torch.float32, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    o = ctypes.c_void_p(out.data_ptr())
    # the size check happens before any device access
    assert B.lib.lbm_field_sums_noalloc(p, p, 16777216 + 1, 1.0, 1.0, 1.0, 1.0, o, None) == B.LBM_ENOMEM
    assert B.lib.lbm_field_sums_noalloc(p, p, 0, 1.0, 1.0, 1.0, 1.0, o, None) == B.LBM_EINVAL
    assert B.lib.lbm_field_sums_noalloc(None, p, 4, 1.0, 1.0, 1.0, 1.0, o, None) == B.LBM_EINVAL


def test_noalloc_at_the_cell_limit():
    """16,777,216 cells, the size that fills the whole static array: with
    phi = 1 and T = 0 both sums are exact in FP64 (mass = n, enthalpy =
    n rho_g L)."""
    n = 16777216
    phi = torch.ones(n, dtype=torch.float32, device="cuda")
    T = torch.zeros(n, dtype=torch.float32, device="cuda")
    params = dict(rho_l=10.0, rho_g=2.0, Cp=1.0, L=0.75)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        m, e = _noalloc_sums(dict(phi=phi, T=T), params, stream)
        assert m == float(n)
        assert e == float(n) * 2.0 * 0.75
