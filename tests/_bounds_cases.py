"""Cases run by test_gpu_bounds.py with both builds of the library.

Each case runs one kernel family on a grid chosen to exercise its edge
handling (ragged last tiles, each wall orientation, a one-cell-wide axis,
periodic wrap, several TMA z blocks) and returns the raw state bytes (or, for
the adjoint, the gradients).  `main(out)` runs them all in the current
process, calls lbm_sync after each (which raises on LBM_EBOUNDS in the
bounds-checking build) and saves the results to `out` (.npz)."""
import sys

import numpy as np
import torch

import workloads as W


def _film(nx, ny, **kw):
    kw.setdefault("phi_wall", (1.0, 0.0))
    return W.film_boiling_2d(nx, ny, rho_ratio=10.0, y0=ny / 3.0, amplitude=2.0, **kw)


def _film3d(nx, ny, nz, z0):
    return W.film_boiling_3d(nx, ny, nz, modes=1, z0=z0, phi_wall=(1.0, 0.0))


def _opt(w, **extra):
    """The workload with the collision / gradient options of rows f2, f3."""
    w.params.update(**extra)
    return w


TRT = dict(collision="trt", trt_magic=(3.0 / 16.0, 0.25, 0.25))
MRT_G = dict(collision="mrt", mrt_rates=(1.4, 1.4, 1.2), mrt_rates_g=(1.3, 1.2, 1.1, 1.25))
BIASED = dict(grad_scheme="biased2")


# name, workload, storage, kernel, steps
STEP_CASES = [
    ("2d_tiled_fp32_ragged_walls", lambda: _film(100, 70), "fp32", "tiled", 12),
    ("2d_tiled_fp16_ragged_walls", lambda: _film(100, 70), "fp16", "tiled", 12),
    ("2d_tiled_x_walls_one_cell_axis", lambda: W.stefan_1d(nx=40, ny=1), "fp32", "tiled", 12),
    ("2d_tiled_periodic", lambda: W.droplet_2d(48, 12.0, T_offset=0.05), "bf16", "tiled", 12),
    ("2d_tma_fp32_ragged_y", lambda: _film(96, 83), "fp32", "tma", 12),
    ("2d_tma_fp16", lambda: _film(128, 96), "fp16", "tma", 12),
    ("3d_tiled_fp32_ragged", lambda: _film3d(44, 13, 37, 12.0), "fp32", "tiled", 6),
    ("3d_tiled_fp16_tiny_z", lambda: _film3d(9, 9, 5, 2.0), "fp16", "tiled", 6),
    ("3d_tma_fp32_ragged", lambda: _film3d(44, 13, 37, 12.0), "fp32", "tma", 6),
    ("3d_tma_fp16_z_blocks", lambda: _film3d(64, 24, 70, 20.0), "fp16", "tma", 6),
    # the separately instantiated collision and gradient options
    ("2d_tiled_biased_ragged_walls", lambda: _opt(_film(100, 70), **BIASED), "fp32", "tiled", 12),
    ("2d_tiled_biased_one_cell_axis", lambda: _opt(W.stefan_1d(nx=40, ny=1), **BIASED), "fp16", "tiled", 12),
    ("2d_tiled_biased_interior_fp32", lambda: _opt(_film(200, 45), **BIASED), "fp32", "tiled", 12),
    ("2d_tiled_biased_interior_fp16", lambda: _opt(_film(200, 45), **BIASED), "fp16", "tiled", 12),
    ("3d_tiled_biased_ragged", lambda: _opt(_film3d(44, 13, 37, 12.0), **BIASED), "fp32", "tiled", 6),
    ("3d_tiled_biased_tiny_z", lambda: _opt(_film3d(9, 9, 5, 2.0), **BIASED), "fp32", "tiled", 6),
    ("2d_tiled_mrt_ragged", lambda: _opt(_film(100, 70), **MRT_G), "fp32", "tiled", 12),
    ("2d_tiled_mrt_periodic", lambda: _opt(W.droplet_2d(48, 12.0, T_offset=0.05), **MRT_G), "fp16", "tiled", 12),
    ("2d_tma_mrt_ragged_y", lambda: _opt(_film(96, 83), **MRT_G), "fp32", "tma", 12),
    ("2d_tiled_trt_ragged", lambda: _opt(_film(100, 70), **TRT), "bf16", "tiled", 12),
    ("3d_tma_trt_ragged", lambda: _opt(_film3d(44, 13, 37, 12.0), **TRT), "fp32", "tma", 6),
    ("3d_tiled_trt_fp16", lambda: _opt(_film3d(44, 13, 37, 12.0), **TRT), "fp16", "tiled", 6),
    ("3d_tma_biased", lambda: _opt(_film3d(64, 12, 37, 12.0), **BIASED), "fp32", "tma", 6),
    ("3d_tma_biased_fp16", lambda: _opt(_film3d(64, 8, 70, 20.0), **BIASED), "fp16", "tma", 6),
    ("3d_tma_mrt_ragged", lambda: _opt(_film3d(44, 13, 37, 12.0), **MRT_G), "fp32", "tma", 6),
    ("3d_tiled_mrt_bf16", lambda: _opt(_film3d(44, 13, 37, 12.0), **MRT_G), "bf16", "tiled", 6),
    ("3d_tma_mrt_biased_fp16", lambda: _opt(_film3d(64, 8, 70, 20.0), **MRT_G, **BIASED), "fp16", "tma", 6),
]

# name, grid size (n, or (nx, ny, nz) for a thin periodic 3D box), storage,
# velocity factor, reversal period, steps
CAC_CASES = [
    ("cac_fp32_ragged", 49, "fp32", 5.0, 30.0, 12),
    ("cac_fp16_ragged", 41, "fp16", 5.0, 0.0, 12),
    # interior, wrapped and ragged 32x8 column tiles of the 3D kernel
    ("cac3d_fp32_interior_ragged", (100, 45, 5), "fp32", 5.0, 30.0, 8),
    ("cac3d_fp16_interior_ragged", (100, 45, 5), "fp16", 5.0, 0.0, 8),
]


def run_step_case(make, storage, kernel, steps):
    from paper_2003_06342_b300 import Solver
    w = make()
    s = Solver(w.n, w.periodic, w.params, storage=storage)
    s.init(w.phi0, w.T0, p0=w.p0)
    s.set_kernel(kernel)
    s.step(steps)
    assert s.kernel() == kernel
    st = s.get_state().cpu().numpy().copy()
    s.sync()
    return st


def run_cac_case(n, storage, speed, period, steps):
    from paper_2003_06342_b300 import Solver
    if isinstance(n, tuple):
        # the vortex disk of the x-y plane repeated along z, uz = 0
        nx, ny, nz = n
        w = W.vortex_disk(n=nx)
        phi0 = np.repeat(w.phi0[None, :ny, :], nz, axis=0)
        u = [np.repeat(uu[None, :ny, :] * speed, nz, axis=0) for uu in w.extra["u"]] + [np.zeros_like(phi0)]
        s = Solver((nx, ny, nz), (True, True, True), w.params, storage=storage)
        s.set_velocity(u, period)
        s.init(phi0, np.ones_like(phi0))
        s.step(steps)
        st = s.get_state().cpu().numpy().copy()
        s.sync()
        return st
    w = W.vortex_disk(n=n)
    u = [uu * speed for uu in w.extra["u"]]
    s = Solver(w.n, w.periodic, w.params, storage=storage)
    s.set_velocity(u, period)
    s.init(w.phi0, w.T0)
    s.step(steps)
    st = s.get_state().cpu().numpy().copy()
    s.sync()
    return st


def run_adjoint_case(biased=False):
    from paper_2003_06342_b300.adjoint import gradients
    w = W.film_boiling_2d(40, 18, rho_ratio=5.0, y0=7.0, amplitude=1.5, phi_wall=(1.0, 0.0), theta_I=0.05)
    if biased:
        # wide enough for interior tiles of the two-ring window
        w = W.film_boiling_2d(96, 24, rho_ratio=5.0, y0=8.0, amplitude=1.5, phi_wall=(1.0, 0.0),
                              theta_I=0.05, grad_scheme="biased2")
    J, g = gradients(w.n, w.periodic, w.params, w.phi0, w.T0, w.phi0.copy(), 8, K=3, p0=w.p0)
    torch.cuda.synchronize()
    return np.concatenate([[J, g["L"], g["M_phi"], g["sigma"]], g["T0"].double().cpu().numpy().ravel()])


def run_noalloc_case():
    """The allocation-free sums on a ragged size (not a multiple of the
    256-cell block)."""
    import ctypes
    from paper_2003_06342_b300 import _binding as B
    n = 100003
    g = torch.Generator().manual_seed(7)
    phi = torch.rand(n, generator=g, dtype=torch.float32).cuda()
    T = (1.0 + 0.1 * torch.rand(n, generator=g, dtype=torch.float32)).cuda()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    B.check(B.lib.lbm_field_sums_noalloc(ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(T.data_ptr()), n,
                                         10.0, 1.0, 1.0, 1.0, ctypes.c_void_p(out.data_ptr()), None),
            "lbm_field_sums_noalloc")
    torch.cuda.synchronize()
    return out.cpu().numpy()


def run_all():
    out = {}
    for name, make, storage, kernel, steps in STEP_CASES:
        out[name] = run_step_case(make, storage, kernel, steps)
    for name, n, storage, speed, period, steps in CAC_CASES:
        out[name] = run_cac_case(n, storage, speed, period, steps)
    out["adjoint"] = run_adjoint_case()
    out["adjoint_biased"] = run_adjoint_case(biased=True)
    out["noalloc"] = run_noalloc_case()
    return out


def main(path):
    from paper_2003_06342_b300 import _binding as B
    assert B.DEBUG and B.LIB_PATH.endswith("liblbmpf_debug.so"), B.LIB_PATH
    np.savez(path, **run_all())
    print("bounds-checked cases ok")


if __name__ == "__main__":
    main(sys.argv[1])
