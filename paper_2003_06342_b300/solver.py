"""Python front end of the C ABI: a `Solver` owning one lattice on one GPU.

PyTorch provides the device memory (the workspace is a uint8 CUDA tensor) and
the CUDA stream; every step of the method runs in the library's kernels.
"""
import ctypes

import numpy as np
import torch

from . import _binding as B

STORAGE = {"fp32": B.LBM_STORE_FP32, "fp16": B.LBM_STORE_FP16, "bf16": B.LBM_STORE_BF16}


def make_params(d, storage="fp32", store_ref=None, store_scale=None):
    """lbm_params from a dictionary of lattice-unit parameters (the keys of
    include/lbm_pf.h).  Default storage references: 0 for f, 1/2 for g and
    T_sat for s; default 16-bit scale 1."""
    p = B.lbm_params()
    for k in ("rho_l", "rho_g", "nu_l", "nu_g", "alpha_l", "alpha_g", "sigma", "W", "M_phi",
              "A", "theta_I", "L", "Cp", "T_sat"):
        setattr(p, k, float(d[k]))
    for k, n in (("gravity", 3), ("body_force", 3), ("phi_wall", 2), ("T_wall", 2)):
        vals = list(d.get(k, [0.0] * n)) + [0.0] * n
        getattr(p, k)[:] = [float(v) for v in vals[:n]]
    p.normal_eps = float(d.get("normal_eps", 1e-3))
    ref = store_ref if store_ref is not None else (0.0, 0.5, float(d["T_sat"]))
    scale = store_scale if store_scale is not None else (1.0, 1.0, 1.0)
    p.store_ref[:] = [float(v) for v in ref]
    p.store_scale[:] = [float(v) for v in scale]
    p.source_on = int(d.get("source_on", 1))
    p.visc_interp = int(d.get("visc_interp", 0))
    p.alpha_interp = int(d.get("alpha_interp", 0))
    p.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    p.model = int(d.get("model", 0))
    coll = d.get("collision", 0)
    p.collision = {"bgk": 0, "trt": 1, "mrt": 2}[coll] if isinstance(coll, str) else int(coll)
    p.trt_magic[:] = [float(v) for v in d.get("trt_magic", (0.25, 0.25, 0.25))]
    p.mrt_rates[:] = [float(v) for v in d.get("mrt_rates", (1.4, 1.4, 1.2))]
    p.mrt_rates_g[:] = [float(v) for v in d.get("mrt_rates_g", (0.0, 0.0, 0.0, 0.0))]
    gs = d.get("grad_scheme", 0)
    p.grad_scheme = {"central": 0, "biased2": 1}[gs] if isinstance(gs, str) else int(gs)
    return p


def make_grid(n, periodic):
    g = B.lbm_grid()
    g.nx, g.ny = int(n[0]), int(n[1])
    g.nz = int(n[2]) if len(n) == 3 else 1
    per = list(periodic) + [True] * (3 - len(periodic))
    g.periodic[:] = [1 if v else 0 for v in per]
    return g


def workspace_bytes(n, periodic, params, storage="fp32"):
    g = make_grid(n, periodic)
    p = make_params(params, storage)
    out = ctypes.c_size_t()
    lat = B.LBM_D2Q9 if len(n) == 2 else B.LBM_D3Q19_D3Q7
    B.check(B.lib.lbm_workspace_bytes(ctypes.byref(g), lat, ctypes.byref(p), ctypes.byref(out)),
            "lbm_workspace_bytes")
    return out.value


class Solver:
    """One phase-field LB lattice.  n = (nx, ny) or (nx, ny, nz); fields are
    arrays of shape reversed(n) ([z][y][x])."""

    def __init__(self, n, periodic, params, storage="fp32", device="cuda", stream=None,
                 store_ref=None, store_scale=None):
        self.n = tuple(int(v) for v in n)
        self.dim = len(self.n)
        self.shape = tuple(reversed(self.n))
        self.cells = int(np.prod(self.n))
        self.device = torch.device(device)
        self.storage = storage
        self.params = dict(params)
        self._grid = make_grid(self.n, periodic)
        self._params = make_params(params, storage, store_ref, store_scale)
        self.lattice = B.LBM_D2Q9 if self.dim == 2 else B.LBM_D3Q19_D3Q7
        nbytes = ctypes.c_size_t()
        B.check(B.lib.lbm_workspace_bytes(ctypes.byref(self._grid), self.lattice,
                                          ctypes.byref(self._params), ctypes.byref(nbytes)),
                "lbm_workspace_bytes")
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        B.check(B.lib.lbm_create(ctypes.byref(self._grid), self.lattice, ctypes.byref(self._params),
                                 ctypes.c_void_p(self.workspace.data_ptr()),
                                 ctypes.c_size_t(nbytes.value),
                                 ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)),
                "lbm_create")
        self._h = h
        self.Qf, self.Qg = (9, 9) if self.dim == 2 else (19, 7)

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            B.lib.lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self.stream = stream
        B.check(B.lib.lbm_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)), "lbm_set_stream")

    # -- helpers
    def _as_device_f32(self, a):
        if a is None:
            return None
        t = torch.as_tensor(a)
        t = t.to(device=self.device, dtype=torch.float32).contiguous()
        if tuple(t.shape) != self.shape:
            raise ValueError(f"field shape {tuple(t.shape)} != {self.shape}")
        return t

    # -- API
    def init(self, phi0, T0, u0=None, p0=None):
        """Populations = barred equilibria of (phi0, T0, u0, p0)."""
        keep = [self._as_device_f32(phi0), self._as_device_f32(T0)]
        u = [None, None, None]
        if u0 is not None:
            for a in range(self.dim):
                u[a] = self._as_device_f32(u0[a])
        p = self._as_device_f32(p0)
        keep += u + [p]
        f = B.lbm_fields()
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        f.phi, f.T = keep[0].data_ptr(), keep[1].data_ptr()
        f.ux = u[0].data_ptr() if u[0] is not None else None
        f.uy = u[1].data_ptr() if u[1] is not None else None
        f.uz = u[2].data_ptr() if u[2] is not None else None
        f.p = p.data_ptr() if p is not None else None
        f.on_device, f.dtype = 1, 0
        B.check(B.lib.lbm_init(self._h, ctypes.byref(f)), "lbm_init")
        self._keep = keep     # inputs stay alive until the init kernel has run
        return self

    @staticmethod
    def _host_array(a, dtype):
        """A C-contiguous host array (numpy or CPU tensor) of `dtype`, kept
        without a copy when it already is one (a pinned float32 tensor stays
        pinned, so its copy to the device runs at the bus rate)."""
        if isinstance(a, torch.Tensor):
            if a.is_cuda:
                raise ValueError("host path: expected a CPU array")
            want = torch.float32 if dtype == np.float32 else torch.float64
            return a if (a.dtype == want and a.is_contiguous()) else a.to(want).contiguous()
        return np.ascontiguousarray(a, dtype=dtype)

    @staticmethod
    def _host_ptr(a):
        return a.data_ptr() if isinstance(a, torch.Tensor) else a.ctypes.data

    def init_host(self, phi0, T0, u0=None, p0=None, dtype=np.float64):
        """Same as init() from host arrays through the host-pointer path of
        lbm_init: float64 (converted on the host) or float32 (copied as is;
        pass pinned CPU tensors for the fastest transfer)."""
        if dtype not in (np.float32, np.float64):
            raise ValueError("dtype must be float32 or float64")
        arrs = [self._host_array(phi0, dtype), self._host_array(T0, dtype)]
        u = [None, None, None]
        if u0 is not None:
            for a in range(self.dim):
                u[a] = self._host_array(u0[a], dtype)
        p = None if p0 is None else self._host_array(p0, dtype)
        f = B.lbm_fields()
        f.phi, f.T = self._host_ptr(arrs[0]), self._host_ptr(arrs[1])
        f.ux = self._host_ptr(u[0]) if u[0] is not None else None
        f.uy = self._host_ptr(u[1]) if u[1] is not None else None
        f.uz = self._host_ptr(u[2]) if u[2] is not None else None
        f.p = self._host_ptr(p) if p is not None else None
        f.on_device, f.dtype = 0, (0 if dtype == np.float32 else 1)
        B.check(B.lib.lbm_init(self._h, ctypes.byref(f)), "lbm_init")
        return self

    def set_velocity(self, u, period=0.0):
        """Phase-field model: the imposed velocity (list of per-axis arrays)
        and its time factor cos(pi n / period) (period 0: constant)."""
        arrs = [np.ascontiguousarray(ua, dtype=np.float64) for ua in u]
        f = B.lbm_fields()
        f.phi = f.T = None
        f.ux = arrs[0].ctypes.data
        f.uy = arrs[1].ctypes.data if len(arrs) > 1 else None
        f.uz = arrs[2].ctypes.data if len(arrs) > 2 else None
        f.p = None
        f.on_device, f.dtype = 0, 1
        B.check(B.lib.lbm_set_velocity(self._h, ctypes.byref(f), float(period)), "lbm_set_velocity")
        return self

    def set_health_check(self, every, phi_excess=0.6):
        """Check phi and the lagged source every `every` steps on the device
        (0: off); a failed check makes sync() raise LBMError(LBM_ENONFINITE)."""
        B.check(B.lib.lbm_set_health_check(self._h, int(every), float(phi_excess)), "lbm_set_health_check")
        return self

    def step(self, n=1):
        B.check(B.lib.lbm_step(self._h, int(n)), "lbm_step")
        return self

    def fields(self):
        """dict(phi, T, u=[ux, uy(, uz)], p) as float32 CUDA tensors."""
        out = {k: torch.empty(self.shape, dtype=torch.float32, device=self.device)
               for k in ("phi", "T", "ux", "uy", "uz", "p")}
        f = B.lbm_fields()
        f.phi, f.T = out["phi"].data_ptr(), out["T"].data_ptr()
        f.ux, f.uy, f.uz = out["ux"].data_ptr(), out["uy"].data_ptr(), out["uz"].data_ptr()
        f.p = out["p"].data_ptr()
        f.on_device, f.dtype = 1, 0
        B.check(B.lib.lbm_get_fields(self._h, ctypes.byref(f)), "lbm_get_fields")
        u = [out["ux"], out["uy"]] + ([out["uz"]] if self.dim == 3 else [])
        return dict(phi=out["phi"], T=out["T"], u=u, p=out["p"])

    def fields_host(self, out=None):
        """dict(phi, T, u=[...], p) on the host through the host-pointer path:
        float64 numpy arrays by default, or written into `out`, a dict of
        float32 CPU buffers (keys phi, T, ux, uy, uz, p; pinned tensors copy
        at the bus rate)."""
        if out is None:
            out = {k: np.empty(self.shape, dtype=np.float64) for k in ("phi", "T", "ux", "uy", "uz", "p")}
            dt = 1
        else:
            dt = 0
        f = B.lbm_fields()
        f.phi, f.T = self._host_ptr(out["phi"]), self._host_ptr(out["T"])
        f.ux, f.uy = self._host_ptr(out["ux"]), self._host_ptr(out["uy"])
        f.uz = self._host_ptr(out["uz"]) if self.dim == 3 else None
        f.p = self._host_ptr(out["p"])
        f.on_device, f.dtype = 0, dt
        B.check(B.lib.lbm_get_fields(self._h, ctypes.byref(f)), "lbm_get_fields")
        u = [out["ux"], out["uy"]] + ([out["uz"]] if self.dim == 3 else [])
        return dict(phi=out["phi"], T=out["T"], u=u, p=out["p"])

    def reduce(self):
        """(sum phi, sum rho (Cp T + phi L)) in FP64; synchronises."""
        m, e = ctypes.c_double(), ctypes.c_double()
        B.check(B.lib.lbm_reduce(self._h, ctypes.byref(m), ctypes.byref(e)), "lbm_reduce")
        return m.value, e.value

    def reduce_async(self, out):
        """Queue the reduction into a float64 CUDA tensor of 2 elements."""
        B.check(B.lib.lbm_reduce_async(self._h, ctypes.c_void_p(out.data_ptr())), "lbm_reduce_async")
        return out

    def state_bytes(self):
        n = ctypes.c_size_t()
        B.check(B.lib.lbm_state_bytes(self._h, ctypes.byref(n)), "lbm_state_bytes")
        return n.value

    def get_state(self, out=None):
        nb = self.state_bytes()
        if out is None:
            out = torch.empty(nb, dtype=torch.uint8, device=self.device)
        B.check(B.lib.lbm_get_state(self._h, ctypes.c_void_p(out.data_ptr()), nb, 1 if out.is_cuda else 0),
                "lbm_get_state")
        return out

    def set_state(self, buf):
        B.check(B.lib.lbm_set_state(self._h, ctypes.c_void_p(buf.data_ptr()), buf.numel(),
                                    1 if buf.is_cuda else 0), "lbm_set_state")
        return self

    def columns_bytes(self, ncols):
        n = ctypes.c_size_t()
        B.check(B.lib.lbm_columns_bytes(self._h, int(ncols), ctypes.byref(n)), "lbm_columns_bytes")
        return n.value

    def pack_columns(self, x0, ncols, out=None):
        """The stored state of columns [x0, x0 + ncols) as a uint8 CUDA tensor
        (queued on the solver's stream)."""
        nb = self.columns_bytes(ncols)
        if out is None:
            out = torch.empty(nb, dtype=torch.uint8, device=self.device)
        B.check(B.lib.lbm_pack_columns(self._h, int(x0), int(ncols), ctypes.c_void_p(out.data_ptr())),
                "lbm_pack_columns")
        return out

    def unpack_columns(self, x0, ncols, buf):
        """Overwrite columns [x0, x0 + ncols) of the state with a block from
        pack_columns (a uint8 CUDA tensor of columns_bytes(ncols) bytes)."""
        if buf.numel() < self.columns_bytes(ncols) or not buf.is_cuda:
            raise ValueError("unpack_columns needs a CUDA buffer of columns_bytes(ncols) bytes")
        B.check(B.lib.lbm_unpack_columns(self._h, int(x0), int(ncols), ctypes.c_void_p(buf.data_ptr())),
                "lbm_unpack_columns")
        return self

    def stream_map(self, which=0):
        Q = self.Qf if which == 0 else self.Qg
        src = torch.empty((Q, self.cells), dtype=torch.int32, device=self.device)
        kind = torch.empty((Q, self.cells), dtype=torch.int8, device=self.device)
        B.check(B.lib.lbm_stream_map(self._h, int(which), ctypes.c_void_p(src.data_ptr()),
                                     ctypes.c_void_p(kind.data_ptr())), "lbm_stream_map")
        return src, kind

    def set_kernel(self, kind):
        """'auto', 'tiled' or 'tma' (2D step kernel variant)."""
        code = {"auto": B.LBM_KERNEL_AUTO, "tiled": B.LBM_KERNEL_TILED, "tma": B.LBM_KERNEL_TMA}[kind]
        B.check(B.lib.lbm_set_kernel(self._h, code), "lbm_set_kernel")
        return self

    def kernel(self):
        v = ctypes.c_int32()
        B.check(B.lib.lbm_get_kernel(self._h, ctypes.byref(v)), "lbm_get_kernel")
        return {B.LBM_KERNEL_TILED: "tiled", B.LBM_KERNEL_TMA: "tma"}.get(v.value, "auto")

    def steps_done(self):
        v = ctypes.c_int64()
        B.check(B.lib.lbm_steps_done(self._h, ctypes.byref(v)), "lbm_steps_done")
        return v.value

    def last_launches(self):
        v = ctypes.c_int32()
        B.check(B.lib.lbm_last_launches(self._h, ctypes.byref(v)), "lbm_last_launches")
        return v.value

    def sync(self):
        B.check(B.lib.lbm_sync(self._h), "lbm_sync")
