"""Gradients of a final-time phase-field misfit through the CUDA adjoint.

J = 1/2 sum_x (phi^N(x) - phi_target(x))^2 after N steps from lbm_init(phi_0,
T_0).  `gradients` runs the forward, keeping a checkpoint of the state every
K steps, then walks the segments backwards: each segment is recomputed from
its checkpoint (storing its K states) and the adjoint kernels
(lbm_adjoint_step) take Lambda^{n+1} to Lambda^n; the initialisation's adjoint
gives dJ/dT_0.  `FinalPhiMisfit` exposes the same as a torch.autograd.Function
of (T_0, L, M_phi, sigma).
"""
import ctypes

import torch

from . import _binding as B
from .solver import Solver


def _f32(a, device):
    return torch.as_tensor(a).to(device=device, dtype=torch.float32).contiguous()


def gradients(n, periodic, params, phi0, T0, phi_target, nsteps, K=100, p0=None, device="cuda"):
    """Returns (J, dict(L=..., M_phi=..., sigma=..., T0=tensor)).  2D, FP32."""
    dev = torch.device(device)
    s = Solver(n, periodic, params, storage="fp32", device=dev)
    phi0_t, T0_t = _f32(phi0, dev), _f32(T0, dev)
    p0_t = None if p0 is None else _f32(p0, dev)
    tgt = _f32(phi_target, dev)
    s.init(phi0_t, T0_t, p0=p0_t)
    adj_bytes, scr_bytes = ctypes.c_size_t(), ctypes.c_size_t()
    B.check(B.lib.lbm_adjoint_bytes(s._h, ctypes.byref(adj_bytes), ctypes.byref(scr_bytes)),
            "lbm_adjoint_bytes")
    nstate = s.state_bytes()
    # forward with checkpoints every K steps
    seg_starts = list(range(0, nsteps, K))
    # device buffers allocated once: one checkpoint per segment and the
    # states of the segment being reversed
    ckpts = torch.empty((len(seg_starts), nstate), dtype=torch.uint8, device=dev)
    seg_states = torch.empty((min(K, max(nsteps, 1)), nstate), dtype=torch.uint8, device=dev)
    for k, start in enumerate(seg_starts):
        s.get_state(ckpts[k])
        s.step(min(K, nsteps - start))
    final = s.get_state()
    lam = torch.zeros(adj_bytes.value // 4, dtype=torch.float32, device=dev)
    lam_next = torch.zeros_like(lam)
    scratch = torch.zeros(scr_bytes.value // 4, dtype=torch.float32, device=dev)
    J = torch.zeros(3, dtype=torch.float64, device=dev)
    dparams = torch.zeros(3, dtype=torch.float64, device=dev)
    vp = lambda t: ctypes.c_void_p(t.data_ptr())
    B.check(B.lib.lbm_adjoint_terminal(s._h, vp(final), vp(tgt), vp(lam_next), vp(J)),
            "lbm_adjoint_terminal")
    stride = seg_states.stride(0)
    for k in reversed(range(len(seg_starts))):
        seg = min(K, nsteps - seg_starts[k])
        # recompute the segment from its checkpoint, keeping every state
        s.set_state(ckpts[k])
        seg_states[0].copy_(ckpts[k])
        if seg > 1:
            B.check(B.lib.lbm_step_record(s._h, seg - 1, vp(seg_states[1]), stride), "lbm_step_record")
        # and walk it backwards in one call; the result sits in lam_next after
        # an even number of steps, in lam after an odd one
        B.check(B.lib.lbm_adjoint_steps(s._h, vp(seg_states), stride, seg, vp(lam_next), vp(lam),
                                        vp(scratch), vp(dparams)), "lbm_adjoint_steps")
        if seg % 2:
            lam, lam_next = lam_next, lam
    dT0 = torch.zeros_like(T0_t)
    f = B.lbm_fields()
    f.phi, f.T = phi0_t.data_ptr(), T0_t.data_ptr()
    f.ux = f.uy = f.uz = None
    f.p = p0_t.data_ptr() if p0_t is not None else None
    f.on_device, f.dtype = 1, 0
    B.check(B.lib.lbm_adjoint_init(s._h, ctypes.byref(f), vp(lam_next), vp(dT0), vp(dparams)),
            "lbm_adjoint_init")
    torch.cuda.synchronize(dev)
    d = dparams.tolist()
    return float(J[0]), dict(L=d[0], M_phi=d[1], sigma=d[2], T0=dT0)


class FinalPhiMisfit(torch.autograd.Function):
    """J(T_0, L, M_phi, sigma) with a CUDA-adjoint backward.  Other inputs:
    grid size n, periodic flags, the remaining parameters, phi_0, phi_target,
    the step count and the checkpoint interval K."""

    @staticmethod
    def forward(ctx, T0, L, M_phi, sigma, n, periodic, params, phi0, phi_target, nsteps, K):
        p = dict(params)
        p.update(L=float(L), M_phi=float(M_phi), sigma=float(sigma))
        J, g = gradients(n, periodic, p, phi0, T0.detach(), phi_target, int(nsteps), int(K),
                         device=T0.device if T0.is_cuda else "cuda")
        ctx.save_for_backward(g["T0"].to(T0.device, T0.dtype))
        ctx.g = (g["L"], g["M_phi"], g["sigma"])
        return torch.tensor(J, dtype=torch.float64, device=T0.device)

    @staticmethod
    def backward(ctx, gJ):
        (dT0,) = ctx.saved_tensors
        dL, dM, dS = ctx.g
        s = float(gJ)
        mk = lambda v: torch.tensor(s * v, dtype=torch.float64)
        return (s * dT0, mk(dL), mk(dM), mk(dS)) + (None,) * 7
