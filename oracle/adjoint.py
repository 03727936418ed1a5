"""Reference gradients of a final-time phase-field misfit (test infrastructure).

J = 1/2 sum_x (phi^N(x) - phi_target(x))^2, with phi^N the phase field after N
steps of `model.step` from `model.init_state(phi_0, T_0)`.  The gradient with
respect to the latent heat L, the mobility M_phi, the surface tension sigma
and the initial temperature field T_0 is taken by torch autograd (reverse
mode) through the float64 oracle itself, so it is the exact discrete adjoint
of the oracle's forward map up to rounding; nothing is derived by hand here.
A central finite-difference helper on the same forward map pins it.
"""
import torch
from torch.utils.checkpoint import checkpoint

from . import model as M

F64 = torch.float64
_KEYS = ("f", "g", "s", "phi_prev", "q_prev")


def _steps(params, grid, n, L, M_phi, sigma, *state):
    """n oracle steps from a state given as tensors (the form autograd
    checkpointing needs)."""
    P = M.Params.from_dict(params)
    P.L, P.M_phi, P.sigma = L, M_phi, sigma
    st = dict(zip(_KEYS, state))
    for _ in range(n):
        st = M.step(st, P, grid)
    return tuple(st[k] for k in _KEYS)


def _forward(phi0, T0, params, grid, nsteps, phi_target, L, M_phi, sigma, p0=None, segment=None):
    P = M.Params.from_dict(params)
    P.L, P.M_phi, P.sigma = L, M_phi, sigma
    st = M.init_state(phi0, T0, P, grid, p0=p0)
    if segment is None:
        for _ in range(nsteps):
            st = M.step(st, P, grid)
    else:
        # the same steps, with autograd keeping only every segment's first
        # state and recomputing the segment in the backward pass (memory
        # only: the forward values and the gradients are those of the loop
        # above)
        state = tuple(st[k] for k in _KEYS)
        done = 0
        while done < nsteps:
            n = min(segment, nsteps - done)
            state = checkpoint(_steps, params, grid, n, L, M_phi, sigma, *state, use_reentrant=False)
            done += n
        st = dict(zip(_KEYS, state))
    phi = M.fields(st, P, grid)["phi"]
    return 0.5 * ((phi - phi_target) ** 2).sum()


def misfit(phi0, T0, params, grid, nsteps, phi_target, p0=None):
    """J for the given inputs (float)."""
    with torch.no_grad():
        J = _forward(torch.as_tensor(phi0, dtype=F64), torch.as_tensor(T0, dtype=F64), params,
                     grid, nsteps, torch.as_tensor(phi_target, dtype=F64),
                     float(params["L"]), float(params["M_phi"]), float(params["sigma"]), p0)
    return float(J)


def gradients(phi0, T0, params, grid, nsteps, phi_target, p0=None, segment=None):
    """(J, dict(L=..., M_phi=..., sigma=..., T0=tensor)) by reverse mode;
    segment=k recomputes k-step segments in the backward pass to bound the
    memory of long runs."""
    L = torch.tensor(float(params["L"]), dtype=F64, requires_grad=True)
    Mp = torch.tensor(float(params["M_phi"]), dtype=F64, requires_grad=True)
    sg = torch.tensor(float(params["sigma"]), dtype=F64, requires_grad=True)
    T0t = torch.as_tensor(T0, dtype=F64).clone().requires_grad_(True)
    J = _forward(torch.as_tensor(phi0, dtype=F64), T0t, params, grid, nsteps,
                 torch.as_tensor(phi_target, dtype=F64), L, Mp, sg, p0, segment)
    J.backward()
    return J.item(), dict(L=float(L.grad), M_phi=float(Mp.grad), sigma=float(sg.grad),
                          T0=T0t.grad.detach().clone())


def central_difference(phi0, T0, params, grid, nsteps, phi_target, name, h, direction=None,
                       p0=None):
    """(J(+h) - J(-h)) / 2h for a scalar parameter `name`, or for T0 along
    `direction` (a field) when name == 'T0'."""
    def J_at(sign):
        p = dict(params)
        T = torch.as_tensor(T0, dtype=F64).clone()
        if name == "T0":
            T = T + sign * h * torch.as_tensor(direction, dtype=F64)
        else:
            p[name] = float(params[name]) + sign * h
        return misfit(phi0, T, p, grid, nsteps, phi_target, p0)
    return (J_at(+1.0) - J_at(-1.0)) / (2.0 * h)
