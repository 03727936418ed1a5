"""Oracle of the phase-field equation alone with an imposed velocity field.

Test infrastructure only (see the package docstring).  This is the
conservative Allen-Cahn lattice Boltzmann scheme of Sec. 3.2 (Eq. LBE for g
with the equilibrium Eq. Geq_Allen-Cahn_Eq, the function Gamma of Eq.
FunctionGamma and the source Eq. SourceTerm_AllenCahn) run without phase
change (q = 0) and with the velocity prescribed instead of computed from the
flow populations -- the setting of the paper's CAC validations (Sec. 4.1:
Zalesak's slotted disk in a rotating field, a disk in a vortex whose
rotation reverses).  The velocity at step n is u(x) * c(n) with c(n) =
cos(pi n / period) when period > 0 (the reversing vortex of Sec. 4.1 uses
period = 2 T_f in steps) and c = 1 otherwise.

State: the post-streaming g populations (Qg, *grid), float64.  The stencils,
the normal, Gamma, the relaxation and the streaming are the coupled oracle's
own functions (oracle.model), so both models share one definition of each.
"""
import math

import torch

from . import model as M
from .lattice import lattices_for

F64 = M.F64


def velocity_factor(n, period):
    return math.cos(math.pi * n / period) if period > 0 else 1.0


def _eq_and_source(phi, u, P, grid):
    """phi Gamma_i(u) and F^g_i = (4/W) phi (1 - phi) w_i e_i.n (no P^g: q = 0)."""
    _, Lg, _ = lattices_for(grid.dim)
    grad, _ = M.gradient_laplacian(phi, grid, P)
    n = M._normal(grad, P.normal_eps)
    G = M.gamma(Lg, u)
    interface = (4.0 / P.W) * phi * (1.0 - phi)
    eq, F = [], []
    for i in range(Lg.Q):
        en = sum(float(Lg.e[i][a]) * n[a] for a in range(grid.dim))
        eq.append(phi * G[i])
        F.append(interface * Lg.wf(i) * en)
    return eq, F


def phase_field(g):
    """phi = sum_i g_i (Eq. Moment_Phi with q = 0)."""
    return g.sum(dim=0)


def init_state(phi0, u, P, grid, period=0.0):
    """Barred equilibria g_i = phi Gamma_i(u c(0)) - F^g_i / 2 (the same
    initialisation reading as the coupled model)."""
    phi0 = torch.as_tensor(phi0, dtype=F64)
    c = velocity_factor(0, period)
    uu = [torch.as_tensor(ua, dtype=F64) * c for ua in u]
    eq, F = _eq_and_source(phi0, uu, P, grid)
    return torch.stack([eq[i] - 0.5 * F[i] for i in range(len(eq))])


def step(g, n, u, P, grid, period=0.0):
    """Step n -> n+1: moments, collision (Eq. LBE with S = F^g), streaming
    (periodic axes; anti bounce-back with the wall's phi on a wall axis)."""
    _, Lg, _ = lattices_for(grid.dim)
    phi = phase_field(g)
    c = velocity_factor(n, period)
    uu = [torch.as_tensor(ua, dtype=F64) * c for ua in u]
    eq, F = _eq_and_source(phi, uu, P, grid)
    tau = P.M_phi / float(Lg.cs2)
    post = torch.stack([M._relax(g[i], eq[i] - 0.5 * F[i], F[i], tau) for i in range(Lg.Q)])
    return M.stream(post, Lg, grid, "g", P)


def run(g, u, P, grid, nsteps, period=0.0, n0=0):
    for n in range(n0, n0 + nsteps):
        g = step(g, n, u, P, grid, period)
    return g
