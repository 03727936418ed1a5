"""Oracle time step of the coupled phase-field / Navier-Stokes / heat LB model.

Test infrastructure only (see the package docstring).  Plain float64 PyTorch
CPU code; every loop over lattice directions runs i = 0..Q-1 in lattice order.

State between steps (all float64 tensors, cells laid out [z][y][x]):
  f, g, s   post-streaming populations fbar_i, gbar_i, sbar_i at time n,
            shapes (Qf, *grid), (Qg, *grid), (Qf, *grid)
  phi_prev  phi at time n-1 (for the backward difference of d(phi)/dt)
  q_prev    the production term mdot'''/rho_g evaluated in the collision of
            step n-1 (lagged source used by the moments at time n)

One step n -> n+1 (Sec. 3):
  1. moments at n: phi (Eq. Moment_Phi), grad/laplacian of phi (Eqs. Grad,
     Laplacian), closures (Eqs. Density, Viscosity, ChemicalPotential,
     SuperficialTensionForce, buoyancy), u and p (Eqs. Velocity, Pressure),
     T (Eq. Moment_Temp);
  2. production rate q^n = mdot'''/rho_g (Eq. ProductionRate);
  3. the three BGK collisions in barred variables (Eq. LBE) with the
     equilibria Eqs. Feq_NS_Incompr, Geq_Allen-Cahn_Eq, Seq_Temp, the function
     Gamma (Eq. FunctionGamma) and the sources Eqs. Forcing, MicroProduction,
     SourceTerm_AllenCahn, Def_SourceTerms_Temp;
  4. streaming with periodic axes, half-way bounce-back for f and anti
     bounce-back Dirichlet for g and s on the wall axis (Sec. 3.3, 4.1).

Readings taken where the paper is silent or inconsistent (each is listed in
the design notes with its reason):
  * grad/laplacian use the stencil lattice's own 1/cs^2 (=3) and its
    neighbours (D2Q9 in 2D, D3Q19 in 3D); the D3Q7 phase-field lattice uses
    cs^2 = 1/4 in Gamma, F^g and tau_g = M_phi/cs^2;
  * buoyancy F_v = (rho(phi) - rho_l) * gravity, gravity pointing down, so the
    light phase rises;
  * S^s_i = -w_i (L/Cp) [d(phi)/dt + div(u phi)] (the sign that makes Eq.
    Moment_Temp the zeroth moment of the variable change, App. C);
  * d(phi)/dt = phi^n - phi^{n-1};  div(u phi) = u.grad(phi) + phi div(u),
    div(u) from Eq. ConservMasse_ChgtPhase;
  * the sources inside the moments at n+1 use the lagged q^n;
  * n = grad(phi) / max(|grad(phi)|, eps), eps = 1e-3 by default: where the
    gradient is below eps (only in the far tails of the profile, more than
    about 7 cells from the centre of a W = 4 interface) the counter term is
    scaled down instead of following the direction of rounding noise;
  * alpha(phi) is interpolated linearly (switch: harmonic);
  * rho(phi), nu(phi) and alpha(phi) are evaluated on phi clipped to [0, 1]
    (the model's range): at density ratio 100 an overshoot phi - 1 > 0.0101
    would otherwise make rho(phi) <= 0;
  * phi ghost value on a wall = the wall's Dirichlet value;
  * initial populations = barred equilibria, theta_bar = theta_eq - S/2,
    with phi_prev = phi_0 and q_prev = q(phi_0, T_0).
"""
from dataclasses import dataclass
from functools import lru_cache

import numpy as np
import torch

from .lattice import lattices_for, D2Q9, D3Q7, D3Q19

F64 = torch.float64

# stream-map kinds (pull view: what lands in direction i of cell x)
KIND_INTERIOR = 0   # from x - e_i, inside the box
KIND_PERIODIC = 1   # from x - e_i wrapped over a periodic axis
KIND_WALL_LO = 2    # bounced at the low wall of the wall axis
KIND_WALL_HI = 3    # bounced at the high wall of the wall axis


@dataclass
class Params:
    """Model parameters in lattice units (dx = dt = 1)."""
    rho_l: float
    rho_g: float
    nu_l: float
    nu_g: float
    alpha_l: float
    alpha_g: float
    sigma: float
    W: float
    M_phi: float
    A: float = 10.0 / 48.0
    theta_I: float = 0.0
    L: float = 1.0
    Cp: float = 1.0
    T_sat: float = 1.0
    gravity: tuple = (0.0, 0.0, 0.0)
    body_force: tuple = (0.0, 0.0, 0.0)
    phi_wall: tuple = (0.0, 0.0)
    T_wall: tuple = (0.0, 0.0)
    source_on: bool = True
    visc_interp: str = "harmonic"     # Eq. Viscosity; "linear" is Eq. Visco_lin
    alpha_interp: str = "linear"
    g_form: str = "source"            # "source": Eq. LBE_PhaseField_Eq;
                                      # "cac_eq": Eq. LBE_PhaseField_Eq_Alternative
    normal_eps: float = 1e-3          # n = grad phi / max(|grad phi|, normal_eps)
    collision: str = "bgk"            # "bgk": Eq. LBE; "trt": two relaxation rates
    grad_scheme: str = "central"      # Eq. DerivDirec_Grad; "biased2": second-order biased
    trt_magic: tuple = (0.25, 0.25, 0.25)   # Lambda of the f, g, s sets (TRT only)
    mrt_rates: tuple = (1.4, 1.4, 1.2)      # s_e, s_eps, s_q of the flow set (MRT only)
    # s_e, s_eps, s_q, s_p of the phase-field set (MRT only; 0: the BGK rate)
    mrt_rates_g: tuple = (0.0, 0.0, 0.0, 0.0)

    @classmethod
    def from_dict(cls, d):
        keys = {k: d[k] for k in cls.__dataclass_fields__ if k in d}
        if "visc_interp" in keys and not isinstance(keys["visc_interp"], str):
            keys["visc_interp"] = "linear" if keys["visc_interp"] else "harmonic"
        if "alpha_interp" in keys and not isinstance(keys["alpha_interp"], str):
            keys["alpha_interp"] = "harmonic" if keys["alpha_interp"] else "linear"
        if "source_on" in keys:
            keys["source_on"] = bool(keys["source_on"])
        if "grad_scheme" in keys and not isinstance(keys["grad_scheme"], str):
            keys["grad_scheme"] = "biased2" if keys["grad_scheme"] else "central"
        if "collision" in keys and not isinstance(keys["collision"], str):
            keys["collision"] = {0: "bgk", 1: "trt", 2: "mrt"}[int(keys["collision"])]
        for k in ("mrt_rates", "mrt_rates_g"):
            if k in keys:
                keys[k] = tuple(float(v) for v in keys[k])
        if "trt_magic" in keys:
            keys["trt_magic"] = tuple(float(v) for v in keys["trt_magic"])
        for k in ("gravity", "body_force", "phi_wall", "T_wall"):
            if k in keys:
                keys[k] = tuple(float(v) for v in keys[k])
        return cls(**keys)


@dataclass(frozen=True)
class Grid:
    n: tuple          # (nx, ny) or (nx, ny, nz)
    periodic: tuple   # one bool per axis (x, y[, z])

    def __post_init__(self):
        if len(self.n) not in (2, 3) or len(self.periodic) != len(self.n):
            raise ValueError("grid must be 2D or 3D with one periodic flag per axis")
        if sum(1 for p in self.periodic if not p) > 1:
            raise ValueError("at most one non-periodic (wall) axis")

    @property
    def dim(self):
        return len(self.n)

    @property
    def shape(self):
        """Tensor shape, slowest axis first: (ny, nx) or (nz, ny, nx)."""
        return tuple(reversed(self.n))

    @property
    def cells(self):
        return int(np.prod(self.n))

    def tdim(self, axis):
        """Tensor dimension of spatial axis (0=x, 1=y, 2=z)."""
        return self.dim - 1 - axis


# ----------------------------------------------------------------------------
# neighbour access and finite differences (Sec. 3.4)
# ----------------------------------------------------------------------------

def _pad(field, grid, lo_val, hi_val, width=1):
    """`width` ghost layers on every axis: the wall's Dirichlet value on the
    wall axis, wrapped values on periodic axes.  The wall axis is padded
    first, so a ghost that is both beyond a wall and beyond a periodic edge
    holds the wall value."""
    out = field
    order = [a for a in range(grid.dim) if not grid.periodic[a]] + \
            [a for a in range(grid.dim) if grid.periodic[a]]
    for a in order:
        d = grid.tdim(a)
        size = out.shape[d]
        if grid.periodic[a]:
            lo = out.index_select(d, torch.tensor([k % size for k in range(-width, 0)]))
            hi = out.index_select(d, torch.tensor([k % size for k in range(width)]))
        else:
            shape = list(out.shape)
            shape[d] = width
            lo = torch.full(shape, lo_val, dtype=out.dtype)
            hi = torch.full(shape, hi_val, dtype=out.dtype)
        out = torch.cat([lo, out, hi], dim=d)
    return out


def _at(padded, grid, e, width=1):
    """Field value at x + e (|e_a| <= width) read from the padded field."""
    out = padded
    for a in range(grid.dim):
        out = out.narrow(grid.tdim(a), width + int(e[a]), grid.n[a])
    return out


def gradient_laplacian(phi, grid, P):
    """grad(phi) by Eqs. DerivDirec_Grad + Grad and lap(phi) by Eqs.
    DerivDirect_Laplacian + Laplacian, over the stencil lattice's directions
    i = 1..Q-1, with prefactor 1/cs^2 of that lattice.  With grad_scheme
    "biased2" the directional derivative in Eq. Grad is the second-order
    biased (upwind) difference of Sec. 3.4,
    e_i . grad(phi) = [-phi(x + 2 e_i) + 4 phi(x + e_i) - 3 phi(x)] / 2,
    read from two ghost layers; the Laplacian stays central."""
    lat = lattices_for(grid.dim)[2]
    biased = P.grad_scheme == "biased2"
    width = 2 if biased else 1
    pad = _pad(phi, grid, P.phi_wall[0], P.phi_wall[1], width)
    grad = [torch.zeros_like(phi) for _ in range(grid.dim)]
    lap = torch.zeros_like(phi)
    for i in range(1, lat.Q):
        e = lat.e[i]
        plus = _at(pad, grid, e, width)
        minus = _at(pad, grid, -e, width)
        if biased:
            plus2 = _at(pad, grid, 2 * e, width)
            directional = (-plus2 + 4.0 * plus - 3.0 * phi) / 2.0
        else:
            directional = (plus - minus) / 2.0         # e_i . grad(phi)
        second = plus - 2.0 * phi + minus              # (e_i . grad)^2 phi
        for a in range(grid.dim):
            if e[a] != 0:
                grad[a] = grad[a] + lat.wf(i) * float(e[a]) * directional
        lap = lap + lat.wf(i) * second
    inv_cs2 = 1.0 / float(lat.cs2)
    return [inv_cs2 * g for g in grad], inv_cs2 * lap


# ----------------------------------------------------------------------------
# closures (Sec. 2)
# ----------------------------------------------------------------------------

def _unit(phi):
    """phi restricted to the model's range 0 <= phi <= 1 (Sec. 2.1) for the
    property closures; overshoot beyond it is numerical."""
    return torch.clamp(phi, 0.0, 1.0)


def density(phi, P):
    """Eq. Density, on phi restricted to [0, 1]."""
    phi = _unit(phi)
    return phi * P.rho_g + (1.0 - phi) * P.rho_l


def viscosity(phi, P):
    """Eq. Viscosity (harmonic mean) or Eq. Visco_lin (linear), on phi
    restricted to [0, 1]."""
    phi = _unit(phi)
    if P.visc_interp == "harmonic":
        return P.nu_l * P.nu_g / (phi * P.nu_l + (1.0 - phi) * P.nu_g)
    return (1.0 - phi) * P.nu_l + phi * P.nu_g


def diffusivity(phi, P):
    """Thermal diffusivity alpha(phi): linear interpolation (reading), or
    harmonic mean as a switch, on phi restricted to [0, 1]."""
    phi = _unit(phi)
    if P.alpha_interp == "harmonic":
        return P.alpha_l * P.alpha_g / (phi * P.alpha_l + (1.0 - phi) * P.alpha_g)
    return phi * P.alpha_g + (1.0 - phi) * P.alpha_l


def chemical_potential(phi, lap, P):
    """Eq. ChemicalPotential with K, H from Eq. Def_K-H."""
    K = 1.5 * P.W * P.sigma
    H = 12.0 * P.sigma / P.W
    return 4.0 * H * phi * (phi - 1.0) * (phi - 0.5) - K * lap


def production_rate(phi, T, P):
    """q = mdot'''/rho_g of Eq. ProductionRate, theta = (Cp/L)(T - T_sat)."""
    if not P.source_on:
        return torch.zeros_like(phi)
    theta = (P.Cp / P.L) * (T - P.T_sat)
    alpha = diffusivity(phi, P)
    return -(4.0 * alpha / (P.A * P.W * P.W)) * (P.theta_I - theta) * phi * (1.0 - phi)


def gamma(lat, u):
    """Eq. FunctionGamma on lattice `lat` (its own cs^2)."""
    cs2 = float(lat.cs2)
    usq = sum(ua * ua for ua in u)
    out = []
    for i in range(lat.Q):
        cu = sum(float(lat.e[i][a]) * u[a] for a in range(len(u)))
        out.append(lat.wf(i) * (1.0 + cu / cs2 + cu * cu / (2.0 * cs2 * cs2) - usq / (2.0 * cs2)))
    return out


def _dot(a, b):
    return sum(x * y for x, y in zip(a, b))


def closures(phi, grid, P):
    """Everything the step derives from phi and its stencils (Sec. 2, 3.4)."""
    grad, lap = gradient_laplacian(phi, grid, P)
    rho = density(phi, P)
    grad_rho = [(P.rho_g - P.rho_l) * ga for ga in grad]
    mu = chemical_potential(phi, lap, P)
    F_tot = []
    for a in range(grid.dim):
        F_s = mu * grad[a]                                   # Eq. SuperficialTensionForce
        F_v = (rho - P.rho_l) * P.gravity[a]                 # buoyancy (reading)
        F_tot.append(F_s + F_v + P.body_force[a])            # Eq. Force_Total (+ body force)
    return dict(grad=grad, lap=lap, rho=rho, grad_rho=grad_rho, mu=mu, F_tot=F_tot)


def _kappa(P):
    """mdot'''(1/rho_g - 1/rho_l) = q * kappa with q = mdot'''/rho_g."""
    return 1.0 - P.rho_g / P.rho_l


# ----------------------------------------------------------------------------
# moments (Eqs. Moment_Phi, Velocity, Pressure, Moment_Temp)
# ----------------------------------------------------------------------------

def moments(st, P, grid):
    """Macroscopic fields at the time of the post-streaming state `st`."""
    Lf, Lg, _ = lattices_for(grid.dim)
    phi = st["g"][0]
    for i in range(1, Lg.Q):
        phi = phi + st["g"][i]
    phi = phi + 0.5 * st["q_prev"]                           # sum_i P^g_i = q
    C = closures(phi, grid, P)
    cs2 = float(Lf.cs2)
    j = [torch.zeros_like(phi) for _ in range(grid.dim)]
    sum_f = st["f"][0]
    sum_s = st["s"][0]
    for i in range(Lf.Q):
        for a in range(grid.dim):
            if Lf.e[i][a] != 0:
                j[a] = j[a] + float(Lf.e[i][a]) * st["f"][i]
        if i > 0:
            sum_f = sum_f + st["f"][i]
            sum_s = sum_s + st["s"][i]
    rho = C["rho"]
    u = [(j[a] / cs2 + 0.5 * C["F_tot"][a]) / rho for a in range(grid.dim)]
    kappa = _kappa(P)
    q_prev = st["q_prev"]
    p = sum_f + 0.5 * (cs2 * _dot(u, C["grad_rho"]) + rho * cs2 * q_prev * kappa)
    dphi_dt = phi - st["phi_prev"]
    T = sum_s - 0.5 * (P.L / P.Cp) * (dphi_dt + _dot(u, C["grad"]) + phi * q_prev * kappa)
    out = dict(C)
    out.update(phi=phi, u=u, p=p, T=T)
    return out


# ----------------------------------------------------------------------------
# equilibria and sources (Sec. 3.1-3.3)
# ----------------------------------------------------------------------------

def _normal(grad, eps):
    """Eq. NormalVector with the regularised norm max(|grad phi|, eps), written
    as sqrt(max(|grad phi|^2, eps^2)) so reverse mode stays finite at 0."""
    sq = sum(g * g for g in grad)
    denom = torch.sqrt(torch.clamp(sq, min=eps * eps))
    return [g / denom for g in grad]


def equilibria_and_sources(phi, phi_prev, u, p, T, q, C, P, grid):
    """Per set, the unbarred equilibria eq_i, the sources S_i of Eq. LBE
    (evaluated with production term q) and the relaxation time."""
    Lf, Lg, _ = lattices_for(grid.dim)
    kappa = _kappa(P)
    rho = C["rho"]
    n = _normal(C["grad"], P.normal_eps)
    usq = _dot(u, u)

    # phase field, Eqs. Geq_Allen-Cahn_Eq and SourceTerm_AllenCahn
    Gg = gamma(Lg, u)
    interface = (4.0 / P.W) * phi * (1.0 - phi)
    g_eq, g_F, g_P = [], [], []
    for i in range(Lg.Q):
        en = sum(float(Lg.e[i][a]) * n[a] for a in range(grid.dim))
        g_eq.append(phi * Gg[i])
        g_F.append(interface * Lg.wf(i) * en)
        g_P.append(Lg.wf(i) * q)
    tau_g = P.M_phi / float(Lg.cs2)

    # flow, Eqs. Feq_NS_Incompr, Forcing, MicroProduction
    cs2 = float(Lf.cs2)
    Gf = gamma(Lf, u)
    nu = viscosity(phi, P)
    f_eq, f_S = [], []
    for i in range(Lf.Q):
        w = Lf.wf(i)
        cu = sum(float(Lf.e[i][a]) * u[a] for a in range(grid.dim))
        f_eq.append(w * (p + rho * cs2 * (cu / cs2 + cu * cu / (2.0 * cs2 * cs2) - usq / (2.0 * cs2))))
        F = torch.zeros_like(phi)
        for a in range(grid.dim):
            F = F + (float(Lf.e[i][a]) - u[a]) * ((Gf[i] - w) * C["grad_rho"][a] * cs2 + Gf[i] * C["F_tot"][a])
        Pf = w * rho * cs2 * q * kappa
        f_S.append(F + Pf)
    tau_f = nu / cs2

    # temperature, Eqs. Seq_Temp and Def_SourceTerms_Temp (sign reading)
    D = (phi - phi_prev) + _dot(u, C["grad"]) + phi * q * kappa
    s_eq, s_S = [], []
    for i in range(Lf.Q):
        s_eq.append(T * Gf[i])
        s_S.append(-Lf.wf(i) * (P.L / P.Cp) * D)
    tau_s = diffusivity(phi, P) / cs2

    return dict(g=(g_eq, g_F, g_P, tau_g, n), f=(f_eq, f_S, tau_f), s=(s_eq, s_S, tau_s))


def _relax(pop, eq_bar, S, tau):
    """Eq. LBE: theta* = theta - (theta - theta_eq_bar)/(tau + 1/2) + S."""
    return pop - (pop - eq_bar) / (tau + 0.5) + S


def _relax_trt(pops, eq_bar, S, tau, magic, lat, transport_odd):
    """Two-relaxation-time collision of one set (the "next" TRT row; not in
    the paper, which uses Eq. LBE).  With the symmetric and antisymmetric
    parts a+_i = (a_i + a_opp(i))/2, a-_i = (a_i - a_opp(i))/2 of the
    populations, of the barred equilibria and of the sources,
        theta*_i = theta_i - w+ (theta+_i - eq_bar+_i) - w- (theta-_i - eq_bar-_i) + S_i,
    which for w+ = w- = 1/(tau + 1/2) is Eq. LBE.  The part that carries the
    set's transport coefficient keeps the BGK rate 1/(tau + 1/2) (the
    symmetric part for the flow, whose viscosity is a second-order moment;
    the antisymmetric part for the phase field and the temperature, whose
    diffusive fluxes are first-order moments); the other rate follows from
    the magic parameter Lambda = (1/w+ - 1/2)(1/w- - 1/2)."""
    tau_other = magic / tau
    tau_p, tau_m = (tau_other, tau) if transport_odd else (tau, tau_other)
    om_p, om_m = 1.0 / (tau_p + 0.5), 1.0 / (tau_m + 0.5)
    out = []
    opp = lat.opposite
    for i in range(lat.Q):
        o = opp[i]
        d_p = 0.5 * ((pops[i] - eq_bar[i]) + (pops[o] - eq_bar[o]))
        d_m = 0.5 * ((pops[i] - eq_bar[i]) - (pops[o] - eq_bar[o]))
        out.append(pops[i] - om_p * d_p - om_m * d_m + S[i])
    return out


def mrt_basis(lat):
    """Orthogonal moment basis of the multiple-relaxation-time collisions,
    built from the lattice vectors (rows: moments, columns: directions; the
    rows are orthogonal under the plain sum over directions).

    D2Q9: rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy with e = 3|c|^2 - 4,
    eps = 4 - 21|c|^2/2 + 9|c|^4/2, q_a = (3|c|^2 - 5) c_a,
    p_xx = c_x^2 - c_y^2, p_xy = c_x c_y.

    D3Q19: rho, e = 19|c|^2 - 30, eps = (21|c|^4 - 53|c|^2 + 24)/2, j_x,
    q_x = (5|c|^2 - 9) c_x, j_y, q_y, j_z, q_z, p_xx = 3c_x^2 - |c|^2,
    pi_xx = (3|c|^2 - 5)(3c_x^2 - |c|^2), p_ww = c_y^2 - c_z^2,
    pi_ww = (3|c|^2 - 5)(c_y^2 - c_z^2), p_xy, p_yz, p_xz,
    m_x = (c_y^2 - c_z^2) c_x, m_y = (c_z^2 - c_x^2) c_y, m_z = (c_x^2 - c_y^2) c_z.

    D3Q7: rho, j_x, j_y, j_z, e = 7|c|^2 - 6, p_xx = 3c_x^2 - |c|^2,
    p_ww = c_y^2 - c_z^2."""
    rows = []
    for i in range(lat.Q):
        c = [float(v) for v in lat.e[i]]
        if lat.name == "D2Q9":
            cx, cy = c
            c2 = cx * cx + cy * cy
            rows.append([1.0, 3.0 * c2 - 4.0, 4.0 - 10.5 * c2 + 4.5 * c2 * c2, cx, (3.0 * c2 - 5.0) * cx,
                         cy, (3.0 * c2 - 5.0) * cy, cx * cx - cy * cy, cx * cy])
        elif lat.name == "D3Q19":
            cx, cy, cz = c
            c2 = cx * cx + cy * cy + cz * cz
            pxx, pww = 3.0 * cx * cx - c2, cy * cy - cz * cz
            rows.append([1.0, 19.0 * c2 - 30.0, (21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0,
                         cx, (5.0 * c2 - 9.0) * cx, cy, (5.0 * c2 - 9.0) * cy, cz, (5.0 * c2 - 9.0) * cz,
                         pxx, (3.0 * c2 - 5.0) * pxx, pww, (3.0 * c2 - 5.0) * pww,
                         cx * cy, cy * cz, cx * cz,
                         (cy * cy - cz * cz) * cx, (cz * cz - cx * cx) * cy, (cx * cx - cy * cy) * cz])
        elif lat.name == "D3Q7":
            cx, cy, cz = c
            c2 = cx * cx + cy * cy + cz * cz
            rows.append([1.0, cx, cy, cz, 7.0 * c2 - 6.0, 3.0 * cx * cx - c2, cy * cy - cz * cz])
        else:
            raise ValueError(f"no moment basis for {lat.name}")
    return torch.tensor(rows, dtype=F64).T          # (moment, direction)


def _relax_moments(pops, eq_bar, S, rates, lat):
    """Collision in the moment space of mrt_basis: with d = theta - eq_bar and
    m = M d, theta*_i = theta_i - (M^-1 diag(s) M d)_i + S_i, where `rates`
    holds one rate s_k per moment (scalars or per-cell tensors) in basis
    order."""
    Mb = mrt_basis(lat)
    d = torch.stack([pops[i] - eq_bar[i] for i in range(lat.Q)])          # (Q, *grid)
    m = torch.tensordot(Mb, d, dims=1)                                    # (Q, *grid)
    norms = (Mb * Mb).sum(dim=1)
    shape = (-1,) + (1,) * (m.dim() - 1)
    s = [r if torch.is_tensor(r) else torch.full_like(m[0], r) for r in rates]
    relaxed = torch.stack([s[k] * m[k] for k in range(len(s))]) / norms.reshape(shape)
    r = torch.tensordot(Mb.T, relaxed, dims=1)                            # M^-1 = M^T diag(1/norms)
    return [pops[i] - r[i] + S[i] for i in range(lat.Q)]


def _relax_mrt(pops, eq_bar, S, tau, rates, lat):
    """Multiple-relaxation-time collision of the flow set (the "next" MRT
    row; not in the paper).  The conserved moment rho and the stress moments
    relax with the BGK rate 1/(tau + 1/2) (the viscosity), e with s_e, the
    fourth-order even moments (eps; in 3D also pi_xx, pi_ww) with s_eps, and
    the odd moments (j, q; in 3D also m) with s_q.  With every rate equal to
    the BGK rate this is Eq. LBE; with s_e = s_eps = 1/(tau + 1/2) every even
    moment relaxes at the BGK rate and every odd one at s_q, which is the TRT
    collision whose antisymmetric rate is s_q."""
    om = 1.0 / (tau + 0.5)
    s_e, s_eps, s_q = rates
    if lat.name == "D2Q9":
        r = [om, s_e, s_eps, s_q, s_q, s_q, s_q, om, om]
    else:   # D3Q19
        r = [om, s_e, s_eps, s_q, s_q, s_q, s_q, s_q, s_q, om, s_eps, om, s_eps, om, om, om, s_q, s_q, s_q]
    return _relax_moments(pops, eq_bar, S, r, lat)


def _relax_mrt_g(pops, eq_bar, S, tau, rates, lat):
    """Multiple-relaxation-time collision of the phase-field set (not in the
    paper): phi and the fluxes j relax with the BGK rate 1/(tau_g + 1/2),
    which carries the mobility M_phi, so the model's transport coefficient
    is that of Eq. LBE; the other moments take s_e (e), s_eps (eps), s_q (q)
    and s_p (the stress moments), a rate of 0 standing for the BGK rate.
    D3Q7 has no eps and no q: e takes s_e, p_xx and p_ww s_p.  With s_q = the
    BGK rate and s_e = s_eps = s_p = w+ this is the TRT collision of g (odd
    moments at the mobility rate, even ones at w+)."""
    om = 1.0 / (tau + 0.5)
    s_e, s_eps, s_q, s_p = [om if r == 0.0 else r for r in rates]
    if lat.name == "D2Q9":
        r = [om, s_e, s_eps, om, s_q, om, s_q, s_p, s_p]
    else:   # D3Q7
        r = [om, om, om, om, s_e, s_p, s_p]
    return _relax_moments(pops, eq_bar, S, r, lat)


def collide(st, M, q, P, grid):
    """Post-collision populations of the three sets at time n."""
    Lf, Lg, _ = lattices_for(grid.dim)
    E = equilibria_and_sources(M["phi"], st["phi_prev"], M["u"], M["p"], M["T"], q, M, P, grid)
    g_eq, g_F, g_P, tau_g, n = E["g"]
    g_bar, g_src = [], []
    for i in range(Lg.Q):
        if P.g_form == "source":
            S = g_F[i] + g_P[i]
            g_bar.append(g_eq[i] - 0.5 * S)
            g_src.append(S)
        else:
            # Eq. Geq_AC-1: phi Gamma_i + M_phi (4/W) phi (1-phi) w_i c_i.n / cs^2
            interface = (4.0 / P.W) * M["phi"] * (1.0 - M["phi"])
            en = sum(float(Lg.e[i][a]) * n[a] for a in range(grid.dim))
            eq_cac = g_eq[i] + P.M_phi * interface * Lg.wf(i) * en / float(Lg.cs2)
            g_bar.append(eq_cac - 0.5 * g_P[i])
            g_src.append(g_P[i])
    f_eq, f_S, tau_f = E["f"]
    f_bar = [f_eq[i] - 0.5 * f_S[i] for i in range(Lf.Q)]
    s_eq, s_S, tau_s = E["s"]
    s_bar = [s_eq[i] - 0.5 * s_S[i] for i in range(Lf.Q)]
    if P.collision == "mrt":
        f_out = _relax_mrt(st["f"], f_bar, f_S, tau_f, P.mrt_rates, Lf)
        g_out = _relax_mrt_g(st["g"], g_bar, g_src, tau_g, P.mrt_rates_g, Lg)
        s_out = [_relax(st["s"][i], s_bar[i], s_S[i], tau_s) for i in range(Lf.Q)]
    elif P.collision == "trt":
        mf, mg, ms = P.trt_magic
        f_out = _relax_trt(st["f"], f_bar, f_S, tau_f, mf, Lf, transport_odd=False)
        g_out = _relax_trt(st["g"], g_bar, g_src, tau_g, mg, Lg, transport_odd=True)
        s_out = _relax_trt(st["s"], s_bar, s_S, tau_s, ms, Lf, transport_odd=True)
    else:
        f_out = [_relax(st["f"][i], f_bar[i], f_S[i], tau_f) for i in range(Lf.Q)]
        g_out = [_relax(st["g"][i], g_bar[i], g_src[i], tau_g) for i in range(Lg.Q)]
        s_out = [_relax(st["s"][i], s_bar[i], s_S[i], tau_s) for i in range(Lf.Q)]
    return torch.stack(f_out), torch.stack(g_out), torch.stack(s_out)


# ----------------------------------------------------------------------------
# streaming (Sec. 3.3 anti bounce-back, Sec. 4.1 half-way bounce-back)
# ----------------------------------------------------------------------------

_LATTICES = {"D2Q9": D2Q9, "D3Q7": D3Q7, "D3Q19": D3Q19}


@lru_cache(maxsize=None)
def _stream_map_cached(lat_name, n, periodic):
    lat = _LATTICES[lat_name]
    dim = len(n)
    shape = tuple(reversed(n))
    idx = np.indices(shape).reshape(dim, -1)        # rows: slowest axis first
    pos = [idx[dim - 1 - a] for a in range(dim)]    # pos[a] = coordinate on axis a
    N = int(np.prod(n))
    own = np.arange(N, dtype=np.int64)
    src = np.empty((lat.Q, N), dtype=np.int64)
    kind = np.empty((lat.Q, N), dtype=np.int8)
    for i in range(lat.Q):
        s = [pos[a] - int(lat.e[i][a]) for a in range(dim)]
        wrapped = np.zeros(N, dtype=bool)
        wall_lo = np.zeros(N, dtype=bool)
        wall_hi = np.zeros(N, dtype=bool)
        for a in range(dim):
            below = s[a] < 0
            above = s[a] >= n[a]
            if periodic[a]:
                wrapped |= below | above
                s[a] = np.mod(s[a], n[a])
            else:
                wall_lo |= below
                wall_hi |= above
        lin = np.zeros(N, dtype=np.int64)
        for a in reversed(range(dim)):
            lin = lin * n[a] + np.clip(s[a], 0, n[a] - 1)
        k = np.full(N, KIND_INTERIOR, dtype=np.int8)
        k[wrapped] = KIND_PERIODIC
        k[wall_lo] = KIND_WALL_LO
        k[wall_hi] = KIND_WALL_HI
        src[i] = np.where(wall_lo | wall_hi, own, lin)
        kind[i] = k
    return src, kind


def stream_map(lat, grid):
    """Pull view of one streaming step: for direction i and destination cell
    x (linear index (z*ny + y)*nx + x), the source cell and the link kind.
    A bounced link's source is x itself (direction opposite(i))."""
    return _stream_map_cached(lat.name, tuple(grid.n), tuple(bool(p) for p in grid.periodic))


@lru_cache(maxsize=None)
def _stream_map_torch(lat_name, n, periodic):
    src, kind = _stream_map_cached(lat_name, n, periodic)
    return torch.from_numpy(src), torch.from_numpy(kind.astype(np.int64))


def stream(post, lat, grid, which, P):
    """Move post-collision populations along e_i.  which = 'f' (half-way
    bounce-back at walls), 'g' or 's' (anti bounce-back with the wall's phi or
    T Dirichlet value: theta_i = -theta*_i' + 2 w_i theta_w)."""
    src_t, kind_t = _stream_map_torch(lat.name, tuple(grid.n), tuple(bool(p) for p in grid.periodic))
    opp = lat.opposite
    Q = lat.Q
    flat = post.reshape(Q, -1)
    wall_vals = {"g": P.phi_wall, "s": P.T_wall}.get(which)
    out = []
    for i in range(Q):
        pulled = flat[i][src_t[i]]
        back = flat[opp[i]]
        if which == "f":
            bounced = back
        else:
            wv = torch.where(kind_t[i] == KIND_WALL_LO,
                             torch.full_like(back, wall_vals[0]),
                             torch.full_like(back, wall_vals[1]))
            bounced = -back + 2.0 * lat.wf(i) * wv
        out.append(torch.where(kind_t[i] <= KIND_PERIODIC, pulled, bounced))
    return torch.stack(out).reshape(post.shape)


# ----------------------------------------------------------------------------
# step, initialisation, outputs
# ----------------------------------------------------------------------------

def step(st, P, grid):
    """One time step n -> n+1; returns the new state dict."""
    Lf, Lg, _ = lattices_for(grid.dim)
    M = moments(st, P, grid)
    q = production_rate(M["phi"], M["T"], P)
    f_post, g_post, s_post = collide(st, M, q, P, grid)
    return dict(
        f=stream(f_post, Lf, grid, "f", P),
        g=stream(g_post, Lg, grid, "g", P),
        s=stream(s_post, Lf, grid, "s", P),
        phi_prev=M["phi"],
        q_prev=q,
    )


def run(st, P, grid, nsteps):
    for _ in range(nsteps):
        st = step(st, P, grid)
    return st


def init_state(phi0, T0, P, grid, u0=None, p0=None):
    """Barred equilibria of the initial fields (reading): theta_bar_i =
    theta_eq_i - S_i/2 with phi_prev = phi_0 and q_prev = q(phi_0, T_0), so
    that `moments` returns phi_0, u_0, p_0 and T_0."""
    phi0 = torch.as_tensor(phi0, dtype=F64)
    T0 = torch.as_tensor(T0, dtype=F64)
    if u0 is None:
        u0 = [torch.zeros_like(phi0) for _ in range(grid.dim)]
    else:
        u0 = [torch.as_tensor(ua, dtype=F64) for ua in u0]
    p0 = torch.zeros_like(phi0) if p0 is None else torch.as_tensor(p0, dtype=F64)
    q = production_rate(phi0, T0, P)
    C = closures(phi0, grid, P)
    E = equilibria_and_sources(phi0, phi0, u0, p0, T0, q, C, P, grid)
    g_eq, g_F, g_P, _, _ = E["g"]
    f_eq, f_S, _ = E["f"]
    s_eq, s_S, _ = E["s"]
    return dict(
        f=torch.stack([f_eq[i] - 0.5 * f_S[i] for i in range(len(f_eq))]),
        g=torch.stack([g_eq[i] - 0.5 * (g_F[i] + g_P[i]) for i in range(len(g_eq))]),
        s=torch.stack([s_eq[i] - 0.5 * s_S[i] for i in range(len(s_eq))]),
        phi_prev=phi0.clone(),
        q_prev=q,
    )


def fields(st, P, grid):
    """phi, u (list per axis), p, T at the state's time."""
    M = moments(st, P, grid)
    return dict(phi=M["phi"], u=M["u"], p=M["p"], T=M["T"])


def reductions(st, P, grid):
    """Global phase-field mass sum(phi) and enthalpy sum(rho (Cp T + phi L))
    (the conserved quantity of Eq. Conservation_Enthalpie with H = Cp T + phi L)."""
    M = moments(st, P, grid)
    mass = float(M["phi"].sum())
    energy = float((M["rho"] * (P.Cp * M["T"] + M["phi"] * P.L)).sum())
    return mass, energy
