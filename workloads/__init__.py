"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This module only builds inputs: grids, parameter dictionaries (lattice units,
dx = dt = 1) and initial fields as float64 numpy arrays laid out [z][y][x].
It holds none of the method's arithmetic; the CUDA path and the oracle each
turn a parameter dictionary into their own parameter structure.

Each workload follows the paper's own cases: film boiling (Sec. 5: heated
bottom wall, vapour film under liquid, periodic side walls, sinusoidal or
multi-mode interface perturbation, Eqs. FilmBoiling_InitCond and
FilmBoiling_InitCond-1), the evaporating droplet, the static droplet of the
Laplace test, the layered Poiseuille channel (Sec. 4.1) and the 1D Stefan
problem (Sec. 4.2).  Random numbers come from numpy's PCG64 with the stated
seed.  The interface profile is the kernel function
phi = 1/2 [1 + tanh(2 zeta / W)] (Eq. Kernel-Function), zeta the signed
distance towards the phi = 1 (gas) side.
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    n: tuple                 # (nx, ny) or (nx, ny, nz)
    periodic: tuple          # per axis
    params: dict
    phi0: np.ndarray         # float64, shape reversed(n)
    T0: np.ndarray
    steps: int = 0           # the paper-scale step count of this case
    p0: np.ndarray = None    # initial pressure (None: zero)
    notes: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def cells(self):
        return int(np.prod(self.n))

    @property
    def dim(self):
        return len(self.n)


def base_params(**over):
    """Film-boiling defaults in lattice units: Table tab:FilmBoiling_Parameters
    converted with dx = 1.25e-3, dt = 7.5e-5 (dt/dx^2 = 48) for the
    diffusivities, mobility, width and surface tension; density and viscosity
    ratios are set per workload."""
    p = dict(
        rho_l=10.0, rho_g=1.0,
        nu_l=0.024, nu_g=0.024,
        alpha_l=0.012, alpha_g=0.12,
        sigma=0.0144, W=4.0, M_phi=0.08,
        A=10.0 / 48.0, theta_I=0.0, L=1.0, Cp=1.0, T_sat=1.0,
        gravity=(0.0, -1.0e-5, 0.0), body_force=(0.0, 0.0, 0.0),
        phi_wall=(1.0, 1.0), T_wall=(1.1, 1.0),
        source_on=1, visc_interp=0, alpha_interp=0, normal_eps=1e-3,
    )
    p.update(over)
    return p


def paper_film_params(**over):
    """Table tab:FilmBoiling_Parameters in lattice units (dx = 1.25e-3,
    dt = 7.5e-5): rho_l/rho_g = 1.658, nu_l = 0.144, nu_g = 0.024,
    alpha_l = 0.012, alpha_g = 0.12, sigma = 0.0144, W = 4, M_phi = 0.0816,
    g = 1.8e-5, wall superheat theta_w = Ja = 0.025, L/Cp = 1."""
    p = base_params(rho_l=1.658, rho_g=1.0, nu_l=0.144, nu_g=0.024, alpha_l=0.012,
                    alpha_g=0.12, sigma=0.0144, W=4.0, M_phi=0.0816,
                    gravity=(0.0, -1.8e-5, 0.0), T_wall=(1.025, 1.0))
    p.update(over)
    return p


def _kernel(zeta, W):
    return 0.5 * (1.0 + np.tanh(2.0 * zeta / W))


def _hydrostatic(phi0, params, axis):
    """Pressure whose gradient along the gravity axis balances the buoyancy of
    the light phase: dp/dh = (rho_l - rho_g) g phi, integrated by a midpoint
    cumulative sum from the low wall and shifted to zero at the high wall."""
    g = -params["gravity"][axis]
    d = phi0.ndim - 1 - axis
    c = (params["rho_l"] - params["rho_g"]) * g
    p = c * (np.cumsum(phi0, axis=d) - 0.5 * phi0)
    top = np.take(p, [p.shape[d] - 1], axis=d)
    return np.ascontiguousarray(p - top)


def _film_fields(n, y_interface, params, axis):
    """phi = 1 (vapour) below the interface height, liquid above; T falls
    linearly from the wall superheat to T_sat across the film; p in
    hydrostatic balance with the buoyancy of the vapour."""
    shape = tuple(reversed(n))
    grids = np.meshgrid(*[np.arange(m, dtype=np.float64) + 0.5 for m in reversed(n)], indexing="ij")
    height = grids[len(n) - 1 - axis]                      # distance from the low wall
    yi = np.broadcast_to(y_interface, shape)
    phi0 = _kernel(yi - height, params["W"])
    superheat = params["T_wall"][0] - params["T_sat"]
    T0 = params["T_sat"] + superheat * np.maximum(0.0, 1.0 - height / yi)
    p0 = _hydrostatic(phi0, params, axis)
    return np.ascontiguousarray(phi0), np.ascontiguousarray(T0), p0


def film_boiling_2d(nx=128, ny=256, rho_ratio=10.0, modes=None, seed=0, y0=32.0,
                    amplitude=2.0, paper=False, **over):
    """2D film boiling (Sec. 5.1).  modes=None: one sine of wavelength nx and
    the given amplitude (Eq. FilmBoiling_InitCond); modes=k: k sines of
    wavenumbers 1..k, amplitudes U[1,4] and phases U[0,2 pi) drawn with `seed`
    (Eq. FilmBoiling_InitCond-1).  paper=True takes the paper's Table
    parameters (paper_film_params) instead of rho_ratio and the defaults."""
    params = paper_film_params(**over) if paper else base_params(rho_l=float(rho_ratio), **over)
    x = np.arange(nx, dtype=np.float64) + 0.5
    if modes is None:
        yi = y0 + amplitude * np.sin(2.0 * np.pi * x / nx)
    else:
        rng = np.random.Generator(np.random.PCG64(seed))
        a = rng.uniform(1.0, 4.0, size=modes)
        psi = rng.uniform(0.0, 2.0 * np.pi, size=modes)
        yi = y0 + sum(a[k] * np.sin(2.0 * np.pi * (k + 1) * x / nx + psi[k]) for k in range(modes))
    phi0, T0, p0 = _film_fields((nx, ny), yi[None, :], params, axis=1)
    return Workload(f"film_boiling_2d_{nx}x{ny}", (nx, ny), (True, False), params, phi0, T0,
                    p0=p0)


def film_boiling_3d(nx=256, ny=256, nz=512, rho_ratio=10.0, modes=4, seed=2, z0=32.0,
                    paper=False, **over):
    """3D film boiling: gravity along z, interface
    z_I = z0 + sum_{k,l=1..modes} a_kl sin(2 pi k x/nx + psi_kl) sin(2 pi l y/ny + chi_kl),
    a ~ U[0.5, 2], phases U[0, 2 pi), numpy PCG64(seed)."""
    if paper:
        params = paper_film_params(gravity=(0.0, 0.0, -1.8e-5), **over)
    else:
        params = base_params(rho_l=float(rho_ratio), gravity=(0.0, 0.0, -1.0e-5), **over)
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.uniform(0.5, 2.0, size=(modes, modes))
    psi = rng.uniform(0.0, 2.0 * np.pi, size=(modes, modes))
    chi = rng.uniform(0.0, 2.0 * np.pi, size=(modes, modes))
    x = np.arange(nx, dtype=np.float64) + 0.5
    y = np.arange(ny, dtype=np.float64) + 0.5
    zi = np.full((ny, nx), z0)
    for k in range(modes):
        for l in range(modes):
            zi = zi + a[k, l] * np.sin(2 * np.pi * (k + 1) * x[None, :] / nx + psi[k, l]) \
                * np.sin(2 * np.pi * (l + 1) * y[:, None] / ny + chi[k, l])
    phi0, T0, p0 = _film_fields((nx, ny, nz), zi[None, :, :], params, axis=2)
    return Workload(f"film_boiling_3d_{nx}x{ny}x{nz}", (nx, ny, nz), (True, True, False),
                    params, phi0, T0, p0=p0)


def gaussian_random_field(shape, corr_len, seed):
    """Zero-mean, unit-variance periodic field with a Gaussian spectrum of
    correlation length corr_len cells (numpy FFT of PCG64 white noise)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    white = rng.standard_normal(shape)
    ks = np.meshgrid(*[np.fft.fftfreq(m) * 2.0 * np.pi for m in shape], indexing="ij")
    k2 = sum(k * k for k in ks)
    field_ = np.real(np.fft.ifftn(np.fft.fftn(white) * np.exp(-0.5 * k2 * corr_len ** 2)))
    field_ = field_ - field_.mean()
    return field_ / field_.std()


def droplet_2d(n=512, radius=40.0, seed=3, T_offset=0.02, T_noise=0.005, corr_len=16.0,
               **over):
    """Evaporating droplet in a periodic box, no gravity: a liquid disk
    (phi = 0 inside) of `radius` at the centre, superheated vapour around it;
    T0 = T_sat + T_offset + T_noise * (Gaussian random field, seed)."""
    params = base_params(gravity=(0.0, 0.0, 0.0), **over)
    c = n / 2.0
    yy, xx = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5, indexing="ij")
    d = np.sqrt((xx - c) ** 2 + (yy - c) ** 2)
    phi0 = _kernel(d - radius, params["W"])
    T0 = params["T_sat"] + T_offset + T_noise * gaussian_random_field((n, n), corr_len, seed)
    return Workload(f"droplet_2d_{n}", (n, n), (True, True), params, phi0, T0,
                    extra=dict(radius=radius))


def static_drop_2d(n=64, radius=12.0, sigma=0.01, rho_l=1.0, rho_g=2.0, nu=0.1, M_phi=0.04,
                   W=5.0):
    """Laplace-law case (Sec. 4.1): a drop of phase phi=1 in phase phi=0,
    periodic box, no gravity, no phase change, uniform T."""
    params = base_params(rho_l=rho_l, rho_g=rho_g, nu_l=nu, nu_g=nu, sigma=sigma, W=W,
                         M_phi=M_phi, gravity=(0.0, 0.0, 0.0), source_on=0)
    c = n / 2.0
    yy, xx = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5, indexing="ij")
    d = np.sqrt((xx - c) ** 2 + (yy - c) ** 2)
    phi0 = _kernel(radius - d, W)
    T0 = np.full((n, n), params["T_sat"])
    return Workload(f"static_drop_{n}_R{radius}", (n, n), (True, True), params, phi0, T0,
                    extra=dict(radius=radius, center=c))


def layered_poiseuille(ny=32, nx=2, nu_A=0.1, nu_B=0.3, rho_A=1.0, rho_B=1.0, u_c=5e-5,
                       W=4.0, M_phi=0.1):
    """Layered Poiseuille channel (Sec. 4.1): fluid A (phi = 0) in the lower
    half, fluid B (phi = 1) in the upper half, no-slip walls on y, periodic x,
    driving force G = u_c (eta_A + eta_B) / h^2 along x."""
    h = ny / 2.0
    eta_A, eta_B = rho_A * nu_A, rho_B * nu_B
    G = u_c * (eta_A + eta_B) / h ** 2
    params = base_params(rho_l=rho_A, rho_g=rho_B, nu_l=nu_A, nu_g=nu_B, sigma=0.0, W=W,
                         M_phi=M_phi, gravity=(0.0, 0.0, 0.0), body_force=(G, 0.0, 0.0),
                         source_on=0, phi_wall=(0.0, 1.0), T_wall=(1.0, 1.0))
    y = np.arange(ny, dtype=np.float64) + 0.5
    phi0 = np.broadcast_to(_kernel(y - h, W)[:, None], (ny, nx)).copy()
    T0 = np.full((ny, nx), 1.0)
    return Workload(f"poiseuille_{ny}", (nx, ny), (True, False), params, phi0, T0,
                    extra=dict(h=h, G=G, eta_A=eta_A, eta_B=eta_B))


def stefan_1d(nx=256, ny=1, alpha_l=0.14, alpha_g=0.14, theta_w=-0.3, theta_inf=0.3,
              theta_I=0.0, W=3.0, M_phi=0.08):
    """1D Stefan problem (Sec. 4.2): walls on x, liquid Dirichlet phi=0 and
    theta_w on the left, gas phi=1 and theta_inf on the right, y periodic, no
    flow (equal densities, no surface tension, no gravity), L = Cp = 1."""
    T_sat = 1.0
    params = base_params(rho_l=1.0, rho_g=1.0, nu_l=0.1, nu_g=0.1, alpha_l=alpha_l,
                         alpha_g=alpha_g, sigma=0.0, W=W, M_phi=M_phi, theta_I=theta_I,
                         gravity=(0.0, 0.0, 0.0), phi_wall=(0.0, 1.0),
                         T_wall=(T_sat + theta_w, T_sat + theta_inf), source_on=1, T_sat=T_sat)
    x = np.arange(nx, dtype=np.float64) + 0.5
    phi0 = np.broadcast_to(_kernel(x, W)[None, :], (ny, nx)).copy()
    T0 = np.full((ny, nx), T_sat + theta_inf)
    return Workload(f"stefan_{nx}", (nx, ny), (False, True), params, phi0, T0,
                    extra=dict(theta_w=theta_w, theta_inf=theta_inf))


# the named workloads of the benchmark and the parity tests
def c1_parity(top_phi=0.0):
    """128 x 256 film boiling, density ratio 10, single-mode perturbation of
    amplitude 2 cells, 1000 steps (the FP64 parity case).  The top wall holds
    the liquid value phi = 0 by default: with the printed phi = 1 the liquid
    layer touching that wall turns into vapour in a violent transient that
    amplifies rounding differences (top_phi=1.0 restores the printed value)."""
    w = film_boiling_2d(128, 256, rho_ratio=10.0, modes=None, amplitude=2.0,
                        phi_wall=(1.0, float(top_phi)))
    w.steps = 1000
    return w


def c2_film_boiling(nx=2048, ny=4096, top_phi=0.0):
    """2048 x 4096 film boiling with the paper's Table parameters (density
    ratio 1.658), modes 1..8 with amplitudes U[1,4] cells, seed 1, 20000
    steps.  (Density ratios 10 to 100 are not stable over this horizon with
    the BGK scheme and central differences.)"""
    w = film_boiling_2d(nx, ny, modes=8, seed=1, y0=64.0, paper=True,
                        phi_wall=(1.0, float(top_phi)))
    w.steps = 20000
    return w


def c3_film_boiling_3d(nx=256, ny=256, nz=512, top_phi=0.0):
    """256 x 256 x 512 3D film boiling at density ratio 10 with the other
    film values of the 128 x 256 case (gravity 1e-5 along z), 2D-mode
    interface perturbation (seed 2), 5000 steps; stable over that horizon."""
    w = film_boiling_3d(nx, ny, nz, rho_ratio=10.0, modes=4, seed=2, z0=32.0,
                        phi_wall=(1.0, float(top_phi)))
    w.steps = 5000
    return w


def c4_droplet(n=512):
    w = droplet_2d(n, 40.0 * n / 512.0, seed=3)
    w.steps = 2000
    return w


def c5_film_boiling_3d_large(top_phi=0.0):
    """512 x 512 x 768 3D film boiling, the physics of c3_film_boiling_3d
    (density ratio 10), 2000 steps, FP16 storage in the measurements."""
    w = film_boiling_3d(512, 512, 768, rho_ratio=10.0, modes=4, seed=2, z0=32.0,
                        phi_wall=(1.0, float(top_phi)))
    w.steps = 2000
    return w


# ----------------------------------------------------------------------------
# phase field alone in an imposed velocity field (Sec. 4.1 CAC validations)
# ----------------------------------------------------------------------------

def cac_params(M_phi=2.0e-3, W=6.0, **over):
    """Lattice-unit parameters of the CAC validations: dx = 5e-3, dt = 1e-4,
    so M_phi = 5e-4 dt / dx^2 = 2e-3 and W = 6 dx = 6 cells; no phase change
    and no body force (the flow populations are not stepped)."""
    return base_params(M_phi=M_phi, W=W, source_on=0, gravity=(0.0, 0.0, 0.0),
                       rho_l=1.0, rho_g=1.0, model=1, **over)


def _disk(n, xc, yc, R, width):
    y, x = np.meshgrid(np.arange(n[1], dtype=np.float64), np.arange(n[0], dtype=np.float64),
                       indexing="ij")
    d = np.sqrt((x - xc) ** 2 + (y - yc) ** 2)
    return 0.5 * (1.0 + np.tanh((R - d) / width)), x, y


def zalesak_disk(n=201, u0=0.7853975, dx=5.0e-3, dt=1.0e-4):
    """Sec. 4.1: a disk of radius R = 80 at the centre of an n x n periodic
    box, phi = [1 + tanh((R - d) / (sqrt(2) W0))] / 2 with W0 = 2, slotted
    (phi = 0) for x_c - R/6 <= x <= x_c + R/6, y_c - 1.1 R <= y <= y_c, in the
    rigid rotation u_x = u0 (2y - 1), u_y = u0 (1 - 2x) (x, y in [0, 1]) that
    turns it once in T_f = 4 (4 / dt steps)."""
    c = (n - 1) / 2.0
    R = 80.0 * (n - 1) / 200.0
    phi, x, y = _disk((n, n), c, c, R, np.sqrt(2.0) * 2.0)
    slot = (x >= c - R / 6.0) & (x <= c + R / 6.0) & (y >= c - 1.1 * R) & (y <= c)
    phi[slot] = 0.0
    L = (n - 1) * dx                                  # box length in physical units
    xs, ys = x * dx / L, y * dx / L                   # in [0, 1]
    scale = dt / dx                                   # physical -> lattice velocity
    ux = u0 * (2.0 * ys - 1.0) * scale
    uy = u0 * (1.0 - 2.0 * xs) * scale
    w = Workload(name=f"zalesak_{n}x{n}", n=(n, n), periodic=(True, True),
                 params=cac_params(), phi0=phi, T0=np.ones_like(phi),
                 steps=int(round(4.0 / dt)))
    w.extra.update(u=(ux, uy), period=0.0)
    return w


def vortex_disk(n=201, u0=0.7853975, dx=5.0e-3, dt=1.0e-4, reverse=True):
    """Sec. 4.1: a disk of radius 40 centred at (100, 60) (for n = 201) in the
    vortex u_x = -u0 cos(pi (x - 1/2)) sin(pi (y - 1/2)),
    u_y = u0 sin(pi (x - 1/2)) cos(pi (y - 1/2)); with `reverse` the field is
    multiplied by cos(pi t / (2 T_f)), T_f = 4, so the disk returns at 2 T_f."""
    s = (n - 1) / 200.0
    phi, x, y = _disk((n, n), 100.0 * s, 60.0 * s, 40.0 * s, np.sqrt(2.0) * 2.0)
    L = (n - 1) * dx
    xs, ys = x * dx / L, y * dx / L
    scale = dt / dx
    ux = -u0 * np.cos(np.pi * (xs - 0.5)) * np.sin(np.pi * (ys - 0.5)) * scale
    uy = u0 * np.sin(np.pi * (xs - 0.5)) * np.cos(np.pi * (ys - 0.5)) * scale
    Tf = int(round(4.0 / dt))
    w = Workload(name=f"vortex_{n}x{n}", n=(n, n), periodic=(True, True),
                 params=cac_params(), phi0=phi, T0=np.ones_like(phi),
                 steps=2 * Tf if reverse else Tf)
    w.extra.update(u=(ux, uy), period=float(2 * Tf) if reverse else 0.0)
    return w
