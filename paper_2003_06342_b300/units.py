"""Conversion of the paper's physical parameters to lattice units.

With space step dx and time step dt (Sec. 5.1): kinematic viscosity,
diffusivity and mobility scale as dt/dx^2, the interface width as 1/dx,
gravity as dt^2/dx, and the surface tension (per unit density) as
dt^2/dx^3; densities and temperatures are unchanged.  Also the
characteristic numbers of the film-boiling problem (Eq. Critical_wavelength
and the Grashof, Prandtl and Jacob numbers of Sec. 5.1).
"""
import math


def to_lattice(phys, dx, dt):
    """phys: dict with rho_l, rho_g, nu_l, nu_g, alpha_l, alpha_g, sigma,
    M_phi, W, g_y (physical units).  Returns the lattice-unit dict."""
    diff = dt / (dx * dx)
    return dict(
        rho_l=phys["rho_l"], rho_g=phys["rho_g"],
        nu_l=phys["nu_l"] * diff, nu_g=phys["nu_g"] * diff,
        alpha_l=phys["alpha_l"] * diff, alpha_g=phys["alpha_g"] * diff,
        M_phi=phys["M_phi"] * diff,
        W=phys["W"] / dx,
        sigma=phys["sigma"] * dt * dt / dx ** 3,
        g_y=phys["g_y"] * dt * dt / dx,
    )


def film_boiling_numbers(rho_l, rho_g, nu_g, alpha_g, sigma, g_y, Cp, L, T_w, T_sat):
    """lambda_s, lambda_c, Gr, Pr, Ja and the time scale t_s = sqrt(lambda_s/g)."""
    lam_s = math.sqrt(sigma / ((rho_l - rho_g) * g_y))
    return dict(lambda_s=lam_s, lambda_c=2.0 * math.pi * lam_s,
                Gr=rho_g * g_y * (rho_l - rho_g) * lam_s ** 3 / (rho_g * rho_g * nu_g * nu_g),
                Pr=nu_g / alpha_g, Ja=Cp * (T_w - T_sat) / L,
                t_s=math.sqrt(lam_s / g_y))
