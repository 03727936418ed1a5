"""Closed forms and constants the paper states (test infrastructure only).

* Stefan problem, Sec. 4.2: interface position (Eq. SolStefan_Position),
  temperature profiles (Eqs. SolStefan_Temp_Liq, SolStefan_Temp_Gas) and the
  transcendental equation for xi (Eq. SolStefan_TranscendEq).  The equation is
  solved with its right-hand side read as -xi sqrt(pi) / (theta_w - theta_I):
  this reduces to the printed -xi sqrt(pi) / theta_w when theta_I = 0 and is
  the form that reproduces the three roots the paper prints for theta_I = 0.05.
* Layered Poiseuille flow, Sec. 4.1 (Eq. AnalyticalSol_Poiseuille-1).  As
  printed, the linear term -(y/h)(eta_A-eta_B)/(eta_A+eta_B) gives non-zero
  velocity at y = -h; the printed expressions satisfy no-slip, continuity of
  velocity and of shear stress only after y -> -y.  The oracle keeps fluid A
  on -h <= y <= 0 and uses +(y/h)(eta_A-eta_B)/(eta_A+eta_B).
* Laplace law, Sec. 4.1 (Eq. LaplaceLaw): p_in - p_out = sigma / R in 2D.
* Coefficient A of Eq. ProductionRate from the four integrals of App. B
  (Eqs. Def_A, Def_Integrals, OurFunctions), evaluated by quadrature.
(The film-boiling characteristic numbers of Sec. 5.1 belong to the package's
unit conversion, which tests them against the printed values.)
"""
import math

import numpy as np
from scipy import integrate, optimize, special


# ----------------------------------------------------------------------------
# Stefan problem
# ----------------------------------------------------------------------------

def stefan_residual(xi, alpha_l, alpha_g, theta_w, theta_inf, theta_I):
    r = alpha_l / alpha_g
    lhs = math.exp(-xi * xi) / special.erf(xi) \
        + math.sqrt(alpha_g / alpha_l) * (theta_I - theta_inf) / (theta_I - theta_w) \
        * math.exp(-xi * xi * r) / special.erfc(xi * math.sqrt(r))
    rhs = -xi * math.sqrt(math.pi) / (theta_w - theta_I)
    return lhs - rhs


def stefan_xi(alpha_l, alpha_g, theta_w, theta_inf, theta_I=0.0):
    """Root xi of the transcendental equation (bracketed on (1e-6, 3))."""
    f = lambda x: stefan_residual(x, alpha_l, alpha_g, theta_w, theta_inf, theta_I)
    return optimize.brentq(f, 1e-6, 3.0, xtol=1e-14, rtol=1e-14)


def stefan_interface(t, xi, alpha_l):
    """x_I(t) = 2 xi sqrt(alpha_l t)."""
    return 2.0 * xi * np.sqrt(alpha_l * t)


def stefan_theta(x, t, xi, alpha_l, alpha_g, theta_w, theta_inf, theta_I=0.0):
    """theta(x, t): liquid profile for x < x_I, gas profile beyond."""
    x = np.asarray(x, dtype=np.float64)
    xI = stefan_interface(t, xi, alpha_l)
    liq = theta_w + (theta_I - theta_w) * special.erf(x / (2.0 * np.sqrt(alpha_l * t))) / special.erf(xi)
    gas = theta_inf + (theta_I - theta_inf) * special.erfc(x / (2.0 * np.sqrt(alpha_g * t))) \
        / special.erfc(xi * np.sqrt(alpha_l / alpha_g))
    return np.where(x < xI, liq, gas)


# ----------------------------------------------------------------------------
# layered Poiseuille flow
# ----------------------------------------------------------------------------

def layered_poiseuille(y, h, G, eta_A, eta_B):
    """u_x(y) for -h <= y <= h, fluid A below y = 0 and fluid B above
    (sign of the linear term per the module docstring)."""
    y = np.asarray(y, dtype=np.float64)
    s = y / h
    ratio = (eta_A - eta_B) / (eta_A + eta_B)
    lower = G * h * h / (2.0 * eta_A) * (-s * s + s * ratio + 2.0 * eta_A / (eta_A + eta_B))
    upper = G * h * h / (2.0 * eta_B) * (-s * s + s * ratio + 2.0 * eta_B / (eta_A + eta_B))
    return np.where(y <= 0.0, lower, upper)


# ----------------------------------------------------------------------------
# Laplace law
# ----------------------------------------------------------------------------

def laplace_pressure_jump(sigma, R):
    """2D Laplace law: p_in - p_out = sigma / R."""
    return sigma / R


# ----------------------------------------------------------------------------
# coefficient A (App. B)
# ----------------------------------------------------------------------------

def A_integrals(W=2.0 * math.sqrt(2.0), span=60.0):
    """The integrals I, J, G, U of Eq. Def_Integrals with phi_0, p_phi^0, h^0
    of Eq. OurFunctions, by adaptive quadrature."""
    phi0 = lambda z: 0.5 * (1.0 + math.tanh(2.0 * z / W))
    dphi0 = lambda z: (1.0 / W) / math.cosh(2.0 * z / W) ** 2
    p_phi = lambda z: phi0(z) * (1.0 - phi0(z))
    inner = lambda z: integrate.quad(phi0, 0.0, z, epsabs=1e-14, epsrel=1e-13)[0]
    kw = dict(epsabs=1e-14, epsrel=1e-12, limit=400)
    I = integrate.quad(lambda z: dphi0(z) ** 2, -span, span, **kw)[0]
    J = integrate.quad(lambda z: dphi0(z) * p_phi(z), -span, span, **kw)[0]
    G = integrate.quad(lambda z: dphi0(z) * p_phi(z) * inner(z), -span, span, **kw)[0]
    U = integrate.quad(phi0, -span, 0.0, **kw)[0]
    return I, J, G, U


def coefficient_A(W=2.0 * math.sqrt(2.0)):
    """Eq. Def_A: A = (G + J U) / (2 I)."""
    I, J, G, U = A_integrals(W)
    return (G + J * U) / (2.0 * I)
