"""Pins of the oracle's closed forms against the numbers the paper prints
(tests/golden/paper_values.json, each entry cites where) and against the
mathematics of each solution (boundary/interface conditions, ODEs)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import closed_forms as CF

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_A_integrals_match_printed_closed_forms():
    I, J, G, U = CF.A_integrals()
    s2 = math.sqrt(2.0)
    assert abs(I - 1.0 / (3.0 * s2)) < 1e-10
    assert abs(J - 1.0 / 6.0) < 1e-10
    assert abs(G - (-(12.0 * math.log(2.0) - 10.0) / (72.0 * s2))) < 1e-10
    assert abs(U - math.log(2.0) / s2) < 1e-10
    assert abs(CF.coefficient_A() - 10.0 / 48.0) < 1e-9
    assert abs(10.0 / 48.0 - GOLD["A"]["decimal"]) < 5e-6


def test_stefan_root_equal_diffusivities():
    g = GOLD["stefan_equal_diffusivity"]
    xi = CF.stefan_xi(0.14, 0.14, g["theta_w"], g["theta_inf"], g["theta_I"])
    assert abs(xi - g["xi"]) < 5e-7
    # with alpha_l = alpha_g and theta_I = 0 the root does not depend on alpha
    assert abs(CF.stefan_xi(0.03, 0.03, g["theta_w"], g["theta_inf"]) - xi) < 1e-12


@pytest.mark.parametrize("case", GOLD["stefan_diffusivity_ratios"]["cases"])
def test_stefan_roots_with_ratios(case):
    g = GOLD["stefan_diffusivity_ratios"]
    alpha_l = case["alpha_l"]
    alpha_g = alpha_l / case["ratio"]
    xi = CF.stefan_xi(alpha_l, alpha_g, g["theta_w"], g["theta_inf"], g["theta_I"])
    assert abs(xi - case["xi"]) < 5e-7


def test_printed_rhs_does_not_reproduce_ratio_roots():
    """Why the right-hand side is read with (theta_w - theta_I): taken
    literally as -xi sqrt(pi)/theta_w the first printed root is missed."""
    g = GOLD["stefan_diffusivity_ratios"]
    c = g["cases"][0]
    a_l, a_g = c["alpha_l"], c["alpha_l"] / c["ratio"]
    r = a_l / a_g

    def literal(xi):
        from scipy import special
        return math.exp(-xi * xi) / special.erf(xi) + math.sqrt(a_g / a_l) \
            * (g["theta_I"] - g["theta_inf"]) / (g["theta_I"] - g["theta_w"]) \
            * math.exp(-xi * xi * r) / special.erfc(xi * math.sqrt(r)) \
            + xi * math.sqrt(math.pi) / g["theta_w"]
    from scipy import optimize
    xi_lit = optimize.brentq(literal, 1e-6, 3.0)
    assert abs(xi_lit - c["xi"]) > 1e-2


@pytest.mark.parametrize("a_l,a_g,th_I", [(0.14, 0.14, 0.0), (0.14, 0.014, 0.05), (0.08, 0.04, 0.05)])
def test_stefan_profiles_satisfy_problem(a_l, a_g, th_I):
    """Eqs. Stefan_EqLiq/EqGas, Stefan_CondInterface1/2 (rho = Cp = L = 1,
    conductivities = diffusivities) hold for the closed form with the root."""
    th_w, th_inf = -0.3, 0.3
    xi = CF.stefan_xi(a_l, a_g, th_w, th_inf, th_I)
    t = 5000.0
    xI = CF.stefan_interface(t, xi, a_l)
    f = lambda x, tt=t: CF.stefan_theta(x, tt, xi, a_l, a_g, th_w, th_inf, th_I)
    h = 1e-4
    assert abs(f(0.0) - th_w) < 1e-12
    assert abs(f(xI - 1e-9) - th_I) < 1e-7 and abs(f(xI + 1e-9) - th_I) < 1e-7
    assert abs(f(1e6) - th_inf) < 1e-9
    dxdt = xi * math.sqrt(a_l / t)
    lhs = a_l * ((f(xI - h) - f(xI - 2 * h)) / h) - a_g * ((f(xI + 2 * h) - f(xI + h)) / h)
    assert abs(lhs - dxdt) < 1e-3 * abs(dxdt) + 1e-7
    # heat equation in each phase: d theta/dt = alpha d2 theta/dx2
    for x, a in ((0.5 * xI, a_l), (2.0 * xI, a_g)):
        dtt = (f(x, t + 1.0) - f(x, t - 1.0)) / 2.0
        dxx = (f(x + 0.01) - 2 * f(x) + f(x - 0.01)) / 1e-4
        assert abs(dtt - a * dxx) < 1e-6


def test_layered_poiseuille_closed_form():
    """No slip at y = +-h, continuous velocity and shear stress at y = 0,
    and eta u'' = -G in each layer."""
    h, G, eA, eB = 16.0, 2e-7, 0.1, 0.3
    u = lambda y: CF.layered_poiseuille(y, h, G, eA, eB)
    assert abs(u(-h)) < 1e-18 and abs(u(h)) < 1e-18
    # the literal printed sign of the linear term violates no-slip at y = -h
    s = -1.0
    literal = G * h * h / (2 * eA) * (-s * s - s * (eA - eB) / (eA + eB) + 2 * eA / (eA + eB))
    assert abs(literal) > 1e-6
    e = 1e-6
    assert abs(u(-1e-13) - u(1e-13)) < 1e-16
    sA = eA * (u(0.0) - u(-e)) / e
    sB = eB * (u(e) - u(0.0)) / e
    assert abs(sA - sB) < 1e-5 * abs(sA)
    for y, eta in ((-8.0, eA), (8.0, eB)):
        d2 = (u(y + 0.5) - 2 * u(y) + u(y - 0.5)) / 0.25
        assert abs(eta * d2 + G) < 1e-12
