"""The package's physical -> lattice conversion against the lattice values of
Table tab:FilmBoiling_Parameters (dx = 1.25e-3, dt = 7.5e-5) and the derived
numbers printed in Sec. 5.1."""
import json
import os

from paper_2003_06342_b300 import units

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_lattice_conversion():
    ph = GOLD["film_boiling"]["physical"]
    lat = units.to_lattice(ph, ph["dx"], ph["dt"])
    assert abs(lat["nu_l"] - 0.144) < 1e-12 and abs(lat["nu_g"] - 0.024) < 1e-12
    assert abs(lat["alpha_l"] - 0.012) < 1e-12 and abs(lat["alpha_g"] - 0.12) < 1e-12
    assert abs(lat["M_phi"] - 0.0816) < 1e-12
    assert abs(lat["W"] - 4.0) < 1e-12
    assert abs(lat["g_y"] - 1.8e-5) < 1e-15
    assert abs(lat["sigma"] - 0.0144) < 1e-12


def test_characteristic_numbers():
    fb = GOLD["film_boiling"]
    ph = fb["physical"]
    n = units.film_boiling_numbers(ph["rho_l"], ph["rho_g"], ph["nu_g"], ph["alpha_g"], ph["sigma"],
                                   ph["g_y"], 1.0, 1.0, 1.0 + ph["theta_w"], 1.0)
    assert abs(n["lambda_s"] - fb["lambda_s"]) / fb["lambda_s"] < 2e-4
    assert abs(n["Pr"] - 0.2) < 1e-12 and abs(n["Ja"] - 0.025) < 1e-12
    assert abs(n["t_s"] - fb["t_s"]) < 5e-5
