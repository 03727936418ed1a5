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
                                   ph["g_y"], 1.0, ph["L_over_Cp"], 1.0 + ph["theta_w"], 1.0)
    # printed truncated to four significant figures (lambda_s = 0.0435855
    # appears as 4.358e-2, lambda_c = 0.273856 as 0.2738)
    assert abs(n["lambda_s"] - fb["lambda_s"]) / fb["lambda_s"] < 2e-4
    assert abs(n["lambda_c"] - fb["lambda_c"]) / fb["lambda_c"] < 5e-4
    assert abs(n["Pr"] - fb["Pr"]) < 1e-12 and abs(n["Pr"] - 0.2) < 1e-12
    assert abs(n["Ja"] - fb["Ja"]) < 1e-12 and abs(n["Ja"] - 0.025) < 1e-12
    assert abs(n["t_s"] - fb["t_s"]) < 5e-5
    # the paper's Gr follows from its rounded lambda_s = 4.358e-2
    Gr_rounded = ph["rho_g"] * ph["g_y"] * (ph["rho_l"] - ph["rho_g"]) * fb["lambda_s"] ** 3 \
        / (ph["rho_g"] ** 2 * ph["nu_g"] ** 2)
    assert abs(Gr_rounded - fb["Gr"]) / fb["Gr"] < 1e-4
    assert abs(n["Gr"] - fb["Gr"]) / fb["Gr"] < 1e-3
