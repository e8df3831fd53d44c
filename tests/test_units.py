"""The dimensional front end (Sec. 2.1) against Table 1 of the paper, on both sides: the oracle's
restatement and the library's lee_units_from_dimensional (host code, no GPU needed)."""
import json
import math
import os

import pytest

import oracle
from oracle import units

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table1.json")))


@pytest.mark.parametrize("row", GOLD["rows"])
def test_oracle_reproduces_table1(row):
    dim = GOLD["dimensional"]
    r = units.run_length(dim["set"], dim["rho0"], dim["theta0"], GOLD["domain_length"], row["N"], dim["t_end"])
    assert r["T"] == pytest.approx(math.sqrt(21 / 5), rel=1e-15)
    assert r["eps"] == pytest.approx(2.0 / row["N"], rel=1e-15)
    # printed with three significant digits
    assert r["mismatch"] == pytest.approx(row["mismatch"], rel=5e-3)


def test_oracle_scales_invert_the_definitions():
    sc = units.scales("D2Q5_DI", 1.7, 0.9, x_star=2.5)
    s = oracle.velset("D2Q5_DI")
    assert sc["rho_star"] * s.rho0 == pytest.approx(1.7)
    assert sc["theta_star"] * s.theta0 == pytest.approx(0.9)
    assert sc["u_star"] ** 2 == pytest.approx(sc["theta_star"])
    assert sc["x_star"] / sc["t_star"] == pytest.approx(sc["u_star"])


@pytest.mark.parametrize("row", GOLD["rows"])
def test_library_reproduces_table1(row):
    import paper_1601_08103_gb300 as lee

    dim = GOLD["dimensional"]
    r = lee.lee_units_from_dimensional(dim["set"], dim["rho0"], dim["theta0"], dim["x_star"], GOLD["domain_length"],
                                       row["N"], dim["t_end"])
    assert r["t_end"] == pytest.approx(math.sqrt(21 / 5), rel=1e-15)
    assert r["mismatch"] == pytest.approx(row["mismatch"], rel=5e-3)
    o = units.run_length(dim["set"], dim["rho0"], dim["theta0"], GOLD["domain_length"], row["N"], dim["t_end"])
    assert r["steps"] == o["steps"]


def test_library_rejects_bad_units():
    import paper_1601_08103_gb300 as lee

    with pytest.raises(lee.LeeError):
        lee.lee_units_from_dimensional("D3Q7", -1.0, 1.0, 1.0, 2.0, 10, 1.0)
    with pytest.raises(lee.LeeError):
        lee.lee_units_from_dimensional("D3Q7", 1.0, 1.0, 1.0, 2.0, 0, 1.0)


@pytest.mark.parametrize("name", ["D1Q3", "D2Q5", "D2Q5_DI", "D3Q7", "D3Q19", "D3Q7_DI"])
def test_dimensional_speed_of_sound(name):
    """u_star * sqrt(gamma theta0) = sqrt(gamma theta0_dim): the lattice sound speed maps onto the
    dimensional one for any background and any set (Sec. 2.1 scales, Sec. 8 gamma)."""
    import paper_1601_08103_gb300 as lee

    s = oracle.velset(name)
    for rho0_dim, theta0_dim, x_star in [(1.0, 1.0, 1.0), (1.2, 287.0 * 300.0, 3.0), (0.01, 2.5, 0.1)]:
        for sc in (units.scales(name, rho0_dim, theta0_dim, x_star),
                   lee.lee_units_from_dimensional(name, rho0_dim, theta0_dim, x_star, 1.0, 10, 1.0)):
            assert sc["u_star"] * math.sqrt(s.gamma * s.theta0) == pytest.approx(math.sqrt(s.gamma * theta0_dim),
                                                                                 rel=1e-14)
