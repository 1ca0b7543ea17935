"""Physical units of the graphene runs, pinned to the numbers printed in Part II
("Model and Methods", "Results"): nu = 0.000132 hbar c^2 / eV from eta, n and m* = m_e;
nu = 11.8 hbar v_F^2 / eV; flow speed 1e5 m/s = 0.1 v_F; Re = 6.37 for one impurity of
diameter 0.5 um and 12.74 for two; a 1024 x 256 lattice at 0.038 um spans the 40 um x
10 um sample."""
import math

import pytest

from paper_2205_04658_gb300 import units as U


def test_kinematic_viscosity_matches_the_printed_values():
    assert U.kinematic_viscosity_natural() == pytest.approx(0.000132, rel=5e-3)
    assert U.kinematic_viscosity_vf() == pytest.approx(11.8, rel=1e-2)


def test_reynolds_numbers_of_one_and_two_impurities():
    assert U.reynolds(0.5e-6, 0.1) == pytest.approx(6.37, rel=5e-3)
    assert U.reynolds(2 * 0.5e-6, 0.1) == pytest.approx(12.74, rel=5e-3)


def test_reynolds_scales_linearly_and_inversely():
    base = U.reynolds(0.5e-6, 0.1)
    assert U.reynolds(1.5e-6, 0.1) == pytest.approx(3 * base, rel=1e-14)
    assert U.reynolds(0.5e-6, 0.2) == pytest.approx(2 * base, rel=1e-14)
    nu = U.kinematic_viscosity_vf()
    assert U.reynolds(0.5e-6, 0.1, nu_vf=2 * nu) == pytest.approx(base / 2, rel=1e-14)


def test_lattice_units_of_the_graphene_sample():
    lu = U.LatticeUnits(0.038e-6, courant=0.5)
    assert 1024 * lu.spacing_m == pytest.approx(38.9e-6, rel=1e-3)   # ~40 um long
    assert 256 * lu.spacing_m == pytest.approx(9.73e-6, rel=1e-3)    # ~10 um wide
    assert lu.velocity_lattice(1e5) == pytest.approx(0.1, rel=1e-14)  # 1e5 m/s = 0.1 v_F
    assert lu.velocity_m_s(0.1) == pytest.approx(1e5, rel=1e-14)
    assert lu.step_seconds() == pytest.approx(0.5 * 0.038e-6 / 1e6, rel=1e-14)
    d = lu.diameter_nodes(0.5e-6)  # 13.2 nodes -> 13
    assert d == 13 and d % 2 == 1


def test_natural_length_unit():
    # hbar v_F / eV with v_F = 1e6 m/s is 0.658 nm
    assert U.length_unit_m() == pytest.approx(6.582119569e-10, rel=1e-12)
    assert U.to_natural_length(U.length_unit_m()) == pytest.approx(1.0, rel=1e-15)
    assert math.isclose(U.kinematic_viscosity_vf(v_f=U.C_M_S), U.kinematic_viscosity_natural(), rel_tol=1e-14)


def test_eta_over_s_for_reynolds_round_trip():
    """eta/s from Re, then Re = L U / nu back with nu = (eta/s) / T."""
    es = U.eta_over_s_for_reynolds(6.37, 13, 0.1)
    nu = es / U.temperature_lattice(1.0)
    assert 13 * 0.1 * 0.1 / nu == pytest.approx(6.37, rel=1e-14)
    assert U.temperature_lattice(1.0) == pytest.approx((math.pi ** 2 / 3) ** 0.25, rel=1e-15)
