"""Pins of the oracle's constants, equation of state and reference state (not GPU)."""
import numpy as np
import pytest

from golden_io import read, values
from oracle.reference import GRAV, pressure, reference_profile, sound_speed


def _golden(key):
    for row in read("paper_constants.txt"):
        if row[0] == key:
            return values(row[1:])
    raise KeyError(key)


def test_sound_speed_matches_paper():
    ref = reference_profile(np.array([0.0]), 300.0)
    a = sound_speed(ref["P0"], ref["rho0"])[0]
    assert abs(a - _golden("sound_speed_300K")[0]) < 0.01


@pytest.mark.parametrize("n_bv", [0.0, 0.01, 0.02])
def test_hydrostatic_balance_and_eos(n_bv):
    z = np.linspace(0.0, 15e3, 31)
    h = 0.5
    r = reference_profile(z, 300.0, n_bv)
    rp, rm = reference_profile(z + h, 300.0, n_bv), reference_profile(z - h, 300.0, n_bv)
    dPdz = (rp["P0"] - rm["P0"]) / (2 * h)
    np.testing.assert_allclose(dPdz, -r["rho0"] * GRAV, rtol=1e-7)
    np.testing.assert_allclose(pressure(r["rho0"], r["theta0"]), r["P0"], rtol=1e-13)
    if n_bv > 0:
        dlnth = (np.log(rp["theta0"]) - np.log(rm["theta0"])) / (2 * h)
        np.testing.assert_allclose(GRAV * dlnth, n_bv ** 2, rtol=1e-6)
