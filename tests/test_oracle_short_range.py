"""Pins of the flexible-water stand-in for V_short (CPU; builder's choice, not the paper's)."""

import math

import numpy as np

from oracle import short_range as sr
from workloads import water_box


def test_equilibrium_geometry_has_zero_intramolecular_energy():
    """A rigid workload molecule sits at r_0 and theta_0, so bonds and the angle cost nothing."""
    w = water_box(1, seed=3)
    w.box[:] = 40.0  # one molecule: no O-O pair inside r_cut
    e, F = sr.water_short_range(w.R, w.box, 8.0)
    assert abs(e) < 1e-20
    assert np.abs(F).max() < 1e-12


def test_forces_are_minus_gradient():
    w = water_box(27, seed=8)
    rng = np.random.default_rng(1)
    R = w.R + rng.normal(scale=0.05, size=w.R.shape)
    e0, F = sr.water_short_range(R, w.box, 6.0)
    h = 1e-6
    for i in (0, 1, 2, 30, 50):
        for d in range(3):
            Rp = R.copy(); Rp[i, d] += h
            Rm = R.copy(); Rm[i, d] -= h
            fd = -(sr.water_short_range(Rp, w.box, 6.0)[0] - sr.water_short_range(Rm, w.box, 6.0)[0]) / (2 * h)
            assert abs(fd - F[i, d]) < 1e-6 * max(1.0, abs(fd))
    assert np.abs(F.sum(axis=0)).max() < 1e-10  # momentum conservation


def test_lj_pair_closed_form():
    """Two O atoms (with their H far away in a huge box): E = 4 eps [(s/r)^12 - (s/r)^6]."""
    r = 3.4
    R = np.array([[10.0, 10.0, 10.0], [10.0, 10.9572, 10.0], [10.0, 10.0, 10.9572],
                  [10.0 + r, 10.0, 10.0], [10.0 + r, 10.9572, 10.0], [10.0 + r, 10.0, 10.9572]])
    box = np.array([80.0, 80.0, 80.0])
    e, F = sr.water_short_range(R, box, 9.0)
    # the molecules are bent at 90 deg instead of theta_0: subtract that part exactly
    e_angle = 2 * 0.5 * sr.K_ANGLE * (math.pi / 2 - sr.THETA0) ** 2
    x6 = (sr.LJ_SIGMA / r) ** 6
    assert abs((e - e_angle) - 4 * sr.LJ_EPS * (x6 * x6 - x6)) < 1e-12
