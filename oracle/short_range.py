"""Analytic flexible-water stand-in for V_short (test infrastructure only).

The paper's charge-independent short-range term is a trained HIP-NN model
(Sec. 4).  Its dataset and weights are out of scope, so the MD workloads use
a plain flexible-water potential instead.  This is a builder's choice, not
fixed by the paper (parity unpinned by the paper; pinned here by finite
differences).  Atoms are ordered O, H, H per molecule.

  E_bond  = 1/2 k_b (|r_OH| - r_0)^2                     per O-H bond
  E_angle = 1/2 k_theta (theta_HOH - theta_0)^2           per molecule
  E_LJ    = 4 eps [(s / r)^12 - (s / r)^6]                per O-O pair (all images),
                                                          truncated at r_cut
r_0 = 0.9572 A and theta_0 = 104.52 deg are the workload geometry.  k_b,
k_theta, eps and s are the SPC/Fw values (Wu, Tepper & Voth, J. Chem. Phys.
124, 024503 (2006)) converted from kcal/mol: k_b = 1059.162, k_theta = 75.90,
eps = 0.1554, s = 3.165492 A.
"""

from __future__ import annotations

import math

import numpy as np

KCAL_TO_EV = 0.0433641
K_BOND = 1059.162 * KCAL_TO_EV  # eV / A^2
R0_BOND = 0.9572  # A
K_ANGLE = 75.90 * KCAL_TO_EV  # eV / rad^2
THETA0 = math.radians(104.52)
LJ_EPS = 0.1554 * KCAL_TO_EV  # eV
LJ_SIGMA = 3.165492  # A


def _min_image(d, box):
    return d - box * np.round(d / box)


def water_short_range(R, box, r_cut):
    """Energy and forces (N, 3) of the flexible-water terms."""
    R = np.asarray(R, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    n = R.shape[0]
    if n % 3:
        raise ValueError("water ordering needs 3 atoms per molecule")
    F = np.zeros_like(R)
    O, H1, H2 = R[0::3], R[1::3], R[2::3]
    a = _min_image(H1 - O, box)
    b = _min_image(H2 - O, box)
    ra = np.linalg.norm(a, axis=1)
    rb = np.linalg.norm(b, axis=1)
    # bonds
    e = 0.5 * K_BOND * np.sum((ra - R0_BOND) ** 2 + (rb - R0_BOND) ** 2)
    fa = -K_BOND * (ra - R0_BOND)[:, None] * a / ra[:, None]  # on H1
    fb = -K_BOND * (rb - R0_BOND)[:, None] * b / rb[:, None]  # on H2
    F[1::3] += fa
    F[2::3] += fb
    F[0::3] -= fa + fb
    # angle
    cos_t = np.sum(a * b, axis=1) / (ra * rb)
    cos_t = np.clip(cos_t, -1.0, 1.0)
    theta = np.arccos(cos_t)
    e += 0.5 * K_ANGLE * np.sum((theta - THETA0) ** 2)
    sin_t = np.sqrt(np.maximum(1.0 - cos_t * cos_t, 1e-300))
    pref = (K_ANGLE * (theta - THETA0) / sin_t)[:, None]
    dcos_da = b / (ra * rb)[:, None] - cos_t[:, None] * a / (ra * ra)[:, None]
    dcos_db = a / (ra * rb)[:, None] - cos_t[:, None] * b / (rb * rb)[:, None]
    ga = pref * dcos_da  # -dE/da = k (theta - theta0) / sin(theta) dcos/da
    gb = pref * dcos_db
    F[1::3] += ga
    F[2::3] += gb
    F[0::3] -= ga + gb
    # O-O Lennard-Jones over all images within r_cut (brute force)
    m = O.shape[0]
    smax = [int(math.ceil(r_cut / L)) + 1 for L in box]
    shifts = np.array([(i, j, k) for i in range(-smax[0], smax[0] + 1)
                       for j in range(-smax[1], smax[1] + 1)
                       for k in range(-smax[2], smax[2] + 1)], dtype=np.float64) * box
    rc2 = r_cut * r_cut
    s6 = LJ_SIGMA ** 6
    e_lj = 0.0
    FO = np.zeros((m, 3))
    for i in range(m):
        d0 = _min_image(O - O[i], box)  # (m, 3)
        d = d0[:, None, :] + shifts[None, :, :]  # (m, S, 3)
        r2 = np.sum(d * d, axis=2)
        mask = r2 < rc2
        mask[i, np.all(shifts == 0, axis=1)] = False
        r2m = r2[mask]
        inv6 = s6 / r2m ** 3
        e_lj += 0.5 * np.sum(4.0 * LJ_EPS * (inv6 * inv6 - inv6))
        # F_i = sum_j dE/dr * d / r with dE/dr = 4 eps (-12 s^12 / r^13 + 6 s^6 / r^7)
        g = 4.0 * LJ_EPS * (-12.0 * inv6 * inv6 + 6.0 * inv6) / r2m
        FO[i] = np.sum(g[:, None] * d[mask], axis=0)
    F[0::3] += FO
    return float(e + e_lj), F
