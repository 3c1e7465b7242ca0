"""Accuracy-driven Ewald parameters (Sec. 3.2, Sec. 3.3: the OpenMM heuristics), CPU only.

qeq_params_from_tolerance is host code of the library.  Its values are checked
against the rule's definition, and the force error it buys is measured with
the oracle: smooth PME at the chosen alpha and mesh against an exact Ewald sum
(converged k-sum, real space to erfc(alpha r) < 1e-8 over all images).  With
the rule's fifth-order splines the relative RMS force error stays at or below
delta.
"""

import math

import numpy as np
import pytest

import paper_2503_21176_gb300 as qg
from oracle import ewald
from workloads import random_neutral_charges, water_box


def _smooth(k):
    for f in (2, 3, 5, 7):
        while k % f == 0:
            k //= f
    return k == 1


def _params(box, r_cut, order):
    p = qg.qeq_params_default()
    for d in range(3):
        p.box[d] = float(box[d])
    p.r_cut = float(r_cut)
    p.order = int(order)
    return p


@pytest.mark.parametrize("delta", [1e-3, 5e-4, 1e-4, 1e-5, 1e-6])
def test_rule_values(delta):
    box = (14.4, 17.0, 31.1)
    p = qg.qeq_params_from_tolerance(_params(box, 6.0, 5), delta)
    alpha = math.sqrt(-math.log(2 * delta)) / 6.0
    assert abs(p.alpha - alpha) < 1e-15 * alpha
    # the reciprocal Gaussian at k_cut is 2 delta, and erfc(alpha r_c) is about 2 delta
    assert abs(math.exp(-p.k_cut ** 2 / (4 * alpha ** 2)) - 2 * delta) < 1e-12 * delta
    for d in range(3):
        bound = max(5, math.ceil(2 * alpha * box[d] / (3 * delta ** 0.2)))
        K = p.mesh[d]
        assert K >= bound and _smooth(K)
        assert not any(_smooth(k) for k in range(bound, K))  # the smallest such size


def test_rule_rejects_bad_input():
    with pytest.raises(qg.QeqError):
        qg.qeq_params_from_tolerance(_params((10, 10, 10), 5.0, 5), 0.0)
    with pytest.raises(qg.QeqError):
        qg.qeq_params_from_tolerance(_params((10, 10, 10), 0.0, 5), 1e-4)
    with pytest.raises(qg.QeqError):  # a mesh above 4096 points per axis
        qg.qeq_params_from_tolerance(_params((1e5, 10, 10), 5.0, 5), 1e-6)


@pytest.fixture(scope="module")
def exact():
    w = water_box(100, seed=5)  # 300 atoms, L 14.4 A
    q = random_neutral_charges(w.n_atoms, seed=3, scale=0.4)
    sig = np.zeros(w.n_atoms)
    a_ref = 0.45  # erfc(a_ref 9 A) = 1.4e-8; exp(-k_cut^2 / 4 a^2) = 1e-16
    ref = ewald.coulomb_apply(w.R, q, sig, w.box, a_ref, 9.0, recip="ewald",
                              k_cut=2 * a_ref * math.sqrt(-math.log(1e-16)), real_method="brute")
    return w, q, sig, ref


@pytest.mark.parametrize("order", [5, 6])
@pytest.mark.parametrize("r_cut", [5.0, 6.0])
def test_measured_force_error_within_delta(exact, order, r_cut):
    w, q, sig, ref = exact
    rms_ref = np.sqrt(np.mean(ref["F"] ** 2))
    errs = []
    for delta in (1e-3, 1e-4, 1e-5):
        p = qg.qeq_params_from_tolerance(_params(w.box, r_cut, order), delta)
        o = ewald.coulomb_apply(w.R, q, sig, w.box, p.alpha, r_cut, recip="pme",
                                mesh=tuple(p.mesh), order=order)
        err = np.sqrt(np.mean((o["F"] - ref["F"]) ** 2)) / rms_ref
        assert err <= 1.1 * delta, f"delta {delta}: relative RMS force error {err:.3e}"
        errs.append(err)
    assert errs[0] > errs[1] > errs[2]
