"""The FP64 real-space kernel's piecewise pair functions, evaluated on the host
exactly as the kernel evaluates them (CPU; no device), against erfc and exp.

F(s) = erfc(alpha sqrt s) / sqrt s is the screened Coulomb pair term of Eq.
ewald_real, G(s) = (dF/dr) / r its field coefficient; the Gaussian-charge
correction erfc(r / gamma) / r is F at alpha = 1 of t = r^2 / gamma^2, over
gamma.  The tables must hold 1e-13 relative, or 1e-15 of the bare 1/r term
where the screened term is below 1e-2 of it.
"""

import numpy as np
import pytest

special = pytest.importorskip("scipy.special")

import paper_2503_21176_gb300 as qg  # noqa: E402


def _reference(alpha, s):
    r = np.sqrt(s)
    F = special.erfc(alpha * r) / r
    G = -(F + 2.0 * alpha / np.sqrt(np.pi) * np.exp(-alpha * alpha * s)) / s
    return F, G


def _check(alpha, s, F, G):
    Fr, Gr = _reference(alpha, s)
    bare = 1.0 / np.sqrt(s)
    fs = np.maximum(np.abs(Fr), 1e-2 * bare)
    gs = np.maximum(np.abs(Gr), 1e-2 * bare / s)
    # 1e-13 for the table plus a few ulp for the double-precision reference
    assert np.max(np.abs(F - Fr) / fs) < 1.2e-13
    assert np.max(np.abs(G - Gr) / gs) < 1.2e-13


def _log_uniform(lo, hi, n, seed):
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), n))


def test_screened_pair_table_r_cut_8():
    """alpha 0.34, r_c 8 (the water workloads): octaves 1/4 .. 64, 32 pieces
    each, all kept; every s in [1/4, 64) is tabulated and accurate."""
    s = np.concatenate([_log_uniform(0.25, 64.0, 20000, 1), 2.0 ** np.arange(-2, 6),
                        np.nextafter(2.0 ** np.arange(-1, 7), 0.0)])
    F, G, inn, kept = qg.qeq_pair_table_eval(0.34, 64.0, 0, s)
    assert kept == 8 * 32
    assert inn.all()
    _check(0.34, s, F, G)


def test_arguments_outside_the_table_take_the_direct_path():
    s = np.array([1e-3, 0.1, np.nextafter(0.25, 0.0), 64.0, 100.0])
    F, G, inn, kept = qg.qeq_pair_table_eval(0.34, 64.0, 0, s)
    assert not inn.any() and np.isnan(F).all() and np.isnan(G).all()


def test_cutoff_sets_the_table_length():
    """r_c^2 = 81: the octave [64, 128) is past the 8 octaves the table holds,
    so its pairs take the direct path; r_c^2 = 20 needs the 7 octaves up to
    [16, 32)."""
    _, _, inn, kept = qg.qeq_pair_table_eval(0.34, 81.0, 0, np.array([63.9, 64.0, 80.0]))
    assert kept == 8 * 32 and inn.tolist() == [1, 0, 0]
    _, _, inn, kept = qg.qeq_pair_table_eval(0.34, 20.0, 0, np.array([15.9, 16.0, 19.9]))
    assert kept == 7 * 32 and inn.tolist() == [1, 1, 1]


@pytest.mark.parametrize("alpha", [0.2, 0.6, 1.5])
def test_screened_pair_table_other_alphas(alpha):
    s = _log_uniform(0.25, 36.0, 5000, int(alpha * 10))
    F, G, inn, kept = qg.qeq_pair_table_eval(alpha, 36.0, 0, s)
    assert 0 < kept <= 8 * 32
    assert inn.any()
    _check(alpha, s[inn == 1], F[inn == 1], G[inn == 1])


def test_gaussian_correction_table():
    """F, G at alpha = 1 of t = r^2 / gamma^2 in [1/32, 6.5^2]: all kept."""
    t = np.concatenate([_log_uniform(1.0 / 32.0, 42.25, 20000, 3), 2.0 ** np.arange(-5, 6)])
    F, G, inn, kept = qg.qeq_pair_table_eval(0.0, 0.0, 1, t)
    assert kept == 11 * 16
    assert inn.all()
    _check(1.0, t, F, G)


def test_bad_arguments_are_rejected():
    with pytest.raises(qg.QeqError):
        qg.qeq_pair_table_eval(0.34, 64.0, 2, np.array([1.0]))
    with pytest.raises(qg.QeqError):
        qg.qeq_pair_table_eval(-1.0, 64.0, 0, np.array([1.0]))
