"""Pins of the oracle's Coulomb operator against closed forms and invariants (CPU only).

Paper passages: Sec. 3.2 (Eqs. ewald_general, ewald_real, ewald_rec, ewald_self and
the derivative forms), Sec. 3.3 (Alg. 2, smooth PME).
"""

import math
import os

import numpy as np
import pytest

from oracle import ewald
from workloads import random_neutral_charges, rocksalt_lattice, water_box

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _madelung():
    with open(os.path.join(GOLDEN, "madelung_nacl.txt")) as fh:
        vals = [ln for ln in fh if ln.strip() and not ln.startswith("#")]
    return float(vals[0])


@pytest.mark.parametrize("n_cells,a,alpha", [(1, 2.0, 1.0), (2, 2.0, 1.0), (2, 2.8201, 0.8),
                                             (3, 2.0, 0.9)])
def test_madelung_rocksalt(n_cells, a, alpha):
    """Direct Ewald (real + explicit k-sum + self) reproduces the NaCl Madelung constant."""
    R, q, L = rocksalt_lattice(n_cells, a)
    box = np.array([L, L, L])
    rc = 6.3 / alpha  # erfc(6.3) ~ 1e-18
    out = ewald.coulomb_apply(R, q, np.zeros(len(q)), box, alpha, rc, recip="ewald")
    m = -out["energy"] / (len(q) / 2) * a / ewald.K_E
    assert abs(m - _madelung()) < 1e-11
    # every ion of one species sees the same potential, -M k_e q / a
    assert np.allclose(out["v"], -_madelung() * ewald.K_E * q / a, rtol=0, atol=1e-9)
    # forces vanish on a perfect lattice
    assert np.abs(out["F"]).max() < 1e-9


def test_madelung_fails_without_self_term():
    """A dropped self term is visible: it shifts the lattice energy by alpha/sqrt(pi) per ion."""
    R, q, L = rocksalt_lattice(1, 2.0)
    box = np.array([L, L, L])
    out = ewald.coulomb_apply(R, q, np.zeros(len(q)), box, 1.0, 6.3, recip="ewald")
    m_wrong = -(out["energy"] - out["energy_self"]) / (len(q) / 2) * 2.0 / ewald.K_E
    assert abs(m_wrong - _madelung()) > 0.1


@pytest.fixture(scope="module")
def small_water():
    w = water_box(27, seed=7)
    q = random_neutral_charges(w.n_atoms, seed=11)
    return w, q


def test_alpha_independence(small_water):
    """Total energy, potentials and fields of the exact lattice sum do not depend on alpha."""
    w, q = small_water
    outs = []
    for alpha in (0.25, 0.34, 0.45):
        rc = 6.25 / alpha  # erfc(6.25) ~ 1e-18: real space converged (multi-image box)
        outs.append(ewald.coulomb_apply(w.R, q, w.sigma, w.box, alpha, rc, recip="ewald"))
    e0 = outs[0]["energy"]
    for o in outs[1:]:
        assert abs(o["energy"] - e0) <= 1e-11 * abs(e0)
        assert np.allclose(o["v"], outs[0]["v"], rtol=0, atol=1e-10)
        assert np.allclose(o["E"], outs[0]["E"], rtol=0, atol=1e-10)


def test_energy_is_half_q_dot_v_and_parts(small_water):
    """E_Coul = 1/2 q.v; the k-sum energy formula agrees with 1/2 q.v_rec."""
    w, q = small_water
    o = ewald.coulomb_apply(w.R, q, w.sigma, w.box, 0.34, 9.0, recip="ewald")
    parts = o["energy_real"] + o["energy_recip"] + o["energy_self"]
    assert abs(parts - o["energy"]) < 1e-11 * abs(o["energy"]) + 1e-12
    assert abs(o["energy_recip"] - o["energy_recip_from_v"]) < 1e-11 * abs(o["energy_recip"])


def test_momentum_conservation_and_translation(small_water):
    """Direct Ewald forces sum to zero; v and E are invariant under a rigid translation."""
    w, q = small_water
    o = ewald.coulomb_apply(w.R, q, w.sigma, w.box, 0.34, 9.0, recip="ewald")
    assert np.abs(o["F"].sum(axis=0)).max() < 1e-11
    shift = np.array([3.3, -7.1, 12.9])
    o2 = ewald.coulomb_apply(w.R + shift, q, w.sigma, w.box, 0.34, 9.0, recip="ewald")
    assert np.allclose(o2["v"], o["v"], rtol=0, atol=1e-11)
    assert np.allclose(o2["E"], o["E"], rtol=0, atol=1e-11)


def test_field_is_minus_gradient_of_energy(small_water):
    """F_i = q_i E_i equals -dE_Coul/dr_i by central differences (direct Ewald)."""
    w, q = small_water
    h = 1e-5
    o = ewald.coulomb_apply(w.R, q, w.sigma, w.box, 0.34, 9.0, recip="ewald")
    for i in (0, 5, 40):
        for d in range(3):
            Rp = w.R.copy(); Rp[i, d] += h
            Rm = w.R.copy(); Rm[i, d] -= h
            ep = ewald.coulomb_apply(Rp, q, w.sigma, w.box, 0.34, 9.0, recip="ewald")["energy"]
            em = ewald.coulomb_apply(Rm, q, w.sigma, w.box, 0.34, 9.0, recip="ewald")["energy"]
            fd = -(ep - em) / (2 * h)
            assert abs(fd - o["F"][i, d]) < 1e-6 * max(1.0, abs(fd))


def test_gaussian_pair_limit():
    """Two Gaussian charges in a huge box interact through erf(r/gamma)/r (closed form)."""
    L = 200.0
    box = np.array([L, L, L])
    r = 1.3
    R = np.array([[10.0, 10.0, 10.0], [10.0 + r, 10.0, 10.0]])
    sigma = np.array([0.7, 0.45])
    q = np.array([1.0, -1.0])
    alpha = 0.05
    o = ewald.coulomb_apply(R, q, sigma, box, alpha, 150.0, recip="ewald")
    gamma = math.hypot(0.7, 0.45)
    # pair energy plus the two point-charge self-image contributions, which vanish as L grows
    pair = -ewald.K_E * math.erf(r / gamma) / r
    assert abs(o["energy"] - pair) < 2e-3 * abs(pair)  # finite-box image terms ~ 1/L
    # gaussian_self adds exactly q_i^2 k_e / (sqrt(2 pi) sigma_i) to the energy
    og = ewald.coulomb_apply(R, q, sigma, box, alpha, 150.0, recip="ewald", gaussian_self=True)
    extra = ewald.K_E * sum(1.0 / (math.sqrt(2 * math.pi) * s) for s in sigma)
    assert abs((og["energy"] - o["energy"]) - extra) < 1e-10


def test_real_space_cells_equal_brute():
    """The cell-list real-space sum equals the brute-force image sum."""
    w = water_box(1000, seed=3)
    q = random_neutral_charges(w.n_atoms, seed=4)
    vb, Eb = ewald.real_space(w.R, q, w.sigma, w.box, 0.34, 8.0, method="brute")
    vc, Ec = ewald.real_space(w.R, q, w.sigma, w.box, 0.34, 8.0, method="cells")
    assert np.allclose(vc, vb, rtol=0, atol=1e-11)
    assert np.allclose(Ec, Eb, rtol=0, atol=1e-11)


def test_real_space_rows_subset():
    w = water_box(64, seed=5)
    q = random_neutral_charges(w.n_atoms, seed=6)
    v, E = ewald.real_space(w.R, q, w.sigma, w.box, 0.34, 9.0, method="brute")
    rows = np.array([3, 100, 7])
    vr, Er = ewald.real_space(w.R, q, w.sigma, w.box, 0.34, 9.0, rows=rows)
    assert np.array_equal(vr, v[rows]) and np.array_equal(Er, E[rows])


# ---------------------------------------------------------------------------
# Smooth PME (Alg. 2)
# ---------------------------------------------------------------------------

def test_bspline_closed_forms():
    """Order-4 cardinal B-spline equals the cubic closed forms; partition of unity for all p."""
    w = np.linspace(0, 1, 17, endpoint=False)
    M, dM = ewald.bspline_table(w, 4)
    assert np.allclose(M[:, 0], w ** 3 / 6, atol=1e-15)
    assert np.allclose(M[:, 1], (-3 * w ** 3 + 3 * w ** 2 + 3 * w + 1) / 6, atol=1e-15)
    assert np.allclose(M[:, 2], (3 * w ** 3 - 6 * w ** 2 + 4) / 6, atol=1e-15)
    assert np.allclose(M[:, 3], (1 - w) ** 3 / 6, atol=1e-15)
    assert np.allclose(dM[:, 0], w ** 2 / 2, atol=1e-15)
    assert np.allclose(dM[:, 3], -(1 - w) ** 2 / 2, atol=1e-15)
    for p in range(2, 9):
        M, dM = ewald.bspline_table(w, p)
        assert np.allclose(M.sum(axis=1), 1.0, atol=1e-14)
        assert np.allclose(dM.sum(axis=1), 0.0, atol=1e-13)
        # derivative by central differences of M_p(w + j)
        h = 1e-6
        Mp, _ = ewald.bspline_table(np.clip(w + h, 0, 1 - 1e-12), p)
        Mm, _ = ewald.bspline_table(np.clip(w - h, 0, 1), p)
        inner = (w > 2 * h) & (w < 1 - 2 * h)
        assert np.allclose(((Mp - Mm) / (2 * h))[inner], dM[inner], atol=1e-7)


def test_bspline_modulus_p4_nyquist():
    """|b(K/2)|^2 for p = 4 is 9 (denominator M(1) - M(2) + M(3) = -1/3)."""
    b = ewald.bspline_modulus(32, 4)
    assert abs(b[16] - 9.0) < 1e-12
    assert abs(b[0] - 1.0) < 1e-14  # sum of M_p(k+1) is 1


@pytest.fixture(scope="module")
def water648():
    w = water_box(216, seed=2503)
    q = random_neutral_charges(w.n_atoms, seed=12)
    ref = ewald.coulomb_apply(w.R, q, w.sigma, w.box, 0.34, 9.0, recip="ewald")
    return w, q, ref


def test_pme_converges_to_direct_ewald(water648):
    """PME error against the explicit k-sum falls monotonically with mesh size and order."""
    w, q, ref = water648
    fref = np.sqrt(np.mean(ref["F"] ** 2))
    errs = {}
    for p in (4, 6):
        prev = None
        for K in (16, 24, 32, 48):
            o = ewald.coulomb_apply(w.R, q, w.sigma, w.box, 0.34, 9.0, recip="pme", mesh=(K, K, K),
                                    order=p)
            e = np.sqrt(np.mean((o["F"] - ref["F"]) ** 2)) / fref
            ev = np.abs(o["v"] - ref["v"]).max()
            if prev is not None:
                assert e < prev[0] and ev < prev[1]
            prev = (e, ev)
            errs[(p, K)] = e
    assert errs[(4, 32)] < 2e-4
    assert errs[(6, 32)] < errs[(4, 32)] / 10
    assert errs[(6, 48)] < 1e-6


def test_pme_energy_equals_half_q_dot_vrec(water648):
    """Mesh energy 1/2 sum G |Qhat|^2 equals 1/2 q.v_rec from the gather (normalisation pin)."""
    w, q, _ = water648
    v, E, en = ewald.pme_reciprocal(w.R, q, w.box, 0.34, (32, 32, 32), 4)
    assert abs(en - 0.5 * q @ v) < 1e-11 * abs(en)


def test_pme_field_is_minus_gradient(water648):
    """PME reciprocal force q_i E_i equals -dE_rec/dr_i by central differences."""
    w, q, _ = water648
    mesh = (24, 24, 24)
    v, E, en = ewald.pme_reciprocal(w.R, q, w.box, 0.34, mesh, 4)
    h = 1e-5
    for i in (0, 17, 300):
        for d in range(3):
            Rp = w.R.copy(); Rp[i, d] += h
            Rm = w.R.copy(); Rm[i, d] -= h
            ep = ewald.pme_reciprocal(Rp, q, w.box, 0.34, mesh, 4)[2]
            em = ewald.pme_reciprocal(Rm, q, w.box, 0.34, mesh, 4)[2]
            assert abs(-(ep - em) / (2 * h) - q[i] * E[i, d]) < 1e-6


def test_pme_orthorhombic_and_anisotropic_mesh():
    """A non-cubic box with a non-cubic mesh still converges to the explicit k-sum."""
    rng = np.random.default_rng(8)
    box = np.array([14.0, 17.5, 21.0])
    R = rng.uniform(0, 1, size=(150, 3)) * box
    q = random_neutral_charges(150, seed=9)
    sigma = np.full(150, 0.6)
    ref = ewald.coulomb_apply(R, q, sigma, box, 0.4, 7.0, recip="ewald")
    o = ewald.coulomb_apply(R, q, sigma, box, 0.4, 7.0, recip="pme", mesh=(40, 48, 60), order=6)
    assert np.abs(o["v"] - ref["v"]).max() < 1e-5 * np.abs(ref["v"]).max()
