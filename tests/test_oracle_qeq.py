"""Pins of the oracle's QEq, shadow-charge, Krylov and integrator functions (CPU only).

Paper passages: Sec. 3.4 (Eqs. qeq_energy_func, linear_qeq and the matrix-free form
C v = u o v + dE/dv), Sec. 3.5 (Eqs. qeq_energy, diag_linear_qeq, the extended
Lagrangian, the adiabatic equations of motion and Eq. Jnddot).
"""

import os

import numpy as np
import pytest

from oracle import ewald, qeq
from workloads import random_neutral_charges, water_box

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ALPHA, RC = 0.34, 9.0


@pytest.fixture(scope="module")
def system():
    w = water_box(12, seed=41)  # 36 atoms, multi-image box
    Phi = ewald.phi_matrix(w.R, w.sigma, w.box, ALPHA, RC, recip="ewald", gaussian_self=True)
    return w, Phi


def _apply_ewald(w):
    def f(R, x, need_field=True):
        o = ewald.coulomb_apply(R, x, w.sigma, w.box, ALPHA, RC, recip="ewald",
                                gaussian_self=True)
        return o["v"], o["E"]
    return f


def test_gaussian_self_energy_makes_qeq_convex():
    """Reading pinned here: the water parameters need the Gaussian self-energy on the diagonal.

    With u = eta and the 1/2 u q^2 convention, diag(u) + Phi without the
    Gaussian self-energy has negative eigenvalues on the neutral subspace, so the
    constrained minimum of Eq. (BO_Min) does not exist.  With k_e sqrt(2/pi) / sigma_i
    added, the neutral spectrum is positive and the QEq charges are physical.
    """
    w = water_box(8, seed=51)
    N = w.n_atoms
    P = np.eye(N) - 1.0 / N
    for gs, sign in ((False, -1), (True, 1)):
        Phi = ewald.phi_matrix(w.R, w.sigma, w.box, ALPHA, RC, recip="ewald", gaussian_self=gs)
        ev = np.sort(np.linalg.eigvalsh(P @ (Phi + np.diag(w.eta)) @ P))
        neutral = ev[np.abs(ev) > 1e-8]  # drop the zero mode along the all-ones vector
        assert np.sign(neutral[0]) == sign
    q, _ = qeq.qeq_dense_solve(Phi, w.chi, w.eta)
    assert np.all(q[w.species == 0] < 0) and np.all(q[w.species == 1] > 0)


def test_phi_matrix_is_symmetric_and_matches_apply(system):
    w, Phi = system
    assert np.abs(Phi - Phi.T).max() < 1e-10
    q = random_neutral_charges(w.n_atoms, seed=1)
    o = ewald.coulomb_apply(w.R, q, w.sigma, w.box, ALPHA, RC, recip="ewald", gaussian_self=True)
    assert np.abs(Phi @ q - o["v"]).max() < 1e-10


def test_dense_qeq_solution(system):
    """Residual of the bordered system, total charge and the minimum property."""
    w, Phi = system
    for q_tot in (0.0, 1.0):
        q, lam = qeq.qeq_dense_solve(Phi, w.chi, w.eta, q_tot)
        res = (Phi + np.diag(w.eta)) @ q + lam + w.chi
        assert np.abs(res).max() < 1e-12 * np.abs(w.chi).max()
        assert abs(q.sum() - q_tot) < 1e-12
        e0 = qeq.qeq_energy(q, w.chi, w.eta, Phi)
        rng = np.random.default_rng(3)
        for _ in range(5):
            d = rng.standard_normal(w.n_atoms)
            d -= d.mean()
            assert qeq.qeq_energy(q + 1e-3 * d, w.chi, w.eta, Phi) > e0


def test_shadow_fixed_point(system):
    """At n = q_min: q[n] = q_min, the shadow energy equals E(q_min), f = 0."""
    w, Phi = system
    qmin, lam = qeq.qeq_dense_solve(Phi, w.chi, w.eta, 0.0)
    qn, lam_n = qeq.shadow_charges(Phi @ qmin, w.chi, w.eta, 0.0)
    assert np.abs(qn - qmin).max() < 1e-12
    assert abs(lam_n - lam) < 1e-10
    es = qeq.shadow_energy(qn, qmin, Phi @ qmin, w.chi, w.eta)
    assert abs(es - qeq.qeq_energy(qmin, w.chi, w.eta, Phi)) < 1e-10


def test_shadow_charges_stationary(system):
    """q[n] is the constrained stationary point of the shadow energy at fixed n."""
    w, Phi = system
    n = random_neutral_charges(w.n_atoms, seed=5, scale=0.3)
    vn = Phi @ n
    q, lam = qeq.shadow_charges(vn, w.chi, w.eta, 0.0)
    grad = w.chi + w.eta * q + vn  # d E_shadow / d q_i
    assert np.abs(grad + lam).max() < 1e-12
    assert abs(q.sum()) < 1e-13


def test_jacobian_by_finite_difference(system):
    """J x equals the derivative of q[n] - n along x (exactly linear)."""
    w, Phi = system
    n = random_neutral_charges(w.n_atoms, seed=6)
    x = random_neutral_charges(w.n_atoms, seed=7)
    eps = 1e-3
    q1, _ = qeq.shadow_charges(Phi @ n, w.chi, w.eta)
    q2, _ = qeq.shadow_charges(Phi @ (n + eps * x), w.chi, w.eta)
    fd = ((q2 - (n + eps * x)) - (q1 - n)) / eps
    assert np.abs(fd - qeq.jacobian_apply(Phi @ x, x, w.eta)).max() < 1e-9


def test_krylov_full_rank_equals_dense_inverse():
    """With a full basis (m = N) the low-rank kernel is J^{-1} f; rank 1 is the 1-D least squares."""
    w = water_box(6, seed=41)  # 18 atoms: short enough that one Gram-Schmidt pass stays orthogonal
    Phi = ewald.phi_matrix(w.R, w.sigma, w.box, ALPHA, RC, recip="ewald")
    n = random_neutral_charges(w.n_atoms, seed=8)
    q, _ = qeq.shadow_charges(Phi @ n, w.chi, w.eta)
    f = q - n
    N = w.n_atoms
    J = np.stack([qeq.jacobian_apply(Phi[:, j], np.eye(N)[j], w.eta) for j in range(N)], axis=1)
    dense = np.linalg.solve(J, f)
    Kf, extra = qeq.krylov_kernel(f, Phi @ f, lambda x: Phi @ x, w.eta, N)
    assert extra == N - 1
    assert np.abs(Kf - dense).max() < 1e-10 * np.abs(dense).max()
    Kf1, _ = qeq.krylov_kernel(f, Phi @ f, lambda x: Phi @ x, w.eta, 1)
    Jf = J @ f
    c = (Jf @ f) / (Jf @ Jf)
    assert np.abs(Kf1 - c * f).max() < 1e-12 * np.abs(f).max()


def test_shadow_forces_are_minus_gradient(system):
    """F = q E^n + n E^f equals -dU/dR at fixed n, U = E_shadow(R, q[n](R), n)."""
    w, _ = system
    coul = _apply_ewald(w)
    n = random_neutral_charges(w.n_atoms, seed=9, scale=0.3)
    sysm = qeq.ShadowSystem(coul, w.chi, w.eta, w.mass, rank=1, dt=0.5)

    def U(R):
        v, _ = coul(R, n)
        q, _ = qeq.shadow_charges(v, w.chi, w.eta)
        return qeq.shadow_energy(q, n, v, w.chi, w.eta)

    ev = sysm.evaluate(w.R, n)
    h = 1e-5
    for i in (0, 4, 20):
        for d in range(3):
            Rp = w.R.copy(); Rp[i, d] += h
            Rm = w.R.copy(); Rm[i, d] -= h
            fd = -(U(Rp) - U(Rm)) / (2 * h)
            assert abs(fd - ev["F"][i, d]) < 1e-6 * max(1.0, abs(fd))


def test_dissipation_table_matches_golden():
    with open(os.path.join(GOLDEN, "xlbomd_dissipation.txt")) as fh:
        rows = [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]
    for r in rows:
        k = int(r[0])
        kappa, a, c = qeq.xlbomd_coefficients(k)
        assert kappa == float(r[1]) and abs(a * 1e3 - float(r[2])) < 1e-12
        assert np.array_equal(c, np.array([float(x) for x in r[3:]]))
        assert c.sum() == 0 and len(c) == k + 1


def test_shadow_md_conserves_charge_and_energy():
    """Short shadow XL-BOMD run: total n and q stay at Q_tot; total energy stays flat."""
    w = water_box(8, seed=51)
    coul = _apply_ewald(w)
    Phi = ewald.phi_matrix(w.R, w.sigma, w.box, ALPHA, RC, recip="ewald", gaussian_self=True)
    qmin, _ = qeq.qeq_dense_solve(Phi, w.chi, w.eta)
    sysm = qeq.ShadowSystem(coul, w.chi, w.eta, w.mass, rank=2, dt=0.5, k_d=5)
    rng = np.random.default_rng(2)
    V = rng.standard_normal(w.R.shape) * np.sqrt(0.0259 / (w.mass[:, None] * qeq.AMU_A2_FS2_IN_EV))
    V -= (w.mass[:, None] * V).sum(0) / w.mass.sum()
    st = sysm.init_state(w.R, V, qmin)
    e0 = st["e_kin"] + st["e_pot"]
    es = []
    for _ in range(40):
        st = sysm.step(st)
        assert abs(st["hist"][0].sum()) < 1e-11
        assert abs(st["q"].sum()) < 1e-11
        es.append(st["e_kin"] + st["e_pot"])
    es = np.array(es)
    # 20 fs of NVE: the shadow total energy drifts by far less than the kinetic energy (~1 eV)
    assert np.abs(es - e0).max() < 2e-4


def test_gmres_converges_to_dense_solution(system):
    """The oracle GMRES of the bordered system reaches the dense LU solution; looser
    tolerances stop earlier with the requested true relative residual."""
    w, Phi = system
    qd, lam = qeq.qeq_dense_solve(Phi, w.chi, w.eta)
    prev_iters = -1
    for tol in (1e-1, 1e-3, 1e-6, 1e-12):
        q, l, info = qeq.qeq_gmres(lambda x: Phi @ x, w.chi, w.eta, np.zeros(w.n_atoms), tol)
        assert info["rel_residual"] <= tol
        assert info["iterations"] >= prev_iters
        prev_iters = info["iterations"]
        A_res = np.concatenate([(Phi + np.diag(w.eta)) @ q + l + w.chi, [q.sum()]])
        b = np.concatenate([-w.chi, [0.0]])
        assert abs(np.linalg.norm(A_res) / np.linalg.norm(b) - info["rel_residual"]) < 1e-10
    assert np.abs(q - qd).max() < 1e-10 and abs(l - lam) < 1e-9
    assert info["iterations"] <= w.n_atoms + 1


def test_gmres_warm_start_is_cheaper(system):
    """A guess near the solution (as in MD, from the previous step) converges in fewer iterations."""
    w, Phi = system
    qd, lam = qeq.qeq_dense_solve(Phi, w.chi, w.eta)
    rng = np.random.default_rng(4)
    guess = qd + 1e-3 * rng.standard_normal(w.n_atoms)
    _, _, cold = qeq.qeq_gmres(lambda x: Phi @ x, w.chi, w.eta, np.zeros(w.n_atoms), 1e-6)
    _, _, warm = qeq.qeq_gmres(lambda x: Phi @ x, w.chi, w.eta, guess, 1e-6, lam0=lam)
    assert warm["iterations"] < cold["iterations"]


def test_adaptive_krylov_stops_at_tolerance(system):
    w, Phi = system
    n = random_neutral_charges(w.n_atoms, seed=3, scale=0.3)
    q, _ = qeq.shadow_charges(Phi @ n, w.chi, w.eta)
    f = q - n
    for tol in (0.5, 0.1, 1e-3):
        Kf, extra = qeq.krylov_kernel(f, Phi @ f, lambda x: Phi @ x, w.eta, 8, tol)
        N = w.n_atoms
        J = np.stack([qeq.jacobian_apply(Phi[:, j], np.eye(N)[j], w.eta) for j in range(N)], axis=1)
        assert np.linalg.norm(J @ Kf - f) <= tol * np.linalg.norm(f) * (1 + 1e-9) or extra == 7


# ---------------------------------------------------------------------------
# Regular BO-MD (Sec. 3.4): the oracle's BOSystem, pinned by identities that do
# not restate its own energy expression
# ---------------------------------------------------------------------------

def _bo_system(w, tol, short=True):
    from oracle import short_range

    coul = _apply_ewald(w)
    sr = (lambda R: short_range.water_short_range(R, w.box, RC)) if short else None
    return qeq.BOSystem(coul, w.chi, w.eta, w.mass, dt=0.5, tol=tol, short=sr)


def test_bo_energy_is_half_q_chi_at_the_solution(system):
    """At the constrained minimum of Eq. (qeq_energy_func), (diag(u) + Phi) q = -chi - lambda,
    so with Q_tot = 0 the BO energy collapses to 1/2 q.chi.  BOSystem.evaluate must
    reach the dense LU charges and report that energy (plus V_short); a dropped or
    doubled 1/2 on either quadratic term, or a v taken from other charges, breaks it."""
    from oracle import short_range

    w, Phi = system
    qd, lam = qeq.qeq_dense_solve(Phi, w.chi, w.eta, 0.0)
    e_short = short_range.water_short_range(w.R, w.box, RC)[0]
    ev = _bo_system(w, 1e-13).evaluate(w.R, np.zeros(w.n_atoms))
    assert np.abs(ev["q"] - qd).max() < 1e-10
    assert abs(ev["lam"] - lam) < 1e-9
    assert abs((ev["e_pot"] - e_short) - 0.5 * qd @ w.chi) < 1e-10 * abs(0.5 * qd @ w.chi)
    # and the BO energy is below the QEq energy of any other neutral charge vector
    rng = np.random.default_rng(12)
    for _ in range(3):
        d = rng.standard_normal(w.n_atoms)
        d -= d.mean()
        q2 = qd + 1e-2 * d
        e2 = float(q2 @ w.chi + 0.5 * np.sum(w.eta * q2 * q2) + 0.5 * q2 @ Phi @ q2)
        assert e2 > ev["e_pot"] - e_short


def test_bo_forces_are_minus_gradient_of_the_bo_energy(system):
    """F = q o E[q] + F_short equals -dU_BO/dR, with U_BO(R) the energy at the solved
    charges of each displaced geometry (the charge response drops out at the
    minimum).  Central differences, solver tolerance 1e-12."""
    w, _ = system
    bo = _bo_system(w, 1e-12)
    ev = bo.evaluate(w.R, np.zeros(w.n_atoms))
    h = 1e-5
    for i in (0, 7, 31):
        for d in range(3):
            e = []
            for sgn in (1.0, -1.0):
                R = w.R.copy()
                R[i, d] += sgn * h
                e.append(bo.evaluate(R, ev["q"], ev["lam"])["e_pot"])
            fd = -(e[0] - e[1]) / (2 * h)
            assert abs(fd - ev["F"][i, d]) < 1e-6 * max(1.0, abs(fd))


def test_bo_md_conserves_energy():
    """40 regular BO-MD steps (0.5 fs, tolerance 1e-10, Coulomb only): the total energy
    stays within the bound of the shadow run (measured 1.0e-5 eV) and the charges stay
    neutral.  A second half kick with the forces of the previous geometry leaves it by
    a factor of about 14, a doubled 1/2 q.v by about 160.  (The stiff bonds of the
    flexible-water V_short add a Verlet fluctuation of about 1e-2 eV at this step, so
    V_short is pinned by the force test instead.)"""
    w = water_box(8, seed=51)
    bo = _bo_system(w, 1e-10, short=False)
    rng = np.random.default_rng(2)
    V = rng.standard_normal(w.R.shape) * np.sqrt(0.0259 / (w.mass[:, None] * qeq.AMU_A2_FS2_IN_EV))
    V -= (w.mass[:, None] * V).sum(0) / w.mass.sum()
    st = bo.init_state(w.R, V, np.zeros(w.n_atoms))
    e0 = st["e_kin"] + st["e_pot"]
    es, kin = [], []
    for _ in range(40):
        st = bo.step(st)
        assert abs(st["q"].sum()) < 1e-9
        es.append(st["e_kin"] + st["e_pot"])
        kin.append(st["e_kin"])
    es = np.array(es)
    assert np.ptp(kin) > 1e-2  # energy really moves between kinetic and potential
    assert np.abs(es - e0).max() < 2e-4
