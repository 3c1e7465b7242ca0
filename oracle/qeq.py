"""Charge equilibration and shadow XL-BOMD (Sec. 3.4, Sec. 3.5) -- test infrastructure only.

Readings of the paper used here:

* The Coulomb block of the QEq matrix is C = diag(u) + Phi.  The printed
  element formula in Sec. 3.4 carries a sign slip.  The matrix-free form
  C v = u o v + dE_Coul/dv fixes the sign.
* In Eq. (diag_linear_qeq), row i has u_i and sums over j != i.  The printed
  ``u_1`` and ``j != 1`` in row 2 are typesetting slips.
* The shadow energy (Eq. qeq_energy) is
  E = sum q chi + 1/2 sum u q^2 + q.Phi n - 1/2 n.Phi n.  At fixed n its
  stationary q is the closed form of Eq. (diag_linear_qeq).
* The Jacobian of the residual q[n] - n acts as J x = (dq/dn) x - x with
  (dq/dn x)_i = -((Phi x)_i + mu) / u_i.  Here mu keeps the charge total fixed:
  mu = -(sum_i (Phi x)_i / u_i) / (sum_i 1 / u_i).
* The kernel K = J^{-1} acts on f = q[n] - n through a rank-m Krylov
  approximation.  The basis starts at w_1 = f / |f| and is extended by
  Gram-Schmidt on r_k = J w_k.  Then K f ~ W c, where c solves the m x m
  normal equations (R^T R) c = R^T f.
* Shadow forces at fixed n: F_i = q_i E^n_i + n_i E^f_i (+ short range).  Here
  E^x is the field of the charges x, and f = q - n.
* The integrator is not printed in the paper.  Positions use velocity Verlet.
  The auxiliary charges use the Verlet form of n'' = -w^2 K(q[n] - n) with the
  dissipation window of Niklasson et al., J. Chem. Phys. 130, 214109 (2009):
  n_{t+1} = 2 n_t - n_{t-1} - kappa (K f)_t + a sum_{k=0}^{K_d} c_k n_{t-k}.
  Those constants come from the literature, not from this paper; parity unpinned.
"""

from __future__ import annotations

import numpy as np

# 1 amu * Angstrom^2 / fs^2 expressed in eV
AMU_A2_FS2_IN_EV = 103.6427

# (kappa, alpha * 1e3, c_0 .. c_K) for dissipation windows K = 3 .. 7
XLBOMD_DISSIPATION = {
    3: (1.69, 150.0, (-2, 3, 0, -1)),
    4: (1.75, 57.0, (-3, 6, -2, -2, 1)),
    5: (1.82, 18.0, (-6, 14, -8, -3, 4, -1)),
    6: (1.84, 5.5, (-14, 36, -27, -2, 12, -6, 1)),
    7: (1.86, 1.6, (-36, 99, -88, 11, 32, -25, 8, -1)),
}


def xlbomd_coefficients(k_d: int):
    kappa, a1e3, c = XLBOMD_DISSIPATION[k_d]
    return kappa, a1e3 * 1e-3, np.asarray(c, dtype=np.float64)


# ---------------------------------------------------------------------------
# Regular QEq (Eq. linear_qeq), dense
# ---------------------------------------------------------------------------

def qeq_dense_solve(Phi, chi, u, q_tot=0.0):
    """Solve [[diag(u) + Phi, 1], [1^T, 0]] [q; lam] = [-chi; Q_tot] by LU (LAPACK gesv)."""
    n = Phi.shape[0]
    A = np.zeros((n + 1, n + 1))
    A[:n, :n] = Phi + np.diag(u)
    A[:n, n] = 1.0
    A[n, :n] = 1.0
    b = np.concatenate([-np.asarray(chi, dtype=np.float64), [q_tot]])
    x = np.linalg.solve(A, b)
    return x[:n], float(x[n])


def qeq_energy(q, chi, u, Phi):
    """E(q) of Eq. (qeq_energy_func) with E_Coul = 1/2 q.Phi q."""
    return float(q @ chi + 0.5 * np.sum(u * q * q) + 0.5 * q @ (Phi @ q))


# ---------------------------------------------------------------------------
# Shadow charges and energy (Eq. qeq_energy, Eq. diag_linear_qeq)
# ---------------------------------------------------------------------------

def shadow_charges(v_n, chi, u, q_tot=0.0):
    """q[n] from the quasi-diagonal system: u_i q_i + lam = -chi_i - v_i[n], sum q = Q_tot."""
    v_n = np.asarray(v_n, dtype=np.float64)
    inv_u = 1.0 / np.asarray(u, dtype=np.float64)
    lam = -(q_tot + np.sum((chi + v_n) * inv_u)) / np.sum(inv_u)
    q = -(chi + v_n + lam) * inv_u
    return q, float(lam)


def shadow_energy(q, n, v_n, chi, u):
    """E(R, q, n) = sum q chi + 1/2 sum u q^2 + q.v[n] - 1/2 n.v[n]."""
    return float(q @ chi + 0.5 * np.sum(u * q * q) + q @ v_n - 0.5 * n @ v_n)


def jacobian_apply(phi_x, x, u):
    """J x for the residual q[n] - n, given Phi x."""
    inv_u = 1.0 / np.asarray(u, dtype=np.float64)
    mu = -np.sum(phi_x * inv_u) / np.sum(inv_u)
    return -(phi_x + mu) * inv_u - x


def krylov_kernel(f, phi_f, apply_phi, u, m, tol=0.0):
    """Rank-m approximation of K f = J^{-1} f.

    ``phi_f`` is Phi f (already computed for the forces).  ``apply_phi(x)``
    returns Phi x.  With tol > 0 the rank grows only until the least-squares
    residual |R c - f| / |f| is <= tol (m is then the largest rank).
    Returns (Kf, number of extra applies).
    """
    nrm = float(np.linalg.norm(f))
    if nrm == 0.0:
        return np.zeros_like(f), 0
    W, Rk = [], []
    w = f / nrm
    phi_w = phi_f / nrm
    applies = 0
    for k in range(m):
        if k > 0:
            phi_w = apply_phi(w)
            applies += 1
        r = jacobian_apply(phi_w, w, u)
        W.append(w)
        Rk.append(r)
        if tol > 0.0:
            Rm = np.stack(Rk, axis=1)
            c = np.linalg.solve(Rm.T @ Rm, Rm.T @ f)
            if np.linalg.norm(Rm @ c - f) <= tol * nrm:
                break
        if k + 1 < m:
            # next basis vector: r orthonormalised against w_1..w_k (modified Gram-Schmidt)
            nv = r.copy()
            for wj in W:
                nv = nv - (wj @ nv) * wj
            nn = float(np.linalg.norm(nv))
            if nn == 0.0:
                break
            w = nv / nn
    Wm = np.stack(W, axis=1)
    Rm = np.stack(Rk, axis=1)
    O = Rm.T @ Rm
    c = np.linalg.solve(O, Rm.T @ f)
    return Wm @ c, applies


# ---------------------------------------------------------------------------
# Shadow XL-BOMD (Sec. 3.5)
# ---------------------------------------------------------------------------

class ShadowSystem:
    """Everything the shadow step needs besides the Coulomb operator.

    ``coulomb(R, x, need_field)`` returns (v, E) for charges x at positions R.
    ``short(R)`` returns (energy, forces) of V_short, or None.
    """

    def __init__(self, coulomb, chi, u, mass, rank, dt, k_d=5, q_tot=0.0, short=None, krylov_tol=0.0):
        self.coulomb = coulomb
        self.chi = np.asarray(chi, dtype=np.float64)
        self.u = np.asarray(u, dtype=np.float64)
        self.mass = np.asarray(mass, dtype=np.float64)
        self.rank = int(rank)
        self.dt = float(dt)
        self.k_d = int(k_d)
        self.q_tot = float(q_tot)
        self.short = short
        self.krylov_tol = float(krylov_tol)
        self.kappa, self.alpha_d, self.c = xlbomd_coefficients(self.k_d)

    def evaluate(self, R, n):
        """Shadow charges, forces, Kf and energies at (R, n); m + 1 Coulomb applies."""
        v_n, E_n = self.coulomb(R, n, True)
        q, lam = shadow_charges(v_n, self.chi, self.u, self.q_tot)
        f = q - n
        phi_f, E_f = self.coulomb(R, f, True)
        F = q[:, None] * E_n + n[:, None] * E_f
        e_short = 0.0
        if self.short is not None:
            e_short, F_short = self.short(R)
            F = F + F_short
        Kf, extra = krylov_kernel(f, phi_f, lambda x: self.coulomb(R, x, False)[0], self.u,
                                  self.rank, self.krylov_tol)
        e_pot = shadow_energy(q, n, v_n, self.chi, self.u) + e_short
        return {"q": q, "F": F, "Kf": Kf, "f": f, "v_n": v_n, "lam": lam,
                "e_shadow": e_pot, "e_short": e_short, "applies": 2 + extra}

    def kinetic(self, V):
        return 0.5 * AMU_A2_FS2_IN_EV * float(np.sum(self.mass[:, None] * V * V))

    def init_state(self, R, V, n0):
        """History window filled with n0; forces and Kf evaluated at (R, n0)."""
        hist = np.tile(np.asarray(n0, dtype=np.float64), (self.k_d + 1, 1))
        ev = self.evaluate(R, hist[0])
        return {"R": np.array(R, dtype=np.float64), "V": np.array(V, dtype=np.float64),
                "hist": hist, "F": ev["F"], "Kf": ev["Kf"], "q": ev["q"],
                "e_pot": ev["e_shadow"], "e_kin": self.kinetic(V)}

    def step(self, st):
        """One velocity-Verlet step for R and one dissipative Verlet step for n."""
        dt = self.dt
        acc = st["F"] / (self.mass[:, None] * AMU_A2_FS2_IN_EV)
        V = st["V"] + 0.5 * dt * acc
        R = st["R"] + dt * V
        h = st["hist"]
        n_new = (2.0 * h[0] - h[1] - self.kappa * st["Kf"]
                 + self.alpha_d * np.tensordot(self.c, h, axes=(0, 0)))
        hist = np.empty_like(h)
        hist[1:] = h[:-1]
        hist[0] = n_new
        ev = self.evaluate(R, n_new)
        acc = ev["F"] / (self.mass[:, None] * AMU_A2_FS2_IN_EV)
        V = V + 0.5 * dt * acc
        return {"R": R, "V": V, "hist": hist, "F": ev["F"], "Kf": ev["Kf"], "q": ev["q"],
                "e_pot": ev["e_shadow"], "e_kin": self.kinetic(V), "applies": ev["applies"]}



# ---------------------------------------------------------------------------
# Regular QEq by GMRES and regular BO-MD (Sec. 3.4, Sec. 4.1)
# ---------------------------------------------------------------------------

def qeq_gmres(apply_phi, chi, u, q0, tol, max_iter=500, restart=40, q_tot=0.0, precond=None,
              final_check=True, lam0=0.0):
    """Restarted GMRES on the bordered QEq system, right-preconditioned by M = diag(d, 1).

    ``apply_phi(x)`` returns Phi x.  ``precond`` is the diagonal d (defaults to u).
    The stopping test is on the true relative residual ||b - A z|| / ||b||, the
    paper's solver tolerance.  The Arnoldi basis is built by modified
    Gram-Schmidt and the least-squares problem by Givens rotations.  Returns
    (q, lambda, info).
    """
    chi = np.asarray(chi, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    n = chi.size
    d = np.asarray(u if precond is None else precond, dtype=np.float64)
    dinv = np.concatenate([1.0 / d, [1.0]])

    def A(z):
        y = np.empty(n + 1)
        y[:n] = u * z[:n] + apply_phi(z[:n]) + z[n]
        y[n] = z[:n].sum()
        return y

    b = np.concatenate([-chi, [q_tot]])
    bnorm = np.linalg.norm(b) or 1.0
    z = np.concatenate([np.asarray(q0, dtype=np.float64), [float(lam0)]])
    iters = applies = 0
    while True:
        r = b - A(z)
        applies += 1
        beta = np.linalg.norm(r)
        relres = beta / bnorm
        if relres <= tol or iters >= max_iter or beta == 0.0:
            break
        V = [r / beta]
        H = np.zeros((restart + 1, restart))
        g = np.zeros(restart + 1)
        g[0] = beta
        cs, sn = np.zeros(restart), np.zeros(restart)
        j = 0
        while j < restart and iters < max_iter:
            w = A(dinv * V[j])
            applies += 1
            iters += 1
            for k in range(j + 1):
                H[k, j] = V[k] @ w
                w = w - H[k, j] * V[k]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V.append(w / H[j + 1, j])
            for k in range(j):
                a, bb = H[k, j], H[k + 1, j]
                H[k, j], H[k + 1, j] = cs[k] * a + sn[k] * bb, -sn[k] * a + cs[k] * bb
            rr = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = (H[j, j] / rr, H[j + 1, j] / rr) if rr > 0 else (1.0, 0.0)
            H[j, j], H[j + 1, j] = rr, 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            j += 1
            if abs(g[j]) / bnorm <= tol or len(V) <= j:
                break
        y = np.linalg.solve(np.triu(H[:j, :j]), g[:j]) if j else np.zeros(0)
        z = z + dinv * (np.stack(V[:j], axis=1) @ y if j else 0.0)
        if (abs(g[j]) / bnorm <= tol or iters >= max_iter) and not final_check:
            relres = abs(g[j]) / bnorm
            break
        if abs(g[j]) / bnorm <= tol or iters >= max_iter:
            r = b - A(z)
            applies += 1
            relres = np.linalg.norm(r) / bnorm
            break
    return z[:n], float(z[n]), {"iterations": iters, "applies": applies, "rel_residual": relres}


class BOSystem:
    """Regular BO-MD: a GMRES QEq solve per step (warm start), forces F = q o E[q] + F_short."""

    def __init__(self, coulomb, chi, u, mass, dt, tol, max_iter=500, short=None, precond=None):
        self.coulomb = coulomb
        self.chi = np.asarray(chi, dtype=np.float64)
        self.u = np.asarray(u, dtype=np.float64)
        self.mass = np.asarray(mass, dtype=np.float64)
        self.dt = float(dt)
        self.tol = float(tol)
        self.max_iter = int(max_iter)
        self.short = short
        self.precond = precond

    def evaluate(self, R, q_guess, lam_guess=0.0):
        q, lam, info = qeq_gmres(lambda x: self.coulomb(R, x, False)[0], self.chi, self.u, q_guess,
                                 self.tol, self.max_iter, precond=self.precond, final_check=False,
                                 lam0=lam_guess)
        v, E = self.coulomb(R, q, True)
        F = q[:, None] * E
        e_short = 0.0
        if self.short is not None:
            e_short, Fs = self.short(R)
            F = F + Fs
        e_pot = float(q @ self.chi + 0.5 * np.sum(self.u * q * q) + 0.5 * q @ v) + e_short
        return {"q": q, "lam": lam, "F": F, "e_pot": e_pot, "applies": info["applies"] + 1,
                "info": info}

    def kinetic(self, V):
        return 0.5 * AMU_A2_FS2_IN_EV * float(np.sum(self.mass[:, None] * V * V))

    def init_state(self, R, V, q0):
        ev = self.evaluate(R, q0)
        return {"R": np.array(R, dtype=np.float64), "V": np.array(V, dtype=np.float64),
                "q": ev["q"], "lam": ev["lam"], "F": ev["F"], "e_pot": ev["e_pot"],
                "e_kin": self.kinetic(V), "applies": ev["applies"]}

    def step(self, st):
        dt = self.dt
        V = st["V"] + 0.5 * dt * st["F"] / (self.mass[:, None] * AMU_A2_FS2_IN_EV)
        R = st["R"] + dt * V
        ev = self.evaluate(R, st["q"], st["lam"])
        V = V + 0.5 * dt * ev["F"] / (self.mass[:, None] * AMU_A2_FS2_IN_EV)
        return {"R": R, "V": V, "q": ev["q"], "lam": ev["lam"], "F": ev["F"], "e_pot": ev["e_pot"],
                "e_kin": self.kinetic(V), "applies": ev["applies"]}
