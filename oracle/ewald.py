"""Periodic Coulomb potential operator v = Phi q and its field (Sec. 3.2, Sec. 3.3).

Test infrastructure only; FP64 throughout.  Two reciprocal parts are provided:

* ``ewald_kspace`` -- the explicit k-vector sum of Eq. (ewald_rec) with the
  derivative forms that follow it.  With a converged k cutoff and a large
  real-space cutoff this is the exact lattice sum under tin-foil boundary
  conditions (Eq. ewald_rec has no dipole term).
* ``pme_reciprocal`` -- smooth PME (Alg. 2): B-spline spreading (step 1), FFT
  (step 2), multiplication by the influence function and the energy sum
  (step 3), inverse FFT (step 4), and the gather of potentials and fields
  with the spline derivative (step 5).  Its FFT is numpy's full complex FFT,
  used as a library primitive.

The real-space part is Eq. (ewald_real) truncated at r_c (strict ``<``, no
shift).  Each pair term subtracts the Gaussian-charge correction
erfc(r / gamma_ij) / r, where gamma_ij = sqrt(sigma_i^2 + sigma_j^2).  So two
Gaussian charges interact through erf(r / gamma_ij) / r.  sigma = 0 denotes a
point charge.  The self term is Eq. (ewald_self) differentiated in q_i:
-2 alpha / sqrt(pi) q_i.  ``gaussian_self`` adds the Gaussian self-energy
derivative sqrt(2/pi) / sigma_i q_i.  That option is off by default, so the
self-energy stays absorbed in the hardness.

Every function returns quantities already multiplied by the Coulomb constant k_e
(eV * Angstrom / e^2 in the water workloads).  The field is E_i = -d v_i / d r_i
with the other charges held fixed, so the Coulomb force is F_i = q_i E_i.
"""

from __future__ import annotations

import math

import numpy as np

from . import native

K_E = 14.3996454784  # eV * Angstrom / e^2


def _c64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ---------------------------------------------------------------------------
# Real space (Eq. ewald_real + Gaussian correction)
# ---------------------------------------------------------------------------

def real_space(R, q, sigma, box, alpha, r_c, k_e=K_E, rows=None, method="auto"):
    """Real-space potential and field for all atoms (or the given rows).

    ``method``: "brute" (every atom and image), "cells" (cell list, all
    rows), or "auto" (brute for small N or row subsets).
    """
    R, q, sigma, box = _c64(R), _c64(q), _c64(sigma), _c64(box)
    n = R.shape[0]
    L = native.lib()
    if method == "auto":
        method = "brute" if (rows is not None or n <= 4000) else "cells"
    if method == "cells":
        if rows is not None:
            raise ValueError("the cell-list form computes all rows")
        v = np.zeros(n)
        E = np.zeros((n, 3))
        rc = L.or_realspace_cells(n, native.dptr(R), native.dptr(q), native.dptr(sigma),
                                  native.dptr(box), float(alpha), float(r_c), native.dptr(v),
                                  native.dptr(E))
        if rc != 0:
            raise MemoryError("or_realspace_cells failed")
        return k_e * v, k_e * E
    if rows is None:
        n_rows, rows_p = n, None
    else:
        rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
        n_rows, rows_p = rows.shape[0], native.i64ptr(rows)
    v = np.zeros(n_rows)
    E = np.zeros((n_rows, 3))
    L.or_realspace_brute(n, native.dptr(R), native.dptr(q), native.dptr(sigma), native.dptr(box),
                         float(alpha), float(r_c), n_rows, rows_p, native.dptr(v), native.dptr(E))
    return k_e * v, k_e * E


def real_space_matrix(R, sigma, box, alpha, r_c, k_e=K_E):
    """Dense real-space block of Phi (small N)."""
    R, sigma, box = _c64(R), _c64(sigma), _c64(box)
    n = R.shape[0]
    out = np.zeros((n, n))
    native.lib().or_realspace_matrix(n, native.dptr(R), native.dptr(sigma), native.dptr(box),
                                     float(alpha), float(r_c), native.dptr(out))
    return k_e * out


# ---------------------------------------------------------------------------
# Self terms (Eq. ewald_self, and the optional Gaussian self-energy)
# ---------------------------------------------------------------------------

def self_potential(q, sigma, alpha, k_e=K_E, gaussian_self=False):
    q = np.asarray(q, dtype=np.float64)
    v = -2.0 * alpha / math.sqrt(math.pi) * q
    if gaussian_self:
        sigma = np.asarray(sigma, dtype=np.float64)
        v = v + math.sqrt(2.0 / math.pi) / sigma * q
    return k_e * v


# ---------------------------------------------------------------------------
# Explicit k-vector reciprocal sum (Eq. ewald_rec and the derivative forms)
# ---------------------------------------------------------------------------

def kspace_cutoff(alpha, tol=1e-16):
    """|k| beyond which exp(-k^2 / 4 alpha^2) < tol."""
    return 2.0 * alpha * math.sqrt(-math.log(tol))


def ewald_kspace(R, q, box, alpha, k_e=K_E, k_cut=None):
    """Reciprocal potential, field and energy by the explicit k-sum."""
    R, q, box = _c64(R), _c64(q), _c64(box)
    n = R.shape[0]
    if k_cut is None:
        k_cut = kspace_cutoff(alpha)
    v = np.zeros(n)
    E = np.zeros((n, 3))
    en = np.zeros(1)
    nk = native.lib().or_ewald_kspace(n, native.dptr(R), native.dptr(q), native.dptr(box),
                                      float(alpha), float(k_cut), native.dptr(v), native.dptr(E),
                                      native.dptr(en))
    if nk < 0:
        raise MemoryError("or_ewald_kspace failed")
    return k_e * v, k_e * E, k_e * float(en[0])


# ---------------------------------------------------------------------------
# Smooth PME (Alg. 2)
# ---------------------------------------------------------------------------

def bspline_table(w, p):
    """Cardinal B-spline M_p(w + j) and M_p'(w + j) for j = 0 .. p-1.

    M_2(u) = 1 - |u - 1| on [0, 2].  The recursion is
    M_n(u) = [u M_{n-1}(u) + (n - u) M_{n-1}(u - 1)] / (n - 1), and the
    derivative is M_n'(u) = M_{n-1}(u) - M_{n-1}(u - 1).  ``w`` holds
    fractional parts in [0, 1).  Returns two arrays of shape w.shape + (p,).
    """
    w = np.asarray(w, dtype=np.float64)
    if p < 2:
        raise ValueError("spline order must be >= 2")
    # level 2: M_2(w) = w, M_2(w + 1) = 1 - w
    M = np.stack([w, 1.0 - w], axis=-1)
    prev = M
    for n in range(3, p + 1):
        prev = M
        nxt = np.zeros(w.shape + (n,))
        for j in range(n):
            u = w + j
            left = prev[..., j] if j < n - 1 else 0.0  # M_{n-1}(w + j)
            right = prev[..., j - 1] if j >= 1 else 0.0  # M_{n-1}(w + j - 1)
            nxt[..., j] = (u * left + (n - u) * right) / (n - 1)
        M = nxt
    # derivative from the order p-1 table
    if p == 2:
        dM = np.stack([np.ones_like(w), -np.ones_like(w)], axis=-1)
    else:
        dM = np.zeros(w.shape + (p,))
        for j in range(p):
            left = prev[..., j] if j < p - 1 else 0.0
            right = prev[..., j - 1] if j >= 1 else 0.0
            dM[..., j] = left - right
    return M, dM


def bspline_modulus(K, p):
    """|b(m)|^2 of the smooth-PME Euler exponential spline, m = 0 .. K-1.

    b(m) = exp(2 pi i (p-1) m / K) / sum_{k=0}^{p-2} M_p(k+1) exp(2 pi i m k / K).
    Where the denominator vanishes (odd p at m = K/2) the modulus is set to 0.
    """
    Mint, _ = bspline_table(np.zeros(1), p)  # M_p(0 + j), j = 0..p-1
    vals = Mint[0]  # M_p(j); M_p(k + 1) = vals[k + 1]
    m = np.arange(K)
    den = np.zeros(K, dtype=np.complex128)
    for k in range(p - 1):
        den += vals[k + 1] * np.exp(2j * math.pi * m * k / K)
    mag2 = np.abs(den) ** 2
    out = np.zeros(K)
    ok = mag2 > 1e-10
    out[ok] = 1.0 / mag2[ok]
    return out


def influence_function(box, mesh, alpha, p, k_e=K_E):
    """G(m) = k_e (4 pi / V) exp(-k^2 / 4 alpha^2) / k^2 * B(m), with G(0) = 0, full mesh."""
    box = np.asarray(box, dtype=np.float64)
    V = float(np.prod(box))
    comps = []
    for d in range(3):
        K = mesh[d]
        m = np.arange(K)
        m = np.where(m <= K // 2, m, m - K)  # centred integer index (Nyquist taken positive)
        comps.append(2.0 * math.pi * m / box[d])
    kx, ky, kz = np.meshgrid(*comps, indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    B = (bspline_modulus(mesh[0], p)[:, None, None] * bspline_modulus(mesh[1], p)[None, :, None]
         * bspline_modulus(mesh[2], p)[None, None, :])
    G = np.zeros_like(k2)
    nz = k2 > 0
    G[nz] = k_e * (4.0 * math.pi / V) * np.exp(-k2[nz] / (4.0 * alpha * alpha)) / k2[nz] * B[nz]
    return G


def _spline_setup(R, box, mesh, p):
    R = np.asarray(R, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    mesh = np.asarray(mesh, dtype=np.int64)
    u = R / box * mesh  # scaled fractional coordinates
    fl = np.floor(u)
    w = u - fl
    base = fl.astype(np.int64)
    Ms, dMs, idx = [], [], []
    for d in range(3):
        M, dM = bspline_table(w[:, d], p)
        Ms.append(M)
        dMs.append(dM)
        # weight M_p(w + j) belongs to mesh point floor(u) - j
        idx.append(np.mod(base[:, d, None] - np.arange(p)[None, :], mesh[d]))
    return Ms, dMs, idx


def pme_reciprocal(R, q, box, alpha, mesh, p, k_e=K_E, chunk=65536):
    """Smooth-PME reciprocal potential, field and energy (Alg. 2, steps 1-5)."""
    R = np.asarray(R, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    K1, K2, K3 = (int(k) for k in mesh)
    n = R.shape[0]
    # step 1: spread q_i M(u_x - kx) M(u_y - ky) M(u_z - kz) onto the mesh
    Q = np.zeros(K1 * K2 * K3)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        Ms, _, idx = _spline_setup(R[s:e], box, mesh, p)
        wgt = (q[s:e, None, None, None] * Ms[0][:, :, None, None] * Ms[1][:, None, :, None]
               * Ms[2][:, None, None, :])
        flat = ((idx[0][:, :, None, None] * K2 + idx[1][:, None, :, None]) * K3
                + idx[2][:, None, None, :])
        Q += np.bincount(flat.ravel(), weights=wgt.ravel(), minlength=K1 * K2 * K3)
    Q = Q.reshape(K1, K2, K3)
    # step 2: forward FFT;  step 3: influence multiply and energy
    Qh = np.fft.fftn(Q)
    G = influence_function(box, (K1, K2, K3), alpha, p, k_e)
    energy = 0.5 * float(np.sum(G * (Qh.real ** 2 + Qh.imag ** 2)))
    # step 4: unnormalised inverse FFT of G * Qh is the mesh potential dE/dQ
    phi = np.fft.ifftn(G * Qh).real * (K1 * K2 * K3)
    phif = phi.ravel()
    # step 5: gather v_i = sum theta_i phi and E_i = -sum grad(theta_i) phi
    v = np.zeros(n)
    E = np.zeros((n, 3))
    scale = np.array([K1, K2, K3], dtype=np.float64) / box
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        Ms, dMs, idx = _spline_setup(R[s:e], box, mesh, p)
        flat = ((idx[0][:, :, None, None] * K2 + idx[1][:, None, :, None]) * K3
                + idx[2][:, None, None, :])
        ph = phif[flat]
        tx = Ms[0][:, :, None, None]
        ty = Ms[1][:, None, :, None]
        tz = Ms[2][:, None, None, :]
        v[s:e] = np.sum(tx * ty * tz * ph, axis=(1, 2, 3))
        E[s:e, 0] = -scale[0] * np.sum(dMs[0][:, :, None, None] * ty * tz * ph, axis=(1, 2, 3))
        E[s:e, 1] = -scale[1] * np.sum(tx * dMs[1][:, None, :, None] * tz * ph, axis=(1, 2, 3))
        E[s:e, 2] = -scale[2] * np.sum(tx * ty * dMs[2][:, None, None, :] * ph, axis=(1, 2, 3))
    return v, E, energy


# ---------------------------------------------------------------------------
# Assembled operator
# ---------------------------------------------------------------------------

def coulomb_apply(R, q, sigma, box, alpha, r_c, k_e=K_E, recip="pme", mesh=None, order=4,
                  k_cut=None, gaussian_self=False, real_method="auto"):
    """v = Phi q, the field E (F = q * E) and the energy parts.

    ``recip`` is "pme" (mesh, order) or "ewald" (explicit k-sum).
    Returns a dict with v, E, energy (= 1/2 q.v) and the real / recip / self parts.
    """
    q = np.asarray(q, dtype=np.float64)
    v_r, E_r = real_space(R, q, sigma, box, alpha, r_c, k_e, method=real_method)
    if recip == "pme":
        v_k, E_k, e_k = pme_reciprocal(R, q, box, alpha, mesh, order, k_e)
    elif recip == "ewald":
        v_k, E_k, e_k = ewald_kspace(R, q, box, alpha, k_e, k_cut)
    else:
        raise ValueError(recip)
    v_s = self_potential(q, sigma, alpha, k_e, gaussian_self)
    v = v_r + v_k + v_s
    E = E_r + E_k
    return {
        "v": v,
        "E": E,
        "F": q[:, None] * E,
        "energy": 0.5 * float(q @ v),
        "energy_real": 0.5 * float(q @ v_r),
        "energy_recip": e_k,
        "energy_recip_from_v": 0.5 * float(q @ v_k),
        "energy_self": 0.5 * float(q @ v_s),
        "v_real": v_r,
        "v_recip": v_k,
    }


def phi_matrix(R, sigma, box, alpha, r_c, k_e=K_E, recip="pme", mesh=None, order=4, k_cut=None,
               gaussian_self=False):
    """Dense Phi (small N): real-space block plus the reciprocal operator applied to unit charges."""
    n = np.asarray(R).shape[0]
    Phi = real_space_matrix(R, sigma, box, alpha, r_c, k_e)
    eye = np.eye(n)
    for j in range(n):
        if recip == "pme":
            vk, _, _ = pme_reciprocal(R, eye[j], box, alpha, mesh, order, k_e)
        else:
            vk, _, _ = ewald_kspace(R, eye[j], box, alpha, k_e, k_cut)
        Phi[:, j] += vk
    Phi += np.diag(self_potential(np.ones(n), sigma, alpha, k_e, gaussian_self))
    return Phi
