"""Differentiation of E(q, R) through the CUDA apply (C4 workload) -- GPU.

dE/dq and dE/dR from the autograd backward are checked against central finite
differences of the same FP64 energy on 64 random atoms (h = 1e-5 A, 1e-6 e).
They are also checked against the oracle's analytic forces: smooth PME on the
same mesh (parity), and the explicit k-sum Ewald (method accuracy).  FP32-mixed
gradients are checked against the FP64 ones.
"""

import numpy as np
import pytest

from gpu_util import cuda_or_skip, dev_tensor, rel_max
from oracle import ewald
from workloads import random_neutral_charges, water_box

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _setup(w, precision, mesh):
    qg = cuda_or_skip()
    p = qg.make_params(w.n_atoms, w.box, alpha=0.34, r_cut=8.0, skin=1.0, mesh=mesh, order=4,
                       precision=precision)
    s = qg.System(p)
    s.neighbor_build(dev_tensor(w.R))
    return qg, s


def _grads(qg, s, w, q):
    R = dev_tensor(w.R).requires_grad_(True)
    qt = dev_tensor(q).requires_grad_(True)
    E = qg.coulomb_energy(s, R, qt, dev_tensor(w.sigma))
    E.backward()
    return float(E.item()), qt.grad.cpu().numpy(), R.grad.cpu().numpy()


@pytest.fixture(scope="module")
def box24k():
    w = water_box(8000, seed=2505)  # 24,000 atoms, L 62.10 A
    q = random_neutral_charges(w.n_atoms, seed=4, scale=0.4)
    return w, q


def test_backward_matches_finite_differences_fp64(box24k):
    w, q = box24k
    qg, s = _setup(w, "fp64", (64, 64, 64))
    E0, gq, gR = _grads(qg, s, w, q)
    R0 = dev_tensor(w.R)
    sig = dev_tensor(w.sigma)
    rng = np.random.default_rng(0)
    atoms = rng.choice(w.n_atoms, 64, replace=False)

    def energy(Rx, qx):
        return float(s.apply(Rx, qx, sig, field=False)[3][0].item())

    qd = dev_tensor(q)
    hq, hr = 1e-6, 1e-5
    # E is quadratic in q, so the central difference in q has no truncation error:
    # what remains is the rounding of a 24k-term energy, about eps * sum|q v| / h.
    noise = 50 * np.finfo(float).eps * float(np.sum(np.abs(q * gq)))
    for i in atoms:
        qp, qm = qd.clone(), qd.clone()
        qp[i] += hq
        qm[i] -= hq
        fd = (energy(R0, qp) - energy(R0, qm)) / (2 * hq)
        assert abs(fd - gq[i]) < noise / hq
    for i in atoms[:16]:
        for d in range(3):
            Rp, Rm = R0.clone(), R0.clone()
            Rp[i, d] += hr
            Rm[i, d] -= hr
            fd = (energy(Rp, qd) - energy(Rm, qd)) / (2 * hr)
            assert abs(fd - gR[i, d]) < noise / hr + 1e-6 * abs(gR[i, d])
    s.close()


def test_backward_matches_oracle_forces(box24k):
    """-dE/dR equals the oracle PME force (parity) and the exact k-sum force (accuracy)."""
    w, q = box24k
    qg, s = _setup(w, "fp64", (64, 64, 64))
    E0, gq, gR = _grads(qg, s, w, q)
    s.close()
    rows = np.random.default_rng(1).choice(w.n_atoms, 64, replace=False)
    vr, Er = ewald.real_space(w.R, q, w.sigma, w.box, 0.34, 8.0, rows=rows)
    vk, Ek, _ = ewald.pme_reciprocal(w.R, q, w.box, 0.34, (64, 64, 64), 4)
    F_pme = q[rows, None] * (Er + Ek[rows])
    assert rel_max(-gR[rows], F_pme) < 1e-10
    vs = ewald.self_potential(q, w.sigma, 0.34, gaussian_self=True)
    assert rel_max(gq[rows], vr + vk[rows] + vs[rows]) < 1e-10
    vk_e, Ek_e, _ = ewald.ewald_kspace(w.R, q, w.box, 0.34, k_cut=ewald.kspace_cutoff(0.34, 1e-10))
    F_ew = q[rows, None] * (Er + Ek_e[rows])
    err = np.sqrt(np.mean((-gR[rows] - F_ew) ** 2) / np.mean(F_ew ** 2))
    assert err < 5e-4


def test_fp32_mixed_backward_close_to_fp64(box24k):
    w, q = box24k
    qg, s64 = _setup(w, "fp64", (64, 64, 64))
    _, gq64, gR64 = _grads(qg, s64, w, q)
    s64.close()
    qg, s32 = _setup(w, "fp32_mixed", (64, 64, 64))
    _, gq32, gR32 = _grads(qg, s32, w, q)
    s32.close()
    assert np.sqrt(np.mean((gR32 - gR64) ** 2) / np.mean(gR64 ** 2)) < 1e-4
    assert rel_max(gq32, gq64) < 1e-5
