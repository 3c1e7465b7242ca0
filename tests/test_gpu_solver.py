"""Regular QEq by GMRES and regular BO-MD on the GPU against the oracle (Sec. 3.4, Sec. 4.1),
and the tolerance-driven shadow Krylov kernel (Sec. 3.5, Eq. Jnddot)."""

import numpy as np
import pytest

from gpu_util import cuda_or_skip, dev_tensor, rel_max
from oracle import ewald, qeq, short_range
from workloads import water_box

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
MESH, RC, ALPHA = (24, 24, 24), 6.0, 0.34


def _coul(w):
    def f(R, x, need_field=True):
        o = ewald.coulomb_apply(R, x, w.sigma, w.box, ALPHA, RC, recip="pme", mesh=MESH, order=4,
                                gaussian_self=True)
        return o["v"], o["E"]
    return f


def _system(qg, w, **kw):
    p = qg.make_params(w.n_atoms, w.box, alpha=ALPHA, r_cut=RC, skin=0.5, mesh=MESH, order=4, **kw)
    s = qg.System(p)
    s.neighbor_build(dev_tensor(w.R))
    return s


def test_gmres_solution_matches_dense_pme_qeq():
    qg = cuda_or_skip()
    w = water_box(40, seed=12)
    Phi = ewald.phi_matrix(w.R, w.sigma, w.box, ALPHA, RC, recip="pme", mesh=MESH, order=4,
                           gaussian_self=True)
    qd, lam = qeq.qeq_dense_solve(Phi, w.chi, w.eta)
    s = _system(qg, w)
    q = torch.zeros(w.n_atoms, dtype=torch.float64, device="cuda")
    info = qg.qeq_solve(s.ctx, dev_tensor(w.R), dev_tensor(w.chi), dev_tensor(w.eta),
                        dev_tensor(w.sigma), q, tol=1e-12)
    assert info["rel_residual"] <= 1e-12
    assert rel_max(q.cpu().numpy(), qd) < 1e-9
    assert abs(info["lambda"] - lam) < 1e-9 * abs(lam)
    s.close()


@pytest.mark.parametrize("restart", [5, 64])
def test_gmres_restarts_reach_dense_solution(restart):
    """Short restarts (several cycles) and the longest basis both reach the dense answer."""
    qg = cuda_or_skip()
    w = water_box(40, seed=16)
    Phi = ewald.phi_matrix(w.R, w.sigma, w.box, ALPHA, RC, recip="pme", mesh=MESH, order=4,
                           gaussian_self=True)
    qd, lam = qeq.qeq_dense_solve(Phi, w.chi, w.eta)
    s = _system(qg, w)
    q = torch.zeros(w.n_atoms, dtype=torch.float64, device="cuda")
    info = qg.qeq_solve(s.ctx, dev_tensor(w.R), dev_tensor(w.chi), dev_tensor(w.eta),
                        dev_tensor(w.sigma), q, tol=1e-11, restart=restart, max_iter=400)
    assert info["rel_residual"] <= 1e-11
    assert rel_max(q.cpu().numpy(), qd) < 1e-8
    s.close()


def test_gmres_iteration_counts_match_oracle():
    """Same algorithm on both sides: the iteration counts to each tolerance agree (+-1)."""
    qg = cuda_or_skip()
    w = water_box(40, seed=13)
    s = _system(qg, w)
    coul = _coul(w)
    d = w.eta + ewald.K_E * np.sqrt(2 / np.pi) / w.sigma  # the library's Jacobi diagonal
    for tol in (1e-1, 1e-3, 1e-6):
        q = torch.zeros(w.n_atoms, dtype=torch.float64, device="cuda")
        info = qg.qeq_solve(s.ctx, dev_tensor(w.R), dev_tensor(w.chi), dev_tensor(w.eta),
                            dev_tensor(w.sigma), q, tol=tol)
        qo, lo, io = qeq.qeq_gmres(lambda x: coul(w.R, x, False)[0], w.chi, w.eta,
                                   np.zeros(w.n_atoms), tol, precond=d)
        assert abs(info["iterations"] - io["iterations"]) <= 1
        assert info["rel_residual"] <= tol
    s.close()


def test_bomd_trajectory_matches_oracle():
    qg = cuda_or_skip()
    w = water_box(27, seed=14)
    rng = np.random.default_rng(2)
    V0 = rng.standard_normal(w.R.shape) * np.sqrt(0.0259 / (w.mass[:, None] * 103.6427))
    s = _system(qg, w, short_range=qg.QEQ_SHORT_WATER, dt=0.4)
    bo = qg.BOMD(s, dev_tensor(w.chi), dev_tensor(w.eta), dev_tensor(w.sigma), dev_tensor(w.mass),
                 dev_tensor(w.R), dev_tensor(V0), torch.zeros(w.n_atoms, dtype=torch.float64,
                                                              device="cuda"), tol=1e-10)
    bo.init()
    d = w.eta + ewald.K_E * np.sqrt(2 / np.pi) / w.sigma
    osys = qeq.BOSystem(_coul(w), w.chi, w.eta, w.mass, dt=0.4, tol=1e-10, precond=d,
                        short=lambda R: short_range.water_short_range(R, w.box, RC))
    st = osys.init_state(w.R, V0, np.zeros(w.n_atoms))
    for _ in range(8):
        bo.step()
        st = osys.step(st)
    assert np.abs(bo.R.cpu().numpy() - st["R"]).max() < 1e-9
    assert rel_max(bo.q.cpu().numpy(), st["q"]) < 1e-7
    e = bo.energy_dict()
    assert abs(e["total"] - (st["e_kin"] + st["e_pot"])) < 1e-7 * abs(st["e_pot"])
    s.close()


@pytest.mark.parametrize("tol,steps", [(0.3, 4), (0.05, 4), (1e-3, 12)])
def test_adaptive_krylov_matches_oracle(tol, steps):
    qg = cuda_or_skip()
    w = water_box(27, seed=15)
    V0 = np.zeros_like(w.R)
    s = _system(qg, w, krylov_rank=6, krylov_tol=tol)
    md = qg.ShadowMD(s, dev_tensor(w.chi), dev_tensor(w.eta), dev_tensor(w.sigma),
                     dev_tensor(w.mass), dev_tensor(w.R), dev_tensor(V0),
                     torch.zeros(w.n_atoms, dtype=torch.float64, device="cuda"))
    md.init()
    osys = qeq.ShadowSystem(_coul(w), w.chi, w.eta, w.mass, rank=6, dt=0.5, k_d=5, krylov_tol=tol)
    st = osys.init_state(w.R, V0, np.zeros(w.n_atoms))
    ev = osys.evaluate(w.R, np.zeros(w.n_atoms))
    assert md.energy_dict()["applies"] == ev["applies"]
    assert rel_max(md.Kf.cpu().numpy(), st["Kf"]) < 1e-8
    for _ in range(steps):
        md.step()
        st = osys.step(st)
        assert md.energy_dict()["applies"] == st["applies"]
    assert rel_max(md.Kf.cpu().numpy(), st["Kf"]) < 1e-7
    assert np.abs(md.R.cpu().numpy() - st["R"]).max() < 1e-10
    s.close()
