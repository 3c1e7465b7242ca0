"""FP32-mixed shadow XL-BOMD steps (Sec. 3.5) against the FP64 oracle step.

FP32-mixed is the throughput mode: the pair sum, spreading, FFT and gather run
in FP32, and the charges, Krylov kernel, reductions and integrator in FP64.
The oracle integrates the same shadow dynamics in FP64 (its own PME on the
same mesh, order and cutoff).  The bounds are those of the mode, stated for a
Coulomb apply (relative RMS force 1e-4, potential 1e-5 of its largest value)
and carried through five steps:

* q = -(chi + v + lambda) / u, so a potential error dv moves q by at most
  2 max|dv| / min(u); the bound takes the mode's 1e-5 max|v|.
* Positions move by dt^2 F / m per step.  Over five steps the sum of the
  drift factors is 15 dt^2, so a relative force error of 1e-4 moves R by at
  most 15 dt^2 1e-4 max|F| / (m_H * mass_unit); the bound keeps that.
* The total energy is a sum of parts that cancel; its error is held to 1e-6
  of the magnitude of the shadow energy's terms (sum |q chi| + sum u q^2 / 2
  + |q.v| + |n.v| / 2).
"""

import numpy as np
import pytest

from gpu_util import cuda_or_skip, dev_tensor
from oracle import ewald, qeq
from workloads import water_box

pytestmark = pytest.mark.gpu

ALPHA, DT, RANK, KD, STEPS = 0.34, 0.5, 2, 5, 5


def _maxwell(w, T_eV, seed):
    rng = np.random.default_rng(seed)
    V = rng.standard_normal(w.R.shape) * np.sqrt(T_eV / (w.mass[:, None] * qeq.AMU_A2_FS2_IN_EV))
    return V - (w.mass[:, None] * V).sum(0) / w.mass.sum()


@pytest.mark.parametrize("n_mol,r_cut,K", [(216, 9.0, 32), (1000, 8.0, 32)])
def test_fp32_mixed_steps_follow_the_fp64_oracle(n_mol, r_cut, K):
    qg = cuda_or_skip()
    w = water_box(n_mol, seed=2503 if n_mol == 216 else 2600)
    mesh = (K, K, K)

    def coul(R, x, need_field=True):
        o = ewald.coulomb_apply(R, x, w.sigma, w.box, ALPHA, r_cut, recip="pme", mesh=mesh,
                                order=4, gaussian_self=True)
        return o["v"], o["E"]

    # n(0): the QEq charges at t = 0 (oracle GMRES to 1e-10), as in a production start
    n0, _, _ = qeq.qeq_gmres(lambda x: coul(w.R, x, False)[0], w.chi, w.eta,
                             np.zeros(w.n_atoms), 1e-10,
                             precond=w.eta + ewald.K_E * np.sqrt(2 / np.pi) / w.sigma)
    V0 = _maxwell(w, 0.025852, seed=11)
    p = qg.make_params(w.n_atoms, w.box, alpha=ALPHA, r_cut=r_cut, skin=1.0, mesh=mesh, order=4,
                       precision="fp32_mixed", krylov_rank=RANK, dissipation_k=KD, dt=DT)
    s = qg.System(p)
    md = qg.ShadowMD(s, dev_tensor(w.chi), dev_tensor(w.eta), dev_tensor(w.sigma),
                     dev_tensor(w.mass), dev_tensor(w.R), dev_tensor(V0), dev_tensor(n0))
    md.init()
    osys = qeq.ShadowSystem(coul, w.chi, w.eta, w.mass, rank=RANK, dt=DT, k_d=KD)
    st = osys.init_state(w.R, V0, n0)
    h_mass = float(w.mass.min()) * qeq.AMU_A2_FS2_IN_EV
    for k in range(STEPS):
        md.step()
        st = osys.step(st)
        q_g, F_g, R_g = md.q.cpu().numpy(), md.F.cpu().numpy(), md.R.cpu().numpy()
        n = st["hist"][0]
        v_n, _ = coul(st["R"], n)
        # relative RMS force
        rms = np.sqrt(np.mean((F_g - st["F"]) ** 2) / np.mean(st["F"] ** 2))
        assert rms < 1e-4, f"step {k + 1}: relative RMS force {rms:.2e}"
        # charges
        q_bound = 2 * 1e-5 * np.abs(v_n).max() / w.eta.min()
        dq = np.abs(q_g - st["q"]).max()
        assert dq < q_bound, f"step {k + 1}: max |dq| {dq:.2e} > {q_bound:.2e}"
        # positions
        steps_done = k + 1
        drift = steps_done * (steps_done + 1) / 2
        R_bound = drift * DT * DT * 1e-4 * np.abs(st["F"]).max() / h_mass
        dR = np.abs(R_g - st["R"]).max()
        assert dR < R_bound, f"step {k + 1}: max |dR| {dR:.2e} > {R_bound:.2e}"
        # total energy
        e = md.energy_dict()
        scale = (np.abs(st["q"] * w.chi).sum() + 0.5 * (w.eta * st["q"] ** 2).sum()
                 + abs(st["q"] @ v_n) + 0.5 * abs(n @ v_n))
        de = abs(e["total"] - (st["e_kin"] + st["e_pot"]))
        assert de < 1e-6 * scale, f"step {k + 1}: |dE| {de:.2e} > {1e-6 * scale:.2e}"
    s.close()
