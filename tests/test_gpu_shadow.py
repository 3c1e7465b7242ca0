"""GPU shadow XL-BOMD step (Sec. 3.5) against the oracle's step, FP64.

The oracle step uses its own smooth PME with the same mesh, order and cutoff,
so both sides integrate the same shadow dynamics.  Differences come only from
rounding order.
"""

import numpy as np
import pytest

from gpu_util import cuda_or_skip, dev_tensor, rel_max
from oracle import ewald, qeq
from workloads import water_box

pytestmark = pytest.mark.gpu


def _maxwell(w, T_eV, seed):
    rng = np.random.default_rng(seed)
    V = rng.standard_normal(w.R.shape) * np.sqrt(T_eV / (w.mass[:, None] * qeq.AMU_A2_FS2_IN_EV))
    return V - (w.mass[:, None] * V).sum(0) / w.mass.sum()


def _run_pair(w, n0, V0, steps, rank, k_d, dt, mesh, r_cut, alpha=0.34, skin=1.0):
    qg = cuda_or_skip()
    p = qg.make_params(w.n_atoms, w.box, alpha=alpha, r_cut=r_cut, skin=skin, mesh=mesh, order=4,
                       krylov_rank=rank, dissipation_k=k_d, dt=dt)
    s = qg.System(p)
    md = qg.ShadowMD(s, dev_tensor(w.chi), dev_tensor(w.eta), dev_tensor(w.sigma),
                     dev_tensor(w.mass), dev_tensor(w.R), dev_tensor(V0), dev_tensor(n0))
    md.init()

    def coul(R, x, need_field=True):
        o = ewald.coulomb_apply(R, x, w.sigma, w.box, alpha, r_cut, recip="pme", mesh=mesh,
                                order=4, gaussian_self=True)
        return o["v"], o["E"]

    osys = qeq.ShadowSystem(coul, w.chi, w.eta, w.mass, rank=rank, dt=dt, k_d=k_d)
    st = osys.init_state(w.R, V0, n0)
    g_e, o_e = [], []
    e = md.energy_dict()
    g_e.append(e["total"])
    o_e.append(st["e_kin"] + st["e_pot"])
    assert abs(e["kinetic"] - st["e_kin"]) < 1e-10 * max(1.0, st["e_kin"])
    assert rel_max(md.q.cpu().numpy(), st["q"]) < 1e-10
    # at an exact QEq fixed point f and Kf are rounding noise: compare on the scale of q
    assert np.abs(md.Kf.cpu().numpy() - st["Kf"]).max() < 1e-9 * np.abs(st["q"]).max()
    for _ in range(steps):
        md.step()
        st = osys.step(st)
        e = md.energy_dict()
        g_e.append(e["total"])
        o_e.append(st["e_kin"] + st["e_pot"])
    out = dict(R=md.R.cpu().numpy(), V=md.V.cpu().numpy(), q=md.q.cpu().numpy(),
               hist=md.n_hist.cpu().numpy(), F=md.F.cpu().numpy(), e=md.energy_dict())
    s.close()
    return out, st, np.array(g_e), np.array(o_e)


def test_shadow_md_648_50_steps():
    """216 molecules, r_c 9, K 32, p 4, dt 0.5 fs, rank 2, K_d 5, 50 steps."""
    w = water_box(216, seed=2503)
    Phi = ewald.phi_matrix(w.R, w.sigma, w.box, 0.34, 9.0, recip="pme", mesh=(32, 32, 32), order=4,
                           gaussian_self=True)
    qmin, _ = qeq.qeq_dense_solve(Phi, w.chi, w.eta, 0.0)
    V0 = _maxwell(w, 0.02585, seed=7)
    g, o, ge, oe = _run_pair(w, qmin, V0, 50, rank=2, k_d=5, dt=0.5, mesh=(32, 32, 32), r_cut=9.0)
    assert np.abs(g["R"] - o["R"]).max() < 1e-9
    assert rel_max(g["V"], o["V"]) < 1e-8
    assert rel_max(g["q"], o["q"]) < 1e-8
    assert rel_max(g["hist"], o["hist"]) < 1e-8
    assert rel_max(g["F"], o["F"]) < 1e-8
    assert np.abs(ge - oe).max() < 1e-8 * np.abs(oe).max()
    # the shadow charges stay neutral and the dynamics conserve energy
    assert abs(g["e"]["sum_q"]) < 1e-10
    assert np.abs(ge - ge[0]).max() < 5e-3


@pytest.mark.parametrize("rank,k_d", [(1, 3), (3, 7), (4, 5), (8, 5)])
def test_shadow_ranks_and_windows(rank, k_d):
    w = water_box(64, seed=rank + 3 * k_d)
    V0 = _maxwell(w, 0.02585, seed=rank)
    n0 = np.zeros(w.n_atoms)
    g, o, ge, oe = _run_pair(w, n0, V0, 6, rank=rank, k_d=k_d, dt=0.4, mesh=(20, 20, 20),
                             r_cut=6.0, skin=0.6)
    assert np.abs(g["R"] - o["R"]).max() < 1e-9
    assert rel_max(g["q"], o["q"]) < 1e-8
    assert rel_max(g["hist"], o["hist"]) < 1e-8


def test_neighbor_rebuild_during_run():
    """A small skin forces rebuilds inside the run; the trajectory still matches."""
    w = water_box(40, seed=21)
    V0 = _maxwell(w, 0.3, seed=3)  # hot, so atoms cross skin / 2 quickly
    g, o, ge, oe = _run_pair(w, np.zeros(w.n_atoms), V0, 12, rank=2, k_d=5, dt=0.5,
                             mesh=(16, 16, 16), r_cut=5.0, skin=0.05)
    assert np.abs(g["R"] - o["R"]).max() < 1e-9
    assert rel_max(g["q"], o["q"]) < 1e-8


def test_shadow_md_with_water_short_range():
    """Shadow MD with the built-in flexible-water V_short matches the oracle's step (FP64)."""
    from oracle import short_range

    qg = cuda_or_skip()
    w = water_box(64, seed=77)
    V0 = _maxwell(w, 0.02585, seed=5)
    n0 = np.zeros(w.n_atoms)
    mesh, r_cut, skin = (20, 20, 20), 6.0, 0.6
    p = qg.make_params(w.n_atoms, w.box, alpha=0.34, r_cut=r_cut, skin=skin, mesh=mesh, order=4,
                       krylov_rank=2, dissipation_k=5, dt=0.5, short_range=qg.QEQ_SHORT_WATER)
    s = qg.System(p)
    md = qg.ShadowMD(s, dev_tensor(w.chi), dev_tensor(w.eta), dev_tensor(w.sigma),
                     dev_tensor(w.mass), dev_tensor(w.R), dev_tensor(V0), dev_tensor(n0))
    md.init()

    def coul(R, x, need_field=True):
        o = ewald.coulomb_apply(R, x, w.sigma, w.box, 0.34, r_cut, recip="pme", mesh=mesh,
                                order=4, gaussian_self=True)
        return o["v"], o["E"]

    osys = qeq.ShadowSystem(coul, w.chi, w.eta, w.mass, rank=2, dt=0.5, k_d=5,
                            short=lambda R: short_range.water_short_range(R, w.box, r_cut))
    st = osys.init_state(w.R, V0, n0)
    e_short_ref = short_range.water_short_range(w.R, w.box, r_cut)[0]
    assert abs(md.energy_dict()["short"] - e_short_ref) < 1e-9 * max(1.0, abs(e_short_ref))
    for _ in range(10):
        md.step()
        st = osys.step(st)
    assert np.abs(md.R.cpu().numpy() - st["R"]).max() < 1e-9
    assert rel_max(md.F.cpu().numpy(), st["F"]) < 1e-8
    e = md.energy_dict()
    assert abs(e["total"] - (st["e_kin"] + st["e_pot"])) < 1e-8 * abs(st["e_pot"])
    s.close()


def test_graph_replay_equals_eager_steps():
    """qeq_shadow_step through the captured CUDA graph gives the eager trajectory."""
    qg = cuda_or_skip()
    import torch

    w = water_box(80, seed=33)
    V0 = _maxwell(w, 0.02585, seed=4)
    out = []
    for graphs in (False, True):
        p = qg.make_params(w.n_atoms, w.box, alpha=0.34, r_cut=6.0, skin=0.4, mesh=(20, 20, 20),
                           order=4, krylov_rank=2, dt=0.5)
        s = qg.System(p)
        qg._lib.qeq_set_graphs(s.ctx, graphs)
        md = qg.ShadowMD(s, dev_tensor(w.chi), dev_tensor(w.eta), dev_tensor(w.sigma),
                         dev_tensor(w.mass), dev_tensor(w.R), dev_tensor(V0),
                         dev_tensor(np.zeros(w.n_atoms)))
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            md.init(stream)
            for _ in range(15):  # the small skin forces rebuilds between replays
                md.step(1, stream)
            stream.synchronize()
        out.append((md.R.cpu().numpy(), md.q.cpu().numpy(), md.energy_dict()["total"],
                    qg.qeq_get_counters(s.ctx)))
        s.close()
    (R0, q0, e0, c0), (R1, q1, e1, c1) = out
    assert np.abs(R1 - R0).max() < 1e-12
    assert rel_max(q1, q0) < 1e-10
    assert abs(e1 - e0) < 1e-10 * abs(e0)
    assert c1[0] == c0[0] and c1[2] == c0[2]  # same kernel and apply counts either way


def test_packed_state_gives_the_same_trajectory():
    """ShadowMD.pack() re-homes the state into one buffer; the steps are unchanged."""
    qg = cuda_or_skip()
    import torch

    w = water_box(100, seed=31)
    V0 = _maxwell(w, 0.025852, 32)
    outs = []
    for packed in (False, True):
        p = qg.make_params(w.n_atoms, w.box, alpha=0.34, r_cut=7.0, skin=1.0, mesh=(24, 24, 24),
                           order=4, precision="fp32_mixed", krylov_rank=2, dt=0.5)
        s = qg.System(p)
        md = qg.ShadowMD(s, dev_tensor(w.chi), dev_tensor(w.eta), dev_tensor(w.sigma),
                         dev_tensor(w.mass), dev_tensor(w.R), dev_tensor(V0),
                         torch.zeros(w.n_atoms, dtype=torch.float64, device="cuda"))
        md.init()
        torch.cuda.synchronize()  # init ran on the default stream, the steps on another
        if packed:
            buf, (n_par, n_state, n_res) = md.pack()
            assert buf.numel() == n_par + n_state + n_res
            assert md.R.data_ptr() == buf[n_par:].data_ptr()
        stream = torch.cuda.Stream()
        for _ in range(6):
            md.step(1, stream)
        torch.cuda.synchronize()
        outs.append((md.R.cpu().numpy(), md.q.cpu().numpy(), md.energy_dict()["total"]))
        s.close()
    # the FP32 mesh spread adds with float atomics in an order that varies from
    # run to run, so the two trajectories agree to that rounding (a mis-homed
    # buffer would differ at O(1))
    np.testing.assert_allclose(outs[0][0], outs[1][0], rtol=0, atol=1e-6)
    np.testing.assert_allclose(outs[0][1], outs[1][1], rtol=0, atol=1e-5)
    assert abs(outs[0][2] - outs[1][2]) <= 1e-7 * abs(outs[0][2])
