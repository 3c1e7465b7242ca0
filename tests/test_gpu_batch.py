"""Batched shadow steps (qeq_batch_step): several systems advanced by one call give the
same trajectories as separate qeq_shadow_step calls (Sec. 3.5 step, serving form).

Each member runs the kernels of its own step, so FP64 results agree to the order of
the PME spread's atomics (1e-10).  Members join and leave between steps, lists are
rebuilt inside the batch, and a tolerance-driven member (no graph) rides along.
"""

import numpy as np
import pytest

from gpu_util import cuda_or_skip, dev_tensor, rel_max
from oracle import qeq
from workloads import serving_mesh_size, water_box

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _maxwell(w, T_eV, seed):
    rng = np.random.default_rng(seed)
    V = rng.standard_normal(w.R.shape) * np.sqrt(T_eV / (w.mass[:, None] * qeq.AMU_A2_FS2_IN_EV))
    return V - (w.mass[:, None] * V).sum(0) / w.mass.sum()


def _member(qg, n_mol, seed, skin=1.0, tol=0.0, T=0.02585):
    w = water_box(n_mol, seed=seed)
    K = serving_mesh_size(w.box[0])
    p = qg.make_params(w.n_atoms, w.box, alpha=0.34, r_cut=min(8.0, 0.49 * w.box[0] + 4.0),
                       skin=skin, mesh=(K, K, K), order=4, krylov_rank=6 if tol else 2,
                       krylov_tol=tol, dt=0.5)
    s = qg.System(p)
    md = qg.ShadowMD(s, dev_tensor(w.chi), dev_tensor(w.eta), dev_tensor(w.sigma),
                     dev_tensor(w.mass), dev_tensor(w.R), dev_tensor(_maxwell(w, T, seed)),
                     torch.zeros(w.n_atoms, dtype=torch.float64, device="cuda"))
    return s, md


def _state(md):
    return (md.R.cpu().numpy(), md.q.cpu().numpy(), md.F.cpu().numpy(), md.energy_dict()["total"])


def _same(a, b):
    assert np.abs(a[0] - b[0]).max() < 1e-10
    assert rel_max(a[1], b[1]) < 1e-10
    assert rel_max(a[2], b[2]) < 1e-10
    assert abs(a[3] - b[3]) < 1e-10 * abs(b[3])


# (molecules, seed, skin, Krylov tolerance): the second member's small skin and high
# temperature force rebuilds inside the batch; the last one has no step graph
SPECS = [(40, 71, 1.0, 0.0), (150, 72, 0.1, 0.0), (300, 73, 1.0, 0.0), (60, 74, 1.0, 0.05)]


def test_batch_steps_equal_separate_steps_with_joins_and_leaves():
    qg = cuda_or_skip()
    stream = torch.cuda.Stream()
    batch = qg.ShadowBatch()
    ref, bat = [], []
    for n_mol, seed, skin, tol in SPECS:
        ref.append(_member(qg, n_mol, seed, skin, tol))
        bat.append(_member(qg, n_mol, seed, skin, tol))
    with torch.cuda.stream(stream):
        for s, md in ref + bat:
            md.init(stream)
        # schedule of members per batch step: joins, leaves and a re-join
        plan = [[0, 1], [0, 1], [0, 1, 2], [0, 1, 2, 3], [0, 1, 2, 3], [1, 2, 3], [1, 2, 3], [0, 2]]
        counts = [0] * len(SPECS)
        for members in plan:
            batch.step([bat[k][1] for k in members], stream)
            for k in members:
                ref[k][1].step(1, stream)
                counts[k] += 1
        stream.synchronize()
    for k in range(len(SPECS)):
        _same(_state(bat[k][1]), _state(ref[k][1]))
    builds, launches = batch.stats()
    # one launch per step; a parent graph per distinct list of graph-replaying members
    # (member 3, tolerance-driven, runs kernel by kernel), or more when a member
    # re-captures its graph after a rebuild that grows or moves its list
    assert launches == len(plan)
    graphed = {tuple(k for k in m if SPECS[k][3] == 0.0) for m in plan}
    assert len(graphed) <= builds <= len(plan)
    rebuilds = qg.qeq_get_counters(bat[1][0].ctx)[1]
    assert rebuilds > 1  # the small-skin member rebuilt its list inside the batch
    batch.close()
    for s, _ in ref + bat:
        s.close()


def test_batch_rejects_bad_members():
    qg = cuda_or_skip()
    stream = torch.cuda.Stream()
    s, md = _member(qg, 20, 81)
    batch = qg.ShadowBatch()
    with torch.cuda.stream(stream):
        md.init(stream)
        with pytest.raises(qg.QeqError):  # the same member twice
            batch.step([md, md], stream)
        with pytest.raises(qg.QeqError):  # the legacy default stream cannot hold the graph
            qg._lib.qeq_batch_step(batch.h, [s.ctx], [md._prm], [md._st], 0)
        batch.step([md], stream)  # still usable
        stream.synchronize()
    assert np.isfinite(md.energy_dict()["total"])
    batch.close()
    s.close()


def test_batch_with_mixed_precision_members():
    """FP32-mixed and FP64 members in one batch: each follows its own separate steps
    (FP64 to 1e-10; FP32-mixed to the rounding order of its float mesh atomics)."""
    qg = cuda_or_skip()
    stream = torch.cuda.Stream()
    batch = qg.ShadowBatch()
    pairs = []
    for n_mol, seed, prec in ((50, 91, "fp32_mixed"), (120, 92, "fp64"), (200, 93, "fp32_mixed")):
        made = []
        for _ in range(2):
            w = water_box(n_mol, seed=seed)
            K = serving_mesh_size(w.box[0])
            p = qg.make_params(w.n_atoms, w.box, alpha=0.34, r_cut=8.0, skin=1.0, mesh=(K, K, K),
                               order=4, precision=prec, krylov_rank=2, dt=0.5)
            s = qg.System(p)
            md = qg.ShadowMD(s, dev_tensor(w.chi), dev_tensor(w.eta), dev_tensor(w.sigma),
                             dev_tensor(w.mass), dev_tensor(w.R), dev_tensor(_maxwell(w, 0.02585, seed)),
                             torch.zeros(w.n_atoms, dtype=torch.float64, device="cuda"))
            made.append((s, md))
        pairs.append((prec, made))
    with torch.cuda.stream(stream):
        for _, made in pairs:
            for s, md in made:
                md.init(stream)
        for _ in range(6):
            batch.step([made[0][1] for _, made in pairs], stream)
            for _, made in pairs:
                made[1][1].step(1, stream)
        stream.synchronize()
    for prec, made in pairs:
        a, b = _state(made[0][1]), _state(made[1][1])
        if prec == "fp64":
            _same(a, b)
        else:
            assert np.abs(a[0] - b[0]).max() < 1e-6 and rel_max(a[1], b[1]) < 1e-5
            assert abs(a[3] - b[3]) < 1e-7 * abs(b[3])
        for s, _ in made:
            s.close()
    batch.close()
