"""User short-range model registered through qeq_set_short_range (FP64).

The callback here returns the oracle's flexible-water energy and forces on
the step's stream.  A run with it on a system whose parameter-selected model
is none must follow the run with the built-in flexible-water term: both add
the same V_short to the shadow potential of Eq. qeq_energy (Sec. 3.5) and to
the regular BO-MD potential (Sec. 3.4).  The tests also check that steps with
a callback are not captured into a CUDA graph, that capture resumes once it is
cleared, and that a failing callback fails the step with QEQ_ERR_INVALID and
its own exception as the cause.
"""

import numpy as np
import pytest

from gpu_util import cuda_or_skip, dev_tensor, rel_max
from oracle import qeq, short_range
from workloads import water_box

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
MESH, RC, SKIN = (20, 20, 20), 6.0, 0.6


def _maxwell(w, T_eV, seed):
    rng = np.random.default_rng(seed)
    V = rng.standard_normal(w.R.shape) * np.sqrt(T_eV / (w.mass[:, None] * qeq.AMU_A2_FS2_IN_EV))
    return V - (w.mass[:, None] * V).sum(0) / w.mass.sum()


def _oracle_model(w, calls):
    def fn(R):
        calls.append(1)
        e, F = short_range.water_short_range(R.cpu().numpy(), w.box, RC)
        return (torch.as_tensor(F, dtype=torch.float64, device=R.device),
                torch.tensor(e, dtype=torch.float64, device=R.device))
    return fn


def _params(qg, w, short):
    return qg.make_params(w.n_atoms, w.box, alpha=0.34, r_cut=RC, skin=SKIN, mesh=MESH, order=4,
                          krylov_rank=2, dissipation_k=5, dt=0.5, short_range=short)


def _shadow(qg, w, V0, short, model=None, steps=10):
    s = qg.System(_params(qg, w, short))
    if model is not None:
        s.set_short_range(model)
    md = qg.ShadowMD(s, dev_tensor(w.chi), dev_tensor(w.eta), dev_tensor(w.sigma),
                     dev_tensor(w.mass), dev_tensor(w.R), dev_tensor(V0),
                     torch.zeros(w.n_atoms, dtype=torch.float64, device="cuda"))
    stream = torch.cuda.Stream()  # graphs need a capturable (non-legacy) stream
    with torch.cuda.stream(stream):
        md.init(stream)
        for _ in range(steps):
            md.step(1, stream)
        stream.synchronize()
    return s, md, stream


def test_callback_follows_the_built_in_model_and_capture_resumes():
    qg = cuda_or_skip()
    w = water_box(64, seed=77)
    V0 = _maxwell(w, 0.02585, seed=5)
    s_ref, md_ref, _ = _shadow(qg, w, V0, qg.QEQ_SHORT_WATER)
    captures_ref, replays_ref = qg.qeq_graph_stats(s_ref.ctx)
    assert captures_ref >= 1 and replays_ref >= 9  # the built-in model runs from a graph

    calls = []
    s, md, stream = _shadow(qg, w, V0, qg.QEQ_SHORT_NONE, _oracle_model(w, calls))
    assert len(calls) == 11  # init + one evaluation per step
    assert qg.qeq_graph_stats(s.ctx) == (0, 0)  # never captured while a callback is set
    assert np.abs(md.R.cpu().numpy() - md_ref.R.cpu().numpy()).max() < 1e-9
    assert rel_max(md.F.cpu().numpy(), md_ref.F.cpu().numpy()) < 1e-8
    assert rel_max(md.q.cpu().numpy(), md_ref.q.cpu().numpy()) < 1e-8
    e, e_ref = md.energy_dict(), md_ref.energy_dict()
    assert abs(e["short"] - e_ref["short"]) < 1e-9 * max(1.0, abs(e_ref["short"]))
    assert abs(e["total"] - e_ref["total"]) < 1e-8 * abs(e_ref["shadow_potential"])

    # cleared: the parameter-selected term (none) is back and steps are captured again
    s.set_short_range(None)
    with torch.cuda.stream(stream):
        for _ in range(4):
            md.step(1, stream)
        stream.synchronize()
    assert len(calls) == 11
    captures, replays = qg.qeq_graph_stats(s.ctx)
    assert captures >= 1 and replays == 4
    assert md.energy_dict()["short"] == 0.0
    s.close()
    s_ref.close()


def test_callback_in_regular_bomd():
    qg = cuda_or_skip()
    w = water_box(27, seed=14)
    V0 = _maxwell(w, 0.0259, seed=2)
    out = []
    for short, model in ((qg.QEQ_SHORT_WATER, None), (qg.QEQ_SHORT_NONE, _oracle_model(w, []))):
        s = qg.System(_params(qg, w, short))
        if model is not None:
            s.set_short_range(model)
        s.neighbor_build(dev_tensor(w.R))
        bo = qg.BOMD(s, dev_tensor(w.chi), dev_tensor(w.eta), dev_tensor(w.sigma),
                     dev_tensor(w.mass), dev_tensor(w.R), dev_tensor(V0),
                     torch.zeros(w.n_atoms, dtype=torch.float64, device="cuda"), tol=1e-10)
        bo.init()
        bo.step()
        out.append((bo.R.cpu().numpy(), bo.F.cpu().numpy(), bo.energy_dict()))
        s.close()
    (R0, F0, e0), (R1, F1, e1) = out
    assert np.abs(R1 - R0).max() < 1e-9
    assert rel_max(F1, F0) < 1e-8
    assert abs(e1["short"] - e0["short"]) < 1e-9 * max(1.0, abs(e0["short"]))
    assert abs(e1["total"] - e0["total"]) < 1e-8 * abs(e0["potential"])


def test_failing_callback_fails_the_step_with_its_cause():
    qg = cuda_or_skip()
    w = water_box(27, seed=19)
    V0 = _maxwell(w, 0.0259, seed=3)
    s, md, stream = _shadow(qg, w, V0, qg.QEQ_SHORT_NONE, _oracle_model(w, []), steps=1)

    class ModelError(RuntimeError):
        pass

    def broken(R):
        raise ModelError("short-range model failed")

    s.set_short_range(broken)
    with torch.cuda.stream(stream):
        with pytest.raises(qg.QeqError) as info:
            md.step(1, stream)
    assert info.value.code == -1  # QEQ_ERR_INVALID
    assert isinstance(info.value.__cause__, ModelError)
    assert s.short_range_error is None  # handed over to the raised error
    # the context stays usable: with the model cleared the next steps run
    s.set_short_range(None)
    with torch.cuda.stream(stream):
        md.step(1, stream)
        stream.synchronize()
    assert np.isfinite(md.energy_dict()["total"])
    s.close()
