"""Serving loop (continuous batching of mixed-size requests) -- GPU.

The results of every request are the same alone and in the mix.  The only
difference allowed is the rounding order of the PME spread's floating-point
atomics: 1e-10 relative in FP64, 1e-5 in FP32-mixed.
"""

import numpy as np
import pytest

from gpu_util import cuda_or_skip, rel_max
from workloads import serving_mesh_size, water_box

pytestmark = pytest.mark.gpu


def _requests(precision):
    from paper_2503_21176_gb300.serve import request_from_box

    reqs = []
    sizes = [34, 120, 500, 80, 1000, 40, 300, 700, 60, 200]  # molecules: 102 .. 3000 atoms
    for k, nm in enumerate(sizes):
        w = water_box(nm, seed=900 + k)
        K = serving_mesh_size(w.box[0])
        rng = np.random.default_rng(k)
        V = rng.standard_normal(w.R.shape) * 0.01
        kind = "md" if k % 2 else "qeq"
        reqs.append(request_from_box(k, kind, w, (K, K, K), V=V, steps=5 if kind == "md" else 0,
                                     arrival=0.002 * k, precision=precision))
    return reqs


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32_mixed", 1e-5)])
def test_results_alone_equal_results_in_mix(precision, tol):
    cuda_or_skip()
    from paper_2503_21176_gb300.serve import Server

    reqs = _requests(precision)
    mixed, stats = Server(max_inflight=4).serve(reqs, realtime=True)
    assert stats["requests"] == len(reqs) and stats["max_concurrent"] >= 2
    # the MD requests were stepped by batched steps (one graph for the members of a step)
    mb = stats["md_batching"]
    assert mb["member_steps"] == sum(r.steps for r in reqs if r.kind == "md")
    assert mb["batch_steps"] <= mb["member_steps"] and mb["parent_graphs_built"] >= 1
    alone = [Server(max_inflight=1).serve([r], realtime=False)[0][0] for r in reqs]
    for a, m in zip(alone, mixed):
        assert a.rid == m.rid
        assert rel_max(m.q, a.q) < tol
        assert rel_max(m.F, a.F) < tol
        assert rel_max(m.R, a.R) < tol
        assert abs(m.energies["total"] - a.energies["total"]) < tol * max(1.0, abs(a.energies["total"]))


def test_admission_by_memory_budget():
    """A budget that fits one request at a time still serves the whole stream, one by one."""
    cuda_or_skip()
    from paper_2503_21176_gb300.serve import Server, estimate_device_bytes

    reqs = _requests("fp32_mixed")[:6]
    budget = max(estimate_device_bytes(r) for r in reqs)
    res, stats = Server(max_inflight=4, hbm_budget=budget).serve(reqs, realtime=False)
    assert stats["requests"] == 6
    assert stats["max_concurrent"] >= 1
    with pytest.raises(MemoryError):
        Server(max_inflight=2, hbm_budget=1024).serve(reqs[:1])


def test_batched_and_unbatched_md_agree():
    """The same stream with MD steps batched across requests and stepped one request at
    a time gives the same results (FP64: to the spread's atomic order)."""
    cuda_or_skip()
    from paper_2503_21176_gb300.serve import Server

    reqs = _requests("fp64")
    a, _ = Server(max_inflight=4, batch_md=True).serve(reqs, realtime=False)
    b, sb = Server(max_inflight=4, batch_md=False).serve(reqs, realtime=False)
    assert sb["md_batching"] is None
    for x, y in zip(a, b):
        assert rel_max(x.R, y.R) < 1e-10 and rel_max(x.q, y.q) < 1e-10
