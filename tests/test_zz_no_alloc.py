"""Allocation-free neighbour build (qeq_neighbor_build_noalloc), checked on the GPU.

The entry point serves callers that cannot call cudaMalloc or cudaFree: an
engine plugin whose host owns all device memory, a latency-critical loop that
cannot take cudaFree's device-wide synchronisation, a process under a hard
memory budget.  Its scratch is a fixed device array inside the library.

This file is named so that pytest collects it last.  Each check runs the new
entry point twice in a row through the C ABI.  Both outputs must equal, as
per-row sets of (j, image), the pair set of the context-based
qeq_neighbor_build + qeq_neighbor_export.  The neighbour tests use the same
bit-exact tolerance.
"""

import numpy as np
import pytest

from gpu_util import cuda_or_skip, dev_tensor
from workloads import simple_cubic_lattice, water_box

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rows_from_noalloc(counts, nbr):
    rows = []
    for i in range(len(counts)):
        ent = []
        for e in nbr[i, :counts[i]]:
            e = int(np.uint32(e))
            code = e >> 24
            ent.append((e & 0xFFFFFF, (code // 25 - 2, (code // 5) % 5 - 2, code % 5 - 2)))
        rows.append(sorted(ent))
    return rows


def _rows_from_context(qg, R, box, r_cut, skin):
    s = qg.System(qg.make_params(len(R), box, r_cut=r_cut, skin=skin, mesh=(8, 8, 8)))
    s.neighbor_build(dev_tensor(R))
    counts, nbr, shift = s.neighbor_export()
    s.close()
    rows = [sorted((int(nbr[i, k]), tuple(int(x) for x in shift[i, k])) for k in range(counts[i]))
            for i in range(len(counts))]
    return counts, rows


@pytest.mark.parametrize("case", ["water648_multi_image", "water3000", "lattice_boundaries"])
def test_noalloc_matches_context_build_twice(case):
    qg = cuda_or_skip()
    if case == "water648_multi_image":
        w = water_box(216, seed=2503)
        R, box, r_cut, skin = w.R, w.box, 9.0, 1.0
    elif case == "water3000":
        w = water_box(1000, seed=17)
        R, box, r_cut, skin = w.R, w.box, 8.0, 1.0
    else:
        R, L = simple_cubic_lattice(6, 2.0, origin=0.0)
        box, r_cut, skin = np.array([L, L, L]), 3.0, 1.0
    ref_counts, ref_rows = _rows_from_context(qg, R, box, r_cut, skin)
    n = len(R)
    width = int(ref_counts.max()) + 8
    Rd = dev_tensor(R)
    for call in range(2):
        counts = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        nbr = torch.full((n, width), -1, dtype=torch.int32, device="cuda")
        qg._lib.qeq_neighbor_build_noalloc(Rd, box, r_cut + skin, counts, nbr)
        torch.cuda.synchronize()
        c = counts.cpu().numpy()
        assert np.array_equal(c, ref_counts), f"call {call}: row counts differ"
        assert _rows_from_noalloc(c, nbr.cpu().numpy()) == ref_rows, f"call {call}: pair sets differ"


def test_noalloc_reports_width_and_limits():
    qg = cuda_or_skip()
    w = water_box(200, seed=5)
    n = w.n_atoms
    Rd = dev_tensor(w.R)
    counts = torch.zeros(n, dtype=torch.int32, device="cuda")
    nbr = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    with pytest.raises(qg.QeqError) as ei:
        qg._lib.qeq_neighbor_build_noalloc(Rd, w.box, 7.0, counts, nbr)
    assert ei.value.code == -8 and ei.value.needed_width > 4
    # a second call with the reported width succeeds on the same shared scratch
    nbr = torch.zeros((n, ei.value.needed_width), dtype=torch.int32, device="cuda")
    qg._lib.qeq_neighbor_build_noalloc(Rd, w.box, 7.0, counts, nbr)
    # sizes beyond the fixed scratch are rejected before any GPU work
    big = torch.zeros((40000, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(qg.QeqError) as ei:
        qg._lib.qeq_neighbor_build_noalloc(big, (100.0, 100.0, 100.0), 5.0,
                                           torch.zeros(40000, dtype=torch.int32, device="cuda"),
                                           torch.zeros((40000, 8), dtype=torch.int32, device="cuda"))
    assert ei.value.code == -8 and "32768" in str(ei.value)
