"""Run-to-run repeatability of the apply (GPU).  The neighbour list, the
real-space sums and the reductions are deterministic; the mesh spread adds
with atomics (FP64: one per point; FP32-mixed: exact integer windows, then a
float reduction into the mesh), so repeated applies agree to that rounding.
The list itself must repeat bit for bit."""

import numpy as np
import pytest

from gpu_util import cuda_or_skip, dev_tensor
from workloads import random_neutral_charges, water_box

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32_mixed", 1e-5)])
def test_apply_repeats(precision, tol):
    qg = cuda_or_skip()
    w = water_box(400, seed=11)
    q = random_neutral_charges(w.n_atoms, seed=12, scale=0.4)
    p = qg.make_params(w.n_atoms, w.box, alpha=0.34, r_cut=8.0, skin=1.0, mesh=(32, 32, 32), order=4,
                       precision=precision)
    s = qg.System(p)
    R, qd, sg = dev_tensor(w.R), dev_tensor(q), dev_tensor(w.sigma)
    outs, lists = [], []
    for _ in range(2):
        s.neighbor_build(R)
        lists.append(s.neighbor_export())
        v, E, F, en = s.apply(R, qd, sg)
        outs.append((v.cpu().numpy().copy(), E.cpu().numpy().copy(), en.cpu().numpy().copy()))
    for a, b in zip(lists[0], lists[1]):
        assert np.array_equal(a, b)
    (v0, E0, e0), (v1, E1, e1) = outs
    assert np.abs(v1 - v0).max() <= tol * np.abs(v0).max()
    assert np.abs(E1 - E0).max() <= tol * np.abs(E0).max()
    assert abs(e1[0] - e0[0]) <= tol * (abs(e0[1]) + abs(e0[2]) + abs(e0[3]))
    s.close()
