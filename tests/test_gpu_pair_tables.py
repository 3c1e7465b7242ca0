"""The FP64 kernel's pair-function tables on the device equal the host
evaluation bit for bit (same tables, same bit indexing, same fused Horner
steps), so the host accuracy checks of tests/test_pair_tables.py hold for
what the kernel computes."""

import numpy as np
import pytest

from gpu_util import cuda_or_skip
from workloads import water_box

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", [0, 1])
def test_device_tables_equal_host_evaluation(which):
    qg = cuda_or_skip()
    import torch

    w = water_box(50, seed=5)
    p = qg.make_params(w.n_atoms, w.box, alpha=0.34, r_cut=7.5, skin=1.0, mesh=(16, 16, 16), order=4,
                       precision="fp64")
    s = qg.System(p)
    rng = np.random.default_rng(which)
    arg = np.concatenate([np.exp(rng.uniform(np.log(1e-3), np.log(100.0), 4000)),
                          2.0 ** np.arange(-6, 7), np.nextafter(2.0 ** np.arange(-6, 7), 0.0)])
    F, G, inn, kept = qg.qeq_pair_table_eval(0.34, 7.5 * 7.5, which, arg)
    assert kept > 0 and inn.any() and not inn.all()
    dev = torch.device("cuda", 0)
    a = torch.as_tensor(arg, device=dev)
    Fd = torch.full_like(a, float("nan"))
    Gd = torch.full_like(a, float("nan"))
    ind = torch.zeros(arg.size, dtype=torch.int32, device=dev)
    qg.qeq_selftest_pair64(s.ctx, which, a, Fd, Gd, ind)
    torch.cuda.synchronize()
    assert np.array_equal(ind.cpu().numpy(), inn)
    m = inn == 1
    assert np.array_equal(Fd.cpu().numpy()[m], F[m])
    assert np.array_equal(Gd.cpu().numpy()[m], G[m])
    s.close()


def test_fp32_context_has_no_pair_tables():
    qg = cuda_or_skip()
    import torch

    w = water_box(50, seed=5)
    p = qg.make_params(w.n_atoms, w.box, alpha=0.34, r_cut=7.5, skin=1.0, mesh=(16, 16, 16), order=4,
                       precision="fp32_mixed")
    s = qg.System(p)
    a = torch.ones(4, dtype=torch.float64, device="cuda")
    with pytest.raises(qg.QeqError):
        qg.qeq_selftest_pair64(s.ctx, 0, a, a.clone(), a.clone(),
                               torch.zeros(4, dtype=torch.int32, device="cuda"))
    s.close()
