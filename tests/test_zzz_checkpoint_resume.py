"""Resuming a shadow XL-BOMD run from its checkpoint continues the trajectory
(GPU, FP64).  The two continuations differ only in summation order (the
resumed run builds its neighbour list at the checkpoint positions, and the
FP64 mesh spread adds with atomics), so they agree to rounding, not bit for
bit."""

import numpy as np
import pytest

from gpu_util import cuda_or_skip, dev_tensor
from workloads import water_box

pytestmark = pytest.mark.gpu

AMU_A2_FS2_IN_EV = 103.6427


def _system(qg, w, dt=0.5):
    p = qg.make_params(w.n_atoms, w.box, alpha=0.34, r_cut=7.0, skin=1.0, mesh=(24, 24, 24), order=4,
                       precision="fp64", krylov_rank=2, dt=dt)
    return qg.System(p)


def test_resume_continues_the_trajectory(tmp_path):
    qg = cuda_or_skip()
    import torch

    w = water_box(100, seed=31)
    rng = np.random.default_rng(32)
    V0 = rng.standard_normal(w.R.shape) * np.sqrt(0.025852 / (w.mass[:, None] * AMU_A2_FS2_IN_EV))
    V0 -= (w.mass[:, None] * V0).sum(0) / w.mass.sum()
    path = tmp_path / "md.npz"

    s1 = _system(qg, w)
    md = qg.ShadowMD(s1, dev_tensor(w.chi), dev_tensor(w.eta), dev_tensor(w.sigma),
                     dev_tensor(w.mass), dev_tensor(w.R), dev_tensor(V0),
                     torch.zeros(w.n_atoms, dtype=torch.float64, device="cuda"))
    md.init()
    torch.cuda.synchronize()
    md.step(4)
    md.checkpoint(path, step=4)
    md.step(4)
    torch.cuda.synchronize()
    R_a, q_a, e_a = md.R.cpu().numpy(), md.q.cpu().numpy(), md.energy_dict()["total"]
    s1.close()

    s2 = _system(qg, w)
    md2, step = qg.ShadowMD.resume(s2, path)
    assert step == 4
    md2.step(4)
    torch.cuda.synchronize()
    np.testing.assert_allclose(md2.R.cpu().numpy(), R_a, rtol=0, atol=1e-9)
    np.testing.assert_allclose(md2.q.cpu().numpy(), q_a, rtol=0, atol=1e-9)
    assert abs(md2.energy_dict()["total"] - e_a) <= 1e-10 * abs(e_a)
    s2.close()

    s3 = _system(qg, w, dt=0.25)
    with pytest.raises(ValueError, match="dt"):
        qg.ShadowMD.resume(s3, path)
    s3.close()
