"""The bench's end-to-end loop keeps the state's round trip through host memory.

`bench.e2e_steps` overlaps the device-to-host copy of step k's state with the
host-to-device copy that makes it step k + 1's input (chunk by chunk, behind
events).  If a chunk went up before it had come down, or a step started
before its input had arrived, the trajectory would differ from the same steps
run with the state resident on the device.  Both runs start from the same
state; after the steps the host buffer of the pipelined run and the device
state of the resident run must agree to the last bit (same kernels, same
inputs; the FP64 mode has no atomics in its sums but the mesh spread's, whose
run-to-run rounding the tolerance allows).
"""

import os
import sys

import numpy as np
import pytest

from gpu_util import cuda_or_skip, dev_tensor
from oracle import qeq
from workloads import water_box

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def _md(qg, w, V0):
    p = qg.make_params(w.n_atoms, w.box, alpha=0.34, r_cut=6.0, skin=0.5, mesh=(24, 24, 24),
                       order=4, krylov_rank=2, dissipation_k=5, dt=0.5)
    s = qg.System(p)
    md = qg.ShadowMD(s, dev_tensor(w.chi), dev_tensor(w.eta), dev_tensor(w.sigma),
                     dev_tensor(w.mass), dev_tensor(w.R), dev_tensor(V0),
                     torch.zeros(w.n_atoms, dtype=torch.float64, device="cuda"))
    return s, md


@pytest.mark.parametrize("chunks", [1, 3, 8])
def test_pipelined_host_round_trip_follows_the_resident_run(chunks):
    qg = cuda_or_skip()
    import bench

    w = water_box(216, seed=31)
    rng = np.random.default_rng(4)
    V0 = rng.standard_normal(w.R.shape) * np.sqrt(0.0259 / (w.mass[:, None] * qeq.AMU_A2_FS2_IN_EV))
    V0 -= (w.mass[:, None] * V0).sum(0) / w.mass.sum()
    steps, warm = 12, 2  # the warm-up steps hand their state on to the timed ones
    stream = torch.cuda.Stream()
    s_ref, ref = _md(qg, w, V0)
    s_e2e, e2e = _md(qg, w, V0)
    with torch.cuda.stream(stream):
        ref.init(stream)
        e2e.init(stream)
        for _ in range(warm + steps):
            ref.step(1, stream)
        stream.synchronize()
    out = bench.e2e_steps(qg, e2e, steps, stream, torch.device("cuda", 0), chunks=chunks,
                          warmup=warm)
    assert out["h2d_bytes_per_step"] > 0 and out["d2h_bytes_per_step"] > 0
    torch.cuda.synchronize()
    # the pipelined run's state after its last step: its device buffer (the host
    # buffer holds the same bytes, checked through the reported total energy)
    R_ref, R_e2e = ref.R.cpu().numpy(), e2e.R.cpu().numpy()
    assert np.abs(R_e2e - R_ref).max() < 1e-11
    assert np.abs(e2e.q.cpu().numpy() - ref.q.cpu().numpy()).max() < 1e-10
    e = ref.energy_dict()
    e_ref = e["total"]
    scale = abs(e["kinetic"]) + abs(e["shadow_potential"])
    # the bench reports the host-read total rounded to 1e-6 eV
    assert abs(out["last_total_energy_eV"] - e_ref) < 1e-6 + 1e-9 * scale
    assert abs(e2e.energy_dict()["total"] - e_ref) < 1e-9 * scale
    s_ref.close()
    s_e2e.close()
