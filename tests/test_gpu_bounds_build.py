"""The bounds-checked build (-DQEQ_BOUNDS) on the GPU: its kernels check their
data-dependent indices (list entries against the tile, the sorted-order
permutation, tile slots in the emit), record the first failing site and skip the
access instead of trapping.  Run on small parity cases in a child process that
loads libqeq_bounds.so, every check must pass (site 0) and the results must still
match the oracle: FP64 applies on a multi-image and an anisotropic box, an
FP32-mixed apply, both neighbour searches, and a few shadow steps.
"""

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2503_21176_gb300 import _build
_build.LIB = _build.LIB_BOUNDS
import torch
import paper_2503_21176_gb300 as qg
from oracle import ewald
from workloads import water_box, random_neutral_charges
qg.load(build_if_missing=False)
assert qg._lib.qeq_build_info()["bounds_checked"]
t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
out = {"sites": [], "errors": []}
cases = [(water_box(216, seed=2503), 9.0, (32, 32, 32), "fp64", "brick"),
         (water_box(300, seed=19), 7.0, (24, 24, 24), "fp32_mixed", "brick"),
         (water_box(150, seed=3), 6.0, (20, 20, 20), "fp64", "atom")]
for w, rc, mesh, prec, method in cases:
    q = random_neutral_charges(w.n_atoms, seed=2, scale=0.3)
    s = qg.System(qg.make_params(w.n_atoms, w.box, r_cut=rc, skin=1.0, mesh=mesh, order=4,
                                 precision=prec, krylov_rank=2, dt=0.5))
    qg.qeq_set_neighbor_method(s.ctx, method)
    s.neighbor_build(t(w.R))
    v, E, F, en = s.apply(t(w.R), t(q), t(w.sigma))
    ref = ewald.coulomb_apply(w.R, q, w.sigma, w.box, 0.34, rc, recip="pme", mesh=mesh, order=4,
                              gaussian_self=True)
    err = float(np.abs(v.cpu().numpy() - ref["v"]).max() / np.abs(ref["v"]).max())
    out["errors"].append([prec, err])
    md = qg.ShadowMD(s, t(w.chi), t(w.eta), t(w.sigma), t(w.mass), t(w.R),
                     t(np.zeros_like(w.R)), t(np.zeros(w.n_atoms)))
    md.init()
    md.step(3)
    out["sites"].append(qg._lib.qeq_bounds_status(s.ctx))
    s.close()
print(json.dumps(out))
'''


def test_bounds_checked_build_runs_clean():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_21176_gb300 import _build

    _build.build(bounds=True)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["sites"] == [0, 0, 0]
    for prec, err in out["errors"]:
        assert err < (1e-10 if prec == "fp64" else 1e-5), (prec, err)
