"""Checkpoint file of a shadow XL-BOMD run: round trip, shape and system checks (CPU)."""

import numpy as np
import pytest

import paper_2503_21176_gb300 as qg
from paper_2503_21176_gb300 import checkpoint as ck


def _params(n=12, dt=0.5):
    p = qg.qeq_params_default()
    p.n_atoms = n
    for d in range(3):
        p.box[d] = 9.0 + d
        p.mesh[d] = 16
    p.dt = dt
    return p


def _arrays(n, kd, seed=0):
    rng = np.random.default_rng(seed)
    shapes = {"R": (n, 3), "V": (n, 3), "F": (n, 3), "Kf": (n,), "q": (n,), "n_hist": (kd + 1, n),
              "energies": (8,), "chi": (n,), "eta": (n,), "sigma": (n,), "mass": (n,)}
    return {k: rng.standard_normal(s) for k, s in shapes.items()}


def test_round_trip(tmp_path):
    p = _params()
    a = _arrays(12, p.dissipation_k)
    path = tmp_path / "md.npz"
    ck.write(path, a, ck.system_signature(p), step=37)
    b, sig, step = ck.read(path)
    assert step == 37
    assert sig == ck.system_signature(p)
    for k in ck.STATE + ck.PARAMS:
        assert np.array_equal(a[k], b[k])
    ck.check_signature(sig, ck.system_signature(_params()))  # same system: no error


def test_other_system_is_rejected(tmp_path):
    p = _params()
    path = tmp_path / "md.npz"
    ck.write(path, _arrays(12, p.dissipation_k), ck.system_signature(p), step=1)
    _, sig, _ = ck.read(path)
    with pytest.raises(ValueError, match="dt"):
        ck.check_signature(sig, ck.system_signature(_params(dt=0.25)))
    q = _params()
    q.mesh[2] = 20
    with pytest.raises(ValueError, match="mesh"):
        ck.check_signature(sig, ck.system_signature(q))


def test_wrong_shapes_and_files_are_rejected(tmp_path):
    p = _params()
    a = _arrays(12, p.dissipation_k)
    a["n_hist"] = a["n_hist"][:-1]  # one history slot short
    with pytest.raises(ValueError, match="n_hist"):
        ck.write(tmp_path / "x.npz", a, ck.system_signature(p), step=0)
    del a["Kf"]
    with pytest.raises(ValueError, match="missing"):
        ck.write(tmp_path / "x.npz", a, ck.system_signature(p), step=0)
    other = tmp_path / "other.npz"
    np.savez(other, meta=np.frombuffer(b'{"format": "something else"}', dtype=np.uint8))
    with pytest.raises(ValueError, match="not a shadow-MD checkpoint"):
        ck.read(other)


def test_user_short_range_model_is_part_of_the_signature(tmp_path):
    """A run started with a user short-range model cannot resume without one (or the
    other way round): the potential would change under the trajectory."""
    p = _params()
    path = tmp_path / "md.npz"
    ck.write(path, _arrays(12, p.dissipation_k), ck.system_signature(p, user_short_range=True),
             step=3)
    _, sig, _ = ck.read(path)
    ck.check_signature(sig, ck.system_signature(_params(), user_short_range=True))
    with pytest.raises(ValueError, match="user_short_range"):
        ck.check_signature(sig, ck.system_signature(_params()))
