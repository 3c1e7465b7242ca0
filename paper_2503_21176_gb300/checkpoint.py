"""Checkpoint and resume of a shadow XL-BOMD run (host file, numpy .npz).

The state one step advances is (R, V, F, Kf, n_hist): positions, velocities,
the forces and the low-rank K f of the current step, and the window of the
K_d + 1 latest extended charges n(t), n(t - dt), ... that the dissipative
n-integrator combines.  The history is shifted in place each step, so the
window is the whole integrator state.  q and the energies are the step's
results and are stored with it.  A checkpoint also stores the per-atom
parameters (chi, eta, sigma, mass), the step count, and the system parameters
that change the trajectory; resuming checks them against the new system and
rebuilds the neighbour list at the stored positions.

This module does file I/O and checks only; the step itself runs in the
library.
"""

from __future__ import annotations

import json

import numpy as np

STATE = ("R", "V", "F", "Kf", "n_hist", "q", "energies")
PARAMS = ("chi", "eta", "sigma", "mass")
FORMAT = "qeq-shadow-md-checkpoint-1"

# qeq_params fields that change the trajectory (the list width is a capacity,
# grown on demand, and does not)
_SCALARS = ("n_atoms", "alpha", "r_cut", "skin", "order", "precision", "krylov_rank",
            "krylov_tol", "dissipation_k", "dt", "mass_unit", "gaussian_self", "k_e", "q_tot",
            "short_range", "recip", "k_cut")


def system_signature(params, user_short_range: bool = False) -> dict:
    """The trajectory-relevant fields of a qeq_params, as plain numbers, and whether a
    user short-range model replaced the parameter-selected one (a run resumed
    without the model it was started with would change its potential)."""
    sig = {"user_short_range": bool(user_short_range)}
    for k in _SCALARS:
        if hasattr(params, k):
            v = getattr(params, k)
            sig[k] = float(v) if isinstance(v, float) else int(v)
    sig["box"] = [float(x) for x in params.box]
    sig["mesh"] = [int(x) for x in params.mesh]
    return sig


def check_signature(saved: dict, current: dict) -> None:
    """Raise ValueError naming every field where the two systems differ."""
    keys = sorted(set(saved) | set(current))
    bad = [k for k in keys if saved.get(k) != current.get(k)]
    if bad:
        detail = ", ".join(f"{k}: {saved.get(k)!r} != {current.get(k)!r}" for k in bad)
        raise ValueError(f"checkpoint was written for another system ({detail})")


def write(path, arrays: dict, signature: dict, step: int) -> None:
    """Write the state and parameter arrays (float64) with the signature and step."""
    missing = [k for k in STATE + PARAMS if k not in arrays]
    if missing:
        raise ValueError(f"checkpoint arrays missing: {missing}")
    n = int(signature["n_atoms"])
    shapes = {"R": (n, 3), "V": (n, 3), "F": (n, 3), "Kf": (n,), "q": (n,),
              "n_hist": (int(signature["dissipation_k"]) + 1, n), "energies": (8,),
              "chi": (n,), "eta": (n,), "sigma": (n,), "mass": (n,)}
    out = {}
    for k in STATE + PARAMS:
        a = np.ascontiguousarray(arrays[k], dtype=np.float64)
        if a.shape != shapes[k]:
            raise ValueError(f"checkpoint array {k} has shape {a.shape}, expected {shapes[k]}")
        out[k] = a
    meta = json.dumps({"format": FORMAT, "step": int(step), "system": signature})
    with open(path, "wb") as fh:
        np.savez(fh, meta=np.frombuffer(meta.encode(), dtype=np.uint8), **out)


def read(path):
    """Return (arrays, signature, step) of a checkpoint file."""
    with np.load(path) as z:
        meta = json.loads(bytes(z["meta"]).decode())
        if meta.get("format") != FORMAT:
            raise ValueError(f"not a shadow-MD checkpoint: {meta.get('format')!r}")
        arrays = {k: z[k].copy() for k in STATE + PARAMS}
    return arrays, meta["system"], int(meta["step"])
