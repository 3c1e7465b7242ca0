"""Seeded request streams for the serving workload (mixed-size periodic water boxes).

Requests arrive as a Poisson process (exponential gaps at ``rate`` per second).
Each is a water box of log-uniform size between ``min_atoms`` and ``max_atoms``
atoms, with fresh seeded chi / eta noise.  Half ask for one QEq charge-plus-force
evaluation ("qeq"), half for ``md_steps`` shadow-MD steps ("md").  The PME mesh
of a request is the smallest 2^k or 3 * 2^k edge with a spacing of at most
1.0 A.
"""

from __future__ import annotations

import math

import numpy as np

from .water import serving_mesh_size, water_box


def serving_stream(n_requests=512, rate=200.0, seed=2506, min_atoms=100, max_atoms=20_000,
                   md_steps=20, temperature_eV=0.025852):
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n_requests)
    arrivals = np.cumsum(gaps) - gaps[0]
    logs = rng.uniform(math.log(min_atoms), math.log(max_atoms), size=n_requests)
    kinds = rng.permutation(np.array(["qeq", "md"] * ((n_requests + 1) // 2))[:n_requests])
    reqs = []
    for k in range(n_requests):
        n_mol = max(1, int(round(math.exp(logs[k]) / 3.0)))
        w = water_box(n_mol, seed=seed * 1000 + k)
        L = float(w.box[0])
        K = serving_mesh_size(L)
        vr = np.random.default_rng(seed * 1000 + k + 7)
        V = vr.standard_normal(w.R.shape) * np.sqrt(temperature_eV / (w.mass[:, None] * 103.6427))
        V -= (w.mass[:, None] * V).sum(0) / w.mass.sum()
        reqs.append({"rid": k, "kind": str(kinds[k]), "arrival": float(arrivals[k]), "box": w,
                     "V": V, "mesh": (K, K, K), "steps": md_steps if kinds[k] == "md" else 0})
    return reqs
