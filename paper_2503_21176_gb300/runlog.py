"""JSON-lines log of an MD run (host side).

One line when the run starts (the caller's metadata), one per logged step
(the step's energies from ShadowMD.energy_dict() or BOMD.energy_dict(),
optionally its device time), and a summary when it closes: the total-energy
drift per atom (last minus first logged total), the largest deviation per
atom from the first total, the applies per step and the p50 / p99 step times.
The paper reports the same quantities for its MD runs (energy fluctuation,
Ewald sums per step, per-component timing).
"""

from __future__ import annotations

import json
import time

import numpy as np


class RunLog:
    def __init__(self, path, n_atoms: int, meta: dict | None = None):
        self.n_atoms = int(n_atoms)
        self._fh = open(path, "a", encoding="utf-8")
        self._totals, self._applies, self._ms = [], [], []
        self._write({"event": "start", "time": time.time(), "n_atoms": self.n_atoms, **(meta or {})})

    def _write(self, rec: dict) -> None:
        self._fh.write(json.dumps(rec) + "\n")
        self._fh.flush()

    def step(self, step: int, energies: dict, step_ms: float | None = None) -> None:
        """Log one step.  energies: an energy_dict() (needs "total"; the other
        keys are copied as they are)."""
        rec = {"event": "step", "step": int(step)}
        rec.update({k: float(v) for k, v in energies.items()})
        if step_ms is not None:
            rec["step_ms"] = float(step_ms)
            self._ms.append(float(step_ms))
        self._totals.append(float(energies["total"]))
        if "applies" in energies:
            self._applies.append(float(energies["applies"]))
        self._write(rec)

    def summary(self) -> dict:
        s = {"event": "summary", "steps_logged": len(self._totals)}
        if self._totals:
            e = np.asarray(self._totals)
            s["drift_per_atom_eV"] = float((e[-1] - e[0]) / self.n_atoms)
            s["max_dev_per_atom_eV"] = float(np.max(np.abs(e - e[0])) / self.n_atoms)
        if self._applies:
            s["applies_per_step"] = float(np.mean(self._applies))
        if self._ms:
            s["step_ms_p50"] = float(np.percentile(self._ms, 50))
            s["step_ms_p99"] = float(np.percentile(self._ms, 99))
        return s

    def close(self) -> dict:
        s = self.summary()
        if not self._fh.closed:
            self._write(s)
            self._fh.close()
        return s

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
