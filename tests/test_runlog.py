"""JSON-lines run log: records, drift per atom, applies and step-time percentiles (CPU)."""

import json

import numpy as np

from paper_2503_21176_gb300.runlog import RunLog


def test_run_log_records_and_summary(tmp_path):
    path = tmp_path / "run.jsonl"
    n = 300
    totals = -100.0 + 0.003 * np.arange(11)  # drifts 0.03 eV over the run
    ms = np.linspace(1.0, 2.0, 11)
    with RunLog(path, n, meta={"workload": "test box", "dt_fs": 0.5}) as log:
        for k, (e, t) in enumerate(zip(totals, ms)):
            log.step(k, {"total": e, "kinetic": 1.0, "shadow_potential": e - 1.0, "sum_q": 0.0,
                         "applies": 3.0}, step_ms=t)
        s = log.summary()
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert lines[0]["event"] == "start" and lines[0]["n_atoms"] == n
    assert lines[0]["workload"] == "test box"
    steps = [x for x in lines if x["event"] == "step"]
    assert len(steps) == 11 and steps[3]["step"] == 3 and steps[3]["applies"] == 3.0
    last = lines[-1]
    assert last["event"] == "summary" and last == s
    assert abs(s["drift_per_atom_eV"] - 0.03 / n) < 1e-15
    assert abs(s["max_dev_per_atom_eV"] - 0.03 / n) < 1e-15
    assert s["applies_per_step"] == 3.0
    assert abs(s["step_ms_p50"] - 1.5) < 1e-12 and s["step_ms_p99"] <= 2.0


def test_empty_log_has_a_summary(tmp_path):
    log = RunLog(tmp_path / "e.jsonl", 10)
    s = log.close()
    assert s == {"event": "summary", "steps_logged": 0}
    assert log.close() == s  # closing twice writes nothing more
    assert len((tmp_path / "e.jsonl").read_text().splitlines()) == 2
