#!/usr/bin/env python
"""Benchmark of the shadow-QEq Coulomb hot path on GB300.

Workload: water box of 100,000 molecules (300,000 atoms, L = 144.13 A, seeded
synthetic recipe), alpha 0.34 1/A, r_c 8 A, skin 1 A, smooth PME 144^3 of
order 4, Krylov rank 2, dissipation window K_d 5, dt 0.5 fs.

A step is one shadow XL-BOMD step.  It covers the integrator, the skin check,
m + 1 = 3 Coulomb applies (neighbour list, real space, PME spread / FFT /
influence / FFT / gather, self term), shadow charges, forces, and the Krylov
kernel.  The headline value is FP32-mixed steps/s.  The same line also
reports the FP64 steps/s, applies/s for both modes, neighbour-build time and
p50 / p99 step times.

Runs: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
N > 1 is launched by torchrun: each rank runs an independent replica on its own
GPU (weak scaling, no collective on the data path).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Coulomb applies/s & shadow-MD steps/s at 300k atoms, FP32-mixed vs FP64; p50/p99 ms"
UNIT = "steps/s"
N_MOL = 100_000
SEED = 2504
ALPHA, R_CUT, SKIN, MESH, ORDER, RANK, KD, DT = 0.34, 8.0, 1.0, 144, 4, 2, 5, 0.5
FLUSH_BYTES = 256 << 20  # > 129 MB L2
# algorithmic work per directed real-space pair inside r_c: about 40 floating-point
# operations (the pair potential and field with the Gaussian correction) and 4
# special-function evaluations (a reciprocal square root, a reciprocal and two
# exponentials of the erfc forms)
PAIR_FLOPS = 40
PAIR_SFU = 4
# DRAM bytes (read + write) per launch of the FP32 real-space kernel (potential
# and field), from an ncu capture of k_real32<1,0> on the 120,000-atom water box
# (78.63 MB read + 1.86 MB written), scaled to the 300,000-atom box by the list
# entries processed (x 2.5).  Valid for the kernel version that capture was
# taken of; None once the kernel changes.
REAL32_TRAFFIC_BYTES = (78.63e6 + 1.86e6) * 2.5
# The same for the FP64 kernel: k_real64<1,0> on the 120,000-atom box moved
# 31.49 GB/s x 2.744 ms = 86.4 MB, x 2.5.
REAL64_TRAFFIC_BYTES = 31.49e9 * 2.744e-3 * 2.5
T_EV = 0.025852  # k_B * 300 K in eV


def workload_config(n_mol=N_MOL):
    from workloads import water_box_length

    L = water_box_length(n_mol)
    return {
        "workload": f"water box {n_mol:,} molecules ({3 * n_mol:,} atoms), L {L:.2f} A, "
                    f"alpha {ALPHA}, r_c {R_CUT} A, skin {SKIN} A, PME {MESH}^3 order {ORDER}, "
                    f"Krylov rank {RANK}, K_d {KD}, dt {DT} fs, shadow XL-BOMD step",
        "n_atoms": 3 * n_mol,
        "box_A": round(L, 4),
        "seed": SEED,
        "l2": "flushed between timed steps (256 MiB write, not timed)",
    }


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            # start timing only once the sampler is producing lines (at most 5 s)
            t_end = time.perf_counter() + 5.0
            while not self.lines and time.perf_counter() < t_end and self.proc.poll() is None:
                time.sleep(0.01)
            self.lines.clear()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def pct(xs, p):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * p / 100.0
    lo, hi = math.floor(k), math.ceil(k)
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


def make_system(qg, w, precision, device):
    import torch

    p = qg.make_params(w.n_atoms, w.box, alpha=ALPHA, r_cut=R_CUT, skin=SKIN,
                       mesh=(MESH, MESH, MESH), order=ORDER, precision=precision,
                       krylov_rank=RANK, dissipation_k=KD, dt=DT)
    with torch.cuda.device(device):
        return qg.System(p, device=device.index)


def initial_state(w, seed):
    """Maxwell-Boltzmann velocities at 300 K (zero total momentum)."""
    rng = np.random.default_rng(seed)
    V = rng.standard_normal(w.R.shape) * np.sqrt(T_EV / (w.mass[:, None] * 103.6427))
    V -= (w.mass[:, None] * V).sum(0) / w.mass.sum()
    return V


def aggregate_over_ranks(local_ms, steps, world, dist=None, device=None):
    """Whole-job throughput of independent replicas: every rank ran `steps` steps in
    `local_ms` ms; the job took the slowest rank's time (max over ranks), and the
    units processed are world * steps.  Returns (value in steps/s, max ms)."""
    total_ms = float(local_ms)
    if dist is not None and world > 1:
        import torch

        t = torch.tensor([total_ms], dtype=torch.float64,
                         device=device if device is not None else "cpu")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return world * steps / (total_ms * 1e-3), total_ms


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_mode(qg, w, precision, device, steps, warmup, stream, flush, profile, q0):
    import torch

    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=device)
    sysm = make_system(qg, w, precision, device)
    R, sigma = t(w.R), t(w.sigma)
    res = {}
    with torch.cuda.stream(stream):
        # neighbour build time (one sync per build is part of the call)
        nl_ms = []
        for k in range(3):
            flush.zero_()
            t0 = time.perf_counter()
            sysm.neighbor_build(R, stream)
            nl_ms.append((time.perf_counter() - t0) * 1e3)
        res["neighbor_build_ms"] = round(min(nl_ms), 3)
        # Coulomb applies (full potential + field)
        q = t(np.random.default_rng(1).standard_normal(w.n_atoms) * 0.3)
        for _ in range(warmup):
            sysm.apply(R, q, sigma, stream=stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            sysm.apply(R, q, sigma, stream=stream)
            ev[k][1].record(stream)
        torch.cuda.synchronize(device)
        ams = [a.elapsed_time(b) for a, b in ev]
        res["apply_ms_p50"] = round(pct(ams, 50), 4)
        res["apply_ms_p99"] = round(pct(ams, 99), 4)
        res["applies_per_s"] = round(1e3 / statistics.mean(ams), 2)

        # shadow MD from n(0) = the converged QEq charges of the initial geometry
        V0 = t(initial_state(w, SEED + 1))
        md = qg.ShadowMD(sysm, t(w.chi), t(w.eta), sigma, t(w.mass), R, V0, q0)
        md.init(stream)
        for _ in range(warmup):
            md.step(1, stream)
        torch.cuda.synchronize(device)

        def timed(n):
            c0 = qg.qeq_get_counters(sysm.ctx)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(n)]
            torch.cuda.synchronize(device)
            for k in range(n):
                flush.zero_()
                ev[k][0].record(stream)
                md.step(1, stream)
                ev[k][1].record(stream)
            torch.cuda.synchronize(device)
            c1 = qg.qeq_get_counters(sysm.ctx)
            return [a.elapsed_time(b) for a, b in ev], [b - a for a, b in zip(c0, c1)]

        # timed region: the production path (each step's evaluation replayed from a
        # CUDA graph), clocks sampled throughout.  A short timed region can end
        # before nvidia-smi reports; the same steps then continue (not timed) until
        # the sampler holds a few samples of this load, at most 5 s.
        sampler = ClockSampler(device.index)
        clock_passes = 1
        with sampler:
            sms, dc = timed(steps)
            t_end = time.perf_counter() + 5.0
            while len(sampler.lines) < 5 and time.perf_counter() < t_end:
                timed(steps)
                clock_passes += 1
        # profiled pass over as many further steps: per-phase device time from CUDA
        # events on the launching stream (the profiler records events between
        # phases, so these steps run un-graphed)
        prof, prof_ms = None, None
        if profile:
            qg.qeq_profile_enable(sysm.ctx, True)
            pms, _ = timed(steps)
            prof = qg.qeq_profile_read(sysm.ctx)
            qg.qeq_profile_enable(sysm.ctx, False)
            prof_ms = statistics.mean(pms)
        e = md.energy_dict()
        res.update({
            "steps_per_s": round(1e3 / statistics.mean(sms), 3),
            "ms_per_step": round(statistics.mean(sms), 4),
            "step_ms_p50": round(pct(sms, 50), 4),
            "step_ms_p99": round(pct(sms, 99), 4),
            "gpu_launches": dc[0],
            "neighbor_rebuilds": dc[1],
            "applies_in_timed_steps": dc[2],
            "ms_per_step_profiled_pass": None if prof_ms is None else round(prof_ms, 4),
            "clocks": dict(sampler.summary(), passes=clock_passes,
                           note="the timed pass, then the same steps repeated (not timed) until "
                                "the sampler held 5 samples"),
            "final_energy_eV": {k: round(v, 6) for k, v in e.items()},
        })
        res["_step_ms_sum"] = float(sum(sms))
        res["_profile"] = prof
        res["_md"] = md
        res["_sys"] = sysm
    return res


def converged_charges(qg, w, device, stream):
    """QEq charges of the initial geometry: FP64 GMRES to a relative residual of 1e-10."""
    import torch

    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=device)
    s0 = qg.System(qg.make_params(w.n_atoms, w.box, alpha=ALPHA, r_cut=R_CUT, skin=SKIN,
                                  mesh=(MESH, MESH, MESH), order=ORDER, precision="fp64"),
                   device=device.index)
    q0 = torch.zeros(w.n_atoms, dtype=torch.float64, device=device)
    with torch.cuda.stream(stream):
        s0.neighbor_build(t(w.R), stream)
        info = qg.qeq_solve(s0.ctx, t(w.R), t(w.chi), t(w.eta), t(w.sigma), q0, tol=1e-10,
                            stream=stream)
        stream.synchronize()
    s0.close()
    return q0, info


def tolerance_steps(qg, w, device, steps, warmup, stream, flush, q0, tol=0.1, max_rank=8):
    """Shadow steps with the Krylov rank grown until the kernel residual |R c - f| / |f| is
    <= tol (the paper's loose shadow tolerance, Sec. 4.2.3), FP32-mixed, from the
    converged start.  Such a step reads the residual on the host after each added
    vector, so it is launched kernel by kernel (no graph)."""
    import torch

    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=device)
    p = qg.make_params(w.n_atoms, w.box, alpha=ALPHA, r_cut=R_CUT, skin=SKIN, mesh=(MESH, MESH, MESH),
                       order=ORDER, precision="fp32_mixed", krylov_rank=max_rank, krylov_tol=tol,
                       dissipation_k=KD, dt=DT)
    sysm = qg.System(p, device=device.index)
    with torch.cuda.stream(stream):
        md = qg.ShadowMD(sysm, t(w.chi), t(w.eta), t(w.sigma), t(w.mass), t(w.R),
                         t(initial_state(w, SEED + 1)), q0)
        md.init(stream)
        for _ in range(warmup):
            md.step(1, stream)
        torch.cuda.synchronize(device)
        ms, applies, resid = [], [], []
        for k in range(steps):
            flush.zero_()
            a0 = qg.qeq_get_counters(sysm.ctx)[2]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            md.step(1, stream)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            applies.append(qg.qeq_get_counters(sysm.ctx)[2] - a0)
            resid.append(round(md.energy_dict()["residual_norm"], 6))
    sysm.close()
    return {"krylov_tol": tol, "max_rank": max_rank, "precision": "fp32_mixed",
            "steps_per_s": round(1e3 / statistics.mean(ms), 3),
            "ms_per_step": round(statistics.mean(ms), 4),
            "step_ms_p50": round(pct(ms, 50), 4), "step_ms_p99": round(pct(ms, 99), 4),
            "applies_per_step": round(statistics.mean(applies), 3),
            "residual_norm_per_step": resid,
            "note": "|q[n] - n| after each timed step; n(0) = converged QEq charges; "
                    "kernel by kernel with one host read per added Krylov vector"}


def neighbor_method_times(qg, w_full, device, stream, reps=3):
    """Neighbour-build time of the brick search and of the per-atom search (the paper's
    one-program-per-atom form, Sec. 3.1) on the bench box and on serving sizes."""
    import torch

    from workloads import water_box

    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=device)
    rows = []
    for n_mol in (100, 1000, 6667, None):
        w = w_full if n_mol is None else water_box(n_mol, seed=2600 + n_mol)
        R = t(w.R)
        row = {"atoms": w.n_atoms}
        for method in ("brick", "atom"):
            s = qg.System(qg.make_params(w.n_atoms, w.box, alpha=ALPHA, r_cut=R_CUT, skin=SKIN,
                                         mesh=(8, 8, 8), order=ORDER, precision="fp32_mixed"),
                          device=device.index)
            qg.qeq_set_neighbor_method(s.ctx, method)
            with torch.cuda.stream(stream):
                s.neighbor_build(R, stream)  # list width settled
                ms = []
                for _ in range(reps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    s.neighbor_build(R, stream)
                    e1.record(stream)
                    e1.synchronize()
                    ms.append(e0.elapsed_time(e1))
            row[f"{method}_ms"] = round(min(ms), 4)
            s.close()
        rows.append(row)
    return {"rows": rows, "r_list_A": R_CUT + SKIN,
            "note": "whole qeq_neighbor_build (wrap, bin, sort, emit, one host read), CUDA events, "
                    "best of 3; both searches write the same list"}


def serving_sample(device, n_requests=128, rate=200.0):
    """A reduced serving stream (the first requests of the 512-request Poisson stream):
    FP32-mixed, MD steps batched across requests; throughput and p50 / p99 latency."""
    from paper_2503_21176_gb300.serve import Server, request_from_box
    from workloads import serving_stream

    stream = serving_stream(n_requests=n_requests, rate=rate)
    reqs = [request_from_box(r["rid"], r["kind"], r["box"], r["mesh"], V=r["V"], steps=r["steps"],
                             arrival=r["arrival"], precision="fp32_mixed") for r in stream]
    # warm-up: one request of each mesh size and kind (cuFFT plans, graph captures,
    # pinned host blocks), then the stream in real time
    seen, warm = set(), []
    for r in reqs:
        if (r.mesh, r.kind) not in seen:
            seen.add((r.mesh, r.kind))
            warm.append(r)
    Server(device=device.index, max_inflight=8).serve(warm + reqs[:8], realtime=False)
    _, st = Server(device=device.index, max_inflight=8).serve(reqs, realtime=True)
    return {"requests": n_requests, "arrival_rate_per_s": rate, "precision": "fp32_mixed",
            "atoms": "100-20,000 log-uniform", "kinds": "half 1 QEq evaluation, half 20 MD steps",
            "throughput_req_per_s": st["throughput_req_per_s"],
            "latency_ms_p50": st["latency_ms_p50"], "latency_ms_p99": st["latency_ms_p99"],
            "failed": st["failed"], "max_concurrent": st["max_concurrent"],
            "md_batching": st["md_batching"], "stage_ms_mean": st["stage_ms_mean"]}


def e2e_steps(qg, md, steps, stream, device, chunks=8, warmup=3):
    """Same step through the C ABI with the state kept in HOST memory: every step
    copies the whole MD state (R, V, F, K f, n history) and the per-atom parameters
    from pinned host memory to the device, runs the step, and copies the advanced
    state, the charges and the energies back to pinned host memory, all inside the
    timed region.  The step works on one contiguous device buffer (ShadowMD.pack);
    two host buffers alternate (the results of step k are the inputs of step
    k + 1), so the trajectory lives on the host with no host copy.

    The host link is full duplex, so the two directions overlap: the state goes
    down (D2H) in `chunks` pieces on one copy stream and each piece comes back up
    (H2D, as step k + 1's input) on another as soon as it has landed, behind an
    event; the parameters go up once step k's compute is done.  Step k + 1 starts
    when all of its input has arrived, so every byte still makes the round trip
    through host memory.  The host reads step k's energies from its host buffer
    (their copy is complete once step k + 1's skin check has synchronised).
    `warmup` steps of the same loop run untimed first (the step graph is
    captured again for the packed buffer)."""
    import torch

    dev_buf, (n_par, n_state, n_res) = md.pack()
    host = [dev_buf.cpu().pin_memory(), torch.empty_like(dev_buf, device="cpu").pin_memory()]
    host[1][:n_par].copy_(host[0][:n_par])  # the parameters, in both buffers
    n_in, n_out = n_par + n_state, n_state + n_res
    h2d, d2h = 8 * n_in, 8 * n_out
    # chunk bounds of the state region [n_par, n_par + n_state)
    bounds = [n_par + (n_state * c) // chunks for c in range(chunks + 1)]
    down = torch.cuda.Stream(device)
    up = torch.cuda.Stream(device)
    ev_down = [torch.cuda.Event() for _ in range(chunks)]
    ev_comp = torch.cuda.Event()
    ev_res = torch.cuda.Event()
    ev_in = torch.cuda.Event()
    e_idx = n_par + n_state + (n_res - md.energies.numel()) + 2  # energies[2]: total
    totals = []

    def run(first, count):
        """Steps first .. first + count - 1 of the pipelined round trip."""
        dev_buf[:n_in].copy_(host[first % 2][:n_in], non_blocking=True)  # the first input
        for k in range(first, first + count):
            src, dst = host[k % 2], host[(k + 1) % 2]
            md.step(1, stream)  # its skin check waited for this step's input
            if k > first:
                totals.append(float(src[e_idx]))  # step k - 1's result, read on the host
            ev_comp.record(stream)
            down.wait_event(ev_comp)
            with torch.cuda.stream(down):
                for c in range(chunks):
                    dst[bounds[c]:bounds[c + 1]].copy_(dev_buf[bounds[c]:bounds[c + 1]], non_blocking=True)
                    ev_down[c].record(down)
                dst[n_par + n_state:].copy_(dev_buf[n_par + n_state:], non_blocking=True)
                ev_res.record(down)
            if k + 1 < first + count:
                up.wait_event(ev_comp)
                with torch.cuda.stream(up):
                    dev_buf[:n_par].copy_(dst[:n_par], non_blocking=True)
                    for c in range(chunks):
                        up.wait_event(ev_down[c])
                        dev_buf[bounds[c]:bounds[c + 1]].copy_(dst[bounds[c]:bounds[c + 1]],
                                                                non_blocking=True)
                    # the results (charges, energies) have landed too before step k + 1
                    # starts, so its skin check tells the host they can be read
                    up.wait_event(ev_res)
                    ev_in.record(up)
                stream.wait_event(ev_in)
            else:
                stream.wait_stream(down)

    with torch.cuda.stream(stream):
        # untimed warm-up: the step graph is captured again for the packed buffer
        run(0, warmup)
        torch.cuda.synchronize(device)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        run(warmup, steps)
        t1.record(stream)
        torch.cuda.synchronize(device)
    totals.append(float(host[(warmup + steps) % 2][e_idx]))
    ms = t0.elapsed_time(t1) / steps
    return {"value": round(1e3 / ms, 3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": round(ms, 4),
            "copies": f"D2H and H2D overlapped in {chunks} chunks on two copy streams",
            "last_total_energy_eV": round(totals[-1], 6)}


def roofline(res, precision, n_pairs_rc, peaks, pipes):
    """Roofline of the dominant phase of the timed steps (CUDA events on the launch stream).

    The real-space kernel is bound by the arithmetic pipes, so its fraction is the
    method's floating-point work (PAIR_FLOPS per directed pair inside r_c) over
    the FP32 (or FP64) FMA rate measured on this GPU by qeq_measure_peaks; the
    special-function work is quoted beside it against the measured MUFU rate."""
    prof = res.get("_profile") or {}
    if not prof:
        return None
    name, (ms, cnt) = max(prof.items(), key=lambda kv: kv[1][0])
    share = ms / max(1e-9, sum(v[0] for v in prof.values()))
    avg_ms = ms / max(1, cnt)
    if name == "real_space":
        fp32 = precision == "fp32_mixed"
        peak = (pipes["fp32_flops"] if fp32 else pipes["fp64_flops"]) / 1e12
        achieved = n_pairs_rc * PAIR_FLOPS / (avg_ms * 1e-3) / 1e12
        sfu = n_pairs_rc * PAIR_SFU / (avg_ms * 1e-3)
        out = {"kernel": name, "bound": "alu", "achieved": round(achieved, 4),
               "peak": round(peak, 3), "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
               "traffic": REAL32_TRAFFIC_BYTES if fp32 else REAL64_TRAFFIC_BYTES,
               "traffic_unit": "DRAM bytes per launch (ncu, scaled from 120k atoms)",
               "algorithmic": f"{PAIR_FLOPS} flop x {n_pairs_rc} directed pairs inside r_c "
                              f"= {PAIR_FLOPS * n_pairs_rc / 1e9:.3f} GFLOP per launch (full list)",
               "peak_source": f"qeq_measure_peaks: {'FP32' if fp32 else 'FP64'} FMA chains on "
                              f"{pipes['sm_count']} SMs, CUDA events, best of 3 (measured)",
               "sfu": {"achieved_ops_per_s": round(sfu, 1), "peak_ops_per_s": round(pipes["mufu_ops"], 1),
                       "frac": round(sfu / pipes["mufu_ops"], 4), "per_pair": PAIR_SFU} if fp32 else None,
               "pairs_per_s": round(n_pairs_rc / (avg_ms * 1e-3), 1),
               "half_list_pairs_per_s": round(0.5 * n_pairs_rc / (avg_ms * 1e-3), 1),
               "list_form": "full list: every unique pair evaluated from both rows, no atomics; "
                            "half_list_pairs_per_s = unique pairs per second of the same launch"}
    else:
        gbs = peaks.get("hbm_gbs", 6800.0)
        out = {"kernel": name, "bound": "hbm", "achieved": None, "peak": gbs, "unit": "GB/s",
               "frac": None, "traffic": None, "peak_source": "MEASURED_PEAKS.json hbm_gbs"}
    out.update({"avg_launch_ms": round(avg_ms, 4), "launches": cnt, "share_of_profiled": round(share, 4),
                "phases_ms": {k: round(v[0], 3) for k, v in prof.items()}})
    return out


def precision_report(s32, s64, w, device, stream):
    """FP32-mixed against FP64 on the same charges and positions.  The FP64 apply
    matches the oracle to 1e-10, so these are the errors against the oracle."""
    import torch

    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=device)
    R, sig = t(w.R), t(w.sigma)
    q = t(np.random.default_rng(7).standard_normal(w.n_atoms) * 0.3)
    out = {}
    for name, sysm in (("fp32", s32), ("fp64", s64)):
        sysm.neighbor_build(R, stream)
        with torch.cuda.stream(stream):
            v, E, F, en = sysm.apply(R, q, sig, stream=stream)
            stream.synchronize()
        out[name] = (v.cpu().numpy().copy(), F.cpu().numpy().copy(), en.cpu().numpy().copy())
    v32, F32, e32 = out["fp32"]
    v64, F64, e64 = out["fp64"]
    return {
        "rel_energy": float(abs(e32[0] - e64[0]) / abs(e64[0])),
        "rel_potential_max": float(np.abs(v32 - v64).max() / np.abs(v64).max()),
        "rel_potential_rms": float(np.sqrt(np.mean((v32 - v64) ** 2) / np.mean(v64 ** 2))),
        "rel_rms_force": float(np.sqrt(np.mean((F32 - F64) ** 2) / np.mean(F64 ** 2))),
        "charges": "N(0, 0.3 e), seed 7",
    }


def drift_bench(args):
    """Total-energy drift per atom of the shadow step, 300k-atom water with the flexible-water
    V_short stand-in, in both precisions; one line of JSON."""
    import torch

    import paper_2503_21176_gb300 as qg
    from workloads import water_box

    qg.load()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    w = water_box(args.n_mol, seed=SEED)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(dev)
    K = MESH if args.n_mol == N_MOL else 4 * math.ceil(float(w.box[0]) / 4.0)
    common = dict(alpha=ALPHA, r_cut=R_CUT, skin=SKIN, mesh=(K, K, K), order=ORDER,
                  dissipation_k=KD, dt=DT, short_range=qg.QEQ_SHORT_WATER)
    # n(0) = the converged QEq charges (GMRES, FP64, relative residual 1e-10): an n(0)
    # away from the ground state starts a charge oscillation whose energy leaks into
    # the atoms in the first tens of steps
    s0 = qg.System(qg.make_params(w.n_atoms, w.box, precision="fp64", **common))
    s0.neighbor_build(t(w.R))
    q0 = torch.zeros(w.n_atoms, dtype=torch.float64, device=dev)
    qg.qeq_solve(s0.ctx, t(w.R), t(w.chi), t(w.eta), t(w.sigma), q0, tol=1e-10)
    torch.cuda.synchronize(dev)
    s0.close()
    rows = {}
    for prec, steps in (("fp32_mixed", args.drift_steps), ("fp64", args.drift_steps_fp64)):
        sysm = qg.System(qg.make_params(w.n_atoms, w.box, precision=prec, krylov_rank=args.drift_rank,
                                        krylov_tol=args.drift_krylov_tol, **common))
        with torch.cuda.stream(stream):
            md = qg.ShadowMD(sysm, t(w.chi), t(w.eta), t(w.sigma), t(w.mass), t(w.R),
                             t(initial_state(w, SEED + 1)), q0.clone())
            md.init(stream)
            e = [md.energies[2].item()]
            qmax = [float(md.q.abs().max().item())]
            res = [md.energies[6].item()]
            c0 = qg.qeq_get_counters(sysm.ctx)
            every = max(1, steps // 100)
            diverged = None
            t0 = time.perf_counter()
            for k in range(steps):
                try:
                    md.step(1, stream)
                except qg.QeqError as exc:  # non-finite positions: the run blew up
                    diverged = {"step": k, "error": str(exc)}
                    break
                if (k + 1) % every == 0:
                    e.append(md.energies[2].item())
                    qmax.append(float(md.q.abs().max().item()))
                    res.append(md.energies[6].item())
                    if not math.isfinite(e[-1]):
                        diverged = {"step": k, "error": "total energy not finite"}
                        break
            stream.synchronize()
            wall = time.perf_counter() - t0
            done = k + 1 if diverged is None else k
            c1 = qg.qeq_get_counters(sysm.ctx)
        sysm.close()
        E = np.array([x for x in e if math.isfinite(x)])
        x = np.arange(len(E)) * every * DT
        slope = float(np.polyfit(x, E, 1)[0]) if len(E) > 2 else 0.0
        rows[prec] = {"atoms": w.n_atoms, "mesh": K, "steps": done, "fs": done * DT,
                      "drift_per_atom_eV": float((E[-1] - E[0]) / w.n_atoms),
                      "slope_per_atom_eV_per_ps": slope * 1000.0 / w.n_atoms,
                      "std_per_atom_eV": float(np.std(E) / w.n_atoms),
                      "max_abs_q": float(max(qmax)), "ms_per_step": 1e3 * wall / max(1, done),
                      "diverged": diverged, "neighbor_rebuilds": c1[1] - c0[1],
                      "applies_per_step": round((c1[2] - c0[2]) / max(1, done), 3),
                      "krylov_rank": args.drift_rank, "krylov_tol": args.drift_krylov_tol,
                      "residual_norm_trace": [round(float(v), 5) for v in res[:: max(1, len(res) // 20)]],
                      "energy_trace_eV": [round(float(v), 4) for v in e[:: max(1, len(e) // 20)]]}
    print(json.dumps({"experiment": "shadow XL-BOMD total-energy drift, water + V_short stand-in",
                      "config": workload_config(args.n_mol), "rows": rows}))


def count_pairs_within_rc(sysm, w):
    """Directed real-space pairs inside r_c at the positions of the last neighbour build.

    The exported images refer to positions wrapped as x - L floor(x / L).
    """
    counts, nbr, shift = sysm.neighbor_export()
    box = np.asarray(w.box, dtype=np.float64)
    xw = w.R - box * np.floor(w.R / box)
    mask = np.arange(nbr.shape[1])[None, :] < counts[:, None]
    rows = np.nonzero(mask)[0]
    cols = nbr[mask]
    d = xw[cols] - xw[rows] + shift[mask].astype(np.float64) * box
    return int(np.count_nonzero(np.einsum("ij,ij->i", d, d) < R_CUT * R_CUT))


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or "unknown"."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        fields = dict(ln.split(":", 1) for ln in out.splitlines() if ":" in ln)
        name = fields.get("Model name", "").strip()
        vendor = fields.get("Vendor ID", "").strip()
        if name:
            return f"{vendor} {name}".strip()
    except (OSError, subprocess.SubprocessError, ValueError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline(w, q0, budget_s):
    """The oracle's shadow step at full size on the host cores: the initial evaluation,
    then whole steps until the budget is spent (at least one); value = timed steps/s."""
    from oracle import ewald, native, qeq

    def coul(R, x, need_field=True):
        o = ewald.coulomb_apply(R, x, w.sigma, w.box, ALPHA, R_CUT, recip="pme",
                                mesh=(MESH, MESH, MESH), order=ORDER, gaussian_self=True)
        return o["v"], o["E"]

    osys = qeq.ShadowSystem(coul, w.chi, w.eta, w.mass, rank=RANK, dt=DT, k_d=KD)
    t_start = time.perf_counter()
    st = osys.init_state(w.R, initial_state(w, SEED + 1), q0)
    times = []
    while True:
        t0 = time.perf_counter()
        st = osys.step(st)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start + times[-1] > budget_s:
            break
    step_s = statistics.mean(times)
    return {"value": round(1.0 / step_s, 5), "unit": UNIT, "cores": native.num_threads(),
            "cpu_model": cpu_model(), "kind": "oracle",
            "sample": f"{len(times)} full shadow XL-BOMD steps of the {w.n_atoms:,}-atom box after "
                      f"its initial evaluation ({RANK + 1} Coulomb applies per step: cell-list real "
                      f"space in C/OpenMP + numpy PME {MESH}^3 + Krylov), "
                      f"{time.perf_counter() - t_start:.1f} s wall, budget {budget_s:.0f} s"}


def ours(args):
    import torch

    import paper_2503_21176_gb300 as qg
    from workloads import water_box

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.gpus != world:
        raise SystemExit(f"--gpus {args.gpus} but WORLD_SIZE {world}")
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=device)
    qg.load()
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        peaks = {"hbm_gbs": 6800.0, "source": "fallback"}

    w = water_box(args.n_mol, seed=SEED + rank)
    stream = torch.cuda.Stream(device)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    # the pipe rates the real-space roofline divides by, measured on this GPU now
    pipes = qg.qeq_measure_peaks(stream)
    q0, solve_info = converged_charges(qg, w, device, stream)

    modes = ["fp32_mixed"] if args.no_fp64 else ["fp32_mixed", "fp64"]
    results = {}
    for m in modes:
        if dist is not None:
            dist.barrier()
        results[m] = run_mode(qg, w, m, device, args.steps, args.warmup, stream, flush,
                              profile=True, q0=q0)
    tol_run = None
    if not args.no_tolerance_run:
        tol_run = tolerance_steps(qg, w, device, args.steps, args.warmup, stream, flush, q0)
    nl_methods = None if args.no_extras else neighbor_method_times(qg, w, device, stream)
    serving = None if (args.no_extras or rank != 0) else serving_sample(device)

    head = results["fp32_mixed"]
    sysm, md = head["_sys"], head["_md"]
    precision = None
    if "fp64" in results:
        precision = precision_report(results["fp32_mixed"]["_sys"], results["fp64"]["_sys"], w,
                                     device, stream)
    # directed pairs inside r_c at the initial positions (fresh list) for the roofline
    sysm.neighbor_build(torch.as_tensor(w.R, dtype=torch.float64, device=device), stream)
    n_pairs = count_pairs_within_rc(sysm, w)

    e2e = e2e_steps(qg, md, max(3, args.steps // 2), stream, device)

    # max over ranks of the timed region
    value, total_ms = aggregate_over_ranks(head["_step_ms_sum"], args.steps, world, dist, device)
    if dist is not None:
        dist.barrier()

    line = None
    if rank == 0:
        roof = roofline(head, "fp32_mixed", n_pairs, peaks, pipes)
        fp64 = None
        if "fp64" in results:
            r64 = results["fp64"]
            fp64 = {k: v for k, v in r64.items() if not k.startswith("_")}
            fp64["roofline"] = roofline(r64, "fp64", n_pairs, peaks, pipes)
        cfg = workload_config(args.n_mol)
        cfg["parallelism"] = f"replicas x{world}" if world > 1 else "single GPU"
        line = {
            "metric": METRIC,
            "value": round(value, 3),
            "unit": UNIT,
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(total_ms / args.steps, 4),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32 (FP32-mixed: f32 pair/PME math, f64 sums, Krylov, integrator)",
            "data": "synthetic",
            "config": cfg,
            "fp32_mixed": {k: v for k, v in head.items() if not k.startswith("_")},
            "fp64": fp64,
            "directed_pairs_within_rc": n_pairs,
            "precision_fp32_vs_fp64": precision,
            "measured_pipes": {"fp32_tflops": round(pipes["fp32_flops"] / 1e12, 3),
                               "fp64_tflops": round(pipes["fp64_flops"] / 1e12, 4),
                               "mufu_tops": round(pipes["mufu_ops"] / 1e12, 4),
                               "sm_count": pipes["sm_count"],
                               "how": "qeq_measure_peaks: dependency chains on every SM, "
                                      "CUDA events, best of 3"},
            "initial_charges": {"method": "GMRES (FP64, Jacobi) to relative residual 1e-10",
                                "iterations": solve_info["iterations"],
                                "rel_residual": solve_info["rel_residual"]},
            "tolerance_driven_step": tol_run,
            "neighbor_methods": nl_methods,
            "serving_sample": serving,
            "roofline": roof,
            "e2e": e2e,
            "gpu_launches": head["gpu_launches"],
            "clocks": head["clocks"],
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w, q0.cpu().numpy(), args.cpu_budget)
    for m in list(results):
        results[m]["_sys"].close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line))


# ---------------------------------------------------------------------------
# reference arm: the oracle, as it stands, on the host cores
# ---------------------------------------------------------------------------

def reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import ewald, native, qeq
    from workloads import water_box

    w = water_box(args.n_mol, seed=SEED)

    def coul(R, x, need_field=True):
        o = ewald.coulomb_apply(R, x, w.sigma, w.box, ALPHA, R_CUT, recip="pme",
                                mesh=(MESH, MESH, MESH), order=ORDER, gaussian_self=True)
        return o["v"], o["E"]

    osys = qeq.ShadowSystem(coul, w.chi, w.eta, w.mass, rank=RANK, dt=DT, k_d=KD)
    st = osys.init_state(w.R, initial_state(w, SEED + 1), np.zeros(w.n_atoms))
    budget_s = args.reference_budget
    t_start = time.perf_counter()
    times = []
    planned = args.warmup + args.steps
    for k in range(planned):
        t0 = time.perf_counter()
        st = osys.step(st)
        times.append(time.perf_counter() - t0)
        spent = time.perf_counter() - t_start
        if spent + times[-1] > budget_s and k + 1 >= 2:
            break
    timed = times[min(args.warmup, len(times) - 1):] if len(times) > 1 else times
    ms = 1e3 * statistics.mean(timed)
    value = 1e3 / ms
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": round(value, 5),
        "unit": UNIT,
        "n_gpus": args.gpus,
        "steps": len(timed),
        "warmup": len(times) - len(timed),
        "ms_per_step": round(ms, 2),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(args.n_mol),
        "cpu_baseline": {
            "value": round(value, 5), "unit": UNIT, "cores": native.num_threads(),
            "cpu_model": cpu_model(), "kind": "oracle",
            "sample": f"{len(timed)} full shadow XL-BOMD steps of the {w.n_atoms:,}-atom box "
                      f"(FP64 oracle: C/OpenMP cell-list real space + numpy PME), "
                      f"capped at {budget_s:.0f} s total",
        },
        "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def serve_bench(args):
    """Serving workload: Poisson stream of mixed-size water boxes, half QEq evaluations and
    half 20-step shadow-MD runs, FP32-mixed and FP64.  Prints one JSON line."""
    import torch

    import paper_2503_21176_gb300 as qg
    from paper_2503_21176_gb300.serve import Server, request_from_box
    from workloads import serving_stream

    qg.load()
    torch.cuda.set_device(0)
    stream = serving_stream(n_requests=args.serve_requests, rate=args.serve_rate)
    out = {"metric": "serving throughput and p50/p99 latency, mixed-size periodic QEq / shadow-MD "
                     "requests", "unit": "requests/s", "data": "synthetic",
           "config": {"requests": args.serve_requests, "arrival_rate_per_s": args.serve_rate,
                      "atoms": "100-20,000 log-uniform", "kinds": "half 1 QEq evaluation, half 20 MD steps",
                      "mesh": "smallest 2^k or 3*2^k with spacing <= 1.0 A", "r_c": 8.0,
                      "max_inflight": args.serve_inflight}}
    for prec, batch_md in (("fp32_mixed", True), ("fp32_mixed", False), ("fp64", True)):
        reqs = [request_from_box(r["rid"], r["kind"], r["box"], r["mesh"], V=r["V"],
                                 steps=r["steps"], arrival=r["arrival"], precision=prec)
                for r in stream]
        # warm-up (not timed): one request of each mesh size and kind (cuFFT plans,
        # first launches of each kernel, graph captures, pinned host blocks) and the
        # first few requests, then the stream in real time
        seen, warm = set(), []
        for r in reqs:
            if (r.mesh, r.kind) not in seen:
                seen.add((r.mesh, r.kind))
                warm.append(r)
        Server(max_inflight=args.serve_inflight, batch_md=batch_md).serve(warm + reqs[:8],
                                                                           realtime=False)
        res, stats = Server(max_inflight=args.serve_inflight, batch_md=batch_md).serve(reqs, realtime=True)
        out[prec if batch_md else prec + "_unbatched"] = stats
    out["value"] = out["fp32_mixed"]["throughput_req_per_s"]
    print(json.dumps(out))


def table1_bench(args):
    """Analogue of the paper's Table 1 (Sec. 4.1): regular BO-MD (GMRES + Jacobi) against
    shadow MD (Krylov kernel to the same tolerance).  Shared settings: 100 water
    molecules, NVE, 0.4 fs, about 300 K, the flexible-water V_short stand-in.
    Reports Coulomb applies per step and the standard deviation of the total energy."""
    import torch

    import paper_2503_21176_gb300 as qg
    from workloads import water_box

    qg.load()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    w = water_box(100, seed=2507)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    V0 = initial_state(w, 2508)
    mesh, rc, alpha = (24, 24, 24), 7.0, 0.4
    common = dict(alpha=alpha, r_cut=rc, skin=1.0, mesh=mesh, order=4, dt=0.4,
                  short_range=qg.QEQ_SHORT_WATER, precision="fp64")
    # reference charges at t = 0 from a tight solve
    s0 = qg.System(qg.make_params(w.n_atoms, w.box, **common))
    s0.neighbor_build(t(w.R))
    q0 = torch.zeros(w.n_atoms, dtype=torch.float64, device=dev)
    qg.qeq_solve(s0.ctx, t(w.R), t(w.chi), t(w.eta), t(w.sigma), q0, tol=1e-10)
    s0.close()
    rows = []
    for method in ("shadow", "regular"):
        for tol in (1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6):
            if method == "shadow":
                s = qg.System(qg.make_params(w.n_atoms, w.box, krylov_rank=8, krylov_tol=tol, **common))
                md = qg.ShadowMD(s, t(w.chi), t(w.eta), t(w.sigma), t(w.mass), t(w.R), t(V0), q0)
            else:
                s = qg.System(qg.make_params(w.n_atoms, w.box, **common))
                md = qg.BOMD(s, t(w.chi), t(w.eta), t(w.sigma), t(w.mass), t(w.R), t(V0), q0, tol=tol)
            md.init()
            energies, applies = [], []
            diverged = None
            t_start = time.perf_counter()
            for k in range(args.table1_steps):
                try:
                    md.step()
                except qg.QeqError as exc:  # non-finite positions: the run blew up
                    diverged = {"step": k, "error": str(exc)}
                    break
                e = md.energies.cpu().tolist()
                if not math.isfinite(e[2]) or (energies and abs(e[2] - energies[0]) > 1e3):
                    diverged = {"step": k, "error": "total energy diverged"}
                    break
                energies.append(e[2])
                applies.append(e[7])
            wall = time.perf_counter() - t_start
            s.close()
            E = np.array(energies) if energies else np.zeros(1)
            rows.append({"method": method, "tol": tol, "applies_per_step": round(float(np.mean(applies)), 2)
                         if applies else None, "energy_std_eV": float(np.std(E)),
                         "energy_max_dev_eV": float(np.abs(E - E[0]).max()),
                         "ms_per_step": round(1e3 * wall / max(1, len(energies)), 3),
                         "diverged": diverged})
    print(json.dumps({"experiment": "Table 1 analogue: shadow vs regular QEq-MD", "water_molecules": 100,
                      "atoms": w.n_atoms, "steps": args.table1_steps, "dt_fs": 0.4,
                      "settings": {"alpha": alpha, "r_cut": rc, "mesh": mesh, "order": 4,
                                   "short_range": "flexible water stand-in", "precision": "fp64"},
                      "rows": rows}))


def crossover_bench(args):
    """Regular Ewald (explicit k-sum) against PME for the charge-derivative apply, FP64, at
    the paper's Sec. 4.2.2 settings: r_c 10 A, Ewald accuracy 5e-4 (alpha r_c = 2.46,
    k_cut = 2 alpha sqrt(-ln 5e-4)), PME of order 6 with a mesh spacing near 1.3 A.
    Water-like boxes of increasing size; milliseconds per apply (potential + field)."""
    import torch

    import paper_2503_21176_gb300 as qg
    from workloads import water_box

    qg.load()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    r_c = 10.0
    alpha = 2.4566 / r_c  # erfc(alpha r_c) = 5e-4
    k_cut = 2.0 * alpha * math.sqrt(-math.log(5e-4))
    rows = []
    for n_mol in (50, 100, 200, 400, 800, 1600, 3200, 6400):
        w = water_box(n_mol, seed=3000 + n_mol)
        L = float(w.box[0])
        K = max(8, int(math.ceil(L / 1.3 / 4.0)) * 4)
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
        R, sig = t(w.R), t(w.sigma)
        q = t(np.random.default_rng(n_mol).standard_normal(w.n_atoms) * 0.3)
        row = {"atoms": w.n_atoms, "box_A": round(L, 2), "pme_mesh": K}
        for method in ("pme", "ewald"):
            p = qg.make_params(w.n_atoms, w.box, alpha=alpha, r_cut=r_c, skin=0.0, mesh=(K, K, K),
                               order=6, recip=method, k_cut=k_cut)
            s = qg.System(p)
            s.neighbor_build(R)
            for _ in range(3):
                s.apply(R, q, sig)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(10):
                s.apply(R, q, sig)
            e1.record()
            torch.cuda.synchronize()
            row[f"{method}_ms"] = round(e0.elapsed_time(e1) / 10, 4)
            s.close()
        rows.append(row)
    print(json.dumps({"experiment": "regular Ewald vs PME, FP64 charge derivatives and forces",
                      "r_cut": r_c, "alpha": round(alpha, 5), "k_cut": round(k_cut, 4),
                      "pme_order": 6, "rows": rows}))


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n-mol", type=int, default=N_MOL)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tolerance-run", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra measurements (neighbour searches, serving sample)")
    ap.add_argument("--cpu-budget", type=float, default=20.0,
                    help="seconds of oracle work the cpu_baseline sample may spend")
    ap.add_argument("--reference-budget", type=float, default=200.0,
                    help="seconds of oracle work the reference arm may spend")
    ap.add_argument("--serve", action="store_true", help="run the serving workload instead")
    ap.add_argument("--table1", action="store_true",
                    help="run the shadow vs regular QEq-MD tolerance sweep instead")
    ap.add_argument("--table1-steps", type=int, default=2000)
    ap.add_argument("--drift", action="store_true", help="run the energy-drift measurement instead")
    ap.add_argument("--drift-steps", type=int, default=10000)
    ap.add_argument("--drift-steps-fp64", type=int, default=2000)
    ap.add_argument("--drift-rank", type=int, default=8, help="Krylov rank (maximum rank with a tolerance)")
    ap.add_argument("--drift-krylov-tol", type=float, default=0.1,
                    help="relative residual of the Krylov kernel (the paper's loose GMRES tolerance)")
    ap.add_argument("--crossover", action="store_true",
                    help="time the explicit Ewald k-sum against PME over system sizes instead")
    ap.add_argument("--serve-requests", type=int, default=512)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-inflight", type=int, default=8)
    args = ap.parse_args()
    if args.serve:
        serve_bench(args)
        return
    if args.table1:
        table1_bench(args)
        return
    if args.crossover:
        crossover_bench(args)
        return
    if args.drift:
        drift_bench(args)
        return
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        reference(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
