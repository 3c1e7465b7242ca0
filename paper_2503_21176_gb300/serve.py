"""Serving loop: continuous batching of periodic QEq / shadow-MD requests on one GPU.

Requests for systems of uneven size arrive over time.  A dispatcher admits a
request once a slot is free and its estimated device memory fits in the free
HBM left after the requests already running.  Each admitted request runs on a
slot's own CUDA stream in a worker thread.  ctypes releases the GIL, so the
library calls of different requests run at the same time and their kernels
overlap on the device.  A request first creates a stream-ordered context
(qeq_create_async: memory from the device pool, no device-wide
synchronisation).  It uploads its inputs from pinned host memory, builds its
neighbour list, and runs either one shadow evaluation (charges, forces,
energies: the "qeq" kind) or the shadow XL-BOMD steps (the "md" kind) with its
list, mesh and n history resident on the device.  Then it copies the results
back and retires its context on its own stream.  Latency is arrival to
completion.  The loop reports p50 / p99 beside throughput.

MD steps are batched across requests (batch_md, the default).  After its
initial evaluation an MD request joins a stepper thread, which advances every
member in lockstep with qeq_batch_step on its own stream: per step, one host
synchronisation covers all members' skin checks and one CUDA graph launch runs
all their evaluations as parallel branches (the graph is rebuilt only when the
members change).  Systems below `batch_split_atoms` atoms and larger ones go to
two steppers (two threads, two streams), so that a small system never waits in
lockstep for the step of a large one.  A request joins at the next step once its initial evaluation
is done (a CUDA event orders it before the stepper's stream) and leaves when
its steps are done (an event orders its download after them).  A failing
batch step fails the requests stepped in it.

Isolation: the work of a request touches only its own context and tensors,
so its result does not depend on what runs beside it.  The only exception is
the order of floating-point atomics in the PME spread.
"""

from __future__ import annotations

import concurrent.futures as cf
import math
import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import ShadowBatch, ShadowMD, System, make_params


@dataclass
class Request:
    rid: int
    kind: str  # "qeq" or "md"
    R: np.ndarray
    box: np.ndarray
    chi: np.ndarray
    eta: np.ndarray
    sigma: np.ndarray
    mass: np.ndarray
    mesh: tuple
    V: np.ndarray | None = None
    steps: int = 0
    arrival: float = 0.0
    precision: str = "fp32_mixed"
    alpha: float = 0.34
    r_cut: float = 8.0
    skin: float = 1.0
    order: int = 4
    rank: int = 2
    k_d: int = 5
    dt: float = 0.5

    @property
    def n_atoms(self) -> int:
        return int(self.R.shape[0])


@dataclass
class Result:
    rid: int
    kind: str
    n_atoms: int
    q: np.ndarray
    F: np.ndarray
    R: np.ndarray
    energies: dict
    t_arrival: float
    t_admit: float
    t_done: float
    phases_ms: dict = field(default_factory=dict)  # host wall time per stage of the request
    error: str | None = None  # set when the request failed (its arrays are then None)

    @property
    def latency_ms(self) -> float:
        return 1e3 * (self.t_done - self.t_arrival)


def estimate_device_bytes(req: Request) -> int:
    """Device memory one request's context and tensors need (an upper estimate)."""
    n = req.n_atoms
    rl = req.r_cut + req.skin
    V = float(np.prod(req.box))
    width = math.ceil(1.2 * 4.0 / 3.0 * math.pi * rl ** 3 * n / V + 32.0)
    rs = 4 if req.precision == "fp32_mixed" else 8
    K0, K1, K2 = req.mesh
    mesh = K0 * K1 * K2
    meshc = K0 * K1 * (K2 // 2 + 1)
    per_atom = 4 * width + 8 * (3 * 12 + 2 * req.rank + req.k_d + 16) + 16 * rs + 64
    total = n * per_atom + rs * (mesh + 3 * 2 * meshc + 2 * mesh)
    return int(1.25 * total) + (4 << 20)


class _Member:
    """An MD request inside the batch stepper."""

    def __init__(self, md, steps, ready):
        self.md = md
        self.remaining = int(steps)
        self.ready = ready            # CUDA event: the request's set-up is done
        self.done_event = None        # CUDA event on the stepper's stream after its last step
        self.finished = threading.Event()
        self.error = None


class _BatchStepper:
    """Advances every MD request in flight by one step per tick with qeq_batch_step."""

    def __init__(self, device):
        self.device = device
        self.stream = torch.cuda.Stream(device)
        self.batch = ShadowBatch()
        self.cv = threading.Condition()
        self.joining = []
        self.members = []
        self.stop = False
        self.ticks = 0
        self.member_steps = 0
        self.thread = threading.Thread(target=self._run, daemon=True)
        self.thread.start()

    def submit(self, md, steps, ready) -> _Member:
        m = _Member(md, steps, ready)
        with self.cv:
            self.joining.append(m)
            self.cv.notify()
        return m

    def _run(self):
        with torch.cuda.device(self.device):
            while True:
                with self.cv:
                    while not (self.stop or self.joining or self.members):
                        self.cv.wait()
                    if self.stop and not self.joining and not self.members:
                        return
                    new, self.joining = self.joining, []
                for m in new:
                    self.stream.wait_event(m.ready)
                self.members.extend(new)
                try:
                    self.batch.step([m.md for m in self.members], self.stream)
                    self.ticks += 1
                    self.member_steps += len(self.members)
                except Exception as exc:  # every request of this step fails with it
                    for m in self.members:
                        m.error = f"{type(exc).__name__}: {exc}"
                        m.remaining = 0
                keep = []
                for m in self.members:
                    m.remaining -= 1
                    if m.remaining <= 0:
                        ev = torch.cuda.Event()
                        ev.record(self.stream)
                        m.done_event = ev
                        m.finished.set()
                    else:
                        keep.append(m)
                self.members = keep

    def close_thread(self):
        """Stop the thread once its members are done; the batch stays open for its stats."""
        with self.cv:
            self.stop = True
            self.cv.notify()
        self.thread.join()
        torch.cuda.synchronize(self.device)


class Server:
    batch_md = False  # set by __init__ (default on); subclasses with their own executor keep it off
    _stepper = None

    def __init__(self, device=0, max_inflight=8, hbm_budget=None, headroom=2 << 30, batch_md=True,
                 batch_split_atoms=4000):
        self.device = torch.device("cuda", device)
        self.batch_md = bool(batch_md)
        self.batch_split_atoms = int(batch_split_atoms)
        self._stepper = None
        self.max_inflight = int(max_inflight)
        with torch.cuda.device(self.device):
            free, _ = torch.cuda.mem_get_info(self.device)
        self.budget = int(hbm_budget) if hbm_budget is not None else max(0, free - headroom)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(self.max_inflight)]
        self._free_slots = list(range(self.max_inflight))
        self._lock = threading.Lock()
        self._reserved = 0

    # -- one request on one stream ------------------------------------------------
    def _execute(self, req: Request, slot: int, t0: float, t_admit: float) -> Result:
        stream = self.streams[slot]
        dev = self.device
        marks = [("start", time.perf_counter())]
        with torch.cuda.device(dev), torch.cuda.stream(stream):
            def up(a):
                h = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory()
                return h.to(dev, non_blocking=True)

            R, chi, eta, sigma, mass = (up(a) for a in (req.R, req.chi, req.eta, req.sigma,
                                                         req.mass))
            V = up(req.V if req.V is not None else np.zeros_like(req.R))
            p = make_params(req.n_atoms, req.box, alpha=req.alpha, r_cut=req.r_cut, skin=req.skin,
                            mesh=req.mesh, order=req.order, precision=req.precision,
                            krylov_rank=req.rank, dissipation_k=req.k_d, dt=req.dt)
            marks.append(("upload", time.perf_counter()))
            sysm = System(p, device=dev.index, stream=stream)
            marks.append(("create", time.perf_counter()))
            try:
                sysm.neighbor_build(R, stream)
                marks.append(("neighbor_build", time.perf_counter()))
                md = ShadowMD(sysm, chi, eta, sigma, mass, R, V,
                              torch.zeros(req.n_atoms, dtype=torch.float64, device=dev))
                md.init(stream)
                marks.append(("init", time.perf_counter()))
                if req.kind == "md" and req.steps > 0:
                    if self._stepper is not None:
                        ready = torch.cuda.Event()
                        ready.record(stream)
                        stepper = self._stepper[req.n_atoms >= self.batch_split_atoms]
                        member = stepper.submit(md, req.steps, ready)
                        member.finished.wait()
                        if member.error:
                            raise RuntimeError(member.error)
                        stream.wait_event(member.done_event)
                    else:
                        md.step(req.steps, stream)
                    marks.append(("steps", time.perf_counter()))
                out = [t.to("cpu", non_blocking=True) for t in (md.q, md.F, md.R, md.energies)]
                stream.synchronize()
                marks.append(("download", time.perf_counter()))
            finally:
                sysm.close()
                marks.append(("close", time.perf_counter()))
        e = out[3].tolist()
        energies = {"kinetic": e[0], "shadow_potential": e[1], "total": e[2], "lambda": e[4],
                    "sum_q": e[5], "residual_norm": e[6], "applies": e[7]}
        phases = {b[0]: 1e3 * (b[1] - a[1]) for a, b in zip(marks, marks[1:])}
        return Result(req.rid, req.kind, req.n_atoms, out[0].numpy(), out[1].numpy(),
                      out[2].numpy(), energies, t0 + req.arrival, t_admit, time.perf_counter(),
                      phases)

    # -- dispatcher -----------------------------------------------------------------
    def serve(self, requests, realtime=True):
        """Run the stream; returns (results ordered by rid, stats dict)."""
        pending = sorted(requests, key=lambda r: r.arrival)
        est = {r.rid: estimate_device_bytes(r) for r in pending}
        for r in pending:
            if est[r.rid] > self.budget:
                raise MemoryError(f"request {r.rid} needs {est[r.rid]} B > budget {self.budget} B")
        ready = []
        inflight = {}
        results = {}
        max_conc = 0
        pool = cf.ThreadPoolExecutor(max_workers=self.max_inflight)
        if self.batch_md:
            self._stepper = (_BatchStepper(self.device), _BatchStepper(self.device))
        t0 = time.perf_counter()
        try:
            while pending or ready or inflight:
                now = time.perf_counter() - t0
                while pending and (not realtime or pending[0].arrival <= now):
                    ready.append(pending.pop(0))
                # admit in arrival order while a slot and memory are free
                while ready and self._free_slots and self._reserved + est[ready[0].rid] <= self.budget:
                    req = ready.pop(0)
                    slot = self._free_slots.pop()
                    self._reserved += est[req.rid]
                    t_admit = time.perf_counter()
                    fut = pool.submit(self._execute, req, slot, t0, t_admit)
                    inflight[fut] = (req, slot, t_admit)
                    max_conc = max(max_conc, len(inflight))
                if not inflight:
                    if pending:
                        time.sleep(max(0.0, min(0.005, pending[0].arrival - (time.perf_counter() - t0))))
                    continue
                timeout = None
                if pending and realtime:
                    timeout = max(0.0, pending[0].arrival - (time.perf_counter() - t0))
                done, _ = cf.wait(list(inflight), timeout=timeout, return_when=cf.FIRST_COMPLETED)
                for fut in done:
                    req, slot, t_admit = inflight.pop(fut)
                    self._reserved -= est[req.rid]
                    self._free_slots.append(slot)
                    try:
                        results[req.rid] = fut.result()
                    except Exception as exc:  # reported with the request; the others go on
                        results[req.rid] = Result(req.rid, req.kind, req.n_atoms, None, None, None, {},
                                                  t0 + req.arrival, t_admit, time.perf_counter(),
                                                  error=f"{type(exc).__name__}: {exc}")
        finally:
            pool.shutdown(wait=True)
            steppers, self._stepper = self._stepper, None
            batching = None
            if steppers is not None:
                for st in steppers:
                    st.close_thread()
                ticks = sum(st.ticks for st in steppers)
                member_steps = sum(st.member_steps for st in steppers)
                batching = {"batch_steps": ticks, "member_steps": member_steps,
                            "mean_members_per_step": round(member_steps / max(1, ticks), 3),
                            "parent_graphs_built": sum(st.batch.stats()[0] for st in steppers),
                            "steppers": "below / from %d atoms" % self.batch_split_atoms}
                for st in steppers:
                    st.batch.close()
        t_end = time.perf_counter()
        res = [results[r] for r in sorted(results)]
        ok = [r for r in res if r.error is None]
        lat = np.array([r.latency_ms for r in ok]) if ok else np.zeros(1)
        mean = lambda xs: round(float(np.mean(xs)), 3) if len(xs) else 0.0
        stats = {
            "requests": len(res),
            "failed": len(res) - len(ok),
            "throughput_req_per_s": round(len(ok) / max(1e-9, t_end - t0), 3),
            "makespan_s": round(t_end - t0, 4),
            "latency_ms_p50": round(float(np.percentile(lat, 50)), 3),
            "latency_ms_p99": round(float(np.percentile(lat, 99)), 3),
            "latency_ms_max": round(float(lat.max()), 3),
            "max_concurrent": max_conc,
            "atoms_total": int(sum(r.n_atoms for r in ok)),
            "md_steps_total": int(sum(r.steps for r in requests if r.kind == "md")),
            "queue_ms_mean": mean([1e3 * (r.t_admit - r.t_arrival) for r in res]),
            "stage_ms_mean": {k: mean([r.phases_ms.get(k, 0.0) for r in ok])
                              for k in ("upload", "create", "neighbor_build", "init", "steps",
                                        "download", "close")},
            "md_batching": batching,
        }
        return res, stats


def request_from_box(rid, kind, box, mesh, V=None, steps=0, arrival=0.0, precision="fp32_mixed",
                     **kw) -> Request:
    """Wrap a water-box-like object (R, box, chi, eta, sigma, mass) into a Request."""
    return Request(rid=rid, kind=kind, R=box.R, box=np.asarray(box.box), chi=box.chi, eta=box.eta,
                   sigma=box.sigma, mass=box.mass, mesh=tuple(mesh), V=V, steps=steps,
                   arrival=arrival, precision=precision, **kw)
