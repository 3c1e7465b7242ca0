"""GB300-native shadow charge-equilibration Coulomb library (Python side).

The compute path is ``libqeq.so`` (hand-written sm_103a CUDA behind the C ABI in
``include/qeq.h``).  This package only marshals torch tensors into that ABI:

* ``_lib``     -- one function per C entry point, same names (qeq_create,
                  qeq_neighbor_build, qeq_coulomb_apply, qeq_shadow_step, ...)
* ``System``   -- owns one context plus the output tensors of an apply
* ``ShadowMD`` -- owns the caller-side state arrays of the shadow XL-BOMD step
* ``ShadowBatch`` -- steps several ShadowMD systems at once (one sync, one graph)
* ``autograd`` -- ``CoulombEnergy``, a torch.autograd.Function over the apply
"""

from __future__ import annotations

import torch

from . import _lib
from ._lib import (  # noqa: F401
    QEQ_FP32_MIXED,
    QEQ_FP64,
    QEQ_SHORT_NONE,
    QEQ_SHORT_WATER,
    QeqError,
    load,
    md_params,
    md_state,
    qeq_coulomb_apply,
    qeq_create,
    qeq_create_async,
    qeq_destroy,
    qeq_get_counters,
    qeq_get_sizes,
    qeq_graph_stats,
    qeq_set_neighbor_method,
    qeq_measure_peaks,
    qeq_last_error,
    qeq_neighbor_build,
    qeq_neighbor_displacement,
    qeq_neighbor_export,
    qeq_neighbor_plan,
    qeq_pair_table_eval,
    qeq_params,
    qeq_params_default,
    qeq_params_from_tolerance,
    qeq_profile_enable,
    qeq_profile_phase_name,
    qeq_profile_read,
    qeq_bomd_init,
    qeq_bomd_step,
    qeq_shadow_init,
    qeq_shadow_run,
    qeq_selftest_pair64,
    qeq_shadow_step,
    qeq_solve,
)

from .autograd import CoulombEnergy, coulomb_energy  # noqa: E402,F401

PRECISIONS = {"fp64": QEQ_FP64, "fp32_mixed": QEQ_FP32_MIXED}


def make_params(n_atoms, box, alpha=0.34, r_cut=8.0, skin=1.0, mesh=(32, 32, 32), order=4,
                precision="fp64", gaussian_self=True, k_e=14.3996454784, max_neighbors=0,
                krylov_rank=2, q_tot=0.0, dissipation_k=5, dt=0.5, short_range=QEQ_SHORT_NONE,
                mass_unit=103.6427, krylov_tol=0.0, recip="pme", k_cut=0.0) -> qeq_params:
    p = qeq_params_default()
    p.n_atoms = int(n_atoms)
    for d in range(3):
        p.box[d] = float(box[d])
        p.mesh[d] = int(mesh[d])
    p.alpha = float(alpha)
    p.r_cut = float(r_cut)
    p.skin = float(skin)
    p.order = int(order)
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    p.gaussian_self = int(bool(gaussian_self))
    p.k_e = float(k_e)
    p.max_neighbors = int(max_neighbors)
    p.krylov_rank = int(krylov_rank)
    p.krylov_tol = float(krylov_tol)
    p.recip = {"pme": _lib.QEQ_RECIP_PME, "ewald": _lib.QEQ_RECIP_EWALD}[recip] \
        if isinstance(recip, str) else int(recip)
    p.k_cut = float(k_cut)
    p.q_tot = float(q_tot)
    p.dissipation_k = int(dissipation_k)
    p.dt = float(dt)
    p.short_range = int(short_range)
    p.mass_unit = float(mass_unit)
    return p


class System:
    """One periodic system on the current CUDA device, with apply outputs preallocated."""

    short_range_error = None  # the exception of the last failing user short-range call
    _short_cb = None

    def _run(self, fn, *args):
        """Call a library entry point; a failure caused by the user short-range model
        is raised with that model's exception as its cause."""
        try:
            return fn(*args)
        except QeqError as err:
            cause = self.short_range_error
            if cause is not None:
                self.short_range_error = None
                raise err from cause
            raise

    @property
    def has_user_short_range(self) -> bool:
        return self._short_cb is not None

    def __init__(self, params: qeq_params, device=None, stream=None):
        """stream=None: qeq_create; a torch.cuda.Stream: qeq_create_async on that stream."""
        self.params = params
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.n = int(params.n_atoms)
        with torch.cuda.device(self.device):
            self.ctx = qeq_create(params) if stream is None else qeq_create_async(params, stream)
        f64 = dict(dtype=torch.float64, device=self.device)
        self.v = torch.empty(self.n, **f64)
        self.E = torch.empty(self.n, 3, **f64)
        self.F = torch.empty(self.n, 3, **f64)
        self.energy = torch.zeros(4, **f64)

    def close(self):
        if getattr(self, "ctx", None):
            qeq_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def neighbor_build(self, R, stream=None):
        qeq_neighbor_build(self.ctx, R, stream)

    def neighbor_export(self):
        return qeq_neighbor_export(self.ctx)

    def displacement2(self, R, stream=None) -> float:
        return qeq_neighbor_displacement(self.ctx, R, stream)

    def set_short_range(self, fn=None):
        """A user short-range model for the MD steps on this system: fn(R) ->
        (F, E) with R, F CUDA float64 [N, 3] tensors and E a CUDA float64
        scalar tensor, run on the step's stream.  fn None restores the
        parameter-selected model.  Steps are not captured into graphs while it
        is set."""
        self.short_range_error = None
        if fn is None:
            _lib.qeq_set_short_range(self.ctx, None)
            self._short_cb = None
            return
        dev = self.device

        def view(ptr, shape):
            class _Cai:
                __cuda_array_interface__ = {"shape": shape, "typestr": "<f8", "data": (ptr, False),
                                            "version": 3, "strides": None}
            return torch.as_tensor(_Cai(), device=dev)

        def cb(user, n, R_ptr, F_ptr, E_ptr, stream_ptr):
            self.short_range_error = None
            try:
                st = torch.cuda.ExternalStream(stream_ptr, device=dev) if stream_ptr else \
                    torch.cuda.default_stream(dev)
                with torch.cuda.device(dev), torch.cuda.stream(st):
                    F, E = fn(view(R_ptr, (n, 3)))
                    view(F_ptr, (n, 3)).copy_(F)
                    view(E_ptr, (1,)).copy_(torch.as_tensor(E, dtype=torch.float64, device=dev).reshape(1))
                return 0
            except Exception as exc:  # the library reports it as QEQ_ERR_INVALID
                self.short_range_error = exc
                return 1

        self._short_cb = _lib.QEQ_SHORT_FN(cb)  # kept alive while set
        _lib.qeq_set_short_range(self.ctx, self._short_cb)

    def apply(self, R, q, sigma, field=True, stream=None):
        """v = Phi q; returns (v, E, F, energy[4]) views of the preallocated outputs."""
        qeq_coulomb_apply(self.ctx, R, q, sigma, self.v, self.E if field else None,
                          self.F if field else None, self.energy, stream)
        return self.v, self.E, self.F, self.energy


class ShadowMD:
    """Caller-side state of the shadow XL-BOMD step (all tensors on the device)."""

    def __init__(self, system: System, chi, eta, sigma, mass, R, V, n0):
        self.sys = system
        p = system.params
        n = system.n
        f64 = dict(dtype=torch.float64, device=system.device)
        self.chi, self.eta, self.sigma, self.mass = (t.contiguous() for t in (chi, eta, sigma, mass))
        self.R = R.clone().contiguous()
        self.V = V.clone().contiguous()
        self.F = torch.zeros(n, 3, **f64)
        self.Kf = torch.zeros(n, **f64)
        self.n_hist = n0.reshape(1, n).repeat(p.dissipation_k + 1, 1).contiguous()
        self.q = torch.zeros(n, **f64)
        self.energies = torch.zeros(8, **f64)
        self._prm = md_params(self.chi, self.eta, self.sigma, self.mass)
        self._st = md_state(self.R, self.V, self.F, self.Kf, self.n_hist, self.q, self.energies)

    def init(self, stream=None):
        self.sys._run(qeq_shadow_init, self.sys.ctx, self._prm, self._st, stream)

    # order of the tensors in pack(): parameters, then the state the step advances,
    # then its results
    PACK_PARAMS = ("chi", "eta", "sigma", "mass")
    PACK_STATE = ("R", "V", "F", "Kf", "n_hist")
    PACK_RESULTS = ("q", "energies")

    def pack(self):
        """Re-home parameters, state and results into one contiguous float64 device
        buffer [chi, eta, sigma, mass | R, V, F, Kf, n_hist | q, energies] and point
        the step at it.  Returns (buffer, (n_params, n_state, n_results)) in elements,
        so a caller that keeps the state on the host moves it with one copy each way:
        H2D of buffer[:n_params + n_state], D2H of buffer[n_params:].  Waits for the
        device (a one-time set-up step)."""
        names = self.PACK_PARAMS + self.PACK_STATE + self.PACK_RESULTS
        sizes = [getattr(self, k).numel() for k in names]
        buf = torch.empty(sum(sizes), dtype=torch.float64, device=self.sys.device)
        off = 0
        for k, sz in zip(names, sizes):
            t = getattr(self, k)
            view = buf[off:off + sz].view(t.shape)
            view.copy_(t)
            setattr(self, k, view)
            off += sz
        self._prm = md_params(self.chi, self.eta, self.sigma, self.mass)
        self._st = md_state(self.R, self.V, self.F, self.Kf, self.n_hist, self.q, self.energies)
        torch.cuda.synchronize(self.sys.device)  # the copies ran on the current stream
        count = lambda group: sum(getattr(self, k).numel() for k in group)
        return buf, (count(self.PACK_PARAMS), count(self.PACK_STATE), count(self.PACK_RESULTS))

    def step(self, n_steps: int = 1, stream=None):
        if n_steps == 1:
            self.sys._run(qeq_shadow_step, self.sys.ctx, self._prm, self._st, stream)
        else:
            self.sys._run(qeq_shadow_run, self.sys.ctx, self._prm, self._st, n_steps, stream)

    def energy_dict(self):
        e = self.energies.cpu().tolist()
        return {"kinetic": e[0], "shadow_potential": e[1], "total": e[2], "short": e[3],
                "lambda": e[4], "sum_q": e[5], "residual_norm": e[6], "applies": e[7]}

    def checkpoint(self, path, step: int = 0) -> None:
        """Write the MD state, the per-atom parameters, `step` and the system
        signature to the host file `path` (see checkpoint.py).  Waits for the
        device."""
        from . import checkpoint as ck

        torch.cuda.synchronize(self.sys.device)
        arrays = {k: getattr(self, k).cpu().numpy() for k in ck.STATE + ck.PARAMS}
        ck.write(path, arrays, ck.system_signature(self.sys.params, self.sys.has_user_short_range),
                 step)

    @classmethod
    def resume(cls, system: System, path):
        """A ShadowMD on `system` continuing from the checkpoint `path`, and the
        stored step count.  The system must have the checkpoint's parameters
        (ValueError otherwise); its neighbour list is built at the stored
        positions.  Waits for the device."""
        from . import checkpoint as ck

        arrays, signature, step = ck.read(path)
        ck.check_signature(signature, ck.system_signature(system.params,
                                                          system.has_user_short_range))
        t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=system.device).contiguous()
        md = cls(system, t(arrays["chi"]), t(arrays["eta"]), t(arrays["sigma"]), t(arrays["mass"]),
                 t(arrays["R"]), t(arrays["V"]), t(arrays["n_hist"][0]))
        for k in ("F", "Kf", "n_hist", "q", "energies"):
            getattr(md, k).copy_(t(arrays[k]))
        system.neighbor_build(md.R)
        torch.cuda.synchronize(system.device)
        return md, step


class ShadowBatch:
    """Advances several ShadowMD systems by one step each with qeq_batch_step: one host
    synchronisation for all skin checks and one CUDA graph for all evaluations.  The
    members' earlier work must be ordered before `stream`."""

    def __init__(self):
        self.h = _lib.qeq_batch_create()
        self._key = None
        self._arrays = None

    def step(self, mds, stream=None):
        if not mds:
            return
        key = tuple(id(md) for md in mds)
        if key != self._key:  # the argument arrays change only with the member list
            self._arrays = _lib.batch_arrays([md.sys.ctx for md in mds], [md._prm for md in mds],
                                             [md._st for md in mds])
            self._key = key
        _lib.qeq_batch_step_arrays(self.h, self._arrays, stream)

    def stats(self):
        """(parent graphs built, graph launches)."""
        return _lib.qeq_batch_stats(self.h)

    def close(self):
        if getattr(self, "h", None):
            _lib.qeq_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BOMD:
    """Caller-side state of regular Born-Oppenheimer MD with a GMRES QEq solve per step."""

    def __init__(self, system: System, chi, eta, sigma, mass, R, V, q0, tol, max_iter=500):
        self.sys = system
        n = system.n
        f64 = dict(dtype=torch.float64, device=system.device)
        self.chi, self.eta, self.sigma, self.mass = (t.contiguous() for t in (chi, eta, sigma, mass))
        self.R = R.clone().contiguous()
        self.V = V.clone().contiguous()
        self.F = torch.zeros(n, 3, **f64)
        self.q = q0.clone().contiguous()
        self.energies = torch.zeros(8, **f64)
        self.tol = float(tol)
        self.max_iter = int(max_iter)
        self._prm = md_params(self.chi, self.eta, self.sigma, self.mass)
        self._st = _lib._bo_state(self.R, self.V, self.F, self.q, self.energies)

    def init(self, stream=None):
        return self.sys._run(qeq_bomd_init, self.sys.ctx, self._prm, self._st, self.tol,
                             self.max_iter, stream)

    def step(self, stream=None):
        return self.sys._run(qeq_bomd_step, self.sys.ctx, self._prm, self._st, self.tol,
                             self.max_iter, stream)

    def energy_dict(self):
        e = self.energies.cpu().tolist()
        return {"kinetic": e[0], "potential": e[1], "total": e[2], "short": e[3], "lambda": e[4],
                "sum_q": e[5], "rel_residual": e[6], "applies": e[7]}
