"""ctypes binding of ``libqeq.so`` (include/qeq.h): argument marshalling only.

Each function keeps the C name and forwards device pointers taken from torch
tensors (CUDA, float64, contiguous).  Every step of the computation runs in
the CUDA library.  If the library is missing the import fails with an error,
and there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os

import torch

from . import _build

QEQ_OK = 0
QEQ_FP64 = 0
QEQ_FP32_MIXED = 1
QEQ_RECIP_PME = 0
QEQ_RECIP_EWALD = 1
QEQ_SHORT_NONE = 0
QEQ_SHORT_WATER = 1

_ERRORS = {
    -1: "QEQ_ERR_INVALID",
    -2: "QEQ_ERR_UNSUPPORTED",
    -3: "QEQ_ERR_CUDA",
    -4: "QEQ_ERR_CUFFT",
    -5: "QEQ_ERR_NOMEM",
    -6: "QEQ_ERR_NOLIST",
    -7: "QEQ_ERR_NONFINITE",
    -8: "QEQ_ERR_CAPACITY",
    -9: "QEQ_ERR_BOUNDS",
}


class QeqError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRORS.get(code, code)}: {msg}")
        self.code = code


class qeq_params(ctypes.Structure):
    _fields_ = [
        ("n_atoms", ctypes.c_int64),
        ("box", ctypes.c_double * 3),
        ("alpha", ctypes.c_double),
        ("r_cut", ctypes.c_double),
        ("skin", ctypes.c_double),
        ("mesh", ctypes.c_int32 * 3),
        ("order", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("gaussian_self", ctypes.c_int32),
        ("k_e", ctypes.c_double),
        ("max_neighbors", ctypes.c_int32),
        ("krylov_rank", ctypes.c_int32),
        ("krylov_tol", ctypes.c_double),
        ("q_tot", ctypes.c_double),
        ("dissipation_k", ctypes.c_int32),
        ("short_range", ctypes.c_int32),
        ("dt", ctypes.c_double),
        ("mass_unit", ctypes.c_double),
        ("recip", ctypes.c_int32),
        ("k_cut", ctypes.c_double),
    ]


# int (*)(void *user, int64_t n_atoms, const double *R, double *F, double *energy, void *stream)
QEQ_SHORT_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class qeq_nl_plan(ctypes.Structure):
    _fields_ = [
        ("nc", ctypes.c_int32 * 3),
        ("reach", ctypes.c_int32 * 3),
        ("brick", ctypes.c_int32 * 3),
        ("bricks", ctypes.c_int32 * 3),
        ("tile_reach", ctypes.c_int32 * 3),
        ("tile_bricks", ctypes.c_int32),
        ("n_bricks", ctypes.c_int64),
        ("cell_width", ctypes.c_double * 3),
        ("r_list", ctypes.c_double),
        ("band_lo", ctypes.c_float),
        ("band_hi", ctypes.c_float),
    ]


class qeq_md_state(ctypes.Structure):
    _fields_ = [(name, ctypes.c_void_p) for name in ("R", "V", "F", "Kf", "n_hist", "q", "energies")]


class qeq_md_params(ctypes.Structure):
    _fields_ = [(name, ctypes.c_void_p) for name in ("chi", "eta", "sigma", "mass")]


class qeq_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("applies", ctypes.c_int32),
                ("rel_residual", ctypes.c_double), ("lambda_", ctypes.c_double)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libqeq.so (building it first if it is absent and nvcc is available)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise OSError(f"{path} is missing; run __graft_entry__.build() first")
        _build.build()
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    L.qeq_params_default.argtypes = [ctypes.POINTER(qeq_params)]
    L.qeq_params_default.restype = None
    L.qeq_create.argtypes = [ctypes.POINTER(qeq_params), ctypes.POINTER(P)]
    L.qeq_create_async.argtypes = [ctypes.POINTER(qeq_params), P, ctypes.POINTER(P)]
    L.qeq_create_async.restype = ctypes.c_int
    L.qeq_destroy.argtypes = [P]
    L.qeq_destroy.restype = None
    L.qeq_last_error.argtypes = [P]
    L.qeq_last_error.restype = ctypes.c_char_p
    L.qeq_get_sizes.argtypes = [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]
    L.qeq_neighbor_build.argtypes = [P, P, P]
    L.qeq_neighbor_export.argtypes = [P, P, P, P]
    L.qeq_neighbor_displacement.argtypes = [P, P, ctypes.POINTER(ctypes.c_double), P]
    L.qeq_coulomb_apply.argtypes = [P, P, P, P, P, P, P, P, P]
    L.qeq_shadow_init.argtypes = [P, ctypes.POINTER(qeq_md_params), ctypes.POINTER(qeq_md_state), P]
    L.qeq_shadow_step.argtypes = [P, ctypes.POINTER(qeq_md_params), ctypes.POINTER(qeq_md_state), P]
    L.qeq_shadow_run.argtypes = [P, ctypes.POINTER(qeq_md_params), ctypes.POINTER(qeq_md_state),
                                 ctypes.c_int32, P]
    L.qeq_neighbor_build_noalloc.argtypes = [P, ctypes.c_int64, P, ctypes.c_double, ctypes.c_int32,
                                             P, P, ctypes.POINTER(ctypes.c_int32), P]
    L.qeq_neighbor_build_noalloc.restype = ctypes.c_int
    L.qeq_selftest_erfc32.argtypes = [P, P, ctypes.c_int64, P]
    L.qeq_selftest_erfc32.restype = ctypes.c_int
    L.qeq_selftest_erfc64.argtypes = [P, P, P, P, ctypes.c_int64, P]
    L.qeq_selftest_erfc64.restype = ctypes.c_int
    L.qeq_set_short_range.argtypes = [P, QEQ_SHORT_FN, P]
    L.qeq_set_short_range.restype = ctypes.c_int
    L.qeq_build_info.argtypes = [P]
    L.qeq_build_info.restype = ctypes.c_int
    L.qeq_bounds_status.argtypes = [P, P]
    L.qeq_bounds_status.restype = ctypes.c_int
    L.qeq_neighbor_plan.argtypes = [P, P]
    L.qeq_neighbor_plan.restype = ctypes.c_int
    L.qeq_pair_table_eval.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_int64,
                                      P, P, P, P, ctypes.POINTER(ctypes.c_int32)]
    L.qeq_pair_table_eval.restype = ctypes.c_int
    L.qeq_selftest_pair64.argtypes = [P, ctypes.c_int32, P, P, P, P, ctypes.c_int64, P]
    L.qeq_selftest_pair64.restype = ctypes.c_int
    SI = ctypes.POINTER(qeq_solve_info)
    L.qeq_solve.argtypes = [P, P, P, P, P, P, ctypes.c_double, ctypes.c_int32, ctypes.c_int32, SI, P]
    L.qeq_solve.restype = ctypes.c_int
    for name in ("qeq_bomd_init", "qeq_bomd_step"):
        getattr(L, name).argtypes = [P, ctypes.POINTER(qeq_md_params), ctypes.POINTER(qeq_md_state),
                                     ctypes.c_double, ctypes.c_int32, SI, P]
        getattr(L, name).restype = ctypes.c_int
    L.qeq_neighbor_export_coo.argtypes = [P, ctypes.c_int64, P, P, P, ctypes.POINTER(ctypes.c_int64), P]
    L.qeq_neighbor_export_coo.restype = ctypes.c_int
    L.qeq_set_graphs.argtypes = [P, ctypes.c_int]
    L.qeq_set_graphs.restype = ctypes.c_int
    L.qeq_profile_enable.argtypes = [P, ctypes.c_int]
    L.qeq_profile_read.argtypes = [P, P, P, ctypes.c_int]
    L.qeq_profile_phase_name.argtypes = [ctypes.c_int]
    L.qeq_profile_phase_name.restype = ctypes.c_char_p
    L.qeq_get_counters.argtypes = [P, P]
    L.qeq_graph_stats.argtypes = [P, P]
    L.qeq_batch_create.argtypes = [ctypes.POINTER(P)]
    L.qeq_batch_create.restype = ctypes.c_int
    L.qeq_batch_destroy.argtypes = [P]
    L.qeq_batch_destroy.restype = None
    L.qeq_batch_step.argtypes = [P, ctypes.c_int32, P, P, P, P]
    L.qeq_batch_step.restype = ctypes.c_int
    L.qeq_batch_stats.argtypes = [P, P]
    L.qeq_batch_stats.restype = ctypes.c_int
    L.qeq_params_from_tolerance.argtypes = [ctypes.POINTER(qeq_params), ctypes.c_double]
    L.qeq_params_from_tolerance.restype = ctypes.c_int
    L.qeq_set_neighbor_method.argtypes = [P, ctypes.c_int]
    L.qeq_set_neighbor_method.restype = ctypes.c_int
    L.qeq_measure_peaks.argtypes = [P, P]
    L.qeq_measure_peaks.restype = ctypes.c_int
    for name in ("qeq_profile_enable", "qeq_profile_read", "qeq_get_counters", "qeq_graph_stats"):
        getattr(L, name).restype = ctypes.c_int
    for name in ("qeq_create", "qeq_get_sizes", "qeq_neighbor_build", "qeq_neighbor_export",
                 "qeq_neighbor_displacement", "qeq_coulomb_apply", "qeq_shadow_init",
                 "qeq_shadow_step", "qeq_shadow_run"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _dev(t, name, shape=None, allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64:
        raise ValueError(f"{name} must be float64")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _check(ctx, rc):
    if rc != QEQ_OK:
        msg = load().qeq_last_error(ctx)
        raise QeqError(rc, msg.decode() if msg else "")
    return rc


# ---------------------------------------------------------------------------
# the C entry points
# ---------------------------------------------------------------------------

def qeq_params_default() -> qeq_params:
    p = qeq_params()
    load().qeq_params_default(ctypes.byref(p))
    return p


def qeq_create(params: qeq_params):
    h = ctypes.c_void_p()
    rc = load().qeq_create(ctypes.byref(params), ctypes.byref(h))
    _check(None, rc)
    return h


def qeq_create_async(params: qeq_params, stream=None):
    h = ctypes.c_void_p()
    rc = load().qeq_create_async(ctypes.byref(params), _stream(stream), ctypes.byref(h))
    _check(None, rc)
    return h


def qeq_destroy(ctx) -> None:
    if ctx:
        load().qeq_destroy(ctx)


def qeq_last_error(ctx) -> str:
    m = load().qeq_last_error(ctx)
    return m.decode() if m else ""


def qeq_get_sizes(ctx):
    n = ctypes.c_int64()
    w = ctypes.c_int32()
    _check(ctx, load().qeq_get_sizes(ctx, ctypes.byref(n), ctypes.byref(w)))
    return int(n.value), int(w.value)


def qeq_neighbor_build(ctx, R, stream=None) -> None:
    _check(ctx, load().qeq_neighbor_build(ctx, _dev(R, "R"), _stream(stream)))


def qeq_neighbor_export(ctx):
    """Host copies (counts [N], nbr [N, width], shift [N, width, 3]) in original numbering."""
    import numpy as np

    n, w = qeq_get_sizes(ctx)
    counts = np.zeros(n, dtype=np.int32)
    nbr = np.full((n, w), -1, dtype=np.int32)
    shift = np.zeros((n, w, 3), dtype=np.int8)
    _check(ctx, load().qeq_neighbor_export(ctx, counts.ctypes.data_as(ctypes.c_void_p),
                                           nbr.ctypes.data_as(ctypes.c_void_p),
                                           shift.ctypes.data_as(ctypes.c_void_p)))
    return counts, nbr, shift


def qeq_neighbor_displacement(ctx, R, stream=None) -> float:
    d2 = ctypes.c_double()
    _check(ctx, load().qeq_neighbor_displacement(ctx, _dev(R, "R"), ctypes.byref(d2),
                                                 _stream(stream)))
    return float(d2.value)


def qeq_coulomb_apply(ctx, R, q, sigma, v, E=None, F=None, energy=None, stream=None) -> None:
    _check(ctx, load().qeq_coulomb_apply(ctx, _dev(R, "R"), _dev(q, "q"), _dev(sigma, "sigma"),
                                         _dev(v, "v"), _dev(E, "E", allow_none=True),
                                         _dev(F, "F", allow_none=True),
                                         _dev(energy, "energy", allow_none=True),
                                         _stream(stream)))


def md_params(chi, eta, sigma, mass) -> qeq_md_params:
    return qeq_md_params(_dev(chi, "chi"), _dev(eta, "eta"), _dev(sigma, "sigma"), _dev(mass, "mass"))


def md_state(R, V, F, Kf, n_hist, q, energies) -> qeq_md_state:
    return qeq_md_state(_dev(R, "R"), _dev(V, "V"), _dev(F, "F"), _dev(Kf, "Kf"),
                        _dev(n_hist, "n_hist"), _dev(q, "q"), _dev(energies, "energies"))


def qeq_shadow_init(ctx, prm: qeq_md_params, st: qeq_md_state, stream=None) -> None:
    _check(ctx, load().qeq_shadow_init(ctx, ctypes.byref(prm), ctypes.byref(st), _stream(stream)))


def qeq_shadow_step(ctx, prm: qeq_md_params, st: qeq_md_state, stream=None) -> None:
    _check(ctx, load().qeq_shadow_step(ctx, ctypes.byref(prm), ctypes.byref(st), _stream(stream)))


def qeq_shadow_run(ctx, prm: qeq_md_params, st: qeq_md_state, n_steps: int, stream=None) -> None:
    _check(ctx, load().qeq_shadow_run(ctx, ctypes.byref(prm), ctypes.byref(st), int(n_steps),
                                      _stream(stream)))


QEQ_NUM_PHASES = 10


def qeq_profile_enable(ctx, on: bool) -> None:
    _check(ctx, load().qeq_profile_enable(ctx, int(bool(on))))


def qeq_profile_read(ctx):
    """{phase name: (milliseconds, launches)} accumulated since the last read (synchronises)."""
    import numpy as np

    ms = np.zeros(QEQ_NUM_PHASES, dtype=np.float64)
    cnt = np.zeros(QEQ_NUM_PHASES, dtype=np.int64)
    _check(ctx, load().qeq_profile_read(ctx, ms.ctypes.data_as(ctypes.c_void_p),
                                        cnt.ctypes.data_as(ctypes.c_void_p), QEQ_NUM_PHASES))
    return {qeq_profile_phase_name(k): (float(ms[k]), int(cnt[k])) for k in range(QEQ_NUM_PHASES)}


def qeq_profile_phase_name(phase: int) -> str:
    return load().qeq_profile_phase_name(int(phase)).decode()


def qeq_get_counters(ctx):
    """(kernel launches, neighbour builds, Coulomb applies, cuFFT executions)."""
    import numpy as np

    out = np.zeros(4, dtype=np.int64)
    _check(ctx, load().qeq_get_counters(ctx, out.ctypes.data_as(ctypes.c_void_p)))
    return tuple(int(x) for x in out)


def qeq_measure_peaks(stream=None) -> dict:
    """Measured FP32 / FP64 FLOP/s, MUFU ops/s and the SM count of the current device."""
    import numpy as np

    out = np.zeros(4, dtype=np.float64)
    _check(None, load().qeq_measure_peaks(out.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
    return {"fp32_flops": float(out[0]), "fp64_flops": float(out[1]), "mufu_ops": float(out[2]),
            "sm_count": int(out[3])}


def qeq_graph_stats(ctx):
    """(shadow-step graphs captured, steps replayed from a graph) since creation."""
    import numpy as np

    out = np.zeros(2, dtype=np.int64)
    _check(ctx, load().qeq_graph_stats(ctx, out.ctypes.data_as(ctypes.c_void_p)))
    return tuple(int(x) for x in out)


def qeq_neighbor_build_noalloc(R, box, r_list, counts, nbr, stream=None) -> None:
    """Allocation-free neighbour build into caller buffers (see include/qeq.h).

    R: CUDA float64 [N, 3]; counts: CUDA int32 [N]; nbr: CUDA int32 [N, width].
    Raises QeqError (code -8 with the needed width in ``.needed_width``) when a
    row does not fit.
    """
    import numpy as np

    n = int(R.shape[0])
    for t, name, dt in ((counts, "counts", torch.int32), (nbr, "nbr", torch.int32)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous CUDA int32 tensor")
    if tuple(counts.shape) != (n,) or nbr.dim() != 2 or nbr.shape[0] != n:
        raise ValueError("counts must be [N] and nbr [N, width]")
    boxh = np.ascontiguousarray(np.asarray(box, dtype=np.float64))
    need = ctypes.c_int32(0)
    rc = load().qeq_neighbor_build_noalloc(_dev(R, "R"), n, boxh.ctypes.data_as(ctypes.c_void_p),
                                           float(r_list), int(nbr.shape[1]),
                                           ctypes.c_void_p(counts.data_ptr()),
                                           ctypes.c_void_p(nbr.data_ptr()), ctypes.byref(need),
                                           _stream(stream))
    if rc != QEQ_OK:
        err = QeqError(rc, qeq_last_error(None))
        err.needed_width = int(need.value)
        raise err


def qeq_selftest_erfc32(x, out, stream=None) -> None:
    """FP32 erfc of the real-space kernel on CUDA float32 tensors x -> out."""
    for t, name in ((x, "x"), (out, "out")):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
                and t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous CUDA float32 tensor")
    _check(None, load().qeq_selftest_erfc32(ctypes.c_void_p(x.data_ptr()),
                                            ctypes.c_void_p(out.data_ptr()), x.numel(),
                                            _stream(stream)))


def qeq_selftest_erfc64(ctx, x, out, dout, stream=None) -> None:
    """FP64 piecewise erfc and its derivative of the real-space kernel (CUDA float64 tensors)."""
    _check(ctx, load().qeq_selftest_erfc64(ctx, _dev(x, "x"), _dev(out, "out"), _dev(dout, "dout"),
                                           x.numel(), _stream(stream)))


def qeq_set_short_range(ctx, fn, user=None) -> None:
    """Set (fn: a QEQ_SHORT_FN) or clear (fn None) the user short-range model.
    The caller keeps fn alive while it is set."""
    cb = fn if fn is not None else QEQ_SHORT_FN()
    _check(ctx, load().qeq_set_short_range(ctx, cb, user))


def qeq_build_info() -> dict:
    """{"bounds_checked": bool}: whether the loaded library is the bounds-checked build."""
    b = ctypes.c_int32(0)
    _check(None, load().qeq_build_info(ctypes.byref(b)))
    return {"bounds_checked": bool(b.value)}


def qeq_bounds_status(ctx) -> int:
    """First failing bounds-check site since the last call (0: none); raises
    QeqError(QEQ_ERR_BOUNDS) when one failed.  Synchronises."""
    site = ctypes.c_int32(0)
    _check(ctx, load().qeq_bounds_status(ctx, ctypes.byref(site)))
    return int(site.value)


def qeq_neighbor_plan(params: qeq_params) -> dict:
    """Host-only cell / brick decomposition and FP32 prefilter band for params."""
    out = qeq_nl_plan()
    _check(None, load().qeq_neighbor_plan(ctypes.byref(params), ctypes.byref(out)))
    return {"nc": list(out.nc), "reach": list(out.reach), "brick": list(out.brick),
            "bricks": list(out.bricks), "tile_reach": list(out.tile_reach),
            "tile_bricks": int(out.tile_bricks), "n_bricks": int(out.n_bricks),
            "cell_width": list(out.cell_width), "r_list": float(out.r_list),
            "band_lo": float(out.band_lo), "band_hi": float(out.band_hi)}


def qeq_pair_table_eval(alpha, smax, which, arg):
    """Host evaluation of the FP64 kernel's pair-function table (no device).

    arg: float64 array.  Returns (F, G, in_table, kept): F, G are NaN where
    in_table is 0 (outside the kept pieces)."""
    import numpy as np

    a = np.ascontiguousarray(arg, dtype=np.float64)
    F = np.full(a.shape, np.nan)
    G = np.full(a.shape, np.nan)
    inn = np.zeros(a.shape, dtype=np.int32)
    kept = ctypes.c_int32(0)
    ptr = lambda x: ctypes.c_void_p(x.ctypes.data)
    _check(None, load().qeq_pair_table_eval(float(alpha), float(smax), int(which), a.size, ptr(a),
                                            ptr(F), ptr(G), ptr(inn), ctypes.byref(kept)))
    return F, G, inn, int(kept.value)


def qeq_selftest_pair64(ctx, which, arg, F, G, in_table, stream=None) -> None:
    """Device evaluation of an FP64 context's pair-function table (CUDA tensors)."""
    if not (isinstance(in_table, torch.Tensor) and in_table.is_cuda and in_table.dtype == torch.int32
            and in_table.is_contiguous()):
        raise ValueError("in_table must be a contiguous CUDA int32 tensor")
    _check(ctx, load().qeq_selftest_pair64(ctx, int(which), _dev(arg, "arg"), _dev(F, "F"), _dev(G, "G"),
                                           ctypes.c_void_p(in_table.data_ptr()), arg.numel(),
                                           _stream(stream)))


def qeq_solve(ctx, R, chi, eta, sigma, q, tol, max_iter=500, restart=40, stream=None):
    """Regular QEq by GMRES; q (CUDA float64 [N]) is the guess on entry, the solution on exit."""
    info = qeq_solve_info()
    _check(ctx, load().qeq_solve(ctx, _dev(R, "R"), _dev(chi, "chi"), _dev(eta, "eta"),
                                 _dev(sigma, "sigma"), _dev(q, "q"), float(tol), int(max_iter),
                                 int(restart), ctypes.byref(info), _stream(stream)))
    return {"iterations": info.iterations, "applies": info.applies,
            "rel_residual": info.rel_residual, "lambda": info.lambda_}


def _bo_state(R, V, F, q, energies) -> qeq_md_state:
    return qeq_md_state(_dev(R, "R"), _dev(V, "V"), _dev(F, "F"), None, None, _dev(q, "q"),
                        _dev(energies, "energies"))


def qeq_bomd_init(ctx, prm, st, tol, max_iter=500, stream=None):
    info = qeq_solve_info()
    _check(ctx, load().qeq_bomd_init(ctx, ctypes.byref(prm), ctypes.byref(st), float(tol),
                                     int(max_iter), ctypes.byref(info), _stream(stream)))
    return {"iterations": info.iterations, "applies": info.applies,
            "rel_residual": info.rel_residual, "lambda": info.lambda_}


def qeq_bomd_step(ctx, prm, st, tol, max_iter=500, stream=None):
    info = qeq_solve_info()
    _check(ctx, load().qeq_bomd_step(ctx, ctypes.byref(prm), ctypes.byref(st), float(tol),
                                     int(max_iter), ctypes.byref(info), _stream(stream)))
    return {"iterations": info.iterations, "applies": info.applies,
            "rel_residual": info.rel_residual, "lambda": info.lambda_}


def qeq_neighbor_export_coo(ctx, capacity=None, stream=None):
    """Device COO copy of the list: (pair_i, pair_j, image_code) CUDA tensors."""
    n, w = qeq_get_sizes(ctx)
    cap = int(capacity) if capacity is not None else n * w
    dev = torch.device("cuda", torch.cuda.current_device())
    pi = torch.empty(cap, dtype=torch.int32, device=dev)
    pj = torch.empty(cap, dtype=torch.int32, device=dev)
    code = torch.empty(cap, dtype=torch.int8, device=dev)
    npairs = ctypes.c_int64(0)
    _check(ctx, load().qeq_neighbor_export_coo(ctx, cap, ctypes.c_void_p(pi.data_ptr()),
                                               ctypes.c_void_p(pj.data_ptr()),
                                               ctypes.c_void_p(code.data_ptr()), ctypes.byref(npairs),
                                               _stream(stream)))
    m = int(npairs.value)
    return pi[:m], pj[:m], code[:m]


def qeq_batch_create():
    h = ctypes.c_void_p()
    _check(None, load().qeq_batch_create(ctypes.byref(h)))
    return h


def qeq_batch_destroy(h) -> None:
    if h:
        load().qeq_batch_destroy(h)


def batch_arrays(ctxs, prms, sts):
    """The C argument arrays of qeq_batch_step for one member list."""
    n = len(ctxs)
    if not (n == len(prms) == len(sts)):
        raise ValueError("ctxs, prms and sts must have the same length")
    c_arr = (ctypes.c_void_p * n)(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    p_arr = (qeq_md_params * n)(*prms)
    s_arr = (qeq_md_state * n)(*sts)
    return (n, c_arr, p_arr, s_arr, [ctypes.cast(a, ctypes.c_void_p) for a in (c_arr, p_arr, s_arr)])


def qeq_batch_step_arrays(h, arrays, stream=None) -> None:
    """qeq_batch_step with arrays from batch_arrays.  On failure the error message is the
    failing member's, else the library's."""
    n, c_arr, _, _, ptrs = arrays
    rc = load().qeq_batch_step(h, n, ptrs[0], ptrs[1], ptrs[2], _stream(stream))
    if rc != QEQ_OK:
        for c in c_arr:
            msg = load().qeq_last_error(c)
            if msg:
                raise QeqError(rc, msg.decode())
        _check(None, rc)


def qeq_batch_step(h, ctxs, prms, sts, stream=None) -> None:
    """One batched shadow step of the member contexts (see include/qeq.h)."""
    qeq_batch_step_arrays(h, batch_arrays(ctxs, prms, sts), stream)


def qeq_batch_stats(h):
    """(parent graphs built, graph launches) of a batch."""
    import numpy as np

    out = np.zeros(2, dtype=np.int64)
    _check(None, load().qeq_batch_stats(h, out.ctypes.data_as(ctypes.c_void_p)))
    return tuple(int(x) for x in out)


def qeq_params_from_tolerance(params: qeq_params, delta: float) -> qeq_params:
    """Set params.alpha, params.mesh and params.k_cut from the error tolerance delta
    (OpenMM's PME rule; see include/qeq.h).  Host only; returns params."""
    _check(None, load().qeq_params_from_tolerance(ctypes.byref(params), float(delta)))
    return params


QEQ_NL_BRICK, QEQ_NL_ATOM = 0, 1


def qeq_set_neighbor_method(ctx, method) -> None:
    """Neighbour search of the next builds: "brick" (QEQ_NL_BRICK) or "atom" (QEQ_NL_ATOM)."""
    if isinstance(method, str):
        method = {"brick": QEQ_NL_BRICK, "atom": QEQ_NL_ATOM}[method]
    _check(ctx, load().qeq_set_neighbor_method(ctx, int(method)))


def qeq_set_graphs(ctx, on: bool) -> None:
    _check(ctx, load().qeq_set_graphs(ctx, int(bool(on))))
