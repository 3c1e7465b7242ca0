"""Context creation rejects invalid and unsupported parameters before any GPU work (CPU).

qeq_create validates its parameters first, so each case below fails with its
status code and a message naming the field on a host without a GPU.  The
cases are the degenerate and limit sizes (no atoms, more atoms than the
24-bit sorted index holds, a mesh smaller than the spline order) and the
combinations the library does not run.
"""

import pytest

import paper_2503_21176_gb300 as qg
from paper_2503_21176_gb300 import _lib

INVALID, UNSUPPORTED = -1, -2  # QEQ_ERR_INVALID, QEQ_ERR_UNSUPPORTED (include/qeq.h)


def _params(**kw):
    p = qg.make_params(kw.pop("n_atoms", 648), kw.pop("box", (18.63, 18.63, 18.63)))
    for k, v in kw.items():
        if k in ("box", "mesh"):
            for d in range(3):
                getattr(p, k)[d] = v[d]
        else:
            setattr(p, k, v)
    return p


def _fails(code, field, **kw):
    with pytest.raises(qg.QeqError) as info:
        qg.qeq_create(_params(**kw))
    assert info.value.code == code
    assert field in str(info.value)


def test_empty_system_is_rejected():
    _fails(INVALID, "n_atoms", n_atoms=0)


def test_atom_count_above_the_sorted_index_range_is_rejected():
    _fails(INVALID, "n_atoms", n_atoms=(1 << 24))


def test_box_must_be_positive_and_finite():
    _fails(INVALID, "box[1]", box=(18.6, 0.0, 18.6))
    _fails(INVALID, "box[2]", box=(18.6, 18.6, float("inf")))


def test_mesh_limits():
    _fails(INVALID, "mesh[0]", mesh=(3, 32, 32))
    _fails(INVALID, "mesh[1]", mesh=(32, 4097, 32))
    _fails(INVALID, "spline order", mesh=(32, 32, 5), order=6)


def test_spline_order_and_krylov_limits():
    _fails(UNSUPPORTED, "order", order=3, mesh=(32, 32, 32))
    _fails(UNSUPPORTED, "order", order=9, mesh=(32, 32, 32))
    _fails(INVALID, "krylov_rank", krylov_rank=0)
    _fails(INVALID, "krylov_rank", krylov_rank=9)
    _fails(INVALID, "dissipation_k", dissipation_k=2)
    _fails(INVALID, "krylov_tol", krylov_tol=-0.1)


def test_physical_parameters_must_be_positive():
    _fails(INVALID, "alpha", alpha=0.0)
    _fails(INVALID, "r_cut", r_cut=-1.0)
    _fails(INVALID, "skin", skin=-0.1)
    _fails(INVALID, "dt", dt=0.0)


def test_unsupported_combinations():
    _fails(UNSUPPORTED, "FP64 only", recip=_lib.QEQ_RECIP_EWALD, precision=_lib.QEQ_FP32_MIXED)
    _fails(INVALID, "O, H, H", n_atoms=647, short_range=_lib.QEQ_SHORT_WATER)
    _fails(INVALID, "precision", precision=7)
