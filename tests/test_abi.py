"""The C-ABI library loads and exports every entry point that include/qeq.h declares (CPU)."""

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "qeq.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qeq_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_2503_21176_gb300 import _build

    path = _build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert "qeq_coulomb_apply" in names and "qeq_neighbor_build" in names
    assert "qeq_shadow_step" in names
    for name in names:
        assert hasattr(lib, name), f"{name} is declared in qeq.h but not exported"


def test_only_qeq_symbols_are_exported():
    import subprocess

    from paper_2503_21176_gb300 import _build

    out = subprocess.run(["nm", "-D", "--defined-only", _build.build()], capture_output=True,
                         text=True, check=True).stdout
    text_syms = [ln.split()[-1] for ln in out.splitlines() if " T " in ln]
    assert text_syms and all(s.startswith("qeq_") for s in text_syms)
    assert set(text_syms) == set(_declared())


def test_params_default_without_gpu():
    """qeq_params_default touches no device, so it runs on a CPU-only host."""
    import paper_2503_21176_gb300 as qg

    p = qg.qeq_params_default()
    assert abs(p.alpha - 0.34) < 1e-15 and p.order == 4 and p.gaussian_self == 1
    assert abs(p.k_e - 14.3996454784) < 1e-12 and p.dissipation_k == 5


def test_binding_rejects_host_tensors():
    import numpy as np
    import pytest
    import torch

    import paper_2503_21176_gb300 as qg

    with pytest.raises(ValueError):
        qg._lib._dev(torch.zeros(3, dtype=torch.float64), "x")
    with pytest.raises(ValueError):
        qg._lib._dev(np.zeros(3), "x")


def test_short_range_callback_needs_a_context():
    """qeq_set_short_range rejects a NULL context before touching a device."""
    from paper_2503_21176_gb300 import _lib

    assert _lib.load().qeq_set_short_range(None, _lib.QEQ_SHORT_FN(), None) == -1
