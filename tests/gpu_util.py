"""Shared helpers for the GPU parity tests (inputs from workloads/, references from oracle/)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def cuda_or_skip():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_21176_gb300 as qg

    qg.load()
    return qg


def dev_tensor(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def canonical_rows_gpu(counts, nbr, shift):
    rows = []
    for i in range(len(counts)):
        c = int(counts[i])
        ent = sorted((int(nbr[i, k]), tuple(int(x) for x in shift[i, k])) for k in range(c))
        rows.append(ent)
    return rows


def canonical_rows_oracle(off, j, s):
    rows = []
    for i in range(len(off) - 1):
        rows.append([(int(j[k]), tuple(int(x) for x in s[k])) for k in range(off[i], off[i + 1])])
    return rows


def rel_max(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
