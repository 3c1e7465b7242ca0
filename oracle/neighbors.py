"""Neighbour-list definition (Sec. 3.1, Alg. 1): the exact pair set, by brute force.

Test infrastructure only.  The cell-based search of Alg. 1 is an accelerator.
The set it must produce is fixed by geometry: every (i, j, image) whose
displacement is shorter than the list radius.  Here that set is enumerated
over all O(N^2 * images) candidates.

Conventions:

* wrap: ``w = -(L * floor(x / L))``, ``xw = x + w``, one IEEE operation per
  step.  The result can equal L exactly when x is a tiny negative number.
  Such a coordinate is still a valid representative.
* image displacement: ``d = (xw_j - xw_i) + s * L``, ``d2 = (dx*dx + dy*dy) + dz*dz``,
  kept when ``d2 < r_list * r_list``.  The comparison is strict, so a pair
  exactly at the list radius is excluded.  The pair of an atom with itself is
  excluded at s = 0 and kept at other images (multi-image boxes).
* rows are in ascending (j, sx, sy, sz) order.
"""

from __future__ import annotations

import math

import numpy as np

from . import native


def wrap(R: np.ndarray, box: np.ndarray):
    """Wrapped positions and the per-atom offsets that produced them."""
    R = np.asarray(R, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    w = -(box * np.floor(R / box))
    return R + w, w


def image_reach(box, r_list) -> np.ndarray:
    """Largest |s_d| an image within r_list can need for wrapped positions in [0, L]."""
    return np.array([int(math.ceil(r_list / b)) + 1 for b in box], dtype=np.int32)


def brute_force_pairs(R: np.ndarray, box, r_list: float):
    """All (i, j, s) with image distance < r_list.

    Returns ``(offsets, j, s)``: CSR row offsets (N + 1, int64), neighbour
    indices (int32) and image vectors (M, 3) int8, rows ascending in
    (j, sx, sy, sz).
    """
    xw, _ = wrap(R, box)
    xw = np.ascontiguousarray(xw)
    box = np.ascontiguousarray(np.asarray(box, dtype=np.float64))
    n = xw.shape[0]
    smax = image_reach(box, r_list)
    L = native.lib()
    counts = np.zeros(n, dtype=np.int64)
    L.or_pairs_count(n, native.dptr(xw), native.dptr(box), float(r_list), native.i32ptr(smax),
                     native.i64ptr(counts))
    offsets = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    m = int(offsets[-1])
    j = np.zeros(max(m, 1), dtype=np.int32)
    s = np.zeros((max(m, 1), 3), dtype=np.int8)
    L.or_pairs_fill(n, native.dptr(xw), native.dptr(box), float(r_list), native.i32ptr(smax),
                    native.i64ptr(offsets), native.i32ptr(j), native.i8ptr(s))
    return offsets, j[:m], s[:m]


def brute_force_pairs_numpy(R: np.ndarray, box, r_list: float):
    """The same set written with numpy broadcasting (tiny N only).

    This version shares no loop with the C one.  It checks the C loops.
    """
    xw, _ = wrap(R, box)
    box = np.asarray(box, dtype=np.float64)
    n = xw.shape[0]
    smax = image_reach(box, r_list)
    rl2 = r_list * r_list
    rows = []
    sx, sy, sz = np.meshgrid(*[np.arange(-m, m + 1) for m in smax], indexing="ij")
    shifts = np.stack([sx.ravel(), sy.ravel(), sz.ravel()], axis=1)
    for i in range(n):
        b = xw - xw[i]  # (n, 3): xw_j - xw_i
        d = b[:, None, :] + shifts[None, :, :].astype(np.float64) * box  # (n, S, 3)
        d2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
        keep = d2 < rl2
        keep[i, np.all(shifts == 0, axis=1)] = False
        jj, ss = np.nonzero(keep)
        rows.append([(int(a), tuple(int(c) for c in shifts[b_])) for a, b_ in zip(jj, ss)])
    return rows
