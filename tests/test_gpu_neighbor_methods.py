"""The per-atom neighbour search (QEQ_NL_ATOM, Sec. 3.1: the paper's one-program-per-atom
form) against the brute-force pair set, bit-exact, and against the brick search.

Both searches take the same pair decision and write the same list format, so the
pair set must equal the oracle's exactly, every row must keep its three distance
classes in order, and a Coulomb apply over either list must agree to rounding.
"""

import numpy as np
import pytest

from gpu_util import canonical_rows_gpu, canonical_rows_oracle, cuda_or_skip, dev_tensor, rel_max
from oracle import neighbors
from workloads import random_neutral_charges, simple_cubic_lattice, water_box

pytestmark = pytest.mark.gpu


def _build(qg, R, box, r_cut, skin, method, max_neighbors=0, mesh=(8, 8, 8)):
    p = qg.make_params(len(R), box, r_cut=r_cut, skin=skin, mesh=mesh, order=4,
                       max_neighbors=max_neighbors)
    s = qg.System(p)
    qg.qeq_set_neighbor_method(s.ctx, method)
    s.neighbor_build(dev_tensor(R))
    return s


def _classes_in_order(R, box, counts, nbr, shift, r_cut, skin):
    """Rows hold near (d^2 < r_list^2 / 3), inside r_c and skin entries in that order
    (class boundaries decided in FP32 by the kernel: a tolerance band of 1e-5)."""
    rl2 = (r_cut + skin) ** 2
    box = np.asarray(box, dtype=np.float64)
    xw = R - box * np.floor(R / box)
    for i in range(len(counts)):
        c = int(counts[i])
        d = xw[nbr[i, :c]] - xw[i] + shift[i, :c].astype(np.float64) * box
        d2 = np.einsum("ij,ij->i", d, d)
        lo = (d2 >= rl2 / 3 * (1 + 1e-5)).astype(int) + (d2 >= r_cut ** 2 * (1 + 1e-5))
        hi = (d2 >= rl2 / 3 * (1 - 1e-5)).astype(int) + (d2 >= r_cut ** 2 * (1 - 1e-5))
        # some assignment between lo and hi is non-decreasing along the row
        run = 0
        for a, b in zip(lo, hi):
            run = max(run, a)
            assert run <= b, f"row {i}: distance classes out of order"


CASES = [
    ("water_648_multi_image", lambda: water_box(216, seed=2503), 9.0, 1.0, 0),
    ("water_3000_ragged", lambda: water_box(1000, seed=17), 8.0, 1.0, 0),
    ("growth_from_tiny_width", lambda: water_box(150, seed=3), 6.0, 0.5, 8),
]


@pytest.mark.parametrize("name,make,r_cut,skin,width", CASES, ids=[c[0] for c in CASES])
def test_atom_search_is_exact(name, make, r_cut, skin, width):
    qg = cuda_or_skip()
    w = make()
    s = _build(qg, w.R, w.box, r_cut, skin, "atom", max_neighbors=width)
    counts, nbr, shift = s.neighbor_export()
    off, j, sh = neighbors.brute_force_pairs(w.R, w.box, r_cut + skin)
    assert np.array_equal(counts, np.diff(off))
    assert canonical_rows_gpu(counts, nbr, shift) == canonical_rows_oracle(off, j, sh)
    _classes_in_order(w.R, w.box, counts, nbr, shift, r_cut, skin)
    s.close()


def test_atom_search_edge_cases():
    """Sites on cell edges with pairs exactly at r_list, a single atom among its own
    images, and positions several box lengths outside an anisotropic box."""
    qg = cuda_or_skip()
    R, L = simple_cubic_lattice(6, 2.0, origin=0.0)
    rng = np.random.default_rng(9)
    box3 = np.array([13.0, 17.0, 21.5])
    R3 = rng.uniform(-2.0, 3.0, size=(700, 3)) * box3
    for R_, box, r_cut, skin in ((R, np.array([L, L, L]), 3.0, 1.0),
                                 (np.array([[0.3, 1.7, 2.9]]), np.array([5.0, 5.5, 6.0]), 4.5, 1.0),
                                 (R3, box3, 5.0, 0.7)):
        s = _build(qg, R_, box, r_cut, skin, "atom")
        counts, nbr, shift = s.neighbor_export()
        off, j, sh = neighbors.brute_force_pairs(R_, box, r_cut + skin)
        assert canonical_rows_gpu(counts, nbr, shift) == canonical_rows_oracle(off, j, sh)
        s.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32_mixed", 1e-5)])
def test_apply_over_either_list_agrees(precision, tol):
    qg = cuda_or_skip()
    w = water_box(500, seed=23)
    q = dev_tensor(random_neutral_charges(w.n_atoms, seed=4, scale=0.3))
    R, sig = dev_tensor(w.R), dev_tensor(w.sigma)
    out = []
    for method in ("brick", "atom"):
        p = qg.make_params(w.n_atoms, w.box, r_cut=8.0, skin=1.0, mesh=(24, 24, 24), order=4,
                           precision=precision)
        s = qg.System(p)
        qg.qeq_set_neighbor_method(s.ctx, method)
        s.neighbor_build(R)
        v, E, F, en = s.apply(R, q, sig)
        out.append((v.cpu().numpy().copy(), F.cpu().numpy().copy()))
        s.close()
    assert rel_max(out[1][0], out[0][0]) < tol
    assert rel_max(out[1][1], out[0][1]) < tol


def test_unknown_method_is_rejected():
    qg = cuda_or_skip()
    w = water_box(10, seed=1)
    s = qg.System(qg.make_params(w.n_atoms, w.box, r_cut=4.0, skin=0.5, mesh=(8, 8, 8)))
    with pytest.raises(qg.QeqError) as ei:
        qg._lib.load().qeq_set_neighbor_method  # exported
        qg._lib._check(s.ctx, qg._lib.load().qeq_set_neighbor_method(s.ctx, 7))
    assert ei.value.code == -1
    s.close()
