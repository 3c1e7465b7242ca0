"""GPU neighbour list (Sec. 3.1, Alg. 1) against the brute-force pair set: bit-exact.

Every row is compared as a set of (j, image) after sorting both sides by (j, sx, sy, sz).
Several outputs are correct as to the order inside a row, but the set is unique.
"""

import numpy as np
import pytest

from gpu_util import canonical_rows_gpu, canonical_rows_oracle, cuda_or_skip, dev_tensor
from oracle import neighbors
from workloads import simple_cubic_lattice, water_box

pytestmark = pytest.mark.gpu


def _compare(R, box, r_cut, skin, max_neighbors=0):
    qg = cuda_or_skip()
    p = qg.make_params(len(R), box, r_cut=r_cut, skin=skin, mesh=(8, 8, 8), order=4,
                       max_neighbors=max_neighbors)
    s = qg.System(p)
    s.neighbor_build(dev_tensor(R))
    counts, nbr, shift = s.neighbor_export()
    off, j, sh = neighbors.brute_force_pairs(R, box, r_cut + skin)
    got = canonical_rows_gpu(counts, nbr, shift)
    want = canonical_rows_oracle(off, j, sh)
    assert np.array_equal(counts, np.diff(off))
    assert got == want
    s.close()
    return counts


def test_water_648_multi_image():
    """216 molecules, r_list 10 > L/2: pairs appear under two images."""
    w = water_box(216, seed=2503)
    counts = _compare(w.R, w.box, 9.0, 1.0)
    assert counts.mean() > 300


def test_water_3000_atoms_ragged():
    w = water_box(1000, seed=17)  # 3000 atoms: 11.7 blocks of 256 threads
    _compare(w.R, w.box, 8.0, 1.0)


def test_growth_from_tiny_width():
    """Initial width 8: the overflow flag triggers regrowth and the set is still exact."""
    w = water_box(150, seed=3)
    _compare(w.R, w.box, 6.0, 0.5, max_neighbors=8)


def test_lattice_on_cell_boundaries():
    """Sites exactly on cell edges and pairs exactly at the list radius (excluded)."""
    R, L = simple_cubic_lattice(6, 2.0, origin=0.0)
    _compare(R, np.array([L, L, L]), 3.0, 1.0)  # r_list 4.0 = 2 spacings: strict exclusion


def test_single_atom_self_images():
    """N = 1: the only neighbours are the atom's own periodic images.

    With r_list 5.5 the +-x images (5.0) are kept and the +-y images (exactly
    5.5) are excluded by the strict comparison.
    """
    R = np.array([[0.3, 1.7, 2.9]])
    counts = _compare(R, np.array([5.0, 5.5, 6.0]), 4.5, 1.0)
    assert counts[0] == 2


def test_positions_outside_box_and_anisotropic():
    rng = np.random.default_rng(9)
    box = np.array([13.0, 17.0, 21.5])
    R = rng.uniform(-2.0, 3.0, size=(700, 3)) * box  # several box lengths away
    R[0] = [-1e-18, 0.0, box[2]]  # wraps to exactly L / 0
    _compare(R, box, 5.0, 0.7)


def test_nonfinite_position_is_reported():
    qg = cuda_or_skip()
    w = water_box(10, seed=1)
    R = w.R.copy()
    R[4, 1] = np.nan
    s = qg.System(qg.make_params(len(R), w.box, r_cut=4.0, skin=0.5, mesh=(8, 8, 8)))
    with pytest.raises(qg.QeqError) as ei:
        s.neighbor_build(dev_tensor(R))
    assert ei.value.code == -7
    s.close()


def test_coo_export_equals_pair_set():
    """The COO format (Sec. 3.1) holds exactly the brute-force pair set."""
    qg = cuda_or_skip()
    w = water_box(300, seed=19)
    r_cut, skin = 7.0, 1.0
    s = qg.System(qg.make_params(w.n_atoms, w.box, r_cut=r_cut, skin=skin, mesh=(8, 8, 8)))
    s.neighbor_build(dev_tensor(w.R))
    pi, pj, code = qg._lib.qeq_neighbor_export_coo(s.ctx)
    pi, pj, code = pi.cpu().numpy(), pj.cpu().numpy(), code.cpu().numpy().astype(np.int32)
    off, j, sh = neighbors.brute_force_pairs(w.R, w.box, r_cut + skin)
    want = set()
    for i in range(w.n_atoms):
        for k in range(off[i], off[i + 1]):
            want.add((i, int(j[k]), int((sh[k, 0] + 2) * 25 + (sh[k, 1] + 2) * 5 + (sh[k, 2] + 2))))
    got = set(zip(pi.tolist(), pj.tolist(), code.tolist()))
    assert len(got) == len(pi) == len(want)
    assert got == want
    with pytest.raises(qg.QeqError) as ei:
        qg._lib.qeq_neighbor_export_coo(s.ctx, capacity=10)
    assert ei.value.code == -8
    s.close()
