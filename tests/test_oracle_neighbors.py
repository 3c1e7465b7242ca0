"""Pins of the brute-force neighbour set (Sec. 3.1, Alg. 1) -- CPU only."""

import itertools
import math

import numpy as np
import pytest

from oracle import neighbors
from workloads import simple_cubic_lattice, water_box


def _lattice_shell_count(rmax_over_a):
    """Number of nonzero integer vectors with |n| < rmax (lattice points in a ball)."""
    m = int(math.ceil(rmax_over_a)) + 1
    c = 0
    for v in itertools.product(range(-m, m + 1), repeat=3):
        n2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2]
        if 0 < n2 < rmax_over_a * rmax_over_a:
            c += 1
    return c


@pytest.mark.parametrize("n_side,ratio", [(5, 1.5), (5, 1.8), (4, 2.1), (3, 1.8), (2, 2.5),
                                          (1, 1.8)])
def test_simple_cubic_counts(n_side, ratio):
    """Every site of a periodic simple cubic lattice has the lattice-ball count of neighbours.

    Small n_side exercises multi-image rows (the same j under several images, and
    an atom's own images).
    """
    a = 1.7
    R, L = simple_cubic_lattice(n_side, a)
    off, j, s = neighbors.brute_force_pairs(R, np.array([L, L, L]), ratio * a)
    counts = np.diff(off)
    assert np.all(counts == _lattice_shell_count(ratio))


def test_c_loops_match_numpy_definition():
    """The C enumeration equals the numpy broadcast form, row by row, in canonical order."""
    rng = np.random.default_rng(21)
    for n, L, rl in ((40, 9.0, 4.0), (25, 6.0, 5.5), (12, 4.0, 6.0)):
        box = np.array([L, L * 1.1, L * 0.9])
        R = rng.uniform(-0.5 * L, 1.5 * L, size=(n, 3))
        off, j, s = neighbors.brute_force_pairs(R, box, rl)
        rows = neighbors.brute_force_pairs_numpy(R, box, rl)
        for i in range(n):
            got = [(int(j[k]), tuple(int(c) for c in s[k])) for k in range(off[i], off[i + 1])]
            assert got == sorted(rows[i])
            assert got == rows[i]


def test_pair_set_symmetry_and_distances():
    """(i, j, s) in the set iff (j, i, -s) is; every kept image distance is < r_list."""
    w = water_box(40, seed=31)
    rl = 6.5
    off, j, s = neighbors.brute_force_pairs(w.R, w.box, rl)
    xw, _ = neighbors.wrap(w.R, w.box)
    pairs = set()
    for i in range(w.n_atoms):
        for k in range(off[i], off[i + 1]):
            pairs.add((i, int(j[k]), tuple(int(c) for c in s[k])))
            d = xw[j[k]] - xw[i] + s[k] * w.box
            assert np.linalg.norm(d) < rl
    for (i, jj, sv) in pairs:
        assert (jj, i, tuple(-c for c in sv)) in pairs


def test_strict_cutoff_excludes_exact_distance():
    """A pair at exactly the list radius is excluded (strict comparison)."""
    R = np.array([[1.0, 1.0, 1.0], [3.0, 1.0, 1.0]])
    box = np.array([20.0, 20.0, 20.0])
    off, _, _ = neighbors.brute_force_pairs(R, box, 2.0)
    assert off[-1] == 0
    off, _, _ = neighbors.brute_force_pairs(R, box, 2.0 + 1e-12)
    assert off[-1] == 2


def test_wrap_convention():
    """Wrap is x + (-(L floor(x / L))); tiny negatives may land exactly on L."""
    box = np.array([10.0, 10.0, 10.0])
    R = np.array([[-1e-18, 5.0, 10.0], [-10.5, 25.0, 3.0]])
    xw, w = neighbors.wrap(R, box)
    assert xw[0, 0] == 10.0 and xw[0, 2] == 0.0
    assert np.allclose(xw[1], [9.5, 5.0, 3.0])
    assert np.array_equal(xw, R + w)
