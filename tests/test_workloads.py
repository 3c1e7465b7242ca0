"""Synthetic input recipe (CPU): the water box follows its stated geometry and
parameters, and the serving mesh rule picks the smallest 2^k or 3 * 2^k mesh
with spacing <= 1 A."""

import numpy as np
import pytest

from workloads import random_neutral_charges, serving_mesh_size, water_box


@pytest.mark.parametrize("n_mol", [1, 8, 216, 1000, 1500])
def test_water_box_recipe(n_mol):
    w = water_box(n_mol, seed=5)
    assert w.n_atoms == 3 * n_mol
    L = (n_mol / 0.0334) ** (1.0 / 3.0)  # density 0.0334 molecules / A^3
    assert np.allclose(w.box, L, rtol=1e-12)
    O, H1, H2 = w.R[0::3], w.R[1::3], w.R[2::3]
    for H in (H1, H2):  # rigid O-H 0.9572 A (geometry before any wrapping)
        assert np.allclose(np.linalg.norm(H - O, axis=1), 0.9572, atol=1e-9)
    c = np.einsum("ij,ij->i", H1 - O, H2 - O) / 0.9572 ** 2
    assert np.allclose(np.degrees(np.arccos(np.clip(c, -1, 1))), 104.52, atol=1e-6)
    assert np.allclose(w.sigma[0::3], 0.70) and np.allclose(w.sigma[1::3], 0.45)
    assert np.allclose(w.mass[0::3], 15.999) and np.allclose(w.mass[2::3], 1.008)
    # chi, eta: O 8.5 / 14.0, H 4.5 / 12.0 eV plus N(0, 0.1 eV) noise
    for arr, mo, mh in ((w.chi, 8.5, 4.5), (w.eta, 14.0, 12.0)):
        assert np.all(np.abs(arr[0::3] - mo) < 0.6) and np.all(np.abs(arr[1::3] - mh) < 0.6)


def test_water_box_is_seeded():
    a, b, c = water_box(64, seed=1), water_box(64, seed=1), water_box(64, seed=2)
    assert np.array_equal(a.R, b.R) and np.array_equal(a.chi, b.chi)
    assert not np.array_equal(a.R, c.R)


def test_random_neutral_charges():
    q = random_neutral_charges(1000, seed=3, scale=0.4)
    assert abs(q.sum()) < 1e-12 and 0.3 < q.std() < 0.5


@pytest.mark.parametrize("L,K", [(5.0, 6), (8.0, 8), (9.0, 12), (18.63, 24), (24.0, 24),
                                 (24.5, 32), (62.1, 64), (96.0, 96), (144.13, 192)])
def test_serving_mesh_rule(L, K):
    assert serving_mesh_size(L) == K
    # brute force over the allowed forms
    allowed = sorted({2 ** k for k in range(12)} | {3 * 2 ** k for k in range(12)})
    assert K == min(m for m in allowed if L / m <= 1.0)
