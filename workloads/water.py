"""Seeded water-like periodic boxes and other synthetic fixtures.

The water recipe stands in for the paper's randomly generated water-like systems
(Sec. 4.2.1, Sec. 4.2.2) and its large water boxes (Sec. 4.2.3):

* rigid-geometry molecules, O-H 0.9572 A, H-O-H 104.52 deg, uniformly random
  orientation (random unit quaternion);
* oxygens on an ``n_side = ceil(n_mol**(1/3))`` cubic lattice of spacing
  ``L / n_side``; the occupied sites are the first ``n_mol`` of a seeded
  permutation, each jittered uniformly by +-0.1 of the spacing;
* 0.0334 molecules per cubic Angstrom, so ``L = (n_mol / 0.0334)**(1/3)``;
* electronegativity chi (O 8.5, H 4.5 eV) and hardness eta (O 14.0, H 12.0 eV),
  each with N(0, 0.1 eV) noise; Gaussian widths sigma_O 0.70 A, sigma_H 0.45 A.

Atoms are ordered O, H, H per molecule.  Positions are not wrapped into the box.
Units: Angstrom, elementary charge, eV, amu.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

WATER_DENSITY = 0.0334  # molecules per cubic Angstrom
OH_BOND = 0.9572  # Angstrom
HOH_ANGLE_DEG = 104.52
O_MASS = 15.999
H_MASS = 1.008
CHI_O, CHI_H = 8.5, 4.5
ETA_O, ETA_H = 14.0, 12.0
SIGMA_O, SIGMA_H = 0.70, 0.45


@dataclass
class WaterBox:
    """One synthetic water box; every array is float64 (species is int8: 0 = O, 1 = H)."""

    R: np.ndarray  # (N, 3) positions, Angstrom
    box: np.ndarray  # (3,) orthorhombic edge lengths, Angstrom
    chi: np.ndarray  # (N,) electronegativity, eV
    eta: np.ndarray  # (N,) hardness, eV
    sigma: np.ndarray  # (N,) Gaussian charge width, Angstrom
    mass: np.ndarray  # (N,) amu
    species: np.ndarray  # (N,) int8

    @property
    def n_atoms(self) -> int:
        return int(self.R.shape[0])


def water_box_length(n_mol: int, density: float = WATER_DENSITY) -> float:
    """Cubic edge length giving ``density`` molecules per cubic Angstrom."""
    return (n_mol / density) ** (1.0 / 3.0)


def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random rotations from normalised Gaussian quaternions, shape (n, 3, 3)."""
    qv = rng.standard_normal((n, 4))
    qv /= np.linalg.norm(qv, axis=1, keepdims=True)
    w, x, y, z = qv.T
    rot = np.empty((n, 3, 3))
    rot[:, 0, 0] = 1 - 2 * (y * y + z * z)
    rot[:, 0, 1] = 2 * (x * y - z * w)
    rot[:, 0, 2] = 2 * (x * z + y * w)
    rot[:, 1, 0] = 2 * (x * y + z * w)
    rot[:, 1, 1] = 1 - 2 * (x * x + z * z)
    rot[:, 1, 2] = 2 * (y * z - x * w)
    rot[:, 2, 0] = 2 * (x * z - y * w)
    rot[:, 2, 1] = 2 * (y * z + x * w)
    rot[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return rot


def water_box(n_mol: int, seed: int, density: float = WATER_DENSITY,
              param_noise: float = 0.1, jitter: float = 0.1) -> WaterBox:
    """Build ``n_mol`` water molecules (3 * n_mol atoms) in a cubic periodic box."""
    if n_mol < 1:
        raise ValueError("n_mol must be positive")
    rng = np.random.default_rng(seed)
    L = water_box_length(n_mol, density)
    n_side = int(math.ceil(n_mol ** (1.0 / 3.0) - 1e-9))
    while n_side ** 3 < n_mol:
        n_side += 1
    spacing = L / n_side
    sites = rng.permutation(n_side ** 3)[:n_mol]
    ix = sites // (n_side * n_side)
    iy = (sites // n_side) % n_side
    iz = sites % n_side
    grid = np.stack([ix, iy, iz], axis=1).astype(np.float64)
    oxy = (grid + 0.5) * spacing + rng.uniform(-jitter, jitter, size=(n_mol, 3)) * spacing

    half = math.radians(HOH_ANGLE_DEG) / 2.0
    h_local = np.array([[OH_BOND * math.sin(half), 0.0, OH_BOND * math.cos(half)],
                        [-OH_BOND * math.sin(half), 0.0, OH_BOND * math.cos(half)]])
    rot = _random_rotations(rng, n_mol)
    h_pos = oxy[:, None, :] + np.einsum("mij,hj->mhi", rot, h_local)

    R = np.empty((n_mol, 3, 3))
    R[:, 0, :] = oxy
    R[:, 1:, :] = h_pos
    R = R.reshape(-1, 3)

    species = np.tile(np.array([0, 1, 1], dtype=np.int8), n_mol)
    is_o = species == 0
    n = 3 * n_mol
    chi = np.where(is_o, CHI_O, CHI_H) + param_noise * rng.standard_normal(n)
    eta = np.where(is_o, ETA_O, ETA_H) + param_noise * rng.standard_normal(n)
    sigma = np.where(is_o, SIGMA_O, SIGMA_H).astype(np.float64)
    mass = np.where(is_o, O_MASS, H_MASS).astype(np.float64)
    return WaterBox(R=np.ascontiguousarray(R), box=np.array([L, L, L]), chi=chi, eta=eta,
                    sigma=sigma, mass=mass, species=species)


def serving_mesh_size(L: float, max_spacing: float = 1.0) -> int:
    """Smallest mesh edge of the form 2**k or 3 * 2**k with ``L / K <= max_spacing``."""
    best = None
    k = 1
    while k < 1 << 20:
        for cand in (k, 3 * k):
            if L / cand <= max_spacing and (best is None or cand < best):
                best = cand
        if best is not None and k > best:
            break
        k *= 2
    return int(best)


def random_neutral_charges(n: int, seed: int, scale: float = 0.4) -> np.ndarray:
    """Gaussian charges (std ``scale`` e) with their mean removed, so they sum to zero."""
    rng = np.random.default_rng(seed)
    q = scale * rng.standard_normal(n)
    return q - q.mean()


def rocksalt_lattice(n_cells: int, a: float = 2.0):
    """Rock-salt (NaCl) crystal: ``n_cells**3`` conventional cubic cells of edge ``2 * a``.

    Returns positions (N, 3), charges (+1 / -1 alternating on the simple cubic
    sublattice of spacing ``a``) and the box edge ``2 * a * n_cells``.  The
    nearest-neighbour distance is ``a``.
    """
    m = 2 * n_cells
    idx = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"),
                   axis=-1).reshape(-1, 3)
    R = idx.astype(np.float64) * a
    q = np.where(idx.sum(axis=1) % 2 == 0, 1.0, -1.0)
    return R, q, m * a


def simple_cubic_lattice(n_side: int, a: float, origin: float = 0.25):
    """Simple cubic lattice of ``n_side**3`` points, spacing ``a``, offset ``origin * a``."""
    idx = np.stack(np.meshgrid(np.arange(n_side), np.arange(n_side), np.arange(n_side),
                               indexing="ij"), axis=-1).reshape(-1, 3)
    return (idx.astype(np.float64) + origin) * a, n_side * a
