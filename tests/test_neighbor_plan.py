"""Cell / brick decomposition and the FP32 prefilter band of the neighbour
build (host logic, CPU).

Alg. 1 bins atoms into cells so that every pair within r_list = r_cut + skin
lies in neighbouring cells; the build here uses cells of at least r_list / 2
paired into bricks, and a tile of bricks around each brick.  The emit decides
a candidate in FP32 outside a band around r_list^2 and in FP64 (fixed
operation order, no FMA) inside it, so the pair set is the exact one as long
as the band covers the FP32 error.  Both are checked here against their
definitions: the decomposition by brute force over cell offsets, the band by
replaying the emit's FP32 and FP64 arithmetic in numpy on pairs near r_list.
"""

import numpy as np
import pytest

import paper_2503_21176_gb300 as qg


def _params(box, r_cut=8.0, skin=1.0, n=3000):
    p = qg.qeq_params_default()
    p.n_atoms = n
    for d in range(3):
        p.box[d] = float(box[d])
        p.mesh[d] = 16
    p.r_cut, p.skin = float(r_cut), float(skin)
    return p


@pytest.mark.parametrize("seed", range(40))
def test_decomposition_covers_every_pair(seed):
    rng = np.random.default_rng(seed)
    r_cut, skin = rng.uniform(4.0, 10.0), rng.uniform(0.3, 1.5)
    rl = r_cut + skin
    box = rng.uniform(0.55 * rl, 12 * rl, 3)
    try:
        g = qg.qeq_neighbor_plan(_params(box, r_cut, skin))
    except qg.QeqError:
        # refused only where an image index would leave [-2, 2]
        assert min(box) < rl / 2 * 1.0000001
        return
    assert g["r_list"] == pytest.approx(rl, rel=1e-15)
    T = 1
    for d in range(3):
        nc, cw, reach, B, nb, br = (g[k][d] for k in ("nc", "cell_width", "reach", "brick", "bricks",
                                                      "tile_reach"))
        assert cw == pytest.approx(box[d] / nc, rel=1e-14)
        assert cw >= rl / 2 or nc == 1           # cells at least r_list / 2 (one cell if the box is smaller)
        if nc >= 4:
            assert nc % 2 == 0 and B == 2
        else:
            assert B == 1
        assert nb * B == nc
        assert reach * cw >= rl                  # a pair spans at most reach cells
        # every cell within reach of a cell of brick b lies in bricks b - br .. b + br
        for c0 in range(B):
            for off in range(-reach, reach + 1):
                assert -br <= (c0 + off) // B <= br
        T *= 2 * br + 1
    assert g["tile_bricks"] == T and g["n_bricks"] == int(np.prod(g["bricks"]))


def _fma32(a, b, c):
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


@pytest.mark.parametrize("L,r_cut", [(144.13, 8.0), (18.63, 9.0), (600.0, 10.0), (40.0, 5.0)])
def test_fp32_band_covers_the_fp32_error(L, r_cut):
    """Replay the emit: FP32 positions (rounded from the wrapped FP64 ones),
    image shift s L in FP32, d^2 in FP32 (plain or fused order); the FP64
    decision is ((x_j - x_i) + s L)^2 summed in a fixed order without FMA.
    Outside [band_lo, band_hi] the FP32 decision must equal the FP64 one."""
    g = qg.qeq_neighbor_plan(_params([L, L, L], r_cut=r_cut))
    rl = g["r_list"]
    rl2 = rl * rl
    lo, hi = np.float32(g["band_lo"]), np.float32(g["band_hi"])
    assert lo < rl2 < hi
    rng = np.random.default_rng(int(L))
    n = 200000
    xi = rng.uniform(0.0, L, (n, 3))
    u = rng.standard_normal((n, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    # distances within a few band widths of r_list
    width = (float(hi) - float(lo)) / (2 * rl)
    d = u * (rl + rng.uniform(-4, 4, n) * width)[:, None]
    xj_img = xi + d
    s = np.floor(xj_img / L)                     # image shift so that x_j is in [0, L)
    xj = xj_img - s * L
    keep64 = np.zeros(n, dtype=bool)
    d2 = np.zeros(n)
    for k in range(3):
        dk = (xj[:, k] - xi[:, k]) + s[:, k] * L   # the kernel adds +-L or +-2L exactly
        d2 = d2 + dk * dk if k else dk * dk
    keep64 = d2 < rl2
    xi32, xj32 = xi.astype(np.float32), xj.astype(np.float32)
    sh32 = s.astype(np.float32) * np.float32(L)
    dx32 = [(xj32[:, k] - xi32[:, k]) + sh32[:, k] for k in range(3)]
    d2_plain = (dx32[0] * dx32[0] + dx32[1] * dx32[1]) + dx32[2] * dx32[2]
    d2_fused = _fma32(dx32[2], dx32[2], _fma32(dx32[1], dx32[1], dx32[0] * dx32[0]))
    # the cell-by-cell emit folds the shift into the row's position first:
    # d = x_j - (x_i - s L), then d^2 with fused multiply-adds
    dxs = [xj32[:, k] - (xi32[:, k] - sh32[:, k]) for k in range(3)]
    d2_shifted = _fma32(dxs[2], dxs[2], _fma32(dxs[1], dxs[1], dxs[0] * dxs[0]))
    for d2f in (d2_plain, d2_fused, d2_shifted):
        below, above = d2f < lo, d2f > hi
        assert below.any() and above.any() and (~below & ~above).any()
        assert np.all(keep64[below]), "FP32 kept a pair the FP64 test drops"
        assert not np.any(keep64[above]), "FP32 dropped a pair the FP64 test keeps"


def test_box_too_small_is_refused():
    with pytest.raises(qg.QeqError):
        qg.qeq_neighbor_plan(_params([3.0, 20.0, 20.0], r_cut=8.0, skin=1.0))
