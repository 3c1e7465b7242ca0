"""GPU Coulomb apply v = Phi q against the CPU oracle (Sec. 3.2, Sec. 3.3 / Alg. 2, Sec. 3.4).

FP64 mode: v, E, F and the energy parts within 1e-10 relative (max abs error
over max abs value) of the oracle's smooth PME on the same mesh and order,
with the same real-space cutoff.
FP32-mixed mode: relative RMS force error <= 1e-4 and relative potential and
energy errors <= 1e-5 against the same FP64 oracle.
"""

import numpy as np
import pytest

from gpu_util import cuda_or_skip, dev_tensor, rel_max
from oracle import ewald
from workloads import random_neutral_charges, water_box

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def _gpu_apply(w, q, alpha, r_cut, mesh, order, precision="fp64", gaussian_self=True, skin=1.0):
    qg = cuda_or_skip()
    p = qg.make_params(w.n_atoms, w.box, alpha=alpha, r_cut=r_cut, skin=skin, mesh=mesh,
                       order=order, precision=precision, gaussian_self=gaussian_self)
    s = qg.System(p)
    R = dev_tensor(w.R)
    s.neighbor_build(R)
    v, E, F, en = s.apply(R, dev_tensor(q), dev_tensor(w.sigma))
    out = {"v": v.cpu().numpy().copy(), "E": E.cpu().numpy().copy(), "F": F.cpu().numpy().copy(),
           "energy": en.cpu().numpy().copy()}
    s.close()
    return out


def _oracle(w, q, alpha, r_cut, mesh, order, gaussian_self=True):
    return ewald.coulomb_apply(w.R, q, w.sigma, w.box, alpha, r_cut, recip="pme", mesh=mesh,
                               order=order, gaussian_self=gaussian_self)


def _check64(g, o):
    assert rel_max(g["v"], o["v"]) < TOL64
    assert rel_max(g["E"], o["E"]) < TOL64
    assert rel_max(g["F"], o["F"]) < TOL64
    scale = abs(o["energy_real"]) + abs(o["energy_recip"]) + abs(o["energy_self"])
    assert abs(g["energy"][0] - o["energy"]) < TOL64 * scale
    assert abs(g["energy"][1] - o["energy_real"]) < TOL64 * scale
    assert abs(g["energy"][2] - o["energy_recip"]) < TOL64 * scale
    assert abs(g["energy"][3] - o["energy_self"]) < TOL64 * scale


def test_fp64_water_648():
    """216-molecule box, r_c 9, K 32, p 4 (the small water workload)."""
    w = water_box(216, seed=2503)
    q = random_neutral_charges(w.n_atoms, seed=1, scale=0.3)
    _check64(_gpu_apply(w, q, 0.34, 9.0, (32, 32, 32), 4), _oracle(w, q, 0.34, 9.0, (32, 32, 32), 4))


@pytest.mark.parametrize("order,mesh", [(5, (24, 30, 36)), (6, (40, 40, 40)), (8, (20, 32, 27))])
def test_fp64_orders_and_meshes(order, mesh):
    w = water_box(400, seed=order)  # 1200 atoms (ragged: 4.7 blocks)
    q = random_neutral_charges(w.n_atoms, seed=order + 10, scale=0.4)
    _check64(_gpu_apply(w, q, 0.3, 7.5, mesh, order), _oracle(w, q, 0.3, 7.5, mesh, order))


def test_fp64_point_charges_no_gaussian_self():
    """sigma = 0 switches the Gaussian correction off; gaussian_self off."""
    w = water_box(100, seed=4)
    w.sigma[:] = 0.0
    q = random_neutral_charges(w.n_atoms, seed=5)
    g = _gpu_apply(w, q, 0.4, 6.0, (24, 24, 24), 4, gaussian_self=False)
    _check64(g, _oracle(w, q, 0.4, 6.0, (24, 24, 24), 4, gaussian_self=False))


@pytest.mark.parametrize("alpha,r_cut", [(0.45, 9.5), (0.8, 6.0)])
def test_fp64_pair_table_ranges(alpha, r_cut):
    """Uniform random atoms: pairs closer than 0.5 A and pairs beyond r = 8 A go
    past the ends of the FP64 kernel's piecewise pair-function table (direct
    erfc path), the rest cross its octave and piece boundaries; sigma mixes 0,
    small and large widths so that the Gaussian-correction test sees both sides."""
    import types
    rng = np.random.default_rng(int(alpha * 100))
    n, L = 360, 19.0
    sigma = rng.choice([0.0, 0.3, 0.7, 1.6], size=n)
    w = types.SimpleNamespace(n_atoms=n, box=np.array([L, L, L]), R=rng.uniform(0.0, L, (n, 3)),
                              sigma=sigma)
    q = random_neutral_charges(n, seed=7, scale=0.5)
    mesh = (24, 24, 24)
    # gaussian_self off: the Gaussian self energy is undefined at sigma = 0
    _check64(_gpu_apply(w, q, alpha, r_cut, mesh, 4, gaussian_self=False),
             _oracle(w, q, alpha, r_cut, mesh, 4, gaussian_self=False))


def test_fp64_non_neutral_and_single_atom():
    w = water_box(1, seed=2)  # 3 atoms in a 4.5 A box: everything is multi-image
    w.box[:] = 5.0
    q = np.array([0.7, -0.2, 0.1])
    _check64(_gpu_apply(w, q, 0.6, 4.0, (8, 8, 8), 4, skin=0.5),
             _oracle(w, q, 0.6, 4.0, (8, 8, 8), 4))


def test_fp64_against_direct_ewald_accuracy():
    """Method accuracy (not parity): PME K 32 p 4 vs the exact k-sum, RMS force error < 2e-4."""
    w = water_box(216, seed=2503)
    q = random_neutral_charges(w.n_atoms, seed=1, scale=0.3)
    g = _gpu_apply(w, q, 0.34, 9.0, (32, 32, 32), 4)
    ref = ewald.coulomb_apply(w.R, q, w.sigma, w.box, 0.34, 9.0, recip="ewald", gaussian_self=True)
    err = np.sqrt(np.mean((g["F"] - ref["F"]) ** 2) / np.mean(ref["F"] ** 2))
    assert err < 2e-4


def test_fp32_mixed_error_bounds():
    w = water_box(1000, seed=77)
    q = random_neutral_charges(w.n_atoms, seed=3, scale=0.4)
    o = _oracle(w, q, 0.34, 8.0, (32, 32, 32), 4)
    g = _gpu_apply(w, q, 0.34, 8.0, (32, 32, 32), 4, precision="fp32_mixed")
    rms_f = np.sqrt(np.mean((g["F"] - o["F"]) ** 2) / np.mean(o["F"] ** 2))
    assert rms_f < 1e-4
    assert rel_max(g["v"], o["v"]) < 1e-5
    # relative energy error: against the magnitude of the energy's parts (the
    # real-space part alone is small here, the parts cancel)
    scale = abs(o["energy_real"]) + abs(o["energy_recip"]) + abs(o["energy_self"])
    assert abs(g["energy"][0] - o["energy"]) < 1e-6 * scale


def test_potential_only_matches_field_apply():
    """The potential-only apply (E, F null) gives the same v as the full apply."""
    qg = cuda_or_skip()
    w = water_box(300, seed=8)
    q = random_neutral_charges(w.n_atoms, seed=9)
    p = qg.make_params(w.n_atoms, w.box, r_cut=8.0, mesh=(32, 32, 32))
    s = qg.System(p)
    R = dev_tensor(w.R)
    s.neighbor_build(R)
    v1 = s.apply(R, dev_tensor(q), dev_tensor(w.sigma))[0].clone()
    v2 = s.apply(R, dev_tensor(q), dev_tensor(w.sigma), field=False)[0].clone()
    assert rel_max(v2.cpu().numpy(), v1.cpu().numpy()) < 1e-13
    s.close()


def test_apply_without_list_is_an_error():
    qg = cuda_or_skip()
    w = water_box(5, seed=1)
    s = qg.System(qg.make_params(w.n_atoms, w.box, r_cut=4.0, skin=0.5, mesh=(8, 8, 8)))
    with pytest.raises(qg.QeqError) as ei:
        s.apply(dev_tensor(w.R), dev_tensor(np.zeros(w.n_atoms)), dev_tensor(w.sigma))
    assert ei.value.code == -6
    s.close()


def test_invalid_params_are_rejected():
    qg = cuda_or_skip()
    with pytest.raises(qg.QeqError) as ei:
        qg.System(qg.make_params(10, (10, 10, 10), order=3))
    assert ei.value.code == -2
    with pytest.raises(qg.QeqError) as ei:
        qg.System(qg.make_params(10, (10, 10, -1)))
    assert ei.value.code == -1
    with pytest.raises(qg.QeqError):
        qg.System(qg.make_params(10, (3.0, 10, 10), r_cut=8.0, skin=1.0))  # box < r_list / 2


@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
def test_full_size_sampled_rows(precision):
    """300,000-atom box (r_c 8, K 144, p 4) in the benchmark configuration.

    Sampled atoms are compared with the oracle: real space by brute force on
    those rows, plus the oracle PME of the whole box.
    """
    qg = cuda_or_skip()
    w = water_box(100_000, seed=2504)
    q = random_neutral_charges(w.n_atoms, seed=2, scale=0.4)
    mesh = (144, 144, 144)
    p = qg.make_params(w.n_atoms, w.box, alpha=0.34, r_cut=8.0, skin=1.0, mesh=mesh, order=4,
                       precision=precision)
    s = qg.System(p)
    R = dev_tensor(w.R)
    s.neighbor_build(R)
    v, E, F, en = s.apply(R, dev_tensor(q), dev_tensor(w.sigma))
    v = v.cpu().numpy()
    E = E.cpu().numpy()
    s.close()
    rows = np.random.default_rng(0).choice(w.n_atoms, 48, replace=False)
    vr, Er = ewald.real_space(w.R, q, w.sigma, w.box, 0.34, 8.0, rows=rows)
    vk, Ek, _ = ewald.pme_reciprocal(w.R, q, w.box, 0.34, mesh, 4)
    vs = ewald.self_potential(q, w.sigma, 0.34, gaussian_self=True)
    v_ref = vr + vk[rows] + vs[rows]
    E_ref = Er + Ek[rows]
    if precision == "fp64":
        assert rel_max(v[rows], v_ref) < TOL64
        assert rel_max(E[rows], E_ref) < TOL64
    else:
        assert rel_max(v[rows], v_ref) < 1e-5
        assert np.sqrt(np.mean((E[rows] - E_ref) ** 2) / np.mean(E_ref ** 2)) < 1e-4


@pytest.mark.parametrize("n_mol,box_scale", [(216, 1.0), (60, 1.0), (30, 1.3)])
def test_fp64_explicit_ewald_matches_oracle(n_mol, box_scale):
    """The GPU explicit k-vector sum (recip = ewald) against the oracle's k-sum, same k_cut."""
    qg = cuda_or_skip()
    w = water_box(n_mol, seed=n_mol)
    w.box *= box_scale
    q = random_neutral_charges(w.n_atoms, seed=3, scale=0.4)
    k_cut = ewald.kspace_cutoff(0.34, 1e-14)
    p = qg.make_params(w.n_atoms, w.box, alpha=0.34, r_cut=8.0, skin=1.0, mesh=(8, 8, 8),
                       recip="ewald", k_cut=k_cut)
    s = qg.System(p)
    R = dev_tensor(w.R)
    s.neighbor_build(R)
    v, E, F, en = s.apply(R, dev_tensor(q), dev_tensor(w.sigma))
    o = ewald.coulomb_apply(w.R, q, w.sigma, w.box, 0.34, 8.0, recip="ewald", k_cut=k_cut,
                            gaussian_self=True)
    assert rel_max(v.cpu().numpy(), o["v"]) < TOL64
    assert rel_max(F.cpu().numpy(), o["F"]) < TOL64
    e = en.cpu().numpy()
    assert abs(e[2] - o["energy_recip"]) < TOL64 * abs(o["energy_recip"])
    assert abs(e[0] - o["energy"]) < TOL64 * (abs(o["energy_real"]) + abs(o["energy_recip"]))
    s.close()
    with pytest.raises(qg.QeqError):
        qg.System(qg.make_params(w.n_atoms, w.box, recip="ewald", precision="fp32_mixed"))


def _dense_small_box(seed):
    """1000 atoms on a jittered 10^3 lattice in an 8 A cube (about 20x water density)."""
    from workloads import simple_cubic_lattice

    rng = np.random.default_rng(seed)
    R, L = simple_cubic_lattice(10, 0.8)
    R = R + rng.uniform(-0.1, 0.1, size=R.shape)

    class W:
        pass

    w = W()
    w.R, w.box, w.n_atoms = R, np.array([L, L, L]), len(R)
    w.sigma = np.where(np.arange(len(R)) % 3 == 0, 0.7, 0.45)
    return w


@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
def test_dense_small_box_global_tiles(precision):
    """Tiles larger than shared memory: the real-space kernels stage them in global scratch.

    r_list 5.6 in an 8 A box gives 2 cells of 4 A per axis, bricks of one cell
    and a tile of 5^3 cell images: 125 x 1000 / 8 = 15,625 atoms, beyond the
    5,200 (FP64) and 11,400 (FP32) atoms that shared memory holds.  The
    neighbour set is also compared exactly with the brute-force search.
    """
    from gpu_util import canonical_rows_gpu, canonical_rows_oracle
    from oracle import neighbors

    qg = cuda_or_skip()
    w = _dense_small_box(12)
    q = random_neutral_charges(w.n_atoms, seed=4, scale=0.3)
    mesh = (16, 16, 16)
    p = qg.make_params(w.n_atoms, w.box, alpha=0.5, r_cut=5.0, skin=0.6, mesh=mesh, order=4,
                       precision=precision)
    s = qg.System(p)
    R = dev_tensor(w.R)
    s.neighbor_build(R)
    counts, nbr, shift = s.neighbor_export()
    off, j, sh = neighbors.brute_force_pairs(w.R, w.box, 5.6)
    assert canonical_rows_gpu(counts, nbr, shift) == canonical_rows_oracle(off, j, sh)
    v, E, F, en = s.apply(R, dev_tensor(q), dev_tensor(w.sigma))
    g = {"v": v.cpu().numpy().copy(), "E": E.cpu().numpy().copy(), "F": F.cpu().numpy().copy(),
         "energy": en.cpu().numpy().copy()}
    s.close()
    o = _oracle(w, q, 0.5, 5.0, mesh, 4)
    if precision == "fp64":
        _check64(g, o)
    else:
        assert np.sqrt(np.mean((g["F"] - o["F"]) ** 2) / np.mean(o["F"] ** 2)) < 1e-4
        assert rel_max(g["v"], o["v"]) < 1e-5
