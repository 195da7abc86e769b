"""The seeded input generators shared by the oracle and the GPU path: the
geometric guarantees they promise (non-overlap, volume fractions, symmetry,
block replication) and the exact workloads the measurements are quoted on
(phase-map hashes and sizes)."""
import math
from collections import Counter

import numpy as np

import rve_inputs as I


def _min_image_dist(a, b, n):
    d = np.abs(a - b)
    n = np.asarray(n, dtype=float)
    d = np.minimum(d, n - d)
    return np.sqrt((d * d).sum(-1))


def test_rsa_spheres_do_not_overlap_and_are_seeded():
    n = (48, 40, 56)
    r = 4.0
    c1 = I.rsa_sphere_centres(n, r, 25, seed=7)
    c2 = I.rsa_sphere_centres(n, r, 25, seed=7)
    c3 = I.rsa_sphere_centres(n, r, 25, seed=8)
    assert c1.shape == (25, 3) and np.array_equal(c1, c2) and not np.array_equal(c1, c3)
    for i in range(len(c1)):
        d = _min_image_dist(c1[i][None, :], np.delete(c1, i, axis=0), n)
        assert d.min() >= 2 * r - 1e-12


def test_voxelized_volume_fraction_matches_the_spheres():
    n = (64, 64, 64)
    r = 6.0
    count = 40
    ph = I.voxelize_spheres(n, I.rsa_sphere_centres(n, r, count, seed=3), r)
    exact = count * 4.0 / 3.0 * math.pi * r ** 3 / np.prod(n)
    assert ph.dtype == np.uint8 and set(np.unique(ph)) <= {0, 1}
    assert abs(ph.mean() - exact) < 0.03 * exact


def test_disc_is_centred_and_mirror_symmetric():
    for N in (16, 64, 128):
        ph = I.disc_phase_map((N, N), 0.2)
        assert abs(ph.mean() - 0.2) < 0.03
        assert np.array_equal(ph, ph[::-1, :]) and np.array_equal(ph, ph[:, ::-1]) and np.array_equal(ph, ph.T)


def test_upsampled_topology_keeps_the_fraction_exactly():
    base = I.voxelize_spheres((16, 16, 16), np.array([[8.0, 8.0, 8.0]]), 5.0)
    for f in (2, 3):
        up = I.upsample_phase(base, f)
        assert up.shape == (16 * f,) * 3
        assert up.mean() == base.mean()
        assert np.array_equal(up[::f, ::f, ::f], base)


def test_bench_workloads_are_the_documented_ones():
    cfg = I.config_3d_spheres(N=256, radius=10.0, vf=0.25, seed=0, ell_vox=4.0, n_incr=40, dE=1e-3)
    assert cfg.meta["sha256"][:16] == "1d67b6273ffaab29"
    assert cfg.meta["count"] == 1001 and abs(cfg.meta["vf_voxel"] - 0.2499) < 1e-4
    assert cfg.target.shape == (40, 6) and abs(cfg.target[-1][0] - 0.04) < 1e-12
    batch = I.config_batch(32)
    assert Counter(c.n[0] for c in batch) == {64: 6, 96: 10, 128: 16}
    assert sum(int(np.prod(c.n)) for c in batch) == 43974656


def test_uniaxial_path_and_plane_strain_mask():
    ctrl, tgt = I.uniaxial_path(5, 2e-3)
    assert list(ctrl) == [1, 0, 0, 0, 0, 0]
    assert np.allclose(tgt[:, 0], 2e-3 * np.arange(1, 6)) and np.all(tgt[:, 1:] == 0)
    c2 = I.plane_strain_mask(ctrl)
    # 33, 23 and 13 are strain-controlled at zero in plane strain; 22 and 12
    # stay stress-controlled
    assert list(c2) == [1, 0, 1, 1, 1, 0]
