"""Parity at the full 256^3 size of the benchmark, in its launch
configuration (compile-time 256-point rows and register passes).

A 256^3 field obtained by tiling a 16^3 field 16 times along every axis has
Fourier modes only at multiples of 16, where the 256^3 grid's discrete
symbol (cubic voxels of unit size) equals the 16^3 grid's symbol at the same
angles.  So G*, the Helmholtz operator and solve, and a whole load increment
of a tiled 16^3 microstructure at 256^3 reproduce, voxel by voxel, the
oracle's result on the 16^3 cell: a full-size check whose oracle side runs
in seconds."""
import numpy as np
import pytest

import rve_inputs as I
from oracle import rve_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

pkg = None
NS, NB = 16, 256          # small cell, full grid
REP = NB // NS


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global pkg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2103_04770_gb300 as p
    p.lib()
    pkg = p
    yield


def tile(a):
    """(NS, NS, NS, ...) -> (NB, NB, NB, ...) periodic repetition"""
    reps = (REP, REP, REP) + (1,) * (a.ndim - 3)
    return np.tile(a, reps)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda", dtype=torch.float64)


def cm(a, nc):
    return np.ascontiguousarray(a.reshape(-1, nc).T)


def _small_phase():
    return I.voxelize_spheres((NS,) * 3, np.array([[8.0, 8.0, 8.0], [1.0, 2.0, 13.0]]), 3.2)


@pytest.mark.parametrize("prec", [0, 1])
def test_gamma_at_256_matches_tiled_oracle(prec):
    g = O.Grid((NS,) * 3)
    ctrl = np.array([1, 0, 0, 0, 0, 0], dtype=np.uint8)
    mask = 1.0 - ctrl.astype(float)
    rng = np.random.default_rng(11)
    tau = rng.standard_normal(g.shape + (6,)) + np.array([3.0, -1.0, 0.5, 0.2, 0.1, -0.3])
    ref = O.G_apply(tau, g, mask)
    phase = tile(_small_phase())
    h = pkg.rve_create(3, (NB,) * 3, (float(NB),) * 3, prec, 1)
    try:
        pkg.rve_set_phases(h, phase, [I.MATRIX, I.PARTICLE], np.array([[2.0, 0.04]]))
        pkg.rve_set_load_path(h, ctrl, np.zeros((1, 6)))
        out = torch.empty(6, NB ** 3, device="cuda", dtype=torch.float64)
        pkg.rve_op_apply_gamma(h, dev(cm(tile(tau), 6)), out)
        got = out.T.reshape(NB, NB, NB, 6)
        want = dev(tile(ref))
        tol = 1e-12 if prec == 0 else 5e-6
        assert (got - want).abs().max().item() <= tol * np.abs(tau).max()
    finally:
        pkg.rve_free(h)


def test_helmholtz_at_256_matches_tiled_oracle():
    g = O.Grid((NS,) * 3)
    ph = _small_phase()
    ell = np.array([[2.5, 0.05]])
    ell2 = ell[0][ph] ** 2
    alpha = np.random.default_rng(12).random(g.shape) * (ph == 0)
    ref, _ = O.helmholtz_solve(alpha, ell2, g, 1e-13, 3000)
    h = pkg.rve_create(3, (NB,) * 3, (float(NB),) * 3, 0, 1)
    try:
        pkg.rve_set_phases(h, tile(ph), [I.MATRIX, I.PARTICLE], ell)
        out = torch.empty(NB ** 3, device="cuda", dtype=torch.float64)
        pkg.rve_op_helmholtz_solve(h, 0, dev(tile(alpha).ravel()), out, 1e-13, 3000)
        want = dev(tile(ref).ravel())
        assert (out - want).abs().max().item() <= 1e-10 * np.abs(ref).max()
    finally:
        pkg.rve_free(h)


def test_mixed_increments_at_256_match_tiled_oracle():
    """The benchmark's form and launch shapes (mixed precision, 256^3): two
    softening increments of a tiled 16^3 two-sphere cell give the
    homogenised stress, strain and peak damage of the oracle's 16^3 cell
    (stress and strain within 1e-4, damage within 1e-3)."""
    ph = _small_phase()
    ctrl, tgt = I.uniaxial_path(2, 3e-3)
    params = [dict(I.MATRIX, eps_C=0.002, eps_R=0.03), I.PARTICLE]
    ell = np.array([[2.0, 0.04]])
    st = O.make_state(O.Grid((NS,) * 3), ph, O.phases_from_dicts(params), ell)
    recs, prev = [], np.zeros(6)
    for t in tgt:
        recs.append(O.step_increment(st, ctrl, prev, t, O.PARITY_OPTIONS))
        prev = t
    assert recs[-1]["D_max"] > 0.1
    smax = max(abs(r["S"][0]) for r in recs)
    cfg = I.RVEConfig("tiled", (NB,) * 3, (float(NB),) * 3, tile(ph), params, ell, ctrl, tgt, 1)
    with pkg.RVE(cfg, precision=1) as r:
        for rec in recs:
            info = r.step()
            assert np.abs(info["sigma"] - rec["S"]).max() <= 1e-4 * smax
            assert np.abs(info["eps"] - rec["E"]).max() <= 1e-4 * abs(rec["E"][0])
            assert abs(info["D_max"] - rec["D_max"]) <= 1e-3
