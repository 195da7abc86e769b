"""GPU: batched RVEs (streams + graph-replayed Krylov chunks), the FFT
schedule autotuner and the two-variable sphere RVEs, against members run
alone and against the oracle."""
import numpy as np
import pytest

import rve_inputs as I
from oracle import rve_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

pkg = None


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global pkg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2103_04770_gb300 as p
    p.lib()
    pkg = p
    yield


EARLY_DAMAGE_3D = dict(I.MATRIX, eps_C=0.004, eps_R=0.04)
EARLY_CRACKING = dict(I.PARTICLE_CRACKING, eps_C=0.0003, eps_R=0.005)


def _member(n, vf, count, seed, n_incr=4, dE=1.5e-3, prec=1):
    cfg = I.config_spheres_two_var(n, vf, count, seed, ell_m=2.0, ell_p=1.5, n_incr=n_incr, dE=dE,
                                   precision=prec)
    cfg.params = [EARLY_DAMAGE_3D, EARLY_CRACKING]
    return cfg


def _small_batch(prec):
    return [_member((12, 12, 12), 0.2, 2, 0, prec=prec), _member((16, 10, 12), 0.15, 2, 1, prec=prec),
            _member((10, 15, 8), 0.25, 1, 2, prec=prec)]


def _parity_options(prec):
    opt = pkg.rve_default_options(prec)
    if prec == 0:
        o = O.PARITY_OPTIONS
        opt.tol_stag, opt.tol_newton, opt.cg_rtol, opt.pcg_rtol = o.tol_stag, o.tol_newton, o.cg_rtol, o.pcg_rtol
    return opt


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_equals_members_alone(prec):
    """Without autotuning the batch runs each member's exact launch sequence
    (graph replays on its own stream): results are bit-identical to the
    member stepped alone with direct launches."""
    cfgs = _small_batch(prec)
    alone = []
    for c in cfgs:
        with pkg.RVE(c, precision=prec) as r:
            alone.append([(r.step(), r.stress().copy()) for _ in range(c.target.shape[0])])
    with pkg.RVEBatch(cfgs, precision=prec, autotune_reps=0) as b:
        for i in range(cfgs[0].target.shape[0]):
            infos = b.step()
            S = b.stresses()
            for m in range(len(cfgs)):
                ref_info, ref_s = alone[m][i]
                assert infos[m]["status"] == 0
                np.testing.assert_array_equal(S[m], ref_s)
                assert infos[m]["cg_iters"] == ref_info["cg_iters"]
                assert infos[m]["pcg_iters"] == ref_info["pcg_iters"]


_ORACLE = {}


def _oracle_curve(m, cfg):
    """oracle curve of small-batch member m (cached: both precisions use it)"""
    if m in _ORACLE:
        return _ORACLE[m]
    g = O.Grid(cfg.n, cfg.L)
    st = O.make_state(g, cfg.phase, O.phases_from_dicts(cfg.params), cfg.ell)
    prev = np.zeros(6)
    recs = []
    for i in range(cfg.target.shape[0]):
        recs.append(O.step_increment(st, cfg.strain_ctrl, prev, cfg.target[i], O.PARITY_OPTIONS))
        prev = cfg.target[i]
    _ORACLE[m] = (recs, st)
    return recs, st


@pytest.mark.parametrize("prec", [0, 1])
def test_autotuned_batch_matches_oracle(prec):
    """Autotuned schedules change only the rounding order: every member's
    curve stays within the parity tolerance of the oracle (FP64 <= 1e-10,
    mixed <= 1e-4 of max |Sigma11|), two non-local variables included."""
    cfgs = _small_batch(prec)
    opt = _parity_options(prec)
    with pkg.RVEBatch(cfgs, precision=prec, options=opt, autotune_reps=2) as b:
        got = []
        for i in range(cfgs[0].target.shape[0]):
            infos = b.step()
            got.append(([inf["sigma"] for inf in infos], [inf["D_max"] for inf in infos]))
    tol = 1e-10 if prec == 0 else 1e-4
    for m, c in enumerate(cfgs):
        recs, st = _oracle_curve(m, c)
        smax = max(abs(r["S"][0]) for r in recs)
        for i, r in enumerate(recs):
            assert np.abs(np.asarray(got[i][0][m]) - r["S"]).max() <= tol * smax
            assert abs(got[i][1][m] - r["D_max"]) <= (1e-9 if prec == 0 else 1e-3)
        part = st.phase == 1
        assert st.D[part].max() > 0.0 and st.D[~part].max() > 0.0   # both variables damaged


def test_autotune_keeps_the_operator():
    """A tuned schedule (radix orders, tile width) is a valid factorisation
    and leaves G*(C_T : p) unchanged to FP64 round-off."""
    n = (30, 20, 24)                       # 15 = 5*3, 20 = 5*4, 24 = 8*3 or 4*3*2 ...
    cfg = _member(n, 0.2, 2, 3, prec=0)
    rng = np.random.default_rng(4)
    V = int(np.prod(n))
    p = torch.as_tensor(rng.standard_normal((6, V)), device="cuda", dtype=torch.float64)
    with pkg.RVE(cfg, precision=0) as r:
        # a tangent descriptor from a return map of a plastic, damaged state
        eps = 3e-3 * rng.standard_normal((6, V))
        eps[0] += 6e-3
        f = lambda *s: torch.zeros(*s, device="cuda", dtype=torch.float64)
        abar = torch.as_tensor(rng.uniform(0, 0.02, (2, V)), device="cuda", dtype=torch.float64)
        pkg.rve_op_return_map(r.h, torch.as_tensor(eps, device="cuda"), f(6, V), f(V), abar, f(6, V),
                              f(6, V), f(V), f(V), f(2, V))
        a0 = torch.empty_like(p)
        pkg.rve_op_matvec(r.h, p, a0)
        ms, tx, rad = pkg.rve_autotune(r.h, 2)
        assert ms > 0 and tx in (1, 2, 4, 8, 16, 32)
        for N, rr in zip((n[0] // 2, n[1], n[2]), rad):
            assert int(np.prod(rr)) == N and all(x in (2, 3, 4, 5, 8) for x in rr)
        a1 = torch.empty_like(p)
        pkg.rve_op_matvec(r.h, p, a1)
        ref = a0.abs().max().item()
        assert (a1 - a0).abs().max().item() <= 1e-12 * ref
        r.step()                               # stepping after tuning works ...
        with pytest.raises(pkg.RVEError) as e:  # ... and closes tuning
            pkg.rve_autotune(r.h, 2)
        assert e.value.status == pkg.RVE_ERR_STATE


def test_graphs_match_direct_launches():
    """rve_set_graphs on a single handle: identical increments."""
    cfg = _member((12, 12, 12), 0.2, 2, 5, prec=1)
    out = []
    for graphs in (False, True):
        with pkg.RVE(cfg, precision=1) as r:
            pkg.rve_set_graphs(r.h, graphs)
            out.append([(r.step()["cg_iters"], r.stress().copy()) for _ in range(3)])
    for (c0, s0), (c1, s1) in zip(*out):
        assert c0 == c1
        np.testing.assert_array_equal(s0, s1)


@pytest.mark.parametrize("N", [64, 96, 128])
def test_batch_member_grids_mixed_vs_fp64(N):
    """One increment of a full-size member of the batched workload for each
    grid (two variables, runtime mixed-radix FFT schedules with tiles above
    48 KB of shared memory): the mixed form agrees with the FP64 form within
    1e-4 of Sigma11, and both converge."""
    seed = next(s for s in range(64) if I.config_batch_member(s, n_incr=1).n[0] == N)
    cfg = I.config_batch_member(seed, n_incr=1)
    out = {}
    for prec in (0, 1):
        with pkg.RVE(cfg, precision=prec) as r:
            info = r.step()
            assert info["status"] == 0 and info["cg_iters"] > 0 and info["pcg_iters"] > 0
            out[prec] = r.stress().copy()
    assert abs(out[1][0] - out[0][0]) <= 1e-4 * abs(out[0][0])
    assert np.abs(out[1] - out[0]).max() <= 1e-4 * abs(out[0][0])


@pytest.mark.parametrize("prec", [0, 1])
def test_save_and_resume_state(prec):
    """Saving after two increments and resuming on a fresh handle gives the
    same next increments, bit for bit, as continuing."""
    cfg = _member((12, 12, 12), 0.2, 2, 7, n_incr=4, prec=prec)
    with pkg.RVE(cfg, precision=prec) as r:
        r.step()
        r.step()
        img = pkg.rve_save_state(r.h)
        cont = [(r.step()["cg_iters"], r.stress().copy()) for _ in range(2)]
    with pkg.RVE(cfg, precision=prec) as r2:
        pkg.rve_load_state(r2.h, img)
        res = [(r2.step(), r2.stress().copy()) for _ in range(2)]
    for (c0, s0), (info, s1) in zip(cont, res):
        assert info["cg_iters"] == c0
        np.testing.assert_array_equal(s0, s1)
    assert res[0][0]["increment"] == 3
    # the image is FP64 in both forms: the other form resumes from it and
    # agrees with this form's continuation to the mixed-form tolerance
    with pkg.RVE(cfg, precision=1 - prec) as r3:
        pkg.rve_load_state(r3.h, img)
        info = r3.step()
        assert info["increment"] == 3
        s3 = r3.stress()
        assert np.abs(s3 - cont[0][1]).max() <= 1e-4 * abs(cont[0][1][0])
    other = _member((12, 12, 16), 0.2, 2, 7, n_incr=4, prec=prec)
    with pkg.RVE(other, precision=prec) as r4:       # grid mismatch is rejected
        with pytest.raises(pkg.RVEError) as e:
            pkg.rve_load_state(r4.h, img)
        assert e.value.status == pkg.RVE_ERR_ARG
