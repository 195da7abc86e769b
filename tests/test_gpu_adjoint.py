"""GPU adjoint of the load path (rve_adjoint_forward / rve_adjoint_backward
and the autograd Function) against the oracle's adjoint and against central
finite differences of GPU forward runs."""
import numpy as np
import pytest

import rve_inputs as I
from oracle import rve_oracle as O
from oracle import rve_adjoint as OA

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


MAT = dict(I.MATRIX, eps_C=0.003, eps_R=0.03)
PC = dict(I.PARTICLE_CRACKING, eps_C=0.0003, eps_R=0.005)


def _tiny(n=(6, 6, 6), r=1.8, n_incr=3):
    ph = I.voxelize_spheres(n, np.array([[x / 2 for x in n]]), r)
    ctrl, tgt = I.uniaxial_path(n_incr, 1.5e-3)
    return I.RVEConfig("adj_tiny", n, tuple(float(x) for x in n), ph, [MAT, PC],
                       np.array([[1.5, 0.03], [0.02, 1.0]]), ctrl, tgt, 0)


def _opts():
    o = pkg.rve_default_options(0)
    p = O.PARITY_OPTIONS
    o.tol_stag, o.tol_newton, o.cg_rtol, o.pcg_rtol = p.tol_stag, p.tol_newton, p.cg_rtol, p.pcg_rtol
    o.tol_stag = 1e-12
    return o


def _gpu_grad(cfg, every=5, stiff=None):
    J = int(cfg.ell.shape[0])
    h = pkg.rve_create(3, cfg.n, cfg.L, 0, J)
    try:
        pkg.rve_set_options(h, _opts())
        pkg.rve_set_phases(h, cfg.phase, cfg.params, cfg.ell)
        pkg.rve_set_load_path(h, cfg.strain_ctrl, cfg.target)
        if stiff is not None:
            pkg.rve_set_stiffness_field(h, stiff)
        Jv = pkg.rve_adjoint_forward(h, every)
        gp, ge, gs, info = pkg.rve_adjoint_backward(h, 1.0, len(cfg.params), J, int(np.prod(cfg.n)))
        S = pkg.rve_homogenized_stress(h)
    finally:
        pkg.rve_free(h)
    return Jv, gp, ge, gs, info, S


def test_adjoint_matches_oracle_adjoint():
    """Same discrete adjoint on both sides: every parameter, both lengths and
    the per-voxel modulus field agree to 1e-8 relative."""
    cfg = _tiny()
    g = O.Grid(cfg.n)
    ref = OA.adjoint_gradient(g, cfg.phase, cfg.params, cfg.ell, cfg.strain_ctrl, cfg.target,
                              O.PARITY_OPTIONS)
    Jv, gp, ge, gs, info, S = _gpu_grad(cfg)
    assert Jv == pytest.approx(ref["J"], rel=1e-10)
    assert S[0] == pytest.approx(Jv, rel=1e-14)            # left at the final state
    for (q, k), v in ref["theta"].items():
        if cfg.params[q]["law"] == 0:
            continue
        kk = OA.PARAMS.index(k)
        assert gp[q, kk] == pytest.approx(v, rel=1e-8, abs=1e-12 * abs(Jv))
    np.testing.assert_allclose(ge, ref["ell"], rtol=1e-8)
    assert np.abs(gs - ref["stiff"]).max() <= 1e-8 * np.abs(ref["stiff"]).max()
    assert info["increments"] == 3 and info["recomputed"] == 3


def test_checkpoint_spacing_does_not_change_the_gradient():
    cfg = _tiny(n_incr=4)
    out = [_gpu_grad(cfg, every=k) for k in (1, 2, 5)]
    for o in out[1:]:
        np.testing.assert_array_equal(o[1], out[0][1])
        np.testing.assert_array_equal(o[2], out[0][2])
        np.testing.assert_array_equal(o[3], out[0][3])
    assert [o[4]["checkpoints"] for o in out] == [4, 2, 1]


def test_adjoint_matches_gpu_finite_differences():
    """Central differences (h = 1e-5 relative) of GPU forward runs on a 12^3
    sphere RVE: within 1e-5 relative."""
    cfg = _tiny(n=(12, 12, 12), r=3.4, n_incr=3)
    Jv, gp, ge, gs, info, _ = _gpu_grad(cfg)

    def J_of(params, ell, stiff=None):
        c = I.RVEConfig(cfg.name, cfg.n, cfg.L, cfg.phase, params, ell, cfg.strain_ctrl, cfg.target, 0)
        with pkg.RVE(c, precision=0, options=_opts()) as r:
            if stiff is not None:
                pkg.rve_set_stiffness_field(r.h, stiff)
            for _ in range(c.target.shape[0]):
                r.step()
            return r.stress()[0]

    h = 1e-5
    for q, k in [(0, "sigma_y"), (0, "H"), (0, "eps_C"), (0, "eps_R"), (1, "eps_C"), (1, "eps_R")]:
        v = cfg.params[q][k]
        pp = [dict(p) for p in cfg.params]
        pm = [dict(p) for p in cfg.params]
        pp[q][k] = v * (1 + h)
        pm[q][k] = v * (1 - h)
        fd = (J_of(pp, cfg.ell) - J_of(pm, cfg.ell)) / (2 * h * v)
        assert gp[q, OA.PARAMS.index(k)] == pytest.approx(fd, rel=1e-5)
    for j in range(2):
        own = cfg.ell[j].max()
        fd = (J_of(cfg.params, cfg.ell * np.where(np.arange(2)[:, None] == j, 1 + h, 1.0))
              - J_of(cfg.params, cfg.ell * np.where(np.arange(2)[:, None] == j, 1 - h, 1.0))) / (2 * h * own)
        assert ge[j] == pytest.approx(fd, rel=1e-5)
    V = int(np.prod(cfg.n))
    for vox in (0, int(np.argmax(cfg.phase.ravel()))):
        s = np.ones(V)
        s[vox] = 1 + h
        Jp = J_of(cfg.params, cfg.ell, s)
        s[vox] = 1 - h
        Jm = J_of(cfg.params, cfg.ell, s)
        assert gs[vox] == pytest.approx((Jp - Jm) / (2 * h), rel=1e-5)


def test_autograd_function_runs_the_adjoint():
    from paper_2103_04770_gb300.adjoint import FinalStress, final_stress
    cfg = _tiny()
    params = torch.tensor([[d[k] for k in OA.PARAMS] for d in cfg.params], dtype=torch.float64,
                          requires_grad=True)
    ell = torch.tensor([1.5, 1.0], dtype=torch.float64, requires_grad=True)
    stiff = torch.ones(int(np.prod(cfg.n)), dtype=torch.float64, requires_grad=True)
    J = final_stress(cfg, params, ell, stiff, checkpoint_every=2, options=_opts())
    (2.0 * J).backward()
    Jv, gp, ge, gs, info, _ = _gpu_grad(cfg)
    assert J.item() == pytest.approx(Jv, rel=1e-14)
    np.testing.assert_allclose(params.grad.numpy(), 2.0 * gp, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(ell.grad.numpy(), 2.0 * ge, rtol=1e-12)
    np.testing.assert_allclose(stiff.grad.numpy(), 2.0 * gs, rtol=1e-12, atol=1e-18)
    assert FinalStress.last_info["checkpoints"] == 2


def test_adjoint_plane_strain_matches_oracle():
    """2D plane strain (carried components 11, 22, 12; gradient fields in
    two directions): GPU adjoint against the oracle's adjoint."""
    n = (12, 12)
    ph = I.disc_phase_map(n, 0.2)
    ctrl, tgt = I.uniaxial_path(3, 1e-3)
    cfg = I.RVEConfig("adj_2d", n, (12.0, 12.0), ph, [MAT, PC], np.array([[1.5, 0.03], [0.02, 1.0]]),
                      I.plane_strain_mask(ctrl), tgt, 0)
    g = O.Grid(n)
    ref = OA.adjoint_gradient(g, cfg.phase, cfg.params, cfg.ell, cfg.strain_ctrl, cfg.target,
                              O.PARITY_OPTIONS)
    h = pkg.rve_create(2, n, cfg.L, 0, 2)
    try:
        pkg.rve_set_options(h, _opts())
        pkg.rve_set_phases(h, cfg.phase, cfg.params, cfg.ell)
        pkg.rve_set_load_path(h, cfg.strain_ctrl, cfg.target)
        Jv = pkg.rve_adjoint_forward(h, 2)
        gp, ge, gs, info = pkg.rve_adjoint_backward(h, 1.0, 2, 2, g.V)
    finally:
        pkg.rve_free(h)
    assert Jv == pytest.approx(ref["J"], rel=1e-10)
    for (q, k), v in ref["theta"].items():
        assert gp[q, OA.PARAMS.index(k)] == pytest.approx(v, rel=1e-8, abs=1e-12 * abs(Jv))
    np.testing.assert_allclose(ge, ref["ell"], rtol=1e-8, atol=1e-12 * abs(Jv))
    assert np.abs(gs - ref["stiff"]).max() <= 1e-8 * np.abs(ref["stiff"]).max()
