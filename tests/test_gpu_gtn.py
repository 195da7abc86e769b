"""GPU parity of the non-local Gurson-Tvergaard-Needleman model (law 3,
Sections 2.1.1 and 2.2.2, Appendix A.1) against the FP64 oracle.

The GPU solves the local Backward-Euler system by Newton with an analytic
Jacobian and forms the consistent tangent by implicit differentiation; the
oracle uses complex-step derivatives for both, so agreement of the tangents
compares two methods.  Tolerances: FP64 <= 1e-11 on the return map and
<= 1e-10 on homogenised stress of whole increments (staggered counts equal);
the mixed form <= 2e-6 on the FP32 tangent and <= 1e-4 on homogenised stress.
"""
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


GTN = dict(E=70000.0, nu=0.33, sigma_y=100.0, H=500.0, law=3, eps_C=0.0, eps_R=1.0, D_max=0.0, var=0,
           hard=0, N=0.1, q1=1.5, q2=1.0, q3=2.25, f_C=0.15, f_F=0.25, f_N=0.04, eps_N=0.02, s_N=0.01,
           f0=0.02, fstar_max=0.6)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda", dtype=torch.float64)


def host(t):
    return t.detach().cpu().numpy()


def _states(g, seed):
    """Random GTN states: strains with pressures of both signs, plastic
    history, porosity and non-local variables of the last increment and of
    the staggered iterate; about 30 % elastic-particle voxels."""
    rng = np.random.default_rng(seed)
    V = g.V
    nc = 6 if g.d == 3 else 3
    phase = (rng.random(g.shape) < 0.3).astype(np.uint8)
    eps = rng.uniform(0.2, 1.5, (V, 1)) * 1.2e-3 * rng.standard_normal((V, nc))
    eps[:, :min(nc, 2)] += rng.uniform(-1.0, 3.0, (V, 1)) * 1.2e-3
    epsp_n = 2e-4 * rng.standard_normal((V, 6))
    ep_n = np.abs(5e-3 * rng.standard_normal(V))
    abar_n = np.stack([ep_n, rng.uniform(0.0, 2e-3, V)])
    abar = abar_n + np.stack([rng.uniform(0.0, 0.02, V), rng.uniform(0.0, 0.01, V)])
    f_n = rng.uniform(0.0, 0.12, V)
    part = phase.ravel() == 1
    epsp_n[part] = 0.0
    ep_n[part] = 0.0
    f_n[part] = 0.0
    return phase, eps, epsp_n, ep_n, abar, abar_n, f_n


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("hard", [0, 1])
@pytest.mark.parametrize("n", [(24, 20), (12, 10, 8)])
def test_return_map_gtn(n, hard, prec):
    g = O.Grid(n)
    d = g.d
    nc = 6 if d == 3 else 3
    phase, eps, epsp_n, ep_n, abar, abar_n, f_n = _states(g, 3 + hard)
    params = [dict(GTN, hard=hard), I.PARTICLE]
    ell = np.array([[2.0, 0.04], [2.0, 0.04]])
    h = pkg.rve_create(d, n, [float(x) for x in n], prec, 2)
    try:
        pkg.rve_set_phases(h, phase, params, ell)
        rm = O.return_map(O.embed(eps, d), epsp_n, ep_n, abar, phase.ravel().astype(int),
                          O.phases_from_dicts(params), abar_n=abar_n, f_n=f_n)
        V = g.V
        out = {k: torch.empty(sz, device="cuda", dtype=torch.float64)
               for k, sz in (("sigma", (6, V)), ("epsp", (6, V)), ("ep", V), ("D", V), ("alpha", (2, V)), ("f", V))}
        pkg.rve_op_return_map_ex(h, dev(eps.T), dev(epsp_n.T), dev(ep_n), dev(abar), dev(abar_n), dev(f_n),
                                 out["sigma"], out["epsp"], out["ep"], out["D"], out["alpha"], out["f"])
        s_ref = rm["sigma"].T
        assert np.abs(host(out["sigma"]) - s_ref).max() <= 1e-11 * np.abs(s_ref).max()
        assert np.abs(host(out["epsp"]) - rm["epsp"].T).max() <= 1e-14
        assert np.abs(host(out["ep"]) - rm["ep"]).max() <= 1e-14
        assert np.abs(host(out["D"]) - rm["D"]).max() <= 1e-14
        assert np.abs(host(out["f"]) - rm["f"]).max() <= 1e-14
        assert np.abs(host(out["alpha"]) - rm["alpha"]).max() <= 1e-14
        gtn = phase.ravel() == 0
        plastic = gtn & (rm["ep"] > ep_n)
        assert plastic.sum() > 0.1 * V and (gtn & ~plastic).sum() > 0.02 * V
        rng = np.random.default_rng(11)
        p = rng.standard_normal((V, nc))
        comps = O.carried(d)
        tau_ref = np.einsum("vij,vj->vi", rm["C"][:, comps][:, :, comps], p)
        tau = torch.empty(nc, V, device="cuda", dtype=torch.float64)
        pkg.rve_op_tangent_apply(h, dev(p.T), tau)
        tol = 1e-9 if prec == 0 else 2e-6
        assert np.abs(host(tau) - tau_ref.T).max() <= tol * np.abs(tau_ref).max()
    finally:
        pkg.rve_free(h)


def _gtn_cfg(dim, hard=0):
    if dim == 2:
        cfg = I.config_2d_disc(16, ell_vox=3.0, n_incr=6, dE=1e-3)
        cfg.ell = np.array([[3.0, 0.06], [3.0, 0.06]])
    else:
        n = (8, 8, 8)
        ph = I.voxelize_spheres(n, np.array([[4.0, 4.0, 4.0]]), 2.6)
        ctrl, tgt = I.uniaxial_path(5, 1.5e-3)
        cfg = I.RVEConfig("gtn_sphere_8", n, (8.0, 8.0, 8.0), ph, [], np.array([[2.0, 0.04], [2.0, 0.04]]),
                          ctrl, tgt, 0)
    cfg.params = [dict(GTN, hard=hard), I.PARTICLE]
    return cfg


def _fields(h, V, nc, J):
    out = {}
    for name, which, n in (("eps", 0, nc * V), ("D", 2, V), ("abar", 3, J * V), ("ep", 4, V), ("f", 6, V)):
        t = torch.empty(n, device="cuda", dtype=torch.float64)
        pkg.rve_get_field(h, which, t)
        out[name] = host(t)
    return out


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", [(2, 0), (3, 0), (2, 1)], ids=["2d", "3d", "2d_aravas"])
def test_gtn_increments_match_oracle(case, prec):
    dim, hard = case
    cfg = _gtn_cfg(dim, hard)
    g = O.Grid(cfg.n, cfg.L)
    nc = 6 if dim == 3 else 3
    st = O.make_state(g, cfg.phase, O.phases_from_dicts(cfg.params), cfg.ell)
    oopt = O.PARITY_OPTIONS
    opt = pkg.rve_default_options(prec)
    if prec == 0:
        opt.tol_stag, opt.tol_newton, opt.cg_rtol, opt.pcg_rtol = (oopt.tol_stag, oopt.tol_newton,
                                                                   oopt.cg_rtol, oopt.pcg_rtol)
    prev = np.zeros(6)
    recs = []
    with pkg.RVE(cfg, precision=prec, options=opt) as r:
        for i in range(cfg.target.shape[0]):
            info = r.step()
            rec = O.step_increment(st, cfg.strain_ctrl, prev, cfg.target[i], oopt)
            prev = cfg.target[i]
            recs.append(rec)
            smax = max(abs(x["S"][0]) for x in recs)
            tol = 1e-10 if prec == 0 else 1e-4
            assert np.abs(info["sigma"] - rec["S"]).max() <= tol * smax
            assert np.abs(info["eps"] - rec["E"]).max() <= tol * abs(rec["E"][0])
            if prec == 0:
                assert info["staggered_iters"] == rec["stag"]
            fl = _fields(r.h, g.V, nc, 2)
            ftol = 1e-8 if prec == 0 else 5e-3
            assert np.abs(fl["f"] - st.f).max() <= ftol * st.f.max()
            assert np.abs(fl["D"] - st.D).max() <= ftol * st.D.max()
            assert np.abs(fl["ep"] - st.ep).max() <= ftol * max(st.ep.max(), 1e-300)
            assert np.abs(fl["abar"] - st.abar.ravel()).max() <= ftol * np.abs(st.abar).max()
            assert np.abs(fl["eps"] - st.eps.T.ravel()).max() <= (1e-9 if prec == 0 else 1e-3) * np.abs(st.eps).max()
        assert st.f.max() > 0.022                    # porosity grew


def test_gtn_state_image_carries_the_porosity():
    """Save after two increments, resume on a fresh handle: the next
    increment (which reads the stored porosity) repeats bit for bit."""
    cfg = _gtn_cfg(2)
    with pkg.RVE(cfg, precision=0) as r:
        r.step()
        r.step()
        img = pkg.rve_save_state(r.h)
        info = r.step()
        s_cont = r.stress().copy()
    with pkg.RVE(cfg, precision=0) as r2:
        pkg.rve_load_state(r2.h, img)
        info2 = r2.step()
        np.testing.assert_array_equal(r2.stress(), s_cont)
        assert info2["cg_iters"] == info["cg_iters"]


def test_gtn_phase_validation():
    """Law 3 needs two non-local variables and a cap below f_V*."""
    n = (8, 8)
    ph = np.zeros((8, 8), dtype=np.uint8)
    h = pkg.rve_create(2, n, [8.0, 8.0], 0, 1)
    try:
        with pytest.raises(pkg.RVEError):
            pkg.rve_set_phases(h, ph, [GTN], np.array([[1.0]]))        # J = 1
    finally:
        pkg.rve_free(h)
    h = pkg.rve_create(2, n, [8.0, 8.0], 0, 2)
    try:
        with pytest.raises(pkg.RVEError):
            pkg.rve_set_phases(h, ph, [dict(GTN, fstar_max=0.7)], np.array([[1.0], [1.0]]))
        pkg.rve_set_phases(h, ph, [GTN], np.array([[1.0], [1.0]]))
    finally:
        pkg.rve_free(h)
