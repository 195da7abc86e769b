"""Pins of the adjoint oracle: the complex-step local Jacobians against the
return map's own consistent tangent and against central differences, the
gradient fields against the real-space corner stencil, and the whole
reverse recursion against central finite differences of the load path."""
import numpy as np
import pytest

import rve_inputs as I
from oracle import rve_oracle as O
from oracle import rve_adjoint as A
from tests import _stencil as S

MAT = dict(I.MATRIX, eps_C=0.003, eps_R=0.03)
PC = dict(I.PARTICLE_CRACKING, eps_C=0.0003, eps_R=0.005)


def _rand_local(seed, V=400):
    rng = np.random.default_rng(seed)
    phase = rng.integers(0, 2, V)
    amp = rng.uniform(0.05, 1.0, (V, 1)) * 3e-3
    eps = amp * rng.standard_normal((V, 6))
    eps[:, 0] += 1.3 * amp[:, 0]
    epsp = 1e-4 * rng.standard_normal((V, 6))
    epsp[:, :3] -= epsp[:, :3].mean(axis=1, keepdims=True)
    epsp[phase == 1] = 0.0
    ep = np.abs(2e-3 * rng.standard_normal(V))
    abar = np.stack([rng.uniform(0.0, 0.04, V), rng.uniform(0.0, 0.006, V)])
    stiff = rng.uniform(0.8, 1.2, V)
    return eps, epsp, ep, abar, phase, O.phases_from_dicts([MAT, PC]), stiff


def test_local_update_restates_the_return_map():
    eps, epsp, ep, abar, phase, phases, stiff = _rand_local(0)
    rm = O.return_map(eps, epsp, ep, abar, phase, phases, stiff)
    sig, alpha, epsp_new, ep_new = A.local_update(eps, epsp, ep, abar, phase, phases, stiff)
    scale = np.abs(rm["sigma"]).max()
    assert np.abs(sig - rm["sigma"]).max() <= 1e-14 * scale
    np.testing.assert_allclose(alpha, rm["alpha"], rtol=1e-14, atol=1e-18)
    np.testing.assert_allclose(epsp_new, rm["epsp"], rtol=1e-14, atol=1e-18)
    np.testing.assert_allclose(ep_new, rm["ep"], rtol=1e-14, atol=1e-18)


def test_complex_step_tangent_is_the_consistent_tangent():
    """d sigma / d eps by complex step equals the analytic consistent tangent
    C_T of the return map (plastic, elastic, damaged and cracking voxels)."""
    g = O.Grid((20, 20))          # V = 400, 2D carried components
    eps, epsp, ep, abar, phase, phases, stiff = _rand_local(1)
    eps[:, 2:5] = 0.0
    Lj = A.LocalJacobian(O.Grid((20, 20, 1)), eps, epsp, ep, abar, phase, phases, stiff)
    rm = O.return_map(eps, epsp, ep, abar, phase, phases, stiff)
    C = rm["C"]
    for c in range(6):
        col = Lj.cols[("eps", c)][0]
        assert np.abs(col - C[:, :, c]).max() <= 1e-10 * np.abs(C).max()
    plastic = (rm["ep"] > ep) & (phase == 0)
    assert plastic.sum() > 20 and (~plastic & (phase == 0)).sum() > 5
    del g


@pytest.mark.parametrize("key", [("epsp", 0), ("epsp", 3), ("ep",), ("abar", 0), ("abar", 1),
                                 ("theta", 0, "sigma_y"), ("theta", 0, "H"), ("theta", 0, "eps_C"),
                                 ("theta", 1, "eps_R"), ("stiff",)])
def test_complex_step_columns_match_central_differences(key):
    eps, epsp, ep, abar, phase, phases, stiff = _rand_local(2)
    Lj = A.LocalJacobian(O.Grid((20, 20, 1)), eps, epsp, ep, abar, phase, phases, stiff)

    def run(delta):
        a = [eps.copy(), epsp.copy(), ep.copy(), abar.copy(), phase, phases, stiff.copy()]
        dp = None
        if key[0] == "epsp":
            a[1][:, key[1]] += delta
        elif key[0] == "ep":
            a[2] += delta
        elif key[0] == "abar":
            a[3][key[1]] += delta
        elif key[0] == "stiff":
            a[6] += delta
        else:
            dp = {(key[1], key[2]): delta}
        return A.local_update(*a, dparam=dp)

    # steps balancing truncation against round-off for inputs of size ~1e-3
    # (strains), ~1 (stiffness factor) and the parameters' own scale
    h = {"epsp": 1e-7, "ep": 1e-7, "abar": 1e-7, "stiff": 1e-6,
         "theta": 1e-6 * getattr(phases[key[1]], key[2]) if key[0] == "theta" else 0}[key[0]]
    p, m = run(h), run(-h)
    # voxels whose branch flips inside +-h are left out (none expected)
    for k in range(4):
        fd = (p[k] - m[k]) / (2 * h)
        cs = Lj.cols[key][k]
        assert np.abs(fd - cs).max() <= 1e-6 * max(np.abs(cs).max(), 1e-12) + 1e-9


def test_gradient_fields_match_the_corner_stencil():
    n = (6, 5, 4)
    g = O.Grid(n, (3.0, 2.5, 2.0))
    a = np.random.default_rng(3).standard_normal(g.shape)
    G = A.willot_grad(a, g)
    ref = S.corner_grad(a, g.h)
    for j in range(3):
        np.testing.assert_allclose(G[j], ref[j], rtol=0, atol=1e-12 * np.abs(ref[j]).max())


def _tiny():
    n = (6, 6, 6)
    g = O.Grid(n)
    ph = I.voxelize_spheres(n, np.array([[3.0, 3.0, 3.0]]), 1.8)
    ell = np.array([[1.5, 0.03], [0.02, 1.0]])
    ctrl, tgt = I.uniaxial_path(3, 1.5e-3)
    return g, ph, [MAT, PC], ell, ctrl, tgt


def test_adjoint_gradient_matches_central_differences():
    """dJ/dtheta for J = final <sigma>_11 on a 6^3 two-phase, two-variable
    RVE (matrix yields and damages, particle cracks) against central
    differences with h = 1e-5 relative, within 1e-5 relative; every FD pair
    stays on the base run's smooth piece (branch signatures equal)."""
    g, ph, params, ell, ctrl, tgt = _tiny()
    opt = O.PARITY_OPTIONS
    res = A.adjoint_gradient(g, ph, params, ell, ctrl, tgt, opt)
    st0, states0 = A.forward_states(g, ph, params, ell, ctrl, tgt, opt)
    sig0 = A.branch_signature(g, ph, params, states0)
    part = ph.ravel() == 1
    assert st0.D[part].max() > 0 and st0.D[~part].max() > 0
    hrel = 1e-5
    straddle = 0

    def J_of(pp, ee, stiff=None):
        st, states = A.forward_states(g, ph, pp, ee, ctrl, tgt, opt, stiff)
        return O.homogenized_stress(st)[0], A.branch_signature(g, ph, pp, states, stiff)

    checks = []
    for q, k in [(0, "sigma_y"), (0, "H"), (0, "eps_C"), (0, "eps_R"), (1, "eps_C"), (1, "eps_R")]:
        v = params[q][k]
        h = hrel * v
        out = []
        for sgn in (1, -1):
            pp = [dict(p) for p in params]
            pp[q][k] = v + sgn * h
            out.append(J_of(pp, ell))
        checks.append(((out[0][0] - out[1][0]) / (2 * h), res["theta"][(q, k)], out))
    for j in range(2):
        own = ell[j].max()
        h = hrel * own
        out = []
        for sgn in (1, -1):
            ee = ell.copy()
            ee[j] *= (own + sgn * h) / own
            out.append(J_of(params, ee))
        checks.append(((out[0][0] - out[1][0]) / (2 * h), res["ell"][j], out))
    flat = ph.ravel()
    for vox in (int(np.where(flat == 0)[0][0]), int(np.where(flat == 1)[0][0])):
        out = []
        for sgn in (1, -1):
            s = np.ones(g.V)
            s[vox] += sgn * hrel
            out.append(J_of(params, ell, s))
        checks.append(((out[0][0] - out[1][0]) / (2 * hrel), res["stiff"][vox], out))
    for fd, ad, out in checks:
        straddle += sum(int((o[1] != sig0).sum()) for o in out)
        assert abs(ad - fd) <= 1e-5 * abs(fd)
    assert straddle == 0
