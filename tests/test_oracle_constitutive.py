"""Pins of the oracle's Lemaitre return map (Appendix A.2, readings R8-R11)
and mechanics (Section 3.2.2) against closed forms, finite differences,
laminate exact solutions, Voigt/Reuss bounds and a dense Galerkin solve."""
import math

import numpy as np
import pytest

import rve_inputs as I
from oracle import rve_oracle as O
from tests import _stencil as S

MAT = O.phases_from_dicts([I.MATRIX])[0]
ELASTIC_MATRIX = dict(I.MATRIX, law=0, var=-1)


def _yield_fn(sig_eff, ep, ph):
    t = O.mandel_to_tensor(sig_eff)
    dev = t - np.trace(t, axis1=-2, axis2=-1)[..., None, None] * np.eye(3) / 3
    return np.sqrt(np.sum(dev * dev, axis=(-2, -1))) - math.sqrt(2 / 3) * (ph.sigma_y + ph.H * ep)


def test_return_map_consistency():
    """Plastic points land on the yield surface; elastic points obey Hooke."""
    rng = np.random.default_rng(0)
    V = 400
    eps = rng.uniform(0.05, 1.5, (V, 1)) * 2e-3 * rng.standard_normal((V, 6))
    epsp_n = 1e-4 * rng.standard_normal((V, 6))
    epsp_n[:, :3] -= epsp_n[:, :3].mean(axis=1, keepdims=True)     # deviatoric
    ep_n = np.abs(1e-3 * rng.standard_normal(V))
    abar = np.zeros((1, V))
    ph = np.zeros(V, dtype=int)
    rm = O.return_map(eps, epsp_n, ep_n, abar, ph, [MAT])
    f = _yield_fn(rm["sigma"], rm["ep"], MAT)
    plastic = rm["ep"] > ep_n
    assert plastic.sum() > 50 and (~plastic).sum() > 50
    assert np.abs(f[plastic]).max() < 1e-9 * MAT.sigma_y
    assert f[~plastic].max() <= 0
    # elastic points: sigma = C (eps - epsp_n)
    K, mu = MAT.K, MAT.mu
    e = eps - epsp_n
    tr = e[:, :3].sum(axis=1)
    hooke = K * tr[:, None] * O.IVEC + 2 * mu * (e - tr[:, None] * O.IVEC / 3)
    np.testing.assert_allclose(rm["sigma"][~plastic], hooke[~plastic], rtol=1e-12, atol=1e-9)
    # flow is deviatoric and eps_p grows by sqrt(2/3) |d epsp|
    depsp = rm["epsp"] - epsp_n
    assert np.abs(depsp[:, :3].sum(axis=1)).max() < 1e-15
    np.testing.assert_allclose(rm["ep"] - ep_n, math.sqrt(2 / 3) * np.linalg.norm(depsp, axis=1),
                               rtol=1e-12, atol=1e-16)


def test_tangent_matches_finite_differences():
    """C_T = d sigma / d eps (central differences, D frozen: R11)."""
    rng = np.random.default_rng(1)
    V = 60
    eps = 3e-3 * rng.standard_normal((V, 6))
    eps[:, 0] += 4e-3
    epsp_n = np.zeros((V, 6))
    ep_n = np.abs(1e-2 * rng.standard_normal(V))
    abar = np.full((1, V), 0.08)        # D = (0.08 - 0.03)/0.17 in the matrix
    ph = np.zeros(V, dtype=int)
    rm = O.return_map(eps, epsp_n, ep_n, abar, ph, [MAT])
    h = 1e-8
    for c in range(6):
        ep_ = eps.copy()
        em_ = eps.copy()
        ep_[:, c] += h
        em_[:, c] -= h
        sp = O.return_map(ep_, epsp_n, ep_n, abar, ph, [MAT])["sigma"]
        sm = O.return_map(em_, epsp_n, ep_n, abar, ph, [MAT])["sigma"]
        fd = (sp - sm) / (2 * h)
        np.testing.assert_allclose(rm["C"][:, :, c], fd, rtol=2e-5, atol=1e-3)
    assert np.all(rm["D"] == pytest.approx((0.08 - 0.03) / 0.17))


def _uniaxial_closed_form(E11, ph):
    """Uniaxial stress, linear hardening: sigma = E eps below yield, else
    sigma_y + E_t (eps - sigma_y/E), eps_p = (E eps - sigma_y)/(E + H);
    Sigma11 = (1 - D(eps_p)) sigma (uniform fields: abar = alpha)."""
    E, H, sy = ph.E, ph.H, ph.sigma_y
    if E * E11 <= sy:
        return E * E11, 0.0, 0.0
    ep = (E * E11 - sy) / (E + H)
    s = sy + H * ep
    D = min(max((ep - ph.eps_C) / (ph.eps_R - ph.eps_C), 0.0), ph.D_max)
    return (1 - D) * s, ep, D


@pytest.mark.parametrize("dim", [3])
def test_uniaxial_closed_form_through_staggered_loop(dim):
    """Homogeneous damaging RVE under mixed control (E11 given, Sigma = 0
    elsewhere): the full staggered scheme reproduces the closed form along
    the curve, through yield and damage onset."""
    n = (4, 4, 4)
    g = O.Grid(n)
    ph = np.zeros(g.shape, dtype=np.uint8)
    ctrl, tgt = I.uniaxial_path(8, 6e-3)
    ell = np.array([[2.0, 0.04]])
    st = O.run_load_path(g, ph, [I.MATRIX, I.PARTICLE], ell, ctrl, tgt, O.PARITY_OPTIONS)
    for rec, t in zip(st.curve, tgt):
        s11, ep, D = _uniaxial_closed_form(t[0], MAT)
        assert rec["S"][0] == pytest.approx(s11, rel=1e-10)
        assert np.abs(rec["S"][1:]).max() < 1e-9 * abs(s11)
        assert rec["D_max"] == pytest.approx(D, abs=1e-10)
    assert st.curve[-1]["D_max"] > 0.05          # damage was reached
    assert np.abs(st.ep - _uniaxial_closed_form(tgt[-1][0], MAT)[1]).max() < 1e-11


def test_homogeneous_strain_control_needs_no_cg():
    """Uniform strain in a homogeneous RVE: G*(sigma) = 0, zero CG work."""
    g = O.Grid((4, 4, 4))
    ph = np.zeros(g.shape, dtype=np.uint8)
    ctrl = np.ones(6, dtype=np.uint8)
    tgt = np.array([[1e-3, -2e-4, 3e-4, 1e-4, -5e-5, 2e-4]])
    st = O.run_load_path(g, ph, [I.MATRIX, I.PARTICLE], np.array([[1.0, 0.02]]), ctrl, tgt,
                         O.PARITY_OPTIONS)
    assert st.curve[0]["cg"] == 0
    np.testing.assert_allclose(st.curve[0]["E"], tgt[0], atol=1e-16)


@pytest.mark.parametrize("dim", [2, 3])
def test_homogeneous_elastic_mixed_control(dim):
    """Elastic uniaxial stress: 3D Sigma11 = E E11, E22 = -nu E11; plane
    strain Sigma11 = E/(1-nu^2) E11, E22 = -nu/(1-nu) E11, Sigma33 = nu
    Sigma11."""
    n = (4, 4) if dim == 2 else (4, 4, 4)
    g = O.Grid(n)
    ph = np.ones(g.shape, dtype=np.uint8)                 # elastic particle phase
    ctrl, tgt = I.uniaxial_path(1, 1e-3)
    if dim == 2:
        ctrl = I.plane_strain_mask(ctrl)
    st = O.run_load_path(g, ph, [I.MATRIX, I.PARTICLE], np.array([[1.0, 0.02]]), ctrl, tgt,
                         O.PARITY_OPTIONS)
    E, nu = I.PARTICLE["E"], I.PARTICLE["nu"]
    rec = st.curve[0]
    if dim == 3:
        assert rec["S"][0] == pytest.approx(E * 1e-3, rel=1e-12)
        assert rec["E"][1] == pytest.approx(-nu * 1e-3, rel=1e-12)
        assert rec["E"][2] == pytest.approx(-nu * 1e-3, rel=1e-12)
    else:
        s11 = E / (1 - nu * nu) * 1e-3
        assert rec["S"][0] == pytest.approx(s11, rel=1e-12)
        assert rec["E"][1] == pytest.approx(-nu / (1 - nu) * 1e-3, rel=1e-12)
        assert rec["S"][2] == pytest.approx(nu * s11, rel=1e-12)


def _iso_C(E, nu):
    K = E / (3 * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    return K * np.outer(O.IVEC, O.IVEC) + 2 * mu * (np.eye(6) - np.outer(O.IVEC, O.IVEC) / 3)


def _laminate_exact(f1, C0, C1, E):
    """Layers normal to x1, prescribed mean strain E (Mandel, 6): in-plane
    strains (22, 33, 23) are uniform, tractions (11, 13, 12) are uniform.
    Unknowns: the (11, 13, 12) strains of each layer and the common
    traction; solved as one small linear system."""
    a = [0, 4, 5]            # free (jump) components
    b = [1, 2, 3]            # continuous components
    A = np.zeros((9, 9))
    rhs = np.zeros(9)
    # rows 0-2: traction in layer 0 = t ; rows 3-5: traction in layer 1 = t
    # unknowns: x0 (3), x1 (3), t (3)
    for L, (C, off) in enumerate([(C0, 0), (C1, 3)]):
        for r, i in enumerate(a):
            A[3 * L + r, off:off + 3] = C[i, a]
            A[3 * L + r, 6 + r] = -1.0
            rhs[3 * L + r] = -C[i, b] @ E[b]
    # rows 6-8: averages
    for r in range(3):
        A[6 + r, r] = 1 - f1
        A[6 + r, 3 + r] = f1
        rhs[6 + r] = E[a[r]]
    x = np.linalg.solve(A, rhs)
    e0 = E.copy()
    e1 = E.copy()
    e0[a] = x[:3]
    e1[a] = x[3:6]
    return e0, e1


def test_laminate_exact_solution():
    """Two-phase elastic laminate: the Galerkin solution is the exact
    piecewise-uniform one to round-off."""
    n = (8, 3, 2)
    g = O.Grid(n)
    ph = I.laminate_phase_map(n, [(2, 5)])            # 3 of 8 layers are phase 1
    f1 = 3 / 8
    ctrl = np.ones(6, dtype=np.uint8)
    Et = np.array([1e-3, -2e-4, 3e-4, 2e-4, -1e-4, 5e-4])    # tensor shears
    st = O.run_load_path(g, ph, [ELASTIC_MATRIX, I.PARTICLE], np.array([[1.0, 0.02]]), ctrl,
                         Et[None], O.PARITY_OPTIONS)
    C0 = _iso_C(I.MATRIX["E"], I.MATRIX["nu"])
    C1 = _iso_C(I.PARTICLE["E"], I.PARTICLE["nu"])
    e0, e1 = _laminate_exact(f1, C0, C1, Et * O.MANDEL_W)
    eps = st.eps.reshape(g.shape + (6,))
    np.testing.assert_allclose(eps[..., 0, :], np.broadcast_to(e0, eps[..., 0, :].shape), atol=1e-15)
    np.testing.assert_allclose(eps[..., 3, :], np.broadcast_to(e1, eps[..., 3, :].shape), atol=1e-15)


def test_voigt_reuss_bounds():
    """Apparent stiffness of a random two-phase elastic cell lies between the
    Reuss and Voigt bounds (energy sense)."""
    n = (6, 6, 6)
    g = O.Grid(n)
    rng = np.random.default_rng(5)
    ph = (rng.random(g.shape) < 0.3).astype(np.uint8)
    f1 = ph.mean()
    ctrl = np.ones(6, dtype=np.uint8)
    Et = np.array([1e-3, 0, 0, 0, 0, 0])
    st = O.run_load_path(g, ph, [ELASTIC_MATRIX, I.PARTICLE], np.array([[1.0, 0.02]]), ctrl,
                         Et[None], O.PARITY_OPTIONS)
    E = Et * O.MANDEL_W
    W = st.curve[0]["S"] * O.MANDEL_W @ E
    C0 = _iso_C(I.MATRIX["E"], I.MATRIX["nu"])
    C1 = _iso_C(I.PARTICLE["E"], I.PARTICLE["nu"])
    voigt = E @ ((1 - f1) * C0 + f1 * C1) @ E
    reuss = E @ np.linalg.inv((1 - f1) * np.linalg.inv(C0) + f1 * np.linalg.inv(C1)) @ E
    assert reuss < W < voigt


@pytest.mark.parametrize("n", [(4, 4), (4, 2, 3)])
def test_newton_step_matches_dense_galerkin(n):
    """One linearised solve G*(C:de) = -G*(sigma - Sigma_bar) by CG equals the
    dense Galerkin solution over admissible strains built from the stencil."""
    rng = np.random.default_rng(7)
    g = O.Grid(n)
    nc = 6 if g.d == 3 else 3
    mask = np.zeros(nc)
    mask[1] = 1.0
    A = rng.standard_normal(g.shape + (nc, nc))
    C = np.einsum("...ij,...kj->...ik", A, A) + 2 * np.eye(nc)
    sig = rng.standard_normal(g.shape + (nc,))
    sbar = mask * 0.3
    b = -O.G_apply(sig - sbar, g, mask)
    x, it = O.cg(lambda v: O.G_apply(np.einsum("...ij,...j->...i", C, v), g, mask), b, 1e-14, 500)
    B = S.compatible_basis(g.shape, g.h, mask)
    Cbig = np.zeros((B.shape[0], B.shape[0]))
    V = g.V
    Cf = C.reshape(V, nc, nc)
    for v in range(V):
        Cbig[v * nc:(v + 1) * nc, v * nc:(v + 1) * nc] = Cf[v]
    K = B.T @ Cbig @ B
    rhs = -B.T @ (sig - sbar).reshape(-1)
    y = np.linalg.lstsq(K, rhs, rcond=1e-12)[0]
    ref = (B @ y).reshape(x.shape)
    np.testing.assert_allclose(x, ref, atol=1e-10 * np.abs(ref).max())


# ------------------------------------------------- particle cracking (R20)
def _rotation(seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).standard_normal((3, 3)))
    return q * np.sign(np.diag(r))


def test_positive_principal_norm_closed_forms():
    """||<eps>_+|| for diagonal tensors, their rotations and pure shear."""
    diag = np.array([[3e-3, -1e-3, 2e-3], [-2e-3, -1e-3, -5e-4], [1e-3, 1e-3, 1e-3],
                     [4e-3, -4e-3, 0.0]])
    want = np.sqrt(np.sum(np.maximum(diag, 0.0) ** 2, axis=1))
    for k, dg in enumerate(diag):
        Q = _rotation(k)
        T = Q @ np.diag(dg) @ Q.T
        e = O.tensor_to_mandel(T[None])[0]
        assert O.positive_principal_norm(e[None])[0] == pytest.approx(want[k], rel=1e-12, abs=1e-18)
    g = 2.5e-3                               # eps12 = g: eigenvalues g, -g, 0
    e = np.array([[0, 0, 0, 0, 0, math.sqrt(2.0) * g]])
    assert O.positive_principal_norm(e)[0] == pytest.approx(g, rel=1e-13)


def test_particle_cracking_history_is_kept():
    """kappa = max(kappa_n, ||<eps>_+||): a smaller current strain keeps the
    stored history, a larger one replaces it; alpha carries kappa."""
    ph = O.phases_from_dicts([dict(I.PARTICLE_CRACKING, var=0)])
    eps = np.array([[4e-3, -8e-4, -8e-4, 0, 0, 0], [2e-2, -4e-3, -4e-3, 0, 0, 0]])
    ep_n = np.array([1e-2, 1e-2])
    out = O.return_map(eps, np.zeros((2, 6)), ep_n, np.zeros((1, 2)), np.zeros(2, dtype=int), ph)
    np.testing.assert_allclose(out["ep"], [1e-2, 2e-2], rtol=1e-14)
    np.testing.assert_allclose(out["alpha"][0], [1e-2, 2e-2], rtol=1e-14)
    P = ph[0]
    C = _iso_C(P.E, P.nu)
    np.testing.assert_allclose(out["sigma"][0], C @ eps[0], rtol=1e-13, atol=1e-15 * P.E)   # D = 0


def test_particle_cracking_uniaxial_through_staggered_loop():
    """Homogeneous cracking-particle RVE under uniaxial stress: kappa = E11
    (the lateral principal strains are -nu E11 < 0), abar = kappa for a
    uniform field, so Sigma11 = (1 - D(E11)) E E11 in closed form."""
    g = O.Grid((4, 4, 4))
    phm = np.zeros(g.shape, dtype=np.uint8)
    ctrl, tgt = I.uniaxial_path(6, 2.5e-3)
    mat = dict(I.PARTICLE_CRACKING, var=0)
    st = O.run_load_path(g, phm, [mat, I.MATRIX], np.array([[3.0, 0.06]]), ctrl, tgt,
                         O.PARITY_OPTIONS)
    P = O.phases_from_dicts([mat])[0]
    for rec, t in zip(st.curve, tgt):
        D = min(max((t[0] - P.eps_C) / (P.eps_R - P.eps_C), 0.0), P.D_max)
        assert rec["S"][0] == pytest.approx((1.0 - D) * P.E * t[0], rel=1e-10)
        assert rec["D_max"] == pytest.approx(D, abs=1e-10)
        assert rec["E"][1] == pytest.approx(-P.nu * t[0], rel=1e-9)
    assert st.curve[-1]["D_max"] > 0.5
