"""Pins of the oracle's non-local Gurson-Tvergaard-Needleman model (law 3:
Section 2.1.1, Section 2.2.2, Appendix A.1).

  * f_V* = (q1 + sqrt(q1^2 - q3)) / q3 = 2/3 for q1 = 1.5, q3 = 2.25, and the
    cap 0.9 f_V* = 0.6 (the values Section 4 prints);
  * with no porosity (f = f* = 0, no nucleation) the surface is von Mises and
    eps_0^p is the equivalent plastic strain: the update equals the J2 radial
    return of the Lemaitre law with D = 0, tangent included;
  * at plastic points the stress lies on the surface (phi written here from
    Eq. yield_gurson), the plastic strain increment is normal to it (the
    gradient taken by central differences of that phi), and the matrix work
    balance sigma : d eps^p = (1 - f) sigma_0 d eps_0^p holds;
  * the complex-step tangent equals central differences of the stress;
  * a homogeneous cell under hydrostatic strain: the staggered scheme's curve
    equals the Backward-Euler solution of the scalar equations of that case
    (yield on the pressure axis, work balance, porosity update with the
    non-local variables equal to the local ones, pressure from the elastic
    predictor), reduced here to nested scalar bisections.
"""
import math

import numpy as np
import pytest


import rve_inputs as I
from oracle import rve_oracle as O

GTN = dict(E=70000.0, nu=0.33, sigma_y=100.0, H=500.0, law=3, eps_C=0.0, eps_R=1.0, D_max=0.0, var=0,
           hard=0, N=0.1, q1=1.5, q2=1.0, q3=2.25, f_C=0.15, f_F=0.25, f_N=0.04, eps_N=0.1, s_N=0.05,
           f0=0.0, fstar_max=0.6)


def _phase(**kw):
    return O.phases_from_dicts([dict(GTN, **kw)])[0]


def test_fV_and_cap_match_section_4():
    ph = _phase()
    assert O.gtn_fV(ph) == pytest.approx(2.0 / 3.0, rel=1e-15)
    assert 0.9 * O.gtn_fV(ph) == pytest.approx(ph.fstar_max, rel=1e-15)
    f = np.array([0.0, 0.1, 0.15, 0.2, 0.25, 0.4])
    fs = O.gtn_fstar(f, ph)
    slope = (2.0 / 3.0 - 0.15) / (0.25 - 0.15)
    np.testing.assert_allclose(fs, [0.0, 0.1, 0.15, 0.15 + slope * 0.05, 0.6, 0.6], rtol=1e-14)


def _random_strains(V, seed, amp=4e-3):
    rng = np.random.default_rng(seed)
    eps = rng.uniform(0.2, 1.5, (V, 1)) * amp * rng.standard_normal((V, 6))
    eps[:, :3] += rng.uniform(-1.0, 3.0, (V, 1)) * amp            # pressures of both signs
    epsp_n = 2e-4 * rng.standard_normal((V, 6))
    ep_n = np.abs(5e-3 * rng.standard_normal(V))
    return eps, epsp_n, ep_n


@pytest.mark.parametrize("hard", [0, 1])
def test_zero_porosity_is_j2_radial_return(hard):
    V = 200
    eps, epsp_n, ep_n = _random_strains(V, 1)
    epsp_n[:, :3] -= epsp_n[:, :3].mean(axis=1, keepdims=True)   # J2 flow is deviatoric
    g = dict(GTN, f_N=0.0, f0=0.0, hard=hard)
    j2 = dict(I.MATRIX, hard=hard, N=0.1, eps_C=10.0, eps_R=11.0, var=0)
    phm = np.zeros(V, dtype=int)
    z2 = np.zeros((2, V))
    a = O.return_map(eps, epsp_n, ep_n, z2, phm, O.phases_from_dicts([g]), f_n=np.zeros(V))
    b = O.return_map(eps, epsp_n, ep_n, z2[:1], phm, O.phases_from_dicts([j2]))
    assert (b["ep"] > ep_n).sum() > 50
    sc = np.abs(b["sigma"]).max()
    np.testing.assert_allclose(a["sigma"], b["sigma"], rtol=0, atol=1e-10 * sc)
    np.testing.assert_allclose(a["epsp"], b["epsp"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(a["ep"], b["ep"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(a["C"], b["C"], rtol=0, atol=1e-7 * np.abs(b["C"]).max())


def _phi(sig, s0, fs, ph):
    """Eq. yield_gurson from a Mandel stress (rows)."""
    tr = sig[..., 0] + sig[..., 1] + sig[..., 2]
    dev = sig - tr[..., None] * O.IVEC / 3.0
    s = np.sqrt(1.5 * np.sum(dev * dev, axis=-1))
    p = -tr / 3.0
    return (s / s0) ** 2 + 2.0 * fs * ph.q1 * np.cosh(-1.5 * ph.q2 * p / s0) - (1.0 + ph.q3 * fs ** 2)


def _porous_case(V, seed):
    """Random GTN states with porosity driven by the non-local variables."""
    rng = np.random.default_rng(seed)
    eps, epsp_n, ep_n = _random_strains(V, seed, amp=1.2e-3)
    abar_n = np.stack([ep_n, rng.uniform(0.0, 2e-3, V)])
    abar = abar_n + np.stack([rng.uniform(0.0, 0.02, V), rng.uniform(0.0, 0.01, V)])
    f_n = rng.uniform(0.0, 0.12, V)
    return eps, epsp_n, ep_n, abar, abar_n, f_n


@pytest.mark.parametrize("hard", [0, 1])
def test_yield_normality_and_work_balance(hard):
    ph = _phase(hard=hard)
    V = 300
    eps, epsp_n, ep_n, abar, abar_n, f_n = _porous_case(V, 2)
    phm = np.zeros(V, dtype=int)
    rm = O.return_map(eps, epsp_n, ep_n, abar, phm, [ph], abar_n=abar_n, f_n=f_n)
    f = rm["f"]
    fs = rm["D"]
    # porosity of Appendix A.1, written out
    AN = ph.f_N / (ph.s_N * math.sqrt(2 * math.pi)) * np.exp(-0.5 * ((abar[0] - ph.eps_N) / ph.s_N) ** 2)
    dat = abar[1] - abar_n[1]
    np.testing.assert_allclose(f - f_n, AN * (abar[0] - abar_n[0]) + (1 - f) * dat, atol=1e-15)
    plastic = rm["ep"] > ep_n
    assert plastic.sum() > 50 and (~plastic).sum() > 20
    s0 = O.flow_stress(ph, rm["ep"])[0]
    sig = rm["sigma"]
    phi = _phi(sig, s0, fs, ph)
    assert np.abs(phi[plastic]).max() < 1e-10
    s0n = O.flow_stress(ph, ep_n)[0]
    assert _phi(sig[~plastic], s0n[~plastic], fs[~plastic], ph).max() <= 1e-12
    # normality: d eps^p parallel to d phi / d sigma (central differences)
    depsp = rm["epsp"] - epsp_n
    grad = np.zeros((V, 6))
    for c in range(6):
        h = 1e-6 * s0
        sp, sm = sig.copy(), sig.copy()
        sp[:, c] += h
        sm[:, c] -= h
        grad[:, c] = (_phi(sp, s0, fs, ph) - _phi(sm, s0, fs, ph)) / (2 * h)
    gp, dp = grad[plastic], depsp[plastic]
    cosang = np.einsum("ij,ij->i", gp, dp) / (np.linalg.norm(gp, axis=1) * np.linalg.norm(dp, axis=1))
    assert np.abs(cosang - 1.0).max() < 1e-8
    # work balance
    work = np.einsum("ij,ij->i", sig, depsp)
    np.testing.assert_allclose(work[plastic], ((1 - f) * s0 * (rm["ep"] - ep_n))[plastic],
                               rtol=1e-9, atol=1e-12 * ph.sigma_y)
    # alpha: eps_0^p and tr eps^p
    np.testing.assert_allclose(rm["alpha"][0], rm["ep"], rtol=0, atol=0)
    np.testing.assert_allclose(rm["alpha"][1], rm["epsp"][:, :3].sum(axis=1), rtol=0, atol=1e-18)


@pytest.mark.parametrize("hard", [0, 1])
def test_tangent_matches_central_differences(hard):
    ph = _phase(hard=hard)
    V = 120
    eps, epsp_n, ep_n, abar, abar_n, f_n = _porous_case(V, 4)
    phm = np.zeros(V, dtype=int)
    rm = O.return_map(eps, epsp_n, ep_n, abar, phm, [ph], abar_n=abar_n, f_n=f_n)
    assert (rm["ep"] > ep_n).sum() > 30
    for c in range(6):
        h = 1e-8
        ep_, em_ = eps.copy(), eps.copy()
        ep_[:, c] += h
        em_[:, c] -= h
        sp = O.return_map(ep_, epsp_n, ep_n, abar, phm, [ph], abar_n=abar_n, f_n=f_n)["sigma"]
        sm = O.return_map(em_, epsp_n, ep_n, abar, phm, [ph], abar_n=abar_n, f_n=f_n)["sigma"]
        fd = (sp - sm) / (2 * h)
        np.testing.assert_allclose(rm["C"][:, :, c], fd, rtol=1e-5, atol=2e-5 * np.abs(rm["C"]).max())


def _bisect(g, lo, hi, iters=200):
    """Root of a scalar g with g(lo) < 0 < g(hi) (either order of lo, hi)."""
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if g(mid) < 0.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _hydrostatic_reference(ph, e_path, f0):
    """Backward-Euler hydrostatic path of a homogeneous GTN cell under strain
    E I (s = 0, p = p_tr + K d_v).  For a volumetric plastic step d_v the
    porosity law with the non-local variables equal to the local ones,
        f' = (f + A_N(e0') d_e0 + d_v) / (1 + d_v),
    and the work balance (1 - f') sigma_0(e0') d_e0 = -p d_v leave one
    equation in d_e0, increasing from -(-p d_v) < 0 at d_e0 = 0; the yield
    condition on the pressure axis then changes sign in d_v between 0
    (trial point, outside) and -p_tr / K (zero pressure, inside).  Both are
    solved by bisection."""
    K = ph.K
    fv = (ph.q1 + math.sqrt(ph.q1 ** 2 - ph.q3)) / ph.q3
    slope = (fv - ph.f_C) / (ph.f_F - ph.f_C)

    def fstar(f):
        fs = f if f < ph.f_C else (ph.f_C + slope * (f - ph.f_C) if f < ph.f_F else fv)
        return min(max(fs, 0.0), ph.fstar_max)

    def s0_of(e0):
        return ph.sigma_y + ph.H * e0

    def A_N(e0):
        return ph.f_N / (ph.s_N * math.sqrt(2 * math.pi)) * math.exp(-0.5 * ((e0 - ph.eps_N) / ph.s_N) ** 2)

    out = []
    vp, e0, f = 0.0, 0.0, f0          # plastic volume strain, eps_0^p, porosity
    for E in e_path:
        p_tr = -K * (3.0 * E - vp)

        def inner(dv):
            p = p_tr + K * dv

            def fn_of(de0):
                return (f + A_N(e0 + de0) * de0 + dv) / (1.0 + dv)

            def work(de0):
                return (1.0 - fn_of(de0)) * s0_of(e0 + de0) * de0 + p * dv

            de0 = _bisect(work, 0.0, 1.0) if dv > 0.0 else 0.0
            return p, de0, fn_of(de0)

        def phi(dv):
            p, de0, fn = inner(dv)
            fs = fstar(fn)
            return 2.0 * fs * ph.q1 * math.cosh(1.5 * ph.q2 * p / s0_of(e0 + de0)) - (1.0 + ph.q3 * fs ** 2)

        if phi(0.0) > 0.0:
            dv = _bisect(lambda x: -phi(x), 0.0, -p_tr / K)
        else:
            dv = 0.0
        p, de0, fn = inner(dv)
        vp, e0, f = vp + dv, e0 + de0, fn
        out.append(-p)                      # Sigma_11 = -p
    return np.array(out)


def test_hydrostatic_path_through_staggered_loop():
    mat = dict(GTN, f0=0.01, f_N=0.04, eps_N=0.002, s_N=0.001)
    ph = O.phases_from_dicts([mat])[0]
    g = O.Grid((4, 4, 4))
    ctrl = np.ones(6, dtype=np.uint8)
    e_path = np.linspace(2e-4, 4e-3, 14)
    tgt = np.zeros((len(e_path), 6))
    tgt[:, :3] = e_path[:, None]
    st = O.run_load_path(g, np.zeros(g.shape, dtype=np.uint8), [mat, I.PARTICLE],
                         np.array([[2.0, 0.04], [2.0, 0.04]]), ctrl, tgt, O.PARITY_OPTIONS)
    ref = _hydrostatic_reference(ph, e_path, 0.01)
    S = np.array([r["S"][0] for r in st.curve])
    np.testing.assert_allclose(S, ref, rtol=1e-9)
    assert S.max() > 0 and S[-1] < S.max()          # the porous matrix softens
    assert st.f.max() > 0.02                        # nucleation and growth happened
    for r in st.curve:
        np.testing.assert_allclose(r["S"][:3], r["S"][0], rtol=1e-12)
        assert np.abs(r["S"][3:]).max() < 1e-9 * abs(r["S"][0])
