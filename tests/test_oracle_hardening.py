"""Pins of the oracle's Aravas flow stress (Section 4.1, Eq. aravas) and of
the Lemaitre return map with it.

The law sigma_0 / sigma_y = (sigma_0 / sigma_y + 3 mu e0 / sigma_y)^N is
implicit in sigma_0, but its inverse is explicit: for y = sigma_0 / sigma_y,
e0 = sigma_y (y^(1/N) - y) / (3 mu).  The pins pick y, form e0 from that
inverse, and ask the oracle for y back; for N = 1/2 the law is a quadratic
with the closed-form root y = (1 + sqrt(1 + 4c)) / 2.  Under homogeneous
uniaxial stress the J2 solution obeys E11 = sigma_0(e_p) / E + e_p, so a
load path built from chosen y values has the closed-form curve
Sigma11 = (1 - D(e_p)) sigma_y y.
"""
import math

import numpy as np
import pytest

import rve_inputs as I
from oracle import rve_oracle as O

ARAVAS = dict(I.MATRIX, hard=1, N=0.1)


def _inverse(ph, y):
    """e0 with sigma_0(e0) = sigma_y y (the explicit inverse of the law)."""
    return ph.sigma_y * (y ** (1.0 / ph.N) - y) / (3.0 * ph.mu)


@pytest.mark.parametrize("N", [0.1, 0.2, 0.5])
def test_flow_stress_inverts_the_explicit_inverse(N):
    ph = O.phases_from_dicts([dict(ARAVAS, N=N)])[0]
    y = np.array([1.0, 1.001, 1.05, 1.2, 1.5, 2.0])
    e0 = _inverse(ph, y)
    s, _ = O.flow_stress(ph, e0)
    np.testing.assert_allclose(s, ph.sigma_y * y, rtol=1e-14)


def test_flow_stress_half_power_closed_form_and_slope():
    ph = O.phases_from_dicts([dict(ARAVAS, N=0.5)])[0]
    e0 = np.array([0.0, 1e-4, 1e-3, 1e-2, 0.2])
    c = 3.0 * ph.mu * e0 / ph.sigma_y
    s, H = O.flow_stress(ph, e0)
    np.testing.assert_allclose(s, ph.sigma_y * (1.0 + np.sqrt(1.0 + 4.0 * c)) / 2.0, rtol=1e-14)
    # d sigma_0 / d e0 of the closed form: sigma_y * (3 mu / sigma_y) / sqrt(1 + 4c)
    np.testing.assert_allclose(H, 3.0 * ph.mu / np.sqrt(1.0 + 4.0 * c), rtol=1e-12)


def test_flow_stress_slope_matches_central_differences():
    ph = O.phases_from_dicts([ARAVAS])[0]
    e0 = np.array([1e-4, 1e-3, 1e-2, 0.1])
    h = 1e-7 * e0
    _, H = O.flow_stress(ph, e0)
    fd = (O.flow_stress(ph, e0 + h)[0] - O.flow_stress(ph, e0 - h)[0]) / (2 * h)
    np.testing.assert_allclose(H, fd, rtol=1e-6)


def test_linear_law_is_unchanged():
    ph = O.phases_from_dicts([I.MATRIX])[0]
    e0 = np.array([0.0, 0.01, 0.3])
    s, H = O.flow_stress(ph, e0)
    np.testing.assert_allclose(s, ph.sigma_y + ph.H * e0, rtol=0, atol=0)
    assert np.all(H == ph.H)


def _yield(sig_eff, ep, ph):
    t = O.mandel_to_tensor(sig_eff)
    dev = t - np.trace(t, axis1=-2, axis2=-1)[..., None, None] * np.eye(3) / 3
    return np.sqrt(np.sum(dev * dev, axis=(-2, -1))) - math.sqrt(2 / 3) * O.flow_stress(ph, ep)[0]


def test_aravas_return_map_consistency_and_tangent():
    """Plastic points land on the yield surface of the current flow stress;
    the tangent equals central differences of the stress (D frozen)."""
    ph = O.phases_from_dicts([ARAVAS])[0]
    rng = np.random.default_rng(3)
    V = 300
    eps = rng.uniform(0.05, 1.5, (V, 1)) * 2e-3 * rng.standard_normal((V, 6))
    epsp_n = 1e-4 * rng.standard_normal((V, 6))
    epsp_n[:, :3] -= epsp_n[:, :3].mean(axis=1, keepdims=True)
    ep_n = np.abs(2e-3 * rng.standard_normal(V))
    abar = np.full((1, V), 0.06)
    phm = np.zeros(V, dtype=int)
    rm = O.return_map(eps, epsp_n, ep_n, abar, phm, [ph])
    plastic = rm["ep"] > ep_n
    assert plastic.sum() > 50 and (~plastic).sum() > 50
    sig_eff = rm["sigma"] / (1.0 - rm["D"][:, None])
    f = _yield(sig_eff, rm["ep"], ph)
    assert np.abs(f[plastic]).max() < 1e-9 * ph.sigma_y
    assert f[~plastic].max() <= 0
    h = 1e-8
    for c in range(6):
        ep_, em_ = eps.copy(), eps.copy()
        ep_[:, c] += h
        em_[:, c] -= h
        fd = (O.return_map(ep_, epsp_n, ep_n, abar, phm, [ph])["sigma"]
              - O.return_map(em_, epsp_n, ep_n, abar, phm, [ph])["sigma"]) / (2 * h)
        np.testing.assert_allclose(rm["C"][:, :, c], fd, rtol=2e-5, atol=2e-3)


def test_aravas_uniaxial_closed_form_through_staggered_loop():
    """Homogeneous damaging RVE in uniaxial stress with the Aravas flow
    stress: targets E11 = sigma_y y / E + e_p(y) from chosen y give
    Sigma11 = (1 - D(e_p)) sigma_y y along the curve (abar = alpha for a
    uniform field), through the full staggered scheme."""
    mat = dict(ARAVAS, eps_C=0.002, eps_R=0.05)
    ph = O.phases_from_dicts([mat])[0]
    y = np.array([0.5, 0.9, 1.0005, 1.01, 1.03, 1.06, 1.1, 1.15, 1.2, 1.25])
    ep = np.where(y >= 1.0, _inverse(ph, np.maximum(y, 1.0)), 0.0)
    E11 = ph.sigma_y * y / ph.E + ep
    g = O.Grid((4, 4, 4))
    ctrl = np.array([1, 0, 0, 0, 0, 0], dtype=np.uint8)
    tgt = np.zeros((len(y), 6))
    tgt[:, 0] = E11
    st = O.run_load_path(g, np.zeros(g.shape, dtype=np.uint8), [mat, I.PARTICLE], np.array([[2.0, 0.04]]),
                         ctrl, tgt, O.PARITY_OPTIONS)
    for rec, yy, e in zip(st.curve, y, ep):
        D = min(max((e - ph.eps_C) / (ph.eps_R - ph.eps_C), 0.0), ph.D_max)
        assert rec["S"][0] == pytest.approx((1.0 - D) * ph.sigma_y * yy, rel=1e-10)
        assert np.abs(rec["S"][1:]).max() < 1e-9 * ph.sigma_y
    assert st.curve[-1]["D_max"] > 0.05
