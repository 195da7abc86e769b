"""Pins of the oracle's discrete derivative (rotated scheme, Section 3.2.1)
and Galerkin projection (Eq. eqdiscrete2) against real-space stencils,
closed forms and a dense least-squares projection."""
import math

import numpy as np
import pytest

from oracle import rve_oracle as O
from tests import _stencil as S

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

GRIDS = [(6, 5), (8, 8), (4, 3, 5), (4, 4, 6), (6, 2, 3)]


def _rng(seed):
    return np.random.default_rng(seed)


@pytest.mark.parametrize("n", GRIDS)
def test_symbol_is_corner_stencil(n):
    """F^-1(k_j F u) equals the real-space corner-difference stencil (R5)."""
    rng = _rng(1)
    L = tuple(rng.uniform(0.5, 2.0) * x for x in n)
    g = O.Grid(n, L)
    u = rng.standard_normal(g.shape)
    ks = O.willot_k(g)
    ref = S.corner_grad(u, g.h)
    for j in range(g.d):
        out = O.ifft_fields(ks[j] * O.fft_fields(u, g), g)
        assert np.abs(out.imag).max() < 1e-12 * np.abs(ref[j]).max()
        np.testing.assert_allclose(out.real, ref[j], rtol=0, atol=1e-12 * np.abs(ref[j]).max())


@pytest.mark.parametrize("N", [64, 128, 256])
def test_symbol_small_angle_limit(N):
    """k_j -> i xi_j exp(i sum theta/2) (the derivative at the voxel corner,
    a half-voxel shift) with error O(theta^2) for the lowest modes."""
    g = O.Grid((N, N, N), (1.0, 1.0, 1.0))
    ks = O.willot_k(g)
    a = O.willot_a(g)
    theta = 2 * math.pi / N
    xi = 2 * math.pi * 1.0
    shift = np.exp(1j * theta)             # mode q = (1, 1, 0): sum theta/2 = theta
    for j in range(2):
        kv = ks[j][0, 1, 1]
        rel = abs(kv - 1j * xi * shift) / xi
        assert rel < 0.5 * theta ** 2 + 1e-12
        assert rel > 0.05 * theta ** 2          # genuinely second order
        assert abs(a[j][0, 1, 1] - xi) / xi < 0.5 * theta ** 2


def test_hidden_zeros():
    """Modes with two Nyquist indices have k = 0 (and only those, besides
    xi = 0)."""
    g = O.Grid((8, 8, 6))
    a = O.willot_a(g)
    a2 = sum(x * x for x in a)
    nyq = [g.bcast(2 * np.abs(g.signed_index(j)) == g.n[j], j) for j in range(3)]
    count = sum(np.broadcast_to(m, g.shape).astype(int) for m in nyq)
    zero = O.zero_mode_mask(g)
    assert np.all(a2[count >= 2] == 0.0)
    assert np.all(a2[(count < 2) & ~zero] > 0.0)


@pytest.mark.parametrize("n", GRIDS)
def test_gamma_projector_properties(n):
    """G* is idempotent and self-adjoint; compatible fields and stress-mask
    means pass unchanged; the complement is divergence free (stencil)."""
    rng = _rng(2)
    g = O.Grid(n)
    nc = 6 if g.d == 3 else 3
    mask = (rng.random(nc) < 0.5).astype(float)
    a = rng.standard_normal(g.shape + (nc,))
    b = rng.standard_normal(g.shape + (nc,))
    Ga = O.G_apply(a, g, mask)
    Gb = O.G_apply(b, g, mask)
    np.testing.assert_allclose(O.G_apply(Ga, g, mask), Ga, atol=1e-12)
    assert abs(np.sum(Ga * b) - np.sum(a * Gb)) < 1e-10 * np.sqrt(np.sum(a * a) * np.sum(b * b))
    # compatible field + admissible mean
    u = [rng.standard_normal(g.shape) for _ in range(g.d)]
    eps = S.sym_grad_mandel(u, g.h) + mask * rng.standard_normal(nc)
    np.testing.assert_allclose(O.G_apply(eps, g, mask), eps, atol=1e-11 * np.abs(eps).max())
    # complement: divergence free, zero stress-controlled mean
    comp = a - Ga
    for dv in S.div_mandel(comp, g.h):
        assert np.abs(dv).max() < 1e-11 * np.abs(a).max()
    assert np.abs(mask * comp.reshape(-1, nc).mean(axis=0)).max() < 1e-13


@pytest.mark.parametrize("n", [(4, 3), (4, 2, 3), (2, 3, 2)])
def test_gamma_is_least_squares_projection(n):
    """Dense brute force: G*(tau) = B B^+ tau with B spanning the admissible
    strains built from the real-space stencil (no FFT)."""
    rng = _rng(3)
    g = O.Grid(n, tuple(rng.uniform(0.7, 1.3) * x for x in n))
    nc = 6 if g.d == 3 else 3
    mask = np.zeros(nc)
    mask[1] = 1.0
    mask[-1] = 1.0
    B = S.compatible_basis(g.shape, g.h, mask)
    tau = rng.standard_normal(g.shape + (nc,))
    coef, *_ = np.linalg.lstsq(B, tau.reshape(-1), rcond=1e-10)
    ref = (B @ coef).reshape(tau.shape)
    np.testing.assert_allclose(O.G_apply(tau, g, mask), ref, atol=1e-10)
