"""Pins of the oracle's heterogeneous Helmholtz solver (Algorithm 2,
Eqs. LhelmFourier and preconditioner)."""
import math

import numpy as np
import pytest

from oracle import rve_oracle as O
from tests import _stencil as S


@pytest.mark.parametrize("n", [(6, 5), (4, 3, 4), (8, 6)])
def test_pcg_matches_dense_stencil_solve(n):
    """Dense brute force: (I + sum_j D_j^T l^2 D_j) abar = alpha with the
    real-space corner stencil and l^2 at the gradient's voxel index."""
    rng = np.random.default_rng(11)
    g = O.Grid(n, tuple(rng.uniform(0.8, 1.2) * x for x in n))
    ph = (rng.random(g.shape) < 0.4).astype(int)
    ell2 = np.where(ph == 0, 1.5, 0.03) ** 2
    alpha = rng.random(g.shape) * (ph == 0)
    abar, it = O.helmholtz_solve(alpha, ell2, g, 1e-14, 500)
    L = S.dense_helmholtz(g.shape, g.h, ell2)
    ref = np.linalg.solve(L, alpha.ravel()).reshape(g.shape)
    np.testing.assert_allclose(abar, ref, atol=1e-12 * np.abs(ref).max())


def _plane_wave_eigenvalue(g, m):
    """Eigenvalue of sum_j D_j^T D_j on exp(i theta.n), from the stencil."""
    idx = np.meshgrid(*[np.arange(N) for N in reversed(g.n)], indexing="ij")
    ph = sum(2 * math.pi * m[j] * idx[g.d - 1 - j] / g.n[j] for j in range(g.d))
    u = np.exp(1j * ph)
    acc = np.zeros_like(u)
    for j, gj in enumerate(S.corner_grad(u, g.h)):
        acc = acc + S.corner_grad_T(gj, g.h, j)
    return (acc / u).real.mean()


@pytest.mark.parametrize("m", [(1, 0, 0), (2, 3, 1), (4, 0, 5)])
def test_constant_ell_sinusoid_exact_in_one_iteration(m):
    """Uniform l, alpha = cos(2 pi m.x / L): abar = alpha / (1 + l^2 lambda_m)
    exactly, and PCG stops after one iteration (M is the exact inverse)."""
    g = O.Grid((16, 12, 10))
    idx = np.meshgrid(*[np.arange(N) for N in reversed(g.n)], indexing="ij")
    alpha = np.cos(sum(2 * math.pi * m[j] * idx[g.d - 1 - j] / g.n[j] for j in range(3)))
    ell2 = np.full(g.shape, 2.3 ** 2)
    abar, it = O.helmholtz_solve(alpha, ell2, g, 1e-13, 50)
    lam = _plane_wave_eigenvalue(g, m)
    np.testing.assert_allclose(abar, alpha / (1 + 2.3 ** 2 * lam), atol=1e-14)
    assert it == 1


def test_invariants_uniform_source_mean_and_local_limit():
    """Uniform alpha -> abar = alpha for any l(x); <abar> = <alpha>;
    l -> 0 recovers the local field."""
    rng = np.random.default_rng(3)
    g = O.Grid((12, 10, 6))
    ell2 = rng.uniform(0.01, 4.0, g.shape)
    one, _ = O.helmholtz_solve(np.full(g.shape, 0.7), ell2, g, 1e-13, 500)
    np.testing.assert_allclose(one, 0.7, atol=1e-13)
    alpha = rng.random(g.shape)
    abar, _ = O.helmholtz_solve(alpha, ell2, g, 1e-13, 500)
    assert abs(abar.mean() - alpha.mean()) < 1e-13
    loc, _ = O.helmholtz_solve(alpha, np.full(g.shape, 1e-8), g, 1e-13, 500)
    np.testing.assert_allclose(loc, alpha, atol=1e-7)


def _two_phase_1d(x, w1, l1, l2, L):
    """Exact periodic solution of abar - (l^2 abar')' = alpha on [0, L) with
    alpha = 1, l = l1 on |x - L/2| < w1 and alpha = 0, l = l2 elsewhere;
    continuity of abar and of the flux l^2 abar' at the interfaces.  Region 2
    is written as B cosh(t/l2)/cosh(w2/l2) to stay finite for small l2."""
    w2 = L / 2 - w1
    A = np.array([[math.cosh(w1 / l1), -1.0],
                  [l1 * math.sinh(w1 / l1), l2 * math.tanh(w2 / l2)]])
    a, b = np.linalg.solve(A, [-1.0, 0.0])
    s = x - L / 2
    t = np.abs(np.where(s > 0, s - L / 2, s + L / 2))
    ratio2 = np.exp((t - w2) / l2) * (1 + np.exp(-2 * t / l2)) / (1 + math.exp(-2 * w2 / l2))
    return np.where(np.abs(s) < w1, 1 + a * np.cosh(s / l1), b * ratio2)


@pytest.mark.parametrize("ratio", [4.0, 1000.0])
def test_two_phase_laminate_flux_law(ratio):
    """1D two-phase laminate: the discrete solution converges (first order)
    to the exact piecewise-cosh solution with flux continuity
    l1^2 abar'_1 = l2^2 abar'_2 (the interface law of Section 2.2.1); for
    l2 << l1 the field vanishes in phase 2 (Neumann limit).  With l^2 taken at
    the gradient's voxel index the discrete interface sits up to one voxel
    off, so the error is measured away from the interfaces; at moderate
    contrast the maximum error halves with h as well."""
    L, w1, l1 = 1.0, 0.25, 0.08
    l2 = l1 / ratio
    errs, far_errs = [], []
    for N in (128, 256, 512):
        g = O.Grid((N, 2), (L, 2 * L / N))
        x = (np.arange(N) + 0.5) * L / N
        inside = np.abs(x - L / 2) < w1
        ell2 = np.broadcast_to(np.where(inside, l1, l2) ** 2, g.shape).copy()
        alpha = np.broadcast_to(inside.astype(float), g.shape).copy()
        abar, _ = O.helmholtz_solve(alpha, ell2, g, 1e-13, 5000)
        ex = _two_phase_1d(x, w1, l1, l2, L)
        err = np.abs(abar[0] - ex)
        errs.append(err.max())
        far_errs.append(err[np.abs(np.abs(x - L / 2) - w1) > 0.05].max())
        if ratio > 100:
            beyond = np.abs(x - L / 2) > w1 + 2.5 * L / N
            assert np.abs(abar[0][beyond]).max() < 1e-6
    assert far_errs[-1] < 1.5e-2
    assert far_errs[1] < 0.6 * far_errs[0] and far_errs[2] < 0.6 * far_errs[1]
    if ratio < 10:
        assert errs[-1] < 4e-2
        assert errs[1] < 0.6 * errs[0] and errs[2] < 0.6 * errs[1]
