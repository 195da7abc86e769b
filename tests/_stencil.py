"""Real-space finite-difference stencils and dense operators used to pin the
oracle.  Written from the definitions of the rotated scheme (derivative at
the voxel corner n + 1/2 as the mean of the forward differences along the
2^(d-1) cube edges parallel to the axis) and of compatibility/equilibrium;
nothing here uses an FFT, so it is independent of the oracle's spectral
operators.

Arrays use numpy shape (N3, N2, N1) / (N2, N1): physical axis j is numpy
axis d-1-j.
"""
import itertools
import math

import numpy as np

SQ2 = math.sqrt(2.0)
PAIRS = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def carried_pairs(d):
    return PAIRS if d == 3 else [PAIRS[0], PAIRS[1], PAIRS[5]]


def shift(u, d, e):
    """u(n + e) for an integer offset e given per physical axis."""
    out = u
    for j, ej in enumerate(e):
        if ej:
            out = np.roll(out, -ej, axis=d - 1 - j)
    return out


def corner_grad(u, h):
    """Rotated-scheme derivative of a periodic voxel field u, one array per
    physical axis, located at the voxel corner n + 1/2."""
    d = u.ndim
    res = []
    for j in range(d):
        acc = np.zeros_like(u)
        for e in itertools.product([0, 1], repeat=d):
            if e[j]:
                continue
            ep = list(e)
            ep[j] = 1
            acc = acc + shift(u, d, ep) - shift(u, d, e)
        res.append(acc / (h[j] * 2 ** (d - 1)))
    return res


def corner_grad_T(g, h, j):
    """Transpose (adjoint) of the j-th corner derivative."""
    d = g.ndim
    acc = np.zeros_like(g)
    for e in itertools.product([0, 1], repeat=d):
        if e[j]:
            continue
        ep = [-x for x in e]
        ep_j = list(ep)
        ep_j[j] = -1
        acc = acc + shift(g, d, ep_j) - shift(g, d, ep)
    return acc / (h[j] * 2 ** (d - 1))


def dense_grad(shape, h):
    """Dense matrices D_j (V x V) of the corner derivative."""
    d = len(shape)
    V = int(np.prod(shape))
    mats = [np.zeros((V, V)) for _ in range(d)]
    for col in range(V):
        e = np.zeros(V)
        e[col] = 1.0
        g = corner_grad(e.reshape(shape), h)
        for j in range(d):
            mats[j][:, col] = g[j].ravel()
    return mats


def sym_grad_mandel(u_list, h):
    """Compatible strain (carried Mandel comps, last axis) from a displacement
    given as a list of d scalar fields."""
    d = len(u_list)
    G = [corner_grad(u, h) for u in u_list]          # G[i][j] = D_j u_i
    comps = []
    for (i, j) in carried_pairs(d):
        if i == j:
            comps.append(G[i][i])
        else:
            comps.append(SQ2 * 0.5 * (G[i][j] + G[j][i]))
    return np.stack(comps, axis=-1)


def div_mandel(sig, h):
    """Discrete divergence (adjoint of the symmetric corner gradient) of a
    carried-Mandel field: returns d scalar fields; zero iff sig is
    orthogonal to every compatible fluctuation."""
    d = sig.ndim - 1
    pairs = carried_pairs(d)
    out = [np.zeros(sig.shape[:-1]) for _ in range(d)]
    for m, (i, j) in enumerate(pairs):
        if i == j:
            out[i] += corner_grad_T(sig[..., m], h, i)
        else:
            s = sig[..., m] / SQ2
            out[i] += corner_grad_T(s, h, j)
            out[j] += corner_grad_T(s, h, i)
    return out


def compatible_basis(shape, h, stress_mask):
    """Dense matrix whose columns span the admissible strain corrections of
    the mixed-control Galerkin problem: symmetric corner gradients of every
    displacement basis vector, plus uniform fields on the stress-controlled
    components."""
    d = len(shape)
    V = int(np.prod(shape))
    pairs = carried_pairs(d)
    nc = len(pairs)
    Dm = dense_grad(shape, h)
    cols = []
    for i in range(d):
        # displacement component i, all voxels
        blocks = []
        for (a, b) in pairs:
            if a == b:
                blocks.append(Dm[a] if a == i else np.zeros((V, V)))
            else:
                m = np.zeros((V, V))
                if a == i:
                    m = m + SQ2 * 0.5 * Dm[b]
                if b == i:
                    m = m + SQ2 * 0.5 * Dm[a]
                blocks.append(m)
        # (V*nc, V) with component fastest
        B = np.stack(blocks, axis=1).reshape(V * nc, V)
        cols.append(B)
    for c in range(nc):
        if stress_mask[c]:
            col = np.zeros((V, nc))
            col[:, c] = 1.0
            cols.append(col.reshape(V * nc, 1))
    return np.concatenate(cols, axis=1)


def dense_helmholtz(shape, h, ell2):
    """Dense L = I + sum_j D_j^T diag(l^2) D_j (l^2 at the voxel index of the
    corner gradient)."""
    V = int(np.prod(shape))
    Dm = dense_grad(shape, h)
    L = np.eye(V)
    w = ell2.ravel()
    for Dj in Dm:
        L = L + Dj.T @ (w[:, None] * Dj)
    return L
