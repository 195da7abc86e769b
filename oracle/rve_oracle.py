"""Plain FP64 CPU oracle of the staggered FFT scheme for gradient-regularised
ductile damage (Magri, Lucarini, Lemoine, Adam, Segurado, "An FFT framework
for simulating non-local ductile failure in heterogeneous materials").

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import this module.  It shares no code with
the CUDA path: it uses numpy's full complex FFT as a library step and applies
every operator by its definition, vectorised over voxels or Fourier modes,
with no blocking or fusion.

Field layout: numpy shape ``(N2, N1, c)`` in 2D or ``(N3, N2, N1, c)`` in 3D
(x1 fastest), strain/stress components in Mandel notation (order 11, 22, 33,
23, 13, 12, shears times sqrt 2), so that double contractions are plain dot
products.  In 2D (plane strain) the mechanical fields carry the in-plane
components 11, 22, 12 only; the local state is kept in full 3D with
eps33 = eps13 = eps23 = 0.

Readings where the paper is silent or ambiguous (each is a numbered reading
R1..R26 of the design notes):
  R1  Algorithm 1 loops while ERR > TOL.
  R2  ERR uses Mandel components and the Frobenius norm of <eps>; the
      non-local term counts 0 when ||abar|| < 1e-30; at least 2 staggered
      iterations run.
  R4  Newton stops when the residual ||G*(sigma - Sigma_bar)||_2 /
      (sqrt(V) ||<sigma>||) and the last correction max|d eps| / ||<eps>||
      are both below TOL_N.
  R5  Willot rotated-scheme discrete derivative (voxel-corner differences).
  R6  Small-strain Galerkin projection = orthogonal projection onto
      compatible symmetric strains.
  R7  Zero-frequency projector = diagonal projector on the stress-controlled
      components.
  R8  sqrt(2/3) in both the yield function and the eps_p rate.
  R9  Total-form stress update sigma = (1 - D) sigma_eff.
  R10 D = D(abar) without irreversibility, capped at D_max.
  R11 D frozen during the mechanical Newton loop.
  R12 <l^2> = voxel average of l_j^2(x).
  R14 Initial guess eps_n + dE on strain-controlled components, abar_n.
  R15 Helmholtz operator a + conj(k).F(l^2 F^-1(k a)), l^2 taken at the
      voxel index of the corner gradient.
  R24 No clamp on abar.
  R25 CG and PCG stop when (p, A p) <= 0: the operators are symmetric
      positive definite in exact arithmetic, so this only happens once the
      residual has reached the round-off floor; the current iterate is kept.
  R26 The mechanical CG of a Newton step also stops once ||r|| <=
      0.01 TOL_N sqrt(V) ||<sigma>||: the linear solve is not pushed below the
      accuracy the Newton test (R4) can use, where the right-hand side is
      dominated by the round-off of -G*(sigma - Sigma_bar).
  R27 Increment cut-back (Section 4 applies a variable strain increment,
      reduced where the solution needs it, down to a minimum admissible
      size, without printing the rule): the remaining path of an increment
      is tried whole; a solve that runs out of its Newton or staggered
      budget halves the sub-step, a converged one doubles it again (capped
      by what is left), targets are linear along the path, and the sub-step
      never falls below 2^-max_cuts of the path.
  R20 Particle cracking (law 2; not in the paper, an extension of Section
      3.1's multi-variable framework): the local variable is the history
      kappa = max(kappa_n, ||<eps>_+||), the Euclidean norm of the positive
      principal strains; it feeds its own non-local variable, and
      D = clamp((kappa_bar - kappa_C)/(kappa_R - kappa_C), 0, D_max) scales an
      elastic stress, sigma = (1 - D) C : eps, with tangent (1 - D) C (R11).
      kappa_C, kappa_R reuse the eps_C, eps_R slots of the phase.

Parity: every function below is pinned by the CPU tests (closed forms,
invariants, dense brute-force solves built from real-space stencils, finite
differences); none is "parity unpinned".  The staggered loop of Algorithm 1
(step_increment: ERR, stopping rule and commit) is pinned on heterogeneous
damaging cells by checking each committed increment against the monolithic
system it must solve (equilibrium at D(abar), the Helmholtz equations, the
macroscopic targets), with operators assembled from real-space stencils, by
recomputing ERR from the iterates, and by mirror symmetry of centred cells.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SQ2 = math.sqrt(2.0)
# Mandel component -> tensor index pair
MANDEL_PAIRS = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
MANDEL_W = np.array([1.0, 1.0, 1.0, SQ2, SQ2, SQ2])
IDX2D = [0, 1, 5]          # carried Mandel components in plane strain
IVEC = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])


# ============================================================ tensor helpers
def mandel_to_tensor(v):
    """(..., 6) Mandel -> (..., 3, 3) symmetric tensor."""
    t = np.zeros(v.shape[:-1] + (3, 3), dtype=v.dtype)
    for m, (i, j) in enumerate(MANDEL_PAIRS):
        val = v[..., m] / MANDEL_W[m]
        t[..., i, j] = val
        t[..., j, i] = val
    return t


def tensor_to_mandel(t):
    """(..., 3, 3) -> (..., 6) Mandel (symmetric part)."""
    out = np.empty(t.shape[:-2] + (6,), dtype=t.dtype)
    for m, (i, j) in enumerate(MANDEL_PAIRS):
        out[..., m] = 0.5 * (t[..., i, j] + t[..., j, i]) * MANDEL_W[m]
    return out


def carried(d):
    """Mandel components carried by the mechanical fields (d = 2 or 3)."""
    return list(range(6)) if d == 3 else IDX2D


def embed(vc, d):
    """Carried components (..., nc) -> full Mandel (..., 6)."""
    if d == 3:
        return vc
    out = np.zeros(vc.shape[:-1] + (6,), dtype=vc.dtype)
    out[..., IDX2D] = vc
    return out


# ============================================================ grid (Sec 3.2.1)
class Grid:
    """Regular N1 x N2 (x N3) voxel grid of a periodic cell L1 x L2 (x L3)
    (Section 3.2.1).  ``n`` and ``L`` are in physical axis order."""

    def __init__(self, n, L=None):
        self.n = tuple(int(x) for x in n)
        self.d = len(self.n)
        self.L = tuple(float(x) for x in (L if L is not None else self.n))
        self.h = [self.L[j] / self.n[j] for j in range(self.d)]
        self.shape = tuple(reversed(self.n))       # numpy shape, x1 last
        self.V = int(np.prod(self.n))

    def axis(self, j):
        """numpy axis index of physical axis j."""
        return self.d - 1 - j

    def signed_index(self, j):
        """Signed frequency index q of each FFT mode along axis j: the set
        n - N/2 (even N) or n - (N-1)/2 (odd N), n in [0, N-1], of Eq.
        (frequencies), in numpy's FFT storage order."""
        N = self.n[j]
        return np.rint(np.fft.fftfreq(N) * N).astype(np.int64)

    def xi(self, j):
        """Continuous frequency xi_j = 2 pi q / L_j (Eq. frequencies)."""
        return 2.0 * np.pi * self.signed_index(j) / self.L[j]

    def bcast(self, v, j):
        s = [1] * self.d
        s[self.axis(j)] = -1
        return v.reshape(s)


# ========================================= discrete derivative (R5, Sec 3.2.1)
def half_angle(grid, j):
    """sin and cos of theta_j / 2, theta_j = 2 pi q / N_j, with the cosine
    set to exactly zero at the Nyquist index of an even axis."""
    N = grid.n[j]
    q = grid.signed_index(j)
    s = np.sin(np.pi * q / N)
    c = np.cos(np.pi * q / N)
    c[2 * np.abs(q) == N] = 0.0
    return s, c


def willot_k(grid):
    """Modified frequencies of the rotated finite-difference scheme (R5):

        k_j = (2 i / h_j) sin(theta_j/2) prod_{m != j} cos(theta_m/2)
              * prod_m exp(i theta_m / 2)

    i.e. the Fourier symbol of the derivative along x_j evaluated at the
    voxel corner n + 1/2 as the mean of the 2^(d-1) forward differences along
    the cube edges parallel to x_j.  Returns a list of d complex arrays of
    the grid shape."""
    d = grid.d
    S = [grid.bcast(half_angle(grid, j)[0], j) for j in range(d)]
    C = [grid.bcast(half_angle(grid, j)[1], j) for j in range(d)]
    phase = np.ones(grid.shape, dtype=np.complex128)
    for m in range(d):
        phase = phase * (C[m] + 1j * S[m])
    ks = []
    for j in range(d):
        mag = (2.0 / grid.h[j]) * S[j] * np.ones(grid.shape)
        for m in range(d):
            if m != j:
                mag = mag * C[m]
        ks.append(1j * mag * phase)
    return ks


def willot_a(grid):
    """Real direction vector a with k = i exp(i phi) a (same R5 symbol
    without its common phase); Gamma depends on k only through a."""
    d = grid.d
    S = [grid.bcast(half_angle(grid, j)[0], j) for j in range(d)]
    C = [grid.bcast(half_angle(grid, j)[1], j) for j in range(d)]
    out = []
    for j in range(d):
        mag = (2.0 / grid.h[j]) * S[j] * np.ones(grid.shape)
        for m in range(d):
            if m != j:
                mag = mag * C[m]
        out.append(mag)
    return out


def zero_mode_mask(grid):
    """True at xi = 0."""
    m = np.ones(grid.shape, dtype=bool)
    for j in range(grid.d):
        m &= grid.bcast(grid.signed_index(j) == 0, j)
    return m


# =========================== Galerkin projection (R6, R7, Eq. eqdiscrete2)
def gamma_hat_apply(tau_hat, grid, stress_mask):
    """Apply the modified projection symbol G*(xi) to complex Mandel fields
    tau_hat of shape grid.shape + (nc,).

    xi != 0 with a != 0: orthogonal projection onto compatible strains
        G(T) = n (x) (T n) + (T n) (x) n - (n.T.n) n (x) n,  n = a / |a|
    (R6); hidden zeros (a = 0, xi != 0): 0; xi = 0: diagonal projector on the
    stress-controlled components (R7).  ``stress_mask`` is a length-nc 0/1
    vector over the carried components."""
    d = grid.d
    comps = carried(d)
    a = willot_a(grid)
    a2 = sum(x * x for x in a)
    nz = a2 > 0.0
    inv = np.where(nz, 1.0 / np.sqrt(np.where(nz, a2, 1.0)), 0.0)
    nvec = np.zeros(grid.shape + (3,))
    for j in range(d):
        nvec[..., j] = a[j] * inv
    T = mandel_to_tensor(embed(tau_hat, d))
    Tn = np.einsum("...ij,...j->...i", T, nvec)
    nTn = np.einsum("...i,...i->...", nvec, Tn)
    G = (np.einsum("...i,...j->...ij", nvec, Tn)
         + np.einsum("...i,...j->...ij", Tn, nvec)
         - nTn[..., None, None] * np.einsum("...i,...j->...ij", nvec, nvec))
    out = tensor_to_mandel(G)[..., comps]
    out[~nz] = 0.0
    z = zero_mode_mask(grid)
    out[z] = tau_hat[z] * np.asarray(stress_mask, dtype=np.float64)
    return out


# Threads of the FFT library step: None uses numpy's FFT (one thread); an
# integer uses scipy.fft with that many worker threads.  Both are the same
# discrete Fourier transform; only the library call differs.
_FFT_WORKERS = None


def set_fft_workers(n):
    """Run the oracle's FFTs on ``n`` threads (scipy.fft), or on numpy's
    single-threaded FFT when ``n`` is None.  Returns the previous value."""
    global _FFT_WORKERS
    old = _FFT_WORKERS
    if n is not None:
        import scipy.fft  # noqa: F401  (fail here, not inside a solve)
    _FFT_WORKERS = None if n is None else int(n)
    return old


def fft_fields(f, grid):
    axes = tuple(range(grid.d))
    if _FFT_WORKERS is None:
        return np.fft.fftn(f, axes=axes)
    import scipy.fft
    return scipy.fft.fftn(f, axes=axes, workers=_FFT_WORKERS)


def ifft_fields(fh, grid):
    axes = tuple(range(grid.d))
    if _FFT_WORKERS is None:
        return np.fft.ifftn(fh, axes=axes)
    import scipy.fft
    return scipy.fft.ifftn(fh, axes=axes, workers=_FFT_WORKERS)


def G_apply(tau, grid, stress_mask):
    """G*(tau) = F^-1 { G*(xi) : F(tau) } (Eq. eqdiscrete2) for a real
    field tau of shape grid.shape + (nc,)."""
    th = fft_fields(tau, grid)
    return ifft_fields(gamma_hat_apply(th, grid, stress_mask), grid).real


# ======================================== constitutive update (Sec 2.1.2, App A)
@dataclass
class Phase:
    E: float
    nu: float
    sigma_y: float = 0.0
    H: float = 0.0
    law: int = 0            # 0 linear elastic, 1 J2 + Lemaitre damage, 2 particle cracking (R20)
    eps_C: float = 0.0
    eps_R: float = 1.0
    D_max: float = 0.0
    var: int = -1           # non-local variable fed/read by this phase
    hard: int = 0           # flow stress: 0 linear sigma_y + H e, 1 Aravas power law (Eq. aravas)
    N: float = 0.1          # Aravas exponent
    # Gurson-Tvergaard-Needleman (law 3, Section 2.1.1; defaults of Section 4.1)
    q1: float = 1.5
    q2: float = 1.0
    q3: float = 2.25
    f_C: float = 0.15       # onset of coalescence
    f_F: float = 0.25       # porosity at fracture
    f_N: float = 0.04       # Chu-Needleman nucleation amplitude
    eps_N: float = 0.3
    s_N: float = 0.1
    f0: float = 0.0         # initial porosity
    fstar_max: float = 0.6  # cap on f* (Section 4: 0.9 f_V*)

    @property
    def K(self):
        return self.E / (3.0 * (1.0 - 2.0 * self.nu))

    @property
    def mu(self):
        return self.E / (2.0 * (1.0 + self.nu))


PHASE_KEYS = ("E", "nu", "sigma_y", "H", "law", "eps_C", "eps_R", "D_max", "var")
PHASE_OPTIONAL = ("hard", "N", "q1", "q2", "q3", "f_C", "f_F", "f_N", "eps_N", "s_N", "f0", "fstar_max")


def phases_from_dicts(ds):
    return [Phase(**{k: d[k] for k in PHASE_KEYS}, **{k: d[k] for k in PHASE_OPTIONAL if k in d})
            for d in ds]


def _bisect_increasing(g, lo, hi, iters=200):
    """Root of the increasing function g on [lo, hi] (arrays, g(lo) <= 0 <=
    g(hi)) by bisection, element-wise."""
    lo = np.array(lo, dtype=np.float64, copy=True)
    hi = np.array(hi, dtype=np.float64, copy=True)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        up = g(mid) > 0.0
        hi = np.where(up, mid, hi)
        lo = np.where(up, lo, mid)
    return 0.5 * (lo + hi)


def flow_stress(ph, e0):
    """Matrix flow stress sigma_0 and its slope d sigma_0 / d e0 at the
    equivalent plastic strain e0 (array).

    hard 0: linear hardening sigma_0 = sigma_y + H e0 (Section 4).
    hard 1: Aravas power law of Section 4.1 (Eq. aravas),
        sigma_0 / sigma_y = (sigma_0 / sigma_y + 3 mu e0 / sigma_y)^N,
    with mu the phase's shear modulus: y = sigma_0 / sigma_y solves
    g(y) = y - (y + c)^N = 0, c = 3 mu e0 / sigma_y, which is increasing in
    y (g' >= 1 - N) with g(1) <= 0 and g((1 + c)^(N/(1-N))) >= 0; the slope
    follows from differentiating the implicit law."""
    e0 = np.asarray(e0, dtype=np.float64)
    if ph.hard == 0:
        return ph.sigma_y + ph.H * e0, np.full(e0.shape, float(ph.H))
    c = 3.0 * ph.mu * e0 / ph.sigma_y
    N = ph.N
    y = _bisect_increasing(lambda y: y - (y + c) ** N, np.ones(e0.shape), (1.0 + c) ** (N / (1.0 - N)))
    w = N * (y + c) ** (N - 1.0)
    return ph.sigma_y * y, 3.0 * ph.mu * w / (1.0 - w)


def _flow_value(ph, e0):
    """sigma_0(e0) for real or complex-step arguments: a complex e0 = a + i b
    (b the complex-step perturbation) maps to sigma_0(a) + i b sigma_0'(a),
    the first-order expansion that complex-step differentiation evaluates."""
    if np.iscomplexobj(e0):
        s0, hp = flow_stress(ph, e0.real)
        return s0 + 1j * e0.imag * hp
    return flow_stress(ph, e0)[0]


def gtn_fV(ph):
    """Porosity at which the GTN surface shrinks to the origin (Section
    2.1.1): f_V* = (q1 + sqrt(q1^2 - q3)) / q3."""
    return (ph.q1 + math.sqrt(ph.q1 ** 2 - ph.q3)) / ph.q3


def gtn_fstar(f, ph):
    """Effective porosity f*(f) (Eq. effective_porosity), clamped to
    [0, fstar_max] (Section 4 caps it at 0.9 f_V*)."""
    fv = gtn_fV(ph)
    fs = np.where(f < ph.f_C, f, np.where(f < ph.f_F, ph.f_C + (fv - ph.f_C) / (ph.f_F - ph.f_C) * (f - ph.f_C), fv))
    return np.clip(fs, 0.0, ph.fstar_max)


def gtn_nucleation(e0bar, ph):
    """Chu-Needleman nucleation rate A_N (Eq. nucleation)."""
    return ph.f_N / (ph.s_N * math.sqrt(2.0 * math.pi)) * np.exp(-0.5 * ((e0bar - ph.eps_N) / ph.s_N) ** 2)


def gtn_porosity(f_n, a0, a0_n, at, at_n, ph):
    """Backward-Euler porosity of the non-local GTN model (Eq.
    non-local_porosity_gurson, Appendix A.1) with the non-local eps_0^p (a0)
    and tr eps^p (at) held at the staggered iterate:
        f - f_n = A_N(a0) (a0 - a0_n) + (1 - f) (at - at_n)."""
    dat = at - at_n
    return (f_n + gtn_nucleation(a0, ph) * (a0 - a0_n) + dat) / (1.0 + dat)


def _gtn_residual(e, epsp_n, e0_n, fs, f, ph, K, mu, x):
    """Residuals of the Backward-Euler GTN update (Appendix A.1) at x =
    (d_v, d_q, e0): plastic strain increment d eps^p = d_v I/3 + d_q n with n
    the trial flow direction (normality, Eq. flow_rule_gurson); pressure p =
    p_tr + K d_v and Mises stress s = s_tr - 3 mu d_q;
      R1 = phi(s, p, sigma_0(e0), f*)                       (Eq. yield_gurson)
      R2 = sigma_0 (d_v dphi/ds + d_q dphi/dp)   (the normality ratio)
      R3 = [(1 - f) sigma_0 (e0 - e0_n) - sigma : d eps^p] / sigma_0
           (Eq. micro-macro, sigma : d eps^p = -p d_v + s d_q).
    Complex arguments are carried through (complex-step differentiation)."""
    ee = e - epsp_n
    tr = ee[:, 0] + ee[:, 1] + ee[:, 2]
    dev = ee - tr[:, None] * IVEC[None, :] / 3.0
    p_tr = -K * tr
    s_tr = np.sqrt(1.5 * np.sum((2.0 * mu[:, None] * dev) ** 2, axis=1))
    dv, dq, e0 = x[:, 0], x[:, 1], x[:, 2]
    s = s_tr - 3.0 * mu * dq
    p = p_tr + K * dv
    s0 = _flow_value(ph, e0)
    arg = 1.5 * ph.q2 * p / s0
    phi = (s / s0) ** 2 + 2.0 * fs * ph.q1 * np.cosh(arg) - (1.0 + ph.q3 * fs ** 2)
    phi_s = 2.0 * s / s0 ** 2
    phi_p = 3.0 * ph.q1 * ph.q2 * fs / s0 * np.sinh(arg)
    r2 = s0 * (dv * phi_s + dq * phi_p)
    r3 = ((1.0 - f) * s0 * (e0 - e0_n) - (-p * dv + s * dq)) / s0
    return np.stack([phi, r2, r3], axis=1), s_tr, p_tr, dev


def gtn_update(e, epsp_n, e0_n, fs, f, ph, K, mu):
    """Backward-Euler GTN return map (Section 2.1.1, Appendix A.1) with f and
    f* held fixed (they follow the frozen non-local variables).  e: (n, 6)
    total Mandel strain, real or complex (complex step).  Elastic where the
    trial stress satisfies phi <= 0; elsewhere Newton on (d_v, d_q, e0) from
    the elastic predictor with a complex-step Jacobian of the residuals at the
    real iterate and backtracking on the real residual.  Returns sigma,
    epsp, e0."""
    n = e.shape[0]
    x = np.zeros((n, 3), dtype=e.dtype)
    x[:, 2] = e0_n
    R, s_tr, p_tr, dev = _gtn_residual(e, epsp_n, e0_n, fs, f, ph, K, mu, x)
    pl = R[:, 0].real > 0.0
    if np.any(pl):
        sel = np.nonzero(pl)[0]
        xs = x[sel]
        args = (e[sel], epsp_n[sel], e0_n[sel], fs[sel], f[sel], ph, K[sel], mu[sel])
        h = 1e-30
        done = False
        for it in range(100):
            Rs = _gtn_residual(*args, xs)[0]
            xr = xs.real.copy()
            J = np.empty((len(sel), 3, 3))
            for k in range(3):
                xp = xr.astype(np.complex128)
                xp[:, k] += 1j * h
                J[:, :, k] = _gtn_residual(args[0].real, *args[1:], xp)[0].imag / h
            step = np.linalg.solve(J, Rs[..., None])[..., 0]
            lam = np.ones(len(sel))
            r0 = np.linalg.norm(Rs.real, axis=1)
            for _ in range(40):
                xn = xs - lam[:, None] * step
                rn = np.linalg.norm(_gtn_residual(*args, xn)[0].real, axis=1)
                bad = ~(rn <= r0 * (1.0 - 1e-4 * lam)) & (r0 > 1e-15)
                if not np.any(bad):
                    break
                lam = np.where(bad, 0.5 * lam, lam)
            xs = xs - lam[:, None] * step
            if done:
                break
            # quadratic convergence: a relative step of 1e-12 leaves the real
            # part at round-off; one more iteration settles the complex-step
            # part, which follows the real iterate
            done = it >= 1 and bool(np.all(np.abs(step) <= 1e-12 * np.maximum(np.abs(xs), 1e-4)))
        else:
            raise RuntimeError("GTN return map did not converge")
        if np.max(np.abs(_gtn_residual(*args, xs)[0].real)) > 1e-10:
            raise RuntimeError("GTN return map did not converge")
        x[sel] = xs
    K2, mu2 = K[:, None], mu[:, None]
    dv, dq, e0 = x[:, 0], x[:, 1], x[:, 2]
    safe = np.where(s_tr.real > 0.0, s_tr, 1.0)
    nflow = np.where((s_tr.real > 0.0)[:, None], 1.5 * 2.0 * mu2 * dev / safe[:, None], 0.0)
    s = s_tr - 3.0 * mu * dq
    p = p_tr + K * dv
    sigma = -p[:, None] * IVEC[None, :] + (2.0 / 3.0) * s[:, None] * nflow
    # elastic voxels: sigma = C (e - epsp_n) exactly
    el = ~pl
    if np.any(el):
        ee = (e - epsp_n)[el]
        trr = ee[:, 0] + ee[:, 1] + ee[:, 2]
        sigma[el] = K2[el] * trr[:, None] * IVEC[None, :] + 2.0 * mu2[el] * (ee - trr[:, None] * IVEC[None, :] / 3.0)
    epsp = epsp_n + dv[:, None] * IVEC[None, :] / 3.0 + dq[:, None] * nflow
    return sigma, epsp, e0


def damage_of(abar, ph):
    """Linear damage law driven by the non-local equivalent plastic strain
    (Eq. non-local_damage_lemaitre), capped at D_max (Section 4.1, R10); the
    same ramp on the non-local kappa for particle cracking (R20)."""
    if ph.law not in (1, 2):
        return np.zeros_like(abar)
    D = (abar - ph.eps_C) / (ph.eps_R - ph.eps_C)
    return np.clip(D, 0.0, ph.D_max)


def positive_principal_norm(e):
    """||<eps>_+|| for Mandel strains e (n, 6): the Euclidean norm of the
    positive parts of the eigenvalues of the strain tensor (R20)."""
    lam = np.linalg.eigvalsh(mandel_to_tensor(e))
    return np.sqrt(np.sum(np.maximum(lam, 0.0) ** 2, axis=-1))


def return_map(eps, epsp_n, ep_n, abar, phase, phases, stiff=None, abar_n=None, f_n=None):
    """Backward-Euler update of the Lemaitre model (Appendix A.2 with R8-R11)
    at every voxel.

    eps, epsp_n: (V, 6) Mandel; ep_n: (V,); abar: (J, V) non-local variables
    held fixed; phase: (V,) int.  Returns a dict with sigma (V,6), tangent
    C (V,6,6), epsp (V,6), ep (V,), D (V,), alpha (J,V).

      sigma_eff_trial = K tr(e) I + 2 mu dev(e),  e = eps - epsp_n
      f = ||dev sigma_eff_trial|| - sqrt(2/3) (sigma_y + H ep_n)
      f > 0: dlambda = f / (2 mu + 2 H / 3), nhat = dev / ||dev||,
             epsp = epsp_n + dlambda nhat, ep = ep_n + sqrt(2/3) dlambda,
             sigma_eff = sigma_eff_trial - 2 mu dlambda nhat
      D = clamp((abar - eps_C) / (eps_R - eps_C), 0, D_max)
      sigma = (1 - D) sigma_eff
      C = (1 - D) [K I(x)I + 2 mu theta P_dev - 2 mu thetabar nhat(x)nhat]
          theta = 1 - 2 mu dlambda / q, thetabar = 1/(1 + H'/(3 mu)) - (1 - theta)
    (the consistent tangent of radial return with isotropic hardening, H' the
    slope of the flow stress at the end point).  With the Aravas flow stress
    (hard 1) sigma_y + H ep_n above reads sigma_0(ep_n) and dlambda solves
    q - 2 mu dlambda - sqrt(2/3) sigma_0(ep_n + sqrt(2/3) dlambda) = 0.
    Particle cracking (law 2, R20): kappa = max(kappa_n, ||<e>_+||) is kept
    in the ep slot, D from abar of the phase's variable, sigma = (1 - D) C e.
    stiff: optional (V,) field scaling the Young's modulus voxel by voxel
    (K and mu of the voxel's phase times stiff; 1 where absent).
    Gurson-Tvergaard-Needleman (law 3, Section 2.1.1 / 2.2.2, Appendix A.1):
    the phase feeds variables var (alpha = eps_0^p, in the ep slot) and
    var + 1 (alpha = tr eps^p); the porosity f follows the frozen non-local
    variables from f_n (gtn_porosity, with abar_n the converged values of the
    last increment), f* = gtn_fstar(f); gtn_update returns sigma, eps^p and
    eps_0^p; the tangent is the complex-step derivative of that map (the
    consistent tangent with f frozen, as D is for Lemaitre, R11); D reports
    f*.  The dict also carries f (V,).
    """
    Vn = eps.shape[0]
    J = abar.shape[0]
    sigma = np.zeros((Vn, 6))
    C = np.zeros((Vn, 6, 6))
    epsp = epsp_n.copy()
    ep = ep_n.copy()
    D = np.zeros(Vn)
    alpha = np.zeros((J, Vn))
    Pdev = np.eye(6) - np.outer(IVEC, IVEC) / 3.0
    if abar_n is None:
        abar_n = np.zeros_like(abar)
    fout = initial_porosity(phase, phases) if f_n is None else np.array(f_n, dtype=np.float64)
    for q, ph in enumerate(phases):
        sel = phase == q
        if not np.any(sel):
            continue
        sc = np.ones(int(sel.sum())) if stiff is None else np.asarray(stiff, dtype=np.float64)[sel]
        K, mu = ph.K * sc, ph.mu * sc
        if ph.law == 3:
            v0, v1 = ph.var, ph.var + 1
            fq = gtn_porosity(fout[sel], abar[v0][sel], abar_n[v0][sel], abar[v1][sel], abar_n[v1][sel], ph)
            fs = gtn_fstar(fq, ph)
            e_q = eps[sel]
            sig_q, epsp_q, e0_q = gtn_update(e_q, epsp_n[sel], ep_n[sel], fs, fq, ph, K, mu)
            Cq = np.empty((e_q.shape[0], 6, 6))
            hcs = 1e-30
            for c in range(6):
                ec = e_q.astype(np.complex128)
                ec[:, c] += 1j * hcs
                Cq[:, :, c] = gtn_update(ec, epsp_n[sel], ep_n[sel], fs, fq, ph, K, mu)[0].imag / hcs
            sigma[sel] = sig_q
            C[sel] = Cq
            epsp[sel] = epsp_q
            ep[sel] = e0_q
            D[sel] = fs
            fout[sel] = fq
            alpha[v0, sel] = e0_q
            alpha[v1, sel] = epsp_q[:, 0] + epsp_q[:, 1] + epsp_q[:, 2]
            continue
        e = eps[sel] - epsp_n[sel]
        tr = e[:, 0] + e[:, 1] + e[:, 2]
        dev = e - tr[:, None] * IVEC[None, :] / 3.0
        s_tr = 2.0 * mu[:, None] * dev
        sig_tr = K[:, None] * tr[:, None] * IVEC[None, :] + s_tr
        qn = np.sqrt(np.einsum("ij,ij->i", s_tr, s_tr))
        theta = np.ones(qn.shape)
        thetabar = np.zeros(qn.shape)
        nhat = np.zeros_like(s_tr)
        sig_eff = sig_tr
        if ph.law == 1:
            s23 = math.sqrt(2.0 / 3.0)
            f = qn - s23 * flow_stress(ph, ep_n[sel])[0]
            pl = f > 0.0
            if ph.hard == 0:
                dl = np.where(pl, f / (2.0 * mu + 2.0 * ph.H / 3.0), 0.0)
            else:
                # nonlinear hardening: q - 2 mu dl - sqrt(2/3) sigma_0(ep_n +
                # sqrt(2/3) dl) = 0 is decreasing in dl, positive at 0 and
                # negative at q / (2 mu)
                dl = np.where(pl, _bisect_increasing(
                    lambda x: -(qn - 2.0 * mu * x - s23 * flow_stress(ph, ep_n[sel] + s23 * x)[0]),
                    np.zeros(qn.shape), qn / (2.0 * mu)), 0.0)
            Hp = flow_stress(ph, ep_n[sel] + s23 * dl)[1]      # slope at the end point
            safe_q = np.where(pl, qn, 1.0)
            nhat = np.where(pl[:, None], s_tr / safe_q[:, None], 0.0)
            epsp[sel] = epsp_n[sel] + dl[:, None] * nhat
            ep[sel] = ep_n[sel] + s23 * dl
            sig_eff = sig_tr - 2.0 * mu[:, None] * dl[:, None] * nhat
            theta = np.where(pl, 1.0 - 2.0 * mu * dl / safe_q, 1.0)
            thetabar = np.where(pl, 1.0 / (1.0 + Hp / (3.0 * mu)) - (1.0 - theta), 0.0)
            Dq = damage_of(abar[ph.var][sel], ph) if ph.var >= 0 else np.zeros(qn.shape)
            D[sel] = Dq
            if ph.var >= 0:
                alpha[ph.var, sel] = ep[sel]
        elif ph.law == 2:
            kap = np.maximum(ep_n[sel], positive_principal_norm(e))
            ep[sel] = kap
            if ph.var >= 0:
                D[sel] = damage_of(abar[ph.var][sel], ph)
                alpha[ph.var, sel] = kap
        Dq = D[sel]
        sigma[sel] = (1.0 - Dq)[:, None] * sig_eff
        Cq = (K[:, None, None] * np.outer(IVEC, IVEC)[None]
              + 2.0 * (mu * theta)[:, None, None] * Pdev[None]
              - 2.0 * (mu * thetabar)[:, None, None] * np.einsum("vi,vj->vij", nhat, nhat))
        C[sel] = (1.0 - Dq)[:, None, None] * Cq
    return dict(sigma=sigma, C=C, epsp=epsp, ep=ep, D=D, alpha=alpha, f=fout)


def initial_porosity(phase, phases):
    """f0 of each GTN voxel, 0 elsewhere."""
    f = np.zeros(len(phase))
    for q, ph in enumerate(phases):
        if ph.law == 3:
            f[phase == q] = ph.f0
    return f


# ============================================================ Krylov solvers
def cg(A, b, rtol, maxit, dot=None, floor=0.0):
    """Textbook conjugate gradients from x0 = 0; stops when ||r|| <=
    max(rtol ||b||, floor) (the criterion of Algorithm 2, with the absolute
    floor of R26) or when (p, A p) <= 0 (R25).  Returns (x, iterations)."""
    if dot is None:
        def dot(u, v):
            return float(np.sum(u * v))
    x = np.zeros_like(b)
    bn = math.sqrt(dot(b, b))
    tol = max(rtol * bn, floor)
    if bn == 0.0 or bn <= tol:
        return x, 0
    r = b.copy()
    p = r.copy()
    rr = dot(r, r)
    it = 0
    while it < maxit:
        Ap = A(p)
        pAp = dot(p, Ap)
        if not pAp > 0.0:
            break
        alpha = rr / pAp
        x = x + alpha * p
        r = r - alpha * Ap
        it += 1
        rr_new = dot(r, r)
        if math.sqrt(rr_new) <= tol:
            break
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, it


def pcg(A, M, b, rtol, maxit):
    """Preconditioned conjugate gradients on complex vectors with the
    Hermitian inner product (ConjGrad of Algorithm 2), x0 = 0, stop when
    ||A x - b|| <= rtol ||b|| (recursive residual) or (p, A p) <= 0 (R25)."""
    def dot(u, v):
        return complex(np.vdot(u, v)).real
    x = np.zeros_like(b)
    bn = math.sqrt(dot(b, b))
    if bn == 0.0:
        return x, 0
    r = b.copy()
    z = M(r)
    p = z.copy()
    rz = dot(r, z)
    it = 0
    while it < maxit:
        Ap = A(p)
        pAp = dot(p, Ap)
        if not pAp > 0.0:
            break
        alpha = rz / pAp
        x = x + alpha * p
        r = r - alpha * Ap
        it += 1
        if math.sqrt(dot(r, r)) <= rtol * bn:
            break
        z = M(r)
        rz_new = dot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it


# ============================================== Helmholtz (Sec 3.2.3, Alg. 2)
def helmholtz_apply_hat(a_hat, ell2, grid, ks=None):
    """GC of Algorithm 2 with the discrete derivative (R15):
        L(a) = a + sum_j conj(k_j) F( l^2(x) F^-1(k_j a) )."""
    if ks is None:
        ks = willot_k(grid)
    out = a_hat.copy()
    for j in range(grid.d):
        g = ifft_fields(ks[j] * a_hat, grid).real
        out = out + np.conj(ks[j]) * fft_fields(ell2 * g, grid)
    return out


def helmholtz_precond(grid, ell2_mean, ks=None):
    """M of Algorithm 2 / Eq. (preconditioner): 1 / (1 + <l^2> |k|^2), with
    the discrete |k|^2 so that M is the exact inverse for uniform l."""
    if ks is None:
        ks = willot_k(grid)
    k2 = sum(np.abs(k) ** 2 for k in ks)
    return 1.0 / (1.0 + ell2_mean * k2)


def helmholtz_solve(alpha, ell2, grid, rtol, maxit):
    """Algorithm 2: b = F(alpha); x = ConjGrad(GC, M, b, TOL); abar = F^-1 x.
    ``alpha`` and ``ell2`` are real fields of the grid shape.  Returns
    (abar, iterations)."""
    ks = willot_k(grid)
    b = fft_fields(alpha, grid)
    m = helmholtz_precond(grid, float(np.mean(ell2)), ks)
    xh, it = pcg(lambda v: helmholtz_apply_hat(v, ell2, grid, ks), lambda v: m * v,
                 b, rtol, maxit)
    return ifft_fields(xh, grid).real, it


# ========================================= mechanics (Sec 3.2.2, Eq. lin_stress)
@dataclass
class Options:
    tol_stag: float = 1e-6
    tol_newton: float = 1e-6
    cg_rtol: float = 1e-8
    pcg_rtol: float = 1e-8
    max_stag: int = 50
    max_newton: int = 30
    max_cg: int = 2000
    max_pcg: int = 2000
    min_stag: int = 2


PARITY_OPTIONS = Options(tol_stag=1e-11, tol_newton=1e-12, cg_rtol=1e-13, pcg_rtol=1e-13)


def mech_solve(grid, eps_c, epsp_n, ep_n, abar, phase, phases, stress_mask, sig_bar_c, opt, stiff=None,
               abar_n=None, f_n=None):
    """Newton-Raphson on the Galerkin residual at fixed abar (step (i) of
    Algorithm 1, Eq. lin_stress and the CG solve after it):

        CG:  G*(C_T : d eps) = -G*(sigma - Sigma_bar),   eps <- eps + d eps

    eps_c holds the carried components; returns the updated strain, the
    last return-map output and iteration counts."""
    d = grid.d
    comps = carried(d)
    sh = grid.shape
    Vn = grid.V
    eps_c = eps_c.copy()
    newton = 0
    cg_total = 0
    de_rel = None
    while True:
        rm = return_map(embed(eps_c, d).reshape(Vn, 6), epsp_n, ep_n, abar, phase, phases, stiff, abar_n, f_n)
        sig_c = rm["sigma"][:, comps].reshape(sh + (len(comps),))
        Cc = rm["C"][:, comps][:, :, comps].reshape(sh + (len(comps), len(comps)))
        res = -G_apply(sig_c - sig_bar_c, grid, stress_mask)
        smean = np.linalg.norm(sig_c.reshape(-1, len(comps)).mean(axis=0))
        res_rel = np.linalg.norm(res) / (math.sqrt(Vn) * max(smean, 1e-300))
        if res_rel < opt.tol_newton and (de_rel is None or de_rel < opt.tol_newton):
            break
        if newton >= opt.max_newton:
            raise RuntimeError("Newton did not converge")
        dx, it = cg(lambda x: G_apply(np.einsum("...ij,...j->...i", Cc, x), grid, stress_mask),
                    res, opt.cg_rtol, opt.max_cg,
                    floor=0.01 * opt.tol_newton * math.sqrt(Vn) * smean)
        eps_c = eps_c + dx
        cg_total += it
        newton += 1
        emean = np.linalg.norm(eps_c.reshape(-1, len(comps)).mean(axis=0))
        de_rel = float(np.max(np.abs(dx))) / max(emean, 1e-300)
    return eps_c, rm, newton, cg_total


# ========================================================= staggered (Alg. 1)
@dataclass
class State:
    grid: Grid
    phase: np.ndarray           # (V,) int
    phases: list
    ell: np.ndarray             # (J, n_phases)
    eps: np.ndarray             # (V, nc) carried Mandel
    epsp: np.ndarray            # (V, 6)
    ep: np.ndarray              # (V,)
    abar: np.ndarray            # (J, V)
    sigma: np.ndarray           # (V, 6)
    D: np.ndarray               # (V,)
    stiff: np.ndarray = None    # (V,) Young's modulus scaling, None = 1
    f: np.ndarray = None        # (V,) porosity of GTN voxels (law 3)
    n_done: int = 0
    curve: list = field(default_factory=list)


def make_state(grid, phase_map, phases, ell, stiff=None):
    Vn = grid.V
    nc = len(carried(grid.d))
    J = np.asarray(ell).shape[0]
    sf = None if stiff is None else np.asarray(stiff, dtype=np.float64).reshape(Vn)
    ph = np.asarray(phase_map).reshape(Vn).astype(np.int64)
    return State(grid, ph, phases, np.asarray(ell, dtype=np.float64), np.zeros((Vn, nc)), np.zeros((Vn, 6)),
                 np.zeros(Vn), np.zeros((J, Vn)), np.zeros((Vn, 6)), np.zeros(Vn), sf,
                 initial_porosity(ph, phases))


def to_mandel_target(t6):
    """Tensor-shear component vector (11,22,33,23,13,12) -> Mandel."""
    return np.asarray(t6, dtype=np.float64) * MANDEL_W


def ell2_field(st, j):
    return (st.ell[j][st.phase] ** 2).reshape(st.grid.shape)


def step_increment(st, strain_ctrl, target_prev, target, opt, trace=None):
    """One load increment n -> n+1 of Algorithm 1 (iterated staggered scheme).

    strain_ctrl: 6-vector, 1 where E_hk is prescribed, 0 where Sigma_HK is;
    target_prev / target: tensor-shear 6-vectors of increment n and n+1.
    trace: optional callable, given after every staggered iteration a dict
    with the iteration count k, the strain and non-local iterates before and
    after it (eps_prev, eps_new, abar_prev, abar_new) and the ERR it computed
    (a read-only view for tests; nothing it returns is used)."""
    g = st.grid
    d = g.d
    comps = carried(d)
    nc = len(comps)
    sh = g.shape
    Vn = g.V
    ctrl_c = np.asarray(strain_ctrl, dtype=np.float64)[comps]
    stress_mask = 1.0 - ctrl_c
    tm = to_mandel_target(target)[comps]
    tpm = to_mandel_target(target_prev)[comps]
    sig_bar = stress_mask * tm
    # initial guess (R14)
    eps_k = st.eps + ctrl_c * (tm - tpm)
    abar_k = st.abar.copy()
    J = st.abar.shape[0]
    stag = 0
    newton_tot = 0
    cg_tot = 0
    pcg_tot = 0
    err = math.inf
    while True:
        eps_new, rm, nn, nc_it = mech_solve(g, eps_k.reshape(sh + (nc,)), st.epsp, st.ep,
                                            abar_k, st.phase, st.phases, stress_mask,
                                            sig_bar, opt, st.stiff, st.abar, st.f)
        eps_new = eps_new.reshape(Vn, nc)
        newton_tot += nn
        cg_tot += nc_it
        abar_new = np.zeros_like(abar_k)
        for j in range(J):
            sol, it = helmholtz_solve(rm["alpha"][j].reshape(sh), ell2_field(st, j), g,
                                      opt.pcg_rtol, opt.max_pcg)
            abar_new[j] = sol.reshape(Vn)
            pcg_tot += it
        emean = np.linalg.norm(eps_new.mean(axis=0))
        err = float(np.max(np.abs(eps_new - eps_k))) / max(emean, 1e-300)
        for j in range(J):
            an = np.linalg.norm(abar_new[j])
            if an >= 1e-30:
                err = max(err, float(np.linalg.norm(abar_new[j] - abar_k[j]) / an))
        if trace is not None:
            trace(dict(k=stag + 1, eps_prev=eps_k.copy(), eps_new=eps_new.copy(),
                       abar_prev=abar_k.copy(), abar_new=abar_new.copy(), err=err))
        eps_k = eps_new
        abar_k = abar_new
        stag += 1
        if stag >= opt.min_stag and err <= opt.tol_stag:
            break
        if stag >= opt.max_stag:
            raise RuntimeError("staggered scheme did not converge")
    # commit (the last mechanics solve was made at abar_k of the previous
    # iteration; its internal variables are the increment's result)
    st.eps = eps_k
    st.epsp = rm["epsp"]
    st.ep = rm["ep"]
    st.abar = abar_k
    st.sigma = rm["sigma"]
    st.D = rm["D"]
    st.f = rm["f"]
    st.n_done += 1
    rec = dict(E=homogenized_strain(st), S=homogenized_stress(st),
               D_mean=float(st.D.mean()), D_max=float(st.D.max()), stag=stag,
               newton=newton_tot, cg=cg_tot, pcg=pcg_tot, err=err,
               voxel_iterations=Vn * (cg_tot + pcg_tot))
    st.curve.append(rec)
    return rec


def homogenized_stress(st):
    """<sigma> as a tensor-shear 6-vector (order 11,22,33,23,13,12)."""
    return st.sigma.mean(axis=0) / MANDEL_W


def homogenized_strain(st):
    e = embed(st.eps, st.grid.d).mean(axis=0)
    return e / MANDEL_W


def step_increment_adaptive(st, strain_ctrl, target_last, target, opt, max_cuts=7):
    """One increment with cut-back (R27).  target_last: the targets of the
    last converged (sub-)step; target: the increment's.  A failed sub-step
    leaves the state untouched (step_increment commits only on success).
    Returns (record of the last sub-step, converged sub-steps, targets
    reached); raises RuntimeError when the sub-step would fall below
    2^-max_cuts of the path, with the state at the last converged sub-step."""
    T0 = np.asarray(target_last, dtype=np.float64)
    T1 = np.asarray(target, dtype=np.float64)
    n0 = st.n_done
    frac, sub, subs = 0.0, 1.0, 0
    last = T0.copy()
    rec = None
    while frac < 1.0:
        fn = min(1.0, frac + sub)
        T = T1.copy() if fn >= 1.0 else T0 + fn * (T1 - T0)
        try:
            rec = step_increment(st, strain_ctrl, last, T, opt)
        except RuntimeError:
            st.n_done = n0
            if sub * 0.5 < 2.0 ** -max_cuts:
                raise
            sub *= 0.5
            continue
        frac = fn
        subs += 1
        sub *= 2.0
        last = T
    st.n_done = n0 + 1
    return rec, subs, last


def run_load_path(grid, phase_map, phase_dicts, ell, strain_ctrl, target, opt, n_incr=None,
                  stiff=None):
    """Algorithm 1's time loop over a load path; returns the state."""
    st = make_state(grid, phase_map, phases_from_dicts(phase_dicts), ell, stiff)
    tgt = np.asarray(target, dtype=np.float64)
    n = len(tgt) if n_incr is None else n_incr
    prev = np.zeros(6)
    for i in range(n):
        step_increment(st, strain_ctrl, prev, tgt[i], opt)
        prev = tgt[i]
    return st
