"""Seeded synthetic inputs for voxelised RVEs: phase maps, load paths,
material sets and random fields.

This module holds geometry, schedules and random numbers only; none of the
method's arithmetic (no return map, no spectral operator, no solver) lives
here.  Both the CPU oracle's tests and the CUDA path's tests and benchmark
draw their inputs from it, so the two sides see identical data.

Conventions
-----------
* A grid is given in physical axis order ``n = (N1, N2)`` (2D) or
  ``(N1, N2, N3)`` (3D); arrays are stored C-contiguous with x1 fastest, so
  a phase map has numpy shape ``(N2, N1)`` or ``(N3, N2, N1)``.
* Voxel centres sit at ``x_i = (1/2 + n_i) L_i / N_i`` (Section 3.2.1,
  "Discretization").  Lengths are in voxel units unless stated otherwise.
* Phase 0 is the damaging elasto-plastic matrix, phase 1 the elastic
  particles.
* Macroscopic components are ordered 11, 22, 33, 23, 13, 12 with tensor (not
  engineering) shears.  Stresses are in MPa.
"""
from __future__ import annotations

import hashlib
import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------- materials
# Matrix: aluminium-like Lemaitre matrix of the paper's 3D examples
# (Section 4.2: E_M = 70 GPa, nu_M = 0.33; damage thresholds eps_C = 0.03,
# eps_R = 0.2, cap D = 0.99) with sigma_y = 100 MPa and H = 500 MPa.
MATRIX = dict(E=70000.0, nu=0.33, sigma_y=100.0, H=500.0, law=1,
              eps_C=0.03, eps_R=0.2, D_max=0.99, var=0)
# Particle: elastic reinforcement of Section 4.2 (E_I = 400 GPa, nu_I = 0.2).
PARTICLE = dict(E=400000.0, nu=0.2, sigma_y=0.0, H=0.0, law=0,
                eps_C=0.0, eps_R=1.0, D_max=0.0, var=-1)

# Cracking particle (builder extension of Section 3.1's multi-variable
# framework, not in the paper): elastic, damaged by its own non-local
# positive-principal-strain history with thresholds kappa_C = 0.005,
# kappa_R = 0.02 (stored in the eps_C / eps_R slots) and the same cap.
PARTICLE_CRACKING = dict(PARTICLE, law=2, eps_C=0.005, eps_R=0.02, D_max=0.99, var=1)

# ratio between the own-phase and other-phase characteristic length
# (Section 4.1: l_M / l_I = 50)
ELL_CONTRAST = 50.0


def phase_params(matrix=None, particle=None):
    """Return the two-phase parameter list ``[matrix, particle]``."""
    return [dict(MATRIX if matrix is None else matrix),
            dict(PARTICLE if particle is None else particle)]


# ------------------------------------------------------------ phase maps
def _centres(n):
    """Voxel-centre coordinates (voxel units) per physical axis."""
    return [np.arange(N, dtype=np.float64) + 0.5 for N in n]


def disc_phase_map(n, area_fraction=0.2):
    """One centred circular particle in a 2D cell (Section 4.1 geometry).

    Radius R = L sqrt(f / pi) in each axis' voxel units (square cells only).
    A voxel is particle iff its centre lies inside the disc (periodic images
    included; a centred disc never reaches them for f < pi/4).
    """
    n1, n2 = n
    if n1 != n2:
        raise ValueError("disc_phase_map expects a square grid")
    R = n1 * math.sqrt(area_fraction / math.pi)
    x1, x2 = _centres(n)
    c = n1 / 2.0
    d2 = (x1[None, :] - c) ** 2 + (x2[:, None] - c) ** 2
    return (d2 < R * R).astype(np.uint8)


def rsa_sphere_centres(n, radius, count, seed, max_rejects=1_000_000):
    """Random sequential addition of ``count`` non-overlapping spheres.

    Centres are uniform in [0, N_i) per axis, drawn from
    ``numpy.random.default_rng(seed)``; a candidate is accepted when its
    periodic minimum-image distance to every accepted centre is >= 2 r.
    Raises ``RuntimeError`` after ``max_rejects`` consecutive rejections.
    """
    rng = np.random.default_rng(seed)
    box = np.asarray(n, dtype=np.float64)
    acc = np.empty((count, 3))
    k = 0
    rejects = 0
    dmin2 = (2.0 * radius) ** 2
    while k < count:
        c = rng.random(3) * box
        if k:
            d = acc[:k] - c
            d -= box * np.round(d / box)
            if np.min(np.einsum("ij,ij->i", d, d)) < dmin2:
                rejects += 1
                if rejects > max_rejects:
                    raise RuntimeError("RSA jammed: %d of %d spheres placed" % (k, count))
                continue
        acc[k] = c
        k += 1
        rejects = 0
    return acc


def voxelize_spheres(n, centres, radius):
    """Phase map (uint8, shape (N3, N2, N1)) of periodic spheres.

    A voxel is particle (1) iff its centre lies within ``radius`` of a sphere
    centre under the periodic minimum image.
    """
    n1, n2, n3 = n
    ph = np.zeros((n3, n2, n1), dtype=np.uint8)
    r = float(radius)
    span = int(math.ceil(r)) + 1
    off = np.arange(-span, span + 1)
    for c in centres:
        i1 = (np.floor(c[0]).astype(int) + off) % n1
        i2 = (np.floor(c[1]).astype(int) + off) % n2
        i3 = (np.floor(c[2]).astype(int) + off) % n3
        d1 = i1 + 0.5 - c[0]
        d1 -= n1 * np.round(d1 / n1)
        d2 = i2 + 0.5 - c[1]
        d2 -= n2 * np.round(d2 / n2)
        d3 = i3 + 0.5 - c[2]
        d3 -= n3 * np.round(d3 / n3)
        inside = (d3[:, None, None] ** 2 + d2[None, :, None] ** 2
                  + d1[None, None, :] ** 2) < r * r
        sub = ph[np.ix_(i3, i2, i1)]
        ph[np.ix_(i3, i2, i1)] = np.maximum(sub, inside.astype(np.uint8))
    return ph


def sphere_count_for_fraction(n, radius, vf):
    """Number of spheres of ``radius`` giving volume fraction ``vf``."""
    V = float(np.prod(n))
    return int(round(vf * V / (4.0 / 3.0 * math.pi * radius ** 3)))


def sphere_radius_for_count(n, count, vf):
    """Radius giving volume fraction ``vf`` with ``count`` spheres."""
    V = float(np.prod(n))
    return (3.0 * vf * V / (4.0 * math.pi * count)) ** (1.0 / 3.0)


def laminate_phase_map(n, fractions_x1):
    """Layers normal to x1: ``fractions_x1`` is a list of (start, stop) voxel
    index ranges along x1 that belong to phase 1; the rest is phase 0."""
    ph = np.zeros(tuple(reversed(n)), dtype=np.uint8)
    for a, b in fractions_x1:
        ph[..., a:b] = 1
    return ph


def phase_sha256(ph):
    return hashlib.sha256(np.ascontiguousarray(ph).tobytes()).hexdigest()


# ------------------------------------------------------------ load paths
def uniaxial_path(n_incr, dE11):
    """Uniaxial tension: E11 prescribed, the other five Sigma = 0.

    Returns ``(strain_ctrl[6] uint8, target[n_incr, 6] float64)`` in the
    component order 11, 22, 33, 23, 13, 12 (tensor shears).  In 2D the
    out-of-plane components 33, 23, 13 are strain-controlled at zero (plane
    strain), so the same mask works once those entries are set to 1.
    """
    ctrl = np.array([1, 0, 0, 0, 0, 0], dtype=np.uint8)
    tgt = np.zeros((n_incr, 6))
    tgt[:, 0] = dE11 * np.arange(1, n_incr + 1)
    return ctrl, tgt


def plane_strain_mask(ctrl):
    c = np.array(ctrl, dtype=np.uint8).copy()
    c[2] = c[3] = c[4] = 1
    return c


# ------------------------------------------------------------ random fields
def random_strain(shape, seed, amp=2e-3, ncomp=6):
    """Seeded random strain field (Mandel components last) around a uniaxial
    mean, amplitude ``amp``; used for kernel-level parity cases."""
    rng = np.random.default_rng(seed)
    e = amp * rng.standard_normal(tuple(shape) + (ncomp,))
    e[..., 0] += 3 * amp
    return e


def random_field(shape, seed, ncomp=None, scale=1.0):
    rng = np.random.default_rng(seed)
    s = tuple(shape) + ((ncomp,) if ncomp else ())
    return scale * rng.standard_normal(s)


# ------------------------------------------------------------ configs
@dataclass
class RVEConfig:
    """A synthetic workload: grid, cell size, phases, lengths and load path."""
    name: str
    n: tuple
    L: tuple
    phase: np.ndarray
    params: list
    ell: np.ndarray            # [J][n_phases] characteristic lengths, L units
    strain_ctrl: np.ndarray    # [6] uint8
    target: np.ndarray         # [n_incr, 6]
    precision: int = 0         # 0 FP64, 1 mixed FP32/FP64
    meta: dict = field(default_factory=dict)

    @property
    def dim(self):
        return len(self.n)


def _ell_table(ell_matrix, n_phases=2):
    """Single non-local variable (matrix eps_p): l_M in the matrix and
    l_M / 50 elsewhere (Section 4.1)."""
    e = np.full((1, n_phases), ell_matrix / ELL_CONTRAST)
    e[0, 0] = ell_matrix
    return e


def config_2d_disc(N=64, ell_vox=4.0, n_incr=50, dE=1e-3, precision=0):
    """2D plane strain, one centred particle (area fraction 0.2), uniaxial
    tension to n_incr * dE.  ``ell_vox`` is the matrix length in voxels."""
    n = (N, N)
    ph = disc_phase_map(n, 0.2)
    ctrl, tgt = uniaxial_path(n_incr, dE)
    ctrl = plane_strain_mask(ctrl)
    return RVEConfig("2d_disc_%d" % N, n, (float(N), float(N)), ph,
                     phase_params(), _ell_table(ell_vox), ctrl, tgt, precision,
                     dict(area_fraction=0.2, sha256=phase_sha256(ph)))


def config_mesh_objectivity(N, n_incr=50, dE=1e-3):
    """Same cell at N x N with l = L/16 fixed in physical units."""
    return config_2d_disc(N, ell_vox=N / 16.0, n_incr=n_incr, dE=dE)


def config_3d_spheres(N=256, radius=10.0, vf=0.25, seed=0, ell_vox=4.0,
                      n_incr=40, dE=1e-3, precision=1, count=None, grid=None):
    """3D RVE of random non-overlapping elastic spheres (random sequential
    addition) in the damaging matrix; uniaxial tension under mixed control.
    ``grid`` = (N1, N2, N3) replaces the N^3 cube (profiling shapes)."""
    n = tuple(grid) if grid is not None else (N, N, N)
    if count is None:
        count = sphere_count_for_fraction(n, radius, vf)
    cen = rsa_sphere_centres(n, radius, count, seed)
    ph = voxelize_spheres(n, cen, radius)
    ctrl, tgt = uniaxial_path(n_incr, dE)
    name = "3d_spheres_%d" % N if grid is None else "3d_spheres_%dx%dx%d" % n
    return RVEConfig(name, n, tuple(float(x) for x in n), ph, phase_params(),
                     _ell_table(ell_vox), ctrl, tgt, precision,
                     dict(radius=radius, count=count, seed=seed,
                          vf_voxel=float(ph.mean()), sha256=phase_sha256(ph)))


# ------------------------------------------------- two-variable 3D sphere RVEs
def _ell_table_two(ell_matrix, ell_particle):
    """Two non-local variables: 0 = matrix eps_p (l_M in the matrix, l_M/50
    in the particles), 1 = particle-cracking kappa (l_P in the particles,
    l_P/50 in the matrix)."""
    return np.array([[ell_matrix, ell_matrix / ELL_CONTRAST],
                     [ell_particle / ELL_CONTRAST, ell_particle]])


def config_spheres_two_var(n, vf, count, seed, ell_m=3.0, ell_p=6.0, n_incr=40, dE=1e-3,
                           precision=1, name=None):
    """3D RVE of ``count`` random non-overlapping spheres (radius from the
    volume fraction, r = (3 vf V / (4 pi count))^(1/3)) in the damaging
    matrix, the spheres cracking (law 2) with their own non-local variable;
    uniaxial tension E11 in ``n_incr`` steps of ``dE``, other Sigma = 0."""
    n = tuple(int(x) for x in n)
    r = sphere_radius_for_count(n, count, vf)
    cen = rsa_sphere_centres(n, r, count, seed)
    ph = voxelize_spheres(n, cen, r)
    ctrl, tgt = uniaxial_path(n_incr, dE)
    nm = name or "spheres2_%dx%dx%d_s%d" % (n + (seed,))
    return RVEConfig(nm, n, tuple(float(x) for x in n), ph, [dict(MATRIX), dict(PARTICLE_CRACKING)],
                     _ell_table_two(ell_m, ell_p), ctrl, tgt, precision,
                     dict(radius=r, count=count, seed=seed, vf=vf, vf_voxel=float(ph.mean()),
                          sha256=phase_sha256(ph)))


BATCH_GRIDS = (64, 96, 128)


def config_batch_member(seed, n_incr=40, dE=1e-3, precision=1):
    """Member ``seed`` of the batched workload: grid drawn uniformly from
    {64, 96, 128}^3 and sphere volume fraction uniform in [0.10, 0.30] with
    numpy.random.default_rng(seed); 30 spheres; l = 3 (matrix) / 6 (particle)
    voxels."""
    rng = np.random.default_rng(seed)
    N = BATCH_GRIDS[int(rng.integers(len(BATCH_GRIDS)))]
    vf = float(rng.uniform(0.10, 0.30))
    return config_spheres_two_var((N, N, N), vf, 30, seed, n_incr=n_incr, dE=dE, precision=precision,
                                  name="batch_s%d_%d" % (seed, N))


def config_batch(count=32, n_incr=40, dE=1e-3, precision=1):
    """The batched workload: members for seeds 0 .. count-1."""
    return [config_batch_member(s, n_incr, dE, precision) for s in range(count)]


def config_adjoint(N=96, n_incr=30, dE=1e-3, precision=0):
    """The adjoint workload: N^3, 30 spheres at volume fraction 0.20, seed 0,
    two non-local variables, 30 increments of 1e-3, FP64."""
    return config_spheres_two_var((N, N, N), 0.20, 30, 0, n_incr=n_incr, dE=dE, precision=precision,
                                  name="adjoint_%d" % N)


# ------------------------------------------- the paper's parameter studies
# Section 4.1 (2D examples): matrix E_M = 300 GPa, nu_M = 0.3, sigma_Y = 1 GPa;
# Lemaitre with eps_C = 0.03, eps_R = 0.2, linear hardening k = 10 GPa, D
# capped at 0.99; Gurson-Tvergaard-Needleman with q1 = 1.5, q2 = 1, q3 = 2.25,
# f_C = 0.15, f_F = 0.25, f_N = 0.04, eps_N = 0.3, s_N = 0.1, no initial
# porosity, the Aravas flow stress with N = 0.1 and f* capped at 0.9 f_V* =
# 0.6; elastic inclusion E_I = 900 GPa, nu_I = 0.3 occupying 10 % of the cell.
PAPER2D_LEMAITRE = dict(E=300000.0, nu=0.3, sigma_y=1000.0, H=10000.0, law=1, eps_C=0.03, eps_R=0.2,
                        D_max=0.99, var=0)
PAPER2D_GTN = dict(E=300000.0, nu=0.3, sigma_y=1000.0, H=0.0, law=3, eps_C=0.0, eps_R=1.0, D_max=0.0, var=0,
                   hard=1, N=0.1, q1=1.5, q2=1.0, q3=2.25, f_C=0.15, f_F=0.25, f_N=0.04, eps_N=0.3, s_N=0.1,
                   f0=0.0, fstar_max=0.6)
PAPER2D_INCLUSION = dict(E=900000.0, nu=0.3, sigma_y=0.0, H=0.0, law=0, eps_C=0.0, eps_R=1.0, D_max=0.0,
                         var=-1)
# Section 4.2 (3D examples): E_M = 70 GPa, nu_M = 0.33, sigma_Y = 200 MPa,
# Lemaitre as above with k = 10 GPa; GTN with eps_N = 0.1, s_N = 0.05;
# inclusions E_I = 400 GPa, nu_I = 0.2, 30 spheres at 20 % volume fraction.
PAPER3D_LEMAITRE = dict(E=70000.0, nu=0.33, sigma_y=200.0, H=10000.0, law=1, eps_C=0.03, eps_R=0.2,
                        D_max=0.99, var=0)
PAPER3D_GTN = dict(PAPER2D_GTN, E=70000.0, nu=0.33, sigma_y=200.0, eps_N=0.1, s_N=0.05)
PAPER3D_INCLUSION = dict(PARTICLE)


def config_paper2d(N, model="lemaitre", local=False, ell_M=0.05, ell_I=0.001, n_incr=50, dE=2e-3,
                   precision=0):
    """The 2D example of Section 4.1 on N x N: one centred circular
    inclusion of 10 % area (radius L / sqrt(10 pi)), plane strain, uniaxial
    E11 under mixed control.  Lengths in units of the cell L: the non-local
    model takes l_M, l_I (0.05 L and 0.001 L in the paper); the local limit
    takes l_M = l_I = 1e-4 L (smaller than a voxel).  model: "lemaitre" (one
    non-local variable) or "gtn" (two: eps_0^p and tr eps^p)."""
    n = (N, N)
    ph = disc_phase_map(n, 0.1)
    ctrl, tgt = uniaxial_path(n_incr, dE)
    ctrl = plane_strain_mask(ctrl)
    lM, lI = (1e-4, 1e-4) if local else (ell_M, ell_I)
    mat = PAPER2D_GTN if model == "gtn" else PAPER2D_LEMAITRE
    J = 2 if model == "gtn" else 1
    ell = np.array([[lM * N, lI * N]] * J)
    name = "paper2d_%s_%s_%d" % (model, "local" if local else "nonlocal", N)
    return RVEConfig(name, n, (float(N), float(N)), ph, [dict(mat), dict(PAPER2D_INCLUSION)], ell, ctrl, tgt,
                     precision, dict(area_fraction=0.1, ell_M=lM, ell_I=lI, model=model, sha256=phase_sha256(ph)))


def upsample_phase(ph, factor):
    """Each voxel of a phase map becomes a factor^d block (the same topology
    on a finer grid, Section 4.2, 'Convergence for a fixed topology')."""
    out = ph
    for ax in range(ph.ndim):
        out = np.repeat(out, factor, axis=ax)
    return out


def config_fixed_topology(factor, base=32, model="lemaitre", seed=0, n_incr=40, dE=2e-3, precision=1):
    """The 3D RVE of Section 4.2 (30 non-overlapping spheres, 20 % volume
    fraction, random sequential addition with seed) generated on base^3
    and resampled to (factor * base)^3 by voxel replication, so the particle
    arrangement is the same at every resolution.  l_M = 0.05 L, l_I =
    0.001 L; uniaxial E11 under mixed control."""
    n0 = (base, base, base)
    r = sphere_radius_for_count(n0, 30, 0.20)
    ph0 = voxelize_spheres(n0, rsa_sphere_centres(n0, r, 30, seed), r)
    ph = upsample_phase(ph0, factor)
    N = base * factor
    n = (N, N, N)
    ctrl, tgt = uniaxial_path(n_incr, dE)
    mat = PAPER3D_GTN if model == "gtn" else PAPER3D_LEMAITRE
    J = 2 if model == "gtn" else 1
    ell = np.array([[0.05 * N, 0.001 * N]] * J)
    return RVEConfig("topology_%s_%d_from_%d" % (model, N, base), n, tuple(float(x) for x in n), ph,
                     [dict(mat), dict(PAPER3D_INCLUSION)], ell, ctrl, tgt, precision,
                     dict(base=base, factor=factor, radius_base=r, seed=seed, vf_voxel=float(ph.mean()),
                          sha256_base=phase_sha256(ph0), sha256=phase_sha256(ph)))
