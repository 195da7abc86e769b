"""Increment cut-back of the oracle (reading R27 of Section 4's variable
strain increment): the policy's bookkeeping against explicit sub-division,
the increment's macroscopic targets and equilibrium at its end, and the
failure path."""
import dataclasses
import math

import numpy as np
import pytest

import rve_inputs as I
from oracle import rve_oracle as O

N2D = (12, 12)
MAT = dict(I.MATRIX, eps_C=0.003, eps_R=0.03)
ELL = np.array([[1.5, 0.03]])


def _state():
    ph = I.disc_phase_map(N2D, 0.2)
    return O.make_state(O.Grid(N2D), ph, O.phases_from_dicts([MAT, I.PARTICLE]), ELL)


def _ctrl():
    return I.plane_strain_mask(np.array([1, 0, 0, 0, 0, 0], dtype=np.uint8))


def _target(e11):
    t = np.zeros(6)
    t[0] = e11
    return t


def test_large_increment_needs_a_cut():
    """E11 = 3e-3 in one increment stalls Newton (the return map switches
    between elastic and plastic voxels); the cut-back halves it once."""
    st = _state()
    with pytest.raises(RuntimeError):
        O.step_increment(st, _ctrl(), np.zeros(6), _target(3e-3), O.PARITY_OPTIONS)
    assert st.n_done == 0 and not np.any(st.eps)          # nothing committed
    rec, subs, last = O.step_increment_adaptive(st, _ctrl(), np.zeros(6), _target(3e-3),
                                                O.PARITY_OPTIONS, max_cuts=4)
    assert subs == 2 and st.n_done == 1
    np.testing.assert_array_equal(last, _target(3e-3))
    # the same state as the explicit sub-division 1.5e-3, 3e-3
    ref = _state()
    O.step_increment(ref, _ctrl(), np.zeros(6), _target(1.5e-3), O.PARITY_OPTIONS)
    O.step_increment(ref, _ctrl(), _target(1.5e-3), _target(3e-3), O.PARITY_OPTIONS)
    np.testing.assert_array_equal(st.eps, ref.eps)
    np.testing.assert_array_equal(st.epsp, ref.epsp)
    np.testing.assert_array_equal(st.abar, ref.abar)


def test_cut_increment_meets_its_targets_and_equilibrium():
    st = _state()
    rec, subs, _ = O.step_increment_adaptive(st, _ctrl(), np.zeros(6), _target(3e-3),
                                             O.PARITY_OPTIONS, max_cuts=4)
    # prescribed macroscopic strain and stresses (plane strain: 22 and 12
    # stress-free, 33 / 13 / 23 strains zero)
    assert rec["E"][0] == pytest.approx(3e-3, rel=1e-12)
    smax = abs(rec["S"][0])
    assert abs(rec["S"][1]) <= 1e-9 * smax and abs(rec["S"][5]) <= 1e-9 * smax
    assert rec["E"][2] == 0.0 and rec["E"][3] == 0.0 and rec["E"][4] == 0.0
    # discrete equilibrium: the Galerkin residual of the committed stress
    g = st.grid
    comps = O.carried(g.d)
    mask = 1.0 - _ctrl()[comps].astype(float)
    sig = st.sigma[:, comps].reshape(g.shape + (len(comps),))
    res = O.G_apply(sig - 0.0, g, mask)
    assert np.linalg.norm(res) <= 1e-9 * math.sqrt(g.V) * smax
    # plastic flow happened in the matrix, none in the particle
    assert st.ep.max() > 0.0
    assert np.all(st.ep[st.phase == 1] == 0.0)


def test_cut_back_gives_up_at_its_minimum_step():
    """A Newton budget of one iteration never converges: the policy halves
    down to 2^-max_cuts, then raises with nothing committed."""
    st = _state()
    opt = dataclasses.replace(O.PARITY_OPTIONS, max_newton=1)
    with pytest.raises(RuntimeError):
        O.step_increment_adaptive(st, _ctrl(), np.zeros(6), _target(1e-3), opt, max_cuts=3)
    assert st.n_done == 0 and not np.any(st.eps) and not st.curve


def test_converging_increment_takes_one_step():
    st = _state()
    ref = _state()
    rec, subs, _ = O.step_increment_adaptive(st, _ctrl(), np.zeros(6), _target(1e-3), O.PARITY_OPTIONS)
    r2 = O.step_increment(ref, _ctrl(), np.zeros(6), _target(1e-3), O.PARITY_OPTIONS)
    assert subs == 1
    np.testing.assert_array_equal(rec["S"], r2["S"])
