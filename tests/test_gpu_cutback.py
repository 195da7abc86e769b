"""GPU increment cut-back (rve_step_increment_adaptive) against the oracle's
policy (reading R27) in the FP64 form with parity tolerances."""
import numpy as np
import pytest

import rve_inputs as I
from oracle import rve_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

pkg = None
N2D = (12, 12)
MAT = dict(I.MATRIX, eps_C=0.003, eps_R=0.03)
ELL = np.array([[1.5, 0.03]])


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global pkg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2103_04770_gb300 as p
    p.lib()
    pkg = p
    yield


def _opts():
    o = pkg.rve_default_options(0)
    p = O.PARITY_OPTIONS
    o.tol_stag, o.tol_newton, o.cg_rtol, o.pcg_rtol = p.tol_stag, p.tol_newton, p.cg_rtol, p.pcg_rtol
    return o


def _cfg(targets):
    ph = I.disc_phase_map(N2D, 0.2)
    ctrl = I.plane_strain_mask(np.array([1, 0, 0, 0, 0, 0], dtype=np.uint8))
    tg = np.zeros((len(targets), 6))
    tg[:, 0] = targets
    return I.RVEConfig("cut", N2D, (12.0, 12.0), ph, [MAT, I.PARTICLE], ELL, ctrl, tg, 0)


def test_adaptive_increment_matches_oracle():
    """E11 = 3e-3 in one increment, then 4e-3: the first is cut once, the
    second converges whole; sub-step counts, homogenised stress and strain,
    and peak damage agree with the oracle (FP64, 1e-10)."""
    cfg = _cfg([3e-3, 4e-3])
    st = O.make_state(O.Grid(N2D), cfg.phase, O.phases_from_dicts(cfg.params), cfg.ell)
    recs, prev = [], np.zeros(6)
    for t in cfg.target:
        rec, subs, prev = O.step_increment_adaptive(st, cfg.strain_ctrl, prev, t, O.PARITY_OPTIONS, max_cuts=4)
        recs.append((rec, subs))
    with pkg.RVE(cfg, precision=0, options=_opts()) as r:
        with pytest.raises(pkg.RVEError) as ei:
            r.step()                                   # the whole increment stalls
        assert ei.value.status == pkg.RVE_ERR_NOT_CONVERGED
        for rec, subs in recs:
            info = r.step_adaptive(max_cuts=4)
            assert info["substeps"] == subs
            smax = abs(rec["S"][0])
            assert np.abs(info["sigma"] - rec["S"]).max() <= 1e-10 * smax
            assert np.abs(info["eps"] - rec["E"]).max() <= 1e-10 * abs(rec["E"][0])
            assert abs(info["D_max"] - rec["D_max"]) <= 1e-9
    assert [s for _, s in recs] == [2, 1]


def test_adaptive_gives_up_and_keeps_the_state():
    cfg = _cfg([1e-3])
    o = _opts()
    o.max_newton = 1                                   # never converges
    with pkg.RVE(cfg, precision=0, options=o) as r:
        info = r.step_adaptive(max_cuts=2, raise_on_error=False)
        assert info["status"] == pkg.RVE_ERR_NOT_CONVERGED and info["substeps"] == 0
        assert np.all(r.strain() == 0.0)
        # a working budget continues from the untouched state
        pkg.rve_set_options(r.h, _opts())
        info = r.step_adaptive(max_cuts=2)
        assert info["substeps"] == 1 and info["increment"] == 1
