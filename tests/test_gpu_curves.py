"""Whole load paths of the 2D single-particle workloads on the GPU against
the FP64 oracle's curves (stored by tests/golden/make_curves.py, which calls
only the oracle).

64^2 (l = 4 voxels) and 128^2 (l = L/16): a centred disc of area fraction
0.2, plane strain, uniaxial E11 in steps of 1e-3 under mixed control.  The
stored curve ends at the first 10 % stress drop below the peak (the end of
the parity range, reading R23), at the first increment the oracle could not
converge, or at the end of the path; the GPU runs the same increments.

  * FP64 form, parity tolerances: mean stress and strain <= 1e-10 relative to
    the peak stress at every increment, staggered counts within 1, damage and
    non-local fields (rve_get_field) <= 1e-8 at the first damaged increment,
    at the peak and at the last increment;
  * mixed form, production tolerances: mean stress <= 1e-4 relative to the
    peak stress at every increment.
"""
import json
import os

import numpy as np
import pytest

import rve_inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
pkg = None


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global pkg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2103_04770_gb300 as p
    p.lib()
    pkg = p
    yield


def _golden(N):
    path = os.path.join(HERE, "golden", "curve_2d_disc_%d.npz" % N)
    if not os.path.exists(path):
        pytest.skip("no stored curve for %d^2" % N)
    z = np.load(path)
    meta = json.loads(str(z["meta"]))
    if str(meta.get("stop", "")).startswith("running"):
        pytest.skip("stored curve for %d^2 is still being written (%s)" % (N, meta["stop"]))
    return z, meta


def _options(meta, prec):
    o = meta["options"]
    opt = pkg.rve_default_options(prec)
    if prec == 0:
        opt.tol_stag, opt.tol_newton, opt.cg_rtol, opt.pcg_rtol = o["tol_stag"], o["tol_newton"], o["cg_rtol"], \
            o["pcg_rtol"]
        opt.max_stag, opt.max_newton, opt.max_cg, opt.max_pcg = o["max_stag"], o["max_newton"], o["max_cg"], \
            o["max_pcg"]
    else:
        opt.max_stag = o["max_stag"]
    return opt


def _field(h, which, n):
    t = torch.empty(n, device="cuda", dtype=torch.float64)
    pkg.rve_get_field(h, which, t)
    return t.cpu().numpy()


@pytest.mark.parametrize("N", [64, 128])
def test_fp64_curve_matches_oracle(N):
    z, meta = _golden(N)
    n = len(z["S"])
    cfg = I.config_2d_disc(N, ell_vox=meta["ell_vox"], n_incr=meta["n_incr"], dE=meta["dE"])
    assert cfg.meta["sha256"] == str(z["phase_sha256"])
    marks = {int(z["incr_" + k]): k for k in ("first_damage", "peak", "last") if "incr_" + k in z}
    smax = np.abs(z["S"][:, 0]).max()
    V = N * N
    with pkg.RVE(cfg, precision=0, options=_options(meta, 0)) as r:
        for i in range(n):
            info = r.step()
            assert np.abs(info["sigma"] - z["S"][i]).max() <= 1e-10 * smax, i + 1
            assert np.abs(info["eps"] - z["E"][i]).max() <= 1e-10 * abs(z["E"][i][0]), i + 1
            # past the peak the staggered iteration contracts slowly (over
            # 100 iterations at 0.95 per iteration), where round-off can
            # move the count by a few
            assert abs(info["staggered_iters"] - int(z["stag"][i])) <= max(1, 0.05 * int(z["stag"][i])), i + 1
            assert abs(info["D_max"] - float(z["D_max"][i])) <= 1e-8
            if i + 1 in marks:
                k = marks[i + 1]
                D = _field(r.h, 2, V)
                ab = _field(r.h, 3, V)
                assert np.abs(D - z["D_" + k]).max() <= 1e-8, (k, i + 1)
                amax = max(np.abs(z["abar_" + k]).max(), 1e-300)
                assert np.abs(ab - z["abar_" + k].ravel()).max() <= 1e-8 * amax, (k, i + 1)
    assert z["D_max"][-1] > 0.1          # the stored curve reaches well into damage


@pytest.mark.parametrize("N", [64, 128])
def test_mixed_curve_matches_oracle(N):
    z, meta = _golden(N)
    n = len(z["S"])
    cfg = I.config_2d_disc(N, ell_vox=meta["ell_vox"], n_incr=meta["n_incr"], dE=meta["dE"])
    smax = np.abs(z["S"][:, 0]).max()
    errs = []
    with pkg.RVE(cfg, precision=1, options=_options(meta, 1)) as r:
        for i in range(n):
            info = r.step()
            errs.append(np.abs(info["sigma"] - z["S"][i]).max() / smax)
    assert max(errs) <= 1e-4, max(errs)
