"""Write the oracle's reference curves of the 2D single-particle workloads.

For a centred disc of area fraction 0.2 on N x N (plane strain, uniaxial E11
in steps of 1e-3 under mixed control, matrix length l voxels) the FP64
oracle runs Algorithm 1 with the parity tolerances and a staggered budget of
1000 iterations, increment by increment, and stops at the first increment
whose stress has dropped by 10 % or more below the peak (the end of the
parity range, reading R23), at the first increment it cannot converge, or
at the end of the path.  Written to curve_2d_disc_<N>.npz beside this file:
per increment the mean strain and stress (tensor shears), mean and maximum
damage, iteration counts and ERR; the damage and non-local fields at the
first damaged increment, at the peak and at the last increment.

Test infrastructure: calls only the oracle and the input generators.
The file is rewritten after every increment, so a run stopped early keeps
its curve so far.
Usage:  python tests/golden/make_curves.py N [l_vox] [fft_threads] [max_increments]
"""
import dataclasses
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import rve_inputs as I  # noqa: E402
from oracle import rve_oracle as O  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
OPTIONS = dataclasses.replace(O.PARITY_OPTIONS, max_stag=1000)
DROP = 0.10


def run(N, ell_vox, n_incr=50, dE=1e-3, threads=None, log=sys.stderr, max_incr=None):
    cfg = I.config_2d_disc(N, ell_vox=ell_vox, n_incr=n_incr, dE=dE)
    g = O.Grid(cfg.n, cfg.L)
    st = O.make_state(g, cfg.phase, O.phases_from_dicts(cfg.params), cfg.ell)
    if threads:
        O.set_fft_workers(threads)
    keys = ("stag", "newton", "cg", "pcg", "err", "D_mean", "D_max")
    rows = {k: [] for k in keys}
    E, S, fields = [], [], {}
    prev = np.zeros(6)
    peak, peak_i, first_dmg, stop = -np.inf, -1, None, "end of path"
    t0 = time.time()
    path = os.path.join(HERE, "curve_2d_disc_%d.npz" % N)

    def save(stop):
        out = dict(E=np.array(E), S=np.array(S), **{k: np.array(v) for k, v in rows.items()},
                   peak_increment=peak_i + 1, phase_sha256=cfg.meta["sha256"],
                   meta=json.dumps({"grid": [N, N], "ell_vox": ell_vox, "dE": dE, "n_incr": n_incr,
                                    "options": dataclasses.asdict(OPTIONS), "stop": stop,
                                    "seconds": round(time.time() - t0, 1)}))
        for name, (i, D, ab) in fields.items():
            out["incr_" + name] = i + 1
            out["D_" + name] = D
            out["abar_" + name] = ab
        np.savez_compressed(path, **out)

    for i in range(n_incr if max_incr is None else min(n_incr, max_incr)):
        try:
            rec = O.step_increment(st, cfg.strain_ctrl, prev, cfg.target[i], OPTIONS)
        except RuntimeError as e:
            stop = "increment %d: %s" % (i + 1, e)
            break
        prev = cfg.target[i]
        E.append(rec["E"])
        S.append(rec["S"])
        for k in keys:
            rows[k].append(rec[k])
        s11 = rec["S"][0]
        if s11 > peak:
            peak, peak_i = s11, i
            fields["peak"] = (i, st.D.copy(), st.abar.copy())
        if first_dmg is None and rec["D_max"] > 0:
            first_dmg = i
            fields["first_damage"] = (i, st.D.copy(), st.abar.copy())
        fields["last"] = (i, st.D.copy(), st.abar.copy())
        print(json.dumps({"N": N, "incr": i + 1, "s": round(time.time() - t0, 1), "S11": s11,
                          "D_max": rec["D_max"], "stag": rec["stag"]}), file=log, flush=True)
        if s11 <= (1.0 - DROP) * peak:
            stop = "stress dropped %.0f %% below the peak at increment %d" % (100 * DROP, i + 1)
            break
        # the curve so far is kept after every increment
        save("running: %d increments done" % (i + 1))
    else:
        if max_incr is not None and max_incr < n_incr:
            stop = "increment cap %d reached" % max_incr
    save(stop)
    return path, stop


if __name__ == "__main__":
    N = int(sys.argv[1])
    ell = float(sys.argv[2]) if len(sys.argv) > 2 else (4.0 if N == 64 else N / 16.0)
    th = int(sys.argv[3]) if len(sys.argv) > 3 else None
    mx = int(sys.argv[4]) if len(sys.argv) > 4 else None
    print(run(N, ell, threads=th, max_incr=mx))
