#!/usr/bin/env python
"""Benchmark of the staggered FFT non-local damage scheme on one GB300.

Workload: a 256^3 periodic RVE of 1001 random non-overlapping elastic spheres
(radius 10 voxels, 25 % volume fraction, random sequential addition, seed 0)
in the damaging Lemaitre matrix, uniaxial tension under mixed control
(E11 prescribed, the other five Sigma = 0) in increments of 1e-3.  A step is
one load increment: the full iterated staggered scheme (return maps, Newton /
CG FFT-Galerkin mechanics, preconditioned Helmholtz solves, ERR) through the
C ABI.  Metric: voxel-iterations/s = voxels x (mechanical CG iterations +
Helmholtz PCG iterations) / wall time of the timed increments.

Prints one JSON line (rank 0).  Under torchrun each rank runs an independent
replica (a single RVE does not shard); value sums the ranks' work over the
slowest rank's time.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "voxel-iterations/s at 256^3 (mixed FP32/FP64 form; plain FP64 GPU form alongside)"
UNIT = "voxel-iterations/s"
HBM_FALLBACK_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--grid", default=None, help="N1,N2,N3 instead of the n^3 cube (profiling shapes)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-cufft", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default schedule instead of rve_autotune before the first increment")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="increments of the instrumented replay that gives the per-class times (0: all)")
    ap.add_argument("--curve", action="store_true",
                    help="time the whole load path (cut-back steps) instead of the headline rate")
    ap.add_argument("--curve-incr", type=int, default=0, help="--curve: first K increments only (0: all)")
    ap.add_argument("--cpu-iters", type=int, default=2)
    ap.add_argument("--obj-grids", type=lambda v: [int(x) for x in v.split(",")], default=[128, 256, 512])
    ap.add_argument("--obj-incr", type=int, default=50)
    ap.add_argument("--obj-max-cg", type=int, default=20000,
                    help="CG budget per Newton step of the objectivity runs (the count grows with the grid "
                         "in the plastic range)")
    ap.add_argument("--study-models", type=lambda v: v.split(","), default=["lemaitre", "gtn"])
    ap.add_argument("--study-emax", type=float, default=0.1)
    ap.add_argument("--study-de", type=float, default=2e-3)
    ap.add_argument("--study-budget-s", type=float, default=120.0)
    ap.add_argument("--study-profile-e", type=float, default=0.05)
    ap.add_argument("--topology-model", default="lemaitre", choices=["lemaitre", "gtn"])
    ap.add_argument("--workload", default="spheres256",
                    choices=["spheres256", "batch", "adjoint", "objectivity", "studies2d", "topology3d",
                             "formcurve"],
                    help="batch: the 32-RVE {64,96,128}^3 two-variable workload; adjoint: gradients of "
                         "the final stress of the 96^3 two-variable RVE; formcurve: the sphere RVE's load "
                         "path (--n, --curve-incr) in the mixed and the FP64 form, compared increment by "
                         "increment (each its own JSON line)")
    ap.add_argument("--adj-incr", type=int, default=30)
    ap.add_argument("--adj-every", type=int, default=5)
    ap.add_argument("--adj-fd", default="0:sigma_y,ell0",
                    help="comma list of gradients to check by central differences (h = 1e-6 relative)")
    ap.add_argument("--batch-count", type=int, default=32)
    ap.add_argument("--autotune-reps", type=int, default=2)
    ap.add_argument("--no-seq", action="store_true", help="batch: skip the one-at-a-time comparison")
    return ap.parse_args()


def workload(n, grid=None):
    import rve_inputs as I
    g = tuple(int(x) for x in grid.split(",")) if grid else None
    cfg = I.config_3d_spheres(N=n, radius=10.0, vf=0.25, seed=0, ell_vox=4.0, n_incr=40, dE=1e-3, grid=g)
    return cfg


def workload_config(cfg, precision):
    return {"workload": cfg.name, "grid": list(cfg.n), "voxels": int(np.prod(cfg.n)),
            "spheres": cfg.meta["count"], "radius_vox": cfg.meta["radius"],
            "vf": round(cfg.meta["vf_voxel"], 4), "seed": cfg.meta["seed"], "ell_matrix_vox": 4.0,
            "load": "uniaxial E11, 40 x 1e-3, Sigma_other = 0", "precision": precision,
            "phase_sha256": cfg.meta["sha256"][:16],
            "l2": "inputs larger than L2 (>= 5 GB touched per CG iteration)"}


# ------------------------------------------------------------------ ranks
def dist_init():
    """One process per GPU (replicas: a single RVE does not shard).  NCCL on
    GPUs; gloo when the host has none (the CPU tests of this path)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, None
    import torch
    import torch.distributed as dist
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist.init_process_group("gloo")
    return rank, ws, dist


def _on_gpu(dist):
    return dist is not None and dist.get_backend() == "nccl"


def barrier(dist):
    if dist is not None:
        import torch
        dist.barrier()
        if _on_gpu(dist):
            torch.cuda.synchronize()


def allreduce(dist, x, op="max"):
    """max or sum of a per-rank scalar over all ranks (identity on one rank)"""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], device="cuda" if _on_gpu(dist) else "cpu", dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def aggregate(dist, ms, work):
    """Whole-job rate of independent replicas: the ranks' work summed over
    the slowest rank's time.  Returns (rate per second, max ms)."""
    ms_max = allreduce(dist, ms, "max")
    return allreduce(dist, work, "sum") / (ms_max * 1e-3), ms_max


# ------------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self):
        self.proc = None
        self.path = None

    def start(self, device_index=0):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(device_index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for k, name in enumerate(names):
                if parts[5 + k].lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ traffic
DEVICE_SOURCES = ["common.cuh", "fft.cuh", "fft256.cuh", "fft_ct.cuh", "ops.cuh", "tma.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_bytes_per_voxel.txt")


def device_sources_sha16():
    """Hash of the device sources whose kernels the DRAM counters describe."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2103_04770_gb300", "csrc")
    for f in DEVICE_SOURCES:
        h.update(f.encode())
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def dram_bytes_per_voxel():
    """{class: DRAM bytes per voxel of one launch} from the committed record
    of an ncu capture, or ({}, reason) when the kernels changed since."""
    try:
        lines = open(TRAFFIC_FILE).read().splitlines()
    except OSError:
        return {}, "no traffic record"
    sha, grid, out = None, None, {}
    for ln in lines:
        t = ln.split()
        if not t or t[0].startswith("#"):
            continue
        if t[0] == "kernel_sources_sha16":
            sha = t[1]
        elif t[0] == "capture_grid":
            grid = [int(x) for x in t[1].split("x")]
        elif len(t) == 4:
            out[t[0]] = (float(t[2]) + float(t[3]))
    if sha != device_sources_sha16() or not grid:
        return {}, "kernels changed since the traffic record was captured"
    V = float(np.prod(grid))
    return {k: v / V for k, v in out.items()}, "ncu capture on %s, scaled by voxels" % "x".join(map(str, grid))


# ------------------------------------------------------------------ ours
def _events(n):
    import torch
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def _pinned(nbytes):
    import torch
    try:
        return torch.empty(int(nbytes), dtype=torch.uint8, pin_memory=True)
    except RuntimeError:
        return torch.empty(int(nbytes), dtype=torch.uint8)


def cufft_comparison(cfg, stream, reps=10):
    """cuFFT (torch.fft, timed comparison only): the six-component FP32 R2C
    and C2R transforms of the 256^3 field, no operator between them, CUDA
    events on the launching stream."""
    import torch
    n1, n2, n3 = cfg.n
    x = torch.randn(6, n3, n2, n1, device="cuda", dtype=torch.float32)
    with torch.cuda.stream(stream):
        for _ in range(3):
            y = torch.fft.irfftn(torch.fft.rfftn(x, dim=(1, 2, 3)), s=(n3, n2, n1), dim=(1, 2, 3))
        a, b = _events(2)
        a.record(stream)
        for _ in range(reps):
            X = torch.fft.rfftn(x, dim=(1, 2, 3))
            y = torch.fft.irfftn(X, s=(n3, n2, n1), dim=(1, 2, 3))
        b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    err = float((y - x).abs().max())
    del x, y, X
    torch.cuda.empty_cache()
    return ms, err


def cg_iteration_ms(pkg, h, V, nc, iters=24):
    """Device time of one fused mechanical CG iteration of the library
    (x1 R2C with C_T : p and the curvature, y, z with G*, y, x1 C2R with the
    CG step and (r, r)) through rve_op_cg on the handle's current tangent,
    with b = G*(t) for a random t (so b lies in the range of G*)."""
    import torch
    t = torch.randn(nc, V, device="cuda", dtype=torch.float64)
    b = torch.empty_like(t)
    pkg.rve_op_apply_gamma(h, t, b)
    x = torch.empty_like(t)
    pkg.rve_op_cg(h, b, x, 1e-30, 2, allow_budget=True)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = _events(2)
    e0.record(s)
    it = pkg.rve_op_cg(h, b, x, 1e-30, iters, allow_budget=True)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    del t, b, x
    torch.cuda.empty_cache()
    return ms / max(it, 1), it


def tune_schedule(pkg, h, args):
    """rve_autotune on a fresh handle (before its first increment): the FFT
    schedule and the projection pass's tile width, timed on the matvec."""
    if args.no_autotune:
        return {"autotuned": False, "gamma_narrow": pkg.rve_get_gamma_tile(h)}
    ms, tx, _ = pkg.rve_autotune(h, 3)
    return {"autotuned": True, "matvec_ms": round(ms, 4), "strided_tile": tx,
            "gamma_narrow": pkg.rve_get_gamma_tile(h)}


def run_ours(args, rank, ws, dist):
    import torch
    import paper_2103_04770_gb300 as pkg

    torch.cuda.init()
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()
    cfg = workload(args.n, args.grid)
    V = int(np.prod(cfg.n))
    nc = 6 if len(cfg.n) == 3 else 3
    prec = pkg.RVE_MIXED if args.precision == "mixed" else pkg.RVE_FP64
    K = args.steps

    # -------- device-resident timing: graph replay of the Krylov chunks on,
    # no per-launch events in the timed region
    r = pkg.RVE(cfg, precision=prec, stream=stream)
    schedule = tune_schedule(pkg, r.h, args)
    pkg.rve_set_graphs(r.h, True)
    for _ in range(args.warmup):
        r.step()
    nbytes = pkg.rve_state_bytes(r.h)
    start_state = pkg.rve_save_state(r.h, _pinned(nbytes))        # before the timed increments
    # like-for-like FP64 samples: the first, middle and last timed increment
    samples = sorted({0, K // 2, K - 1}) if (not args.no_fp64 and prec == pkg.RVE_MIXED) else []
    snaps = {}
    pkg.rve_profile_reset(r.h)
    clocks = ClockSampler()
    if rank == 0:
        clocks.start(dev)
    barrier(dist)
    torch.cuda.synchronize()
    ev_a, ev_b = _events(K), _events(K)
    e0, e1 = _events(2)
    e0.record(stream)
    infos = []
    for i in range(K):
        ev_a[i].record(stream)
        infos.append(r.step())
        ev_b[i].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    ck = clocks.stop() if rank == 0 else None
    ms = e0.elapsed_time(e1)
    incr_ms = [a.elapsed_time(b) for a, b in zip(ev_a, ev_b)]
    launches = pkg.rve_profile_read(r.h)
    gpu_launches = int(sum(v[1] for v in launches.values()))
    vi = sum(i["voxel_iterations"] for i in infos)
    rate, ms_max = aggregate(dist, ms, vi)

    # -------- per-class device time: an instrumented replay (CUDA events
    # around every launch, direct launches) of the timed increments from the
    # saved state; it also keeps the states before the FP64 samples
    pkg.rve_load_state(r.h, start_state)
    pkg.rve_profile_reset(r.h)
    pkg.rve_profile(r.h, True)
    n_rep = K if args.profile_steps <= 0 else min(args.profile_steps, K)
    last_sample = max(samples) if samples else 0
    rep_infos = []
    prof = None
    for i in range(K):
        if i == n_rep:                                                # replay of n_rep increments done
            prof = pkg.rve_profile_read(r.h)
            pkg.rve_profile(r.h, False)
        if i in samples and i > 0:
            snaps[i] = pkg.rve_save_state(r.h, _pinned(nbytes))       # state before increment i
        if i >= n_rep and i >= last_sample:
            break
        rep_infos.append(r.step())
    if prof is None:
        prof = pkg.rve_profile_read(r.h)
    pkg.rve_profile(r.h, False)
    replay_same = all(a["cg_iters"] == b["cg_iters"] and a["pcg_iters"] == b["pcg_iters"]
                      for a, b in zip(rep_infos, infos))

    # roofline of the dominant kernel class (its CUDA-event time in the replay)
    dom = max((k for k in prof if k not in ("finalize",)), key=lambda k: prof[k][0])
    dms, dlaunch, dbytes = prof[dom]
    peak, peak_src = HBM_FALLBACK_GBS, "fallback"
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        try:
            peak, peak_src = float(json.load(open(pk))["hbm_gbs"]), "measured"
        except Exception:
            pass
    achieved = dbytes / (dms * 1e-3) / 1e9 if dms > 0 else 0.0
    bpv, traffic_note = dram_bytes_per_voxel()
    traffic = None
    if dom in bpv and prec == pkg.RVE_MIXED and len(cfg.n) == 3:
        traffic = round(bpv[dom] * V)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_source": peak_src,
                "traffic": traffic, "traffic_source": traffic_note if traffic is not None else traffic_note,
                "bytes_per_launch": dbytes / max(dlaunch, 1),
                "avg_launch_ms": dms / max(dlaunch, 1), "launches": dlaunch,
                "timing": "CUDA events around every launch of an instrumented replay of the first %d of the "
                          "%d timed increments from the saved state (same iteration counts: %s)"
                          % (n_rep, K, replay_same),
                "classes": {k: {"ms": round(v[0], 3), "launches": v[1],
                                "GBps": round(v[2] / (v[0] * 1e-3) / 1e9, 1) if v[0] > 0 else None}
                            for k, v in prof.items() if v[1] > 0}}

    out = {"metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": ws,
           "steps": K, "warmup": args.warmup, "ms_per_step": ms_max / K,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64" if prec == pkg.RVE_MIXED else "f64", "data": "synthetic",
           "config": workload_config(cfg, args.precision), "schedule": schedule, "roofline": roofline,
           "gpu_launches": gpu_launches, "clocks": ck,
           "timed_region": "increments %d..%d, graph replay of the Krylov chunks, no per-launch events"
                           % (args.warmup + 1, args.warmup + K),
           "increments": [{"incr": i["increment"], "ms": round(t, 2) if t else None, "stag": i["staggered_iters"],
                           "newton": i["newton_iters"], "cg": i["cg_iters"], "pcg": i["pcg_iters"],
                           "S11": i["sigma"][0], "D_max": i["D_max"]} for i, t in zip(infos, incr_ms)]}

    # -------- cuFFT timed comparison beside one fused CG iteration
    if not args.no_cufft and len(cfg.n) == 3:
        cg_ms, cg_it = cg_iteration_ms(pkg, r.h, V, nc)
        cf_ms, cf_err = cufft_comparison(cfg, stream)
        out["cufft_comparison"] = {
            "cufft_r2c_c2r_6comp_fp32_ms": round(cf_ms, 4), "cufft_roundtrip_max_abs_err": cf_err,
            "ours_cg_iteration_ms": round(cg_ms, 4), "ours_cg_iterations_timed": cg_it,
            "ours_over_cufft": round(cg_ms / cf_ms, 3),
            "what": "cuFFT: torch.fft rfftn + irfftn of a (6, N3, N2, N1) FP32 field, nothing between; "
                    "ours: one whole mechanical CG iteration (R2C with C_T:p and the curvature, y, z with "
                    "G*, y, C2R with the CG step and (r, r)) timed through rve_op_cg"}
    r.close()

    # -------- plain FP64 GPU form on the same increments, each from the mixed
    # run's converged state before it
    if samples:
        r3 = pkg.RVE(cfg, precision=pkg.RVE_FP64, stream=stream)
        schedule64 = tune_schedule(pkg, r3.h, args)
        pkg.rve_set_graphs(r3.h, True)
        r3.step()                                                     # kernels loaded, graphs captured
        t64, vi64, tm, vim, errs, rows = 0.0, 0.0, 0.0, 0.0, [], []
        for i in samples:
            pkg.rve_load_state(r3.h, start_state if i == 0 else snaps[i])
            a, b = _events(2)
            torch.cuda.synchronize()
            a.record(stream)
            inf = r3.step()
            b.record(stream)
            torch.cuda.synchronize()
            t = a.elapsed_time(b)
            t64 += t
            vi64 += inf["voxel_iterations"]
            tm += incr_ms[i]
            vim += infos[i]["voxel_iterations"]
            errs.append(abs(infos[i]["sigma"][0] - inf["sigma"][0]) / abs(inf["sigma"][0]))
            rows.append({"incr": inf["increment"], "fp64_ms": round(t, 1), "mixed_ms": round(incr_ms[i], 1),
                         "fp64_cg": inf["cg_iters"], "mixed_cg": infos[i]["cg_iters"], "fp64_pcg": inf["pcg_iters"],
                         "mixed_pcg": infos[i]["pcg_iters"], "S11_fp64": inf["sigma"][0],
                         "S11_mixed": infos[i]["sigma"][0], "D_max": inf["D_max"]})
        r3.close()
        for s in snaps.values():
            del s
        v64 = vi64 / (t64 * 1e-3)
        vmix = vim / (tm * 1e-3)
        out["fp64_form"] = {"value": v64, "unit": UNIT, "schedule": schedule64, "increments": rows,
                            "mixed_same_increments": vmix, "mixed_over_fp64": vmix / v64,
                            "time_ratio_fp64_over_mixed": t64 / tm,
                            "sigma11_rel_err_mixed_vs_fp64": max(errs),
                            "how": "each sampled increment solved by both forms from the same converged state "
                                   "(the mixed run's, FP64 image), CUDA events around the increment"}

    # -------- end to end through the public API with host buffers, the same
    # increments: microstructure, load path and the converged state before
    # the timed increments go host -> device inside the timed region
    if not args.no_e2e:
        r2 = pkg.RVE(cfg, precision=prec, stream=stream)
        pkg.rve_set_gamma_tile(r2.h, schedule["gamma_narrow"])                # the timed handle's schedule
        pkg.rve_set_graphs(r2.h, True)
        r2.step()                                                     # kernels loaded
        phase_host = np.ascontiguousarray(cfg.phase)
        barrier(dist)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pkg.rve_set_phases(r2.h, phase_host, cfg.params, cfg.ell)    # H2D of the microstructure
        pkg.rve_set_load_path(r2.h, cfg.strain_ctrl, cfg.target)
        pkg.rve_load_state(r2.h, start_state)                         # H2D of the converged state
        vi2 = 0.0
        s11 = []
        for _ in range(K):
            inf = pkg.rve_step_increment(r2.h)                        # D2H step record
            s11.append(pkg.rve_homogenized_stress(r2.h)[0])           # D2H result
            vi2 += inf["voxel_iterations"]
        torch.cuda.synchronize()
        t2 = time.perf_counter() - t0
        t2 = allreduce(dist, t2, "max")
        vi2 = allreduce(dist, vi2, "sum")
        r2.close()
        h2d = V + 6 * 8 * cfg.target.shape[0] + 64 * len(cfg.params) + 8 * cfg.ell.size + nbytes
        d2h = 208 + 48
        out["e2e"] = {"value": vi2 / t2, "unit": UNIT, "h2d_bytes_per_step": h2d / K,
                      "d2h_bytes_per_step": d2h, "s": t2,
                      "includes": "rve_set_phases(host map) + rve_set_load_path + rve_load_state(host image "
                                  "of the state before increment %d) + the same %d increments + "
                                  "rve_homogenized_stress per step" % (args.warmup + 1, K),
                      "same_S11_as_device_timed": bool(np.allclose(s11, [i["sigma"][0] for i in infos],
                                                                   rtol=1e-12, atol=0))}
    del start_state
    return out, cfg


# ------------------------------------------------------------------ oracle
def cpu_threads():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


class OracleNewtonSample:
    """A bounded sample of the workload on the host with the FP64 oracle as
    it stands: the first Newton iteration of the first increment (the return
    map of every voxel at the initial guess, the residual -G*(sigma -
    Sigma_bar), then mechanical CG iterations of G*(C_T : d eps) = residual),
    at full size.  The FFT library step runs on ``threads`` host threads
    (scipy.fft); the oracle's other numpy steps run on one."""

    def __init__(self, cfg, threads):
        from oracle import rve_oracle as O
        self.O = O
        self.threads = threads
        O.set_fft_workers(threads)
        self.g = O.Grid(cfg.n, cfg.L)
        self.st = O.make_state(self.g, cfg.phase, O.phases_from_dicts(cfg.params), cfg.ell)
        self.cfg = cfg

    def newton_setup(self):
        """Return map and residual; sets the CG operator and right-hand side."""
        O, g, st, cfg = self.O, self.g, self.st, self.cfg
        ctrl_c = cfg.strain_ctrl.astype(float)[O.carried(g.d)]
        self.mask = 1.0 - ctrl_c
        tm = O.to_mandel_target(cfg.target[0])[O.carried(g.d)]
        eps = st.eps + ctrl_c * tm
        rm = O.return_map(O.embed(eps, g.d), st.epsp, st.ep, st.abar, st.phase, st.phases)
        comps = O.carried(g.d)
        sig = rm["sigma"][:, comps].reshape(g.shape + (len(comps),))
        self.C = rm["C"][:, comps][:, :, comps].reshape(g.shape + (len(comps), len(comps)))
        self.res = -O.G_apply(sig - self.mask * tm, g, self.mask)

    def cg(self, iters):
        O, g = self.O, self.g
        O.cg(lambda x: O.G_apply(np.einsum("...ij,...j->...i", self.C, x), g, self.mask), self.res, 1e-30,
             iters)

    def close(self):
        self.O.set_fft_workers(None)


def oracle_sample(cfg, iters, threads):
    """Timed sample: return map + residual + `iters` CG iterations of the
    first Newton iteration.  Returns (voxel-iterations/s, seconds)."""
    smp = OracleNewtonSample(cfg, threads)
    try:
        t0 = time.perf_counter()
        smp.newton_setup()
        smp.cg(iters)
        t = time.perf_counter() - t0
    finally:
        smp.close()
    return smp.g.V * iters / t, t


def run_reference(args, rank, ws, dist):
    """The oracle, as it stands, on the host cores (FFTs on every host
    thread): the timed run is the first Newton iteration of the first
    increment on the full workload, its return map and residual once, then
    one mechanical CG iteration per step."""
    cfg = workload(args.n, args.grid)
    if rank != 0:
        return None, cfg
    th = cpu_threads()
    smp = OracleNewtonSample(cfg, th)
    try:
        smp.newton_setup()
        smp.cg(args.warmup)                      # warm-up (untimed)
        t0 = time.perf_counter()
        smp.newton_setup()
        for _ in range(args.steps):
            smp.cg(1)
        t = time.perf_counter() - t0
    finally:
        smp.close()
    V = smp.g.V
    v = V * args.steps / t
    sample = ("first Newton iteration of increment 1 on the full %s workload: return map + residual "
              "-G*(sigma - Sigma_bar) once, then one FP64 oracle CG iteration per step; FFTs on %d threads "
              "(scipy.fft), other numpy steps on one" % ("x".join(map(str, cfg.n)), th))
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": workload_config(cfg, args.precision),
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": th, "kind": "oracle", "sample": sample,
                            "host_threads": cpu_threads()},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return out, cfg


# ------------------------------------------------------------------ batch
def run_batch(args, rank, ws, dist):
    """The batched workload: 32 two-variable sphere RVEs (grids drawn from
    {64,96,128}^3, volume fractions 10-30 %, seeds 0..31) advanced together
    (one stream, graph-replayed Krylov chunks and one host worker per member,
    autotuned FFT schedules); the same members stepped one at a time with
    direct launches alongside."""
    import torch
    import rve_inputs as I
    import paper_2103_04770_gb300 as pkg

    torch.cuda.init()
    dev = torch.cuda.current_device()
    cfgs = I.config_batch(args.batch_count)
    Vs = [int(np.prod(c.n)) for c in cfgs]
    t0 = time.time()
    b = pkg.RVEBatch(cfgs, precision=pkg.RVE_MIXED, autotune_reps=args.autotune_reps)
    setup_s = time.time() - t0
    for _ in range(args.warmup):
        b.step()
    clocks = ClockSampler()
    if rank == 0:
        clocks.start(dev)
    barrier(dist)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    steps = [b.step() for _ in range(args.steps)]
    e1.record()
    torch.cuda.synchronize()
    ck = clocks.stop() if rank == 0 else None
    ms = e0.elapsed_time(e1)
    vi = sum(V * (inf["cg_iters"] + inf["pcg_iters"]) for infos in steps for V, inf in zip(Vs, infos))
    S11 = [float(m.stress()[0]) for m in b.members]
    b.close()
    ms_max = allreduce(dist, ms, "max")
    vi_sum = allreduce(dist, vi, "sum")
    value = vi_sum / (ms_max * 1e-3)
    out = {"metric": "voxel-iterations/s, batch of %d two-variable sphere RVEs {64,96,128}^3 (mixed)"
                     % len(cfgs),
           "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": "batch%d_spheres2_64-128" % len(cfgs), "members": len(cfgs),
                      "voxels_total": int(sum(Vs)),
                      "grids": {str(N): sum(1 for c in cfgs if c.n[0] == N) for N in I.BATCH_GRIDS},
                      "spheres_per_member": 30, "vf_range": [0.10, 0.30], "seeds": [0, len(cfgs) - 1],
                      "ell_vox": {"matrix": 3.0, "particle": 6.0}, "precision": "mixed",
                      "autotune_reps": args.autotune_reps, "setup_s": round(setup_s, 2),
                      "l2": "inputs larger than L2 (44 M voxels)"},
           "clocks": ck, "S11_last": S11[:4]}
    if not args.no_seq and ws == 1:
        members = [pkg.RVE(c, precision=pkg.RVE_MIXED) for c in cfgs]
        for _ in range(args.warmup):
            for m in members:
                m.step()
        torch.cuda.synchronize()
        e0.record()
        vi_seq = 0
        for _ in range(args.steps):
            for V, m in zip(Vs, members):
                inf = m.step()
                vi_seq += V * (inf["cg_iters"] + inf["pcg_iters"])
        e1.record()
        torch.cuda.synchronize()
        ms_seq = e0.elapsed_time(e1)
        for m in members:
            m.close()
        out["sequential"] = {"value": vi_seq / (ms_seq * 1e-3), "unit": UNIT, "ms_per_step": ms_seq / args.steps,
                             "how": "same members, fresh handles, one at a time on one stream, "
                                    "direct launches, default schedules"}
        out["batch_over_sequential"] = value / out["sequential"]["value"]
    return out


# ------------------------------------------------------------------ adjoint
def run_adjoint(args):
    """The adjoint workload: 96^3, 30 spheres at 20 %, two non-local
    variables, FP64, checkpoint every 5 increments; d<sigma_N>_11 with
    respect to the per-phase parameters, both lengths and the per-voxel
    modulus field, timed, with central-difference checks."""
    import torch
    import rve_inputs as I
    import paper_2103_04770_gb300 as pkg

    torch.cuda.init()
    cfg = I.config_adjoint(n_incr=args.adj_incr)
    V = int(np.prod(cfg.n))
    J = int(cfg.ell.shape[0])
    opt = pkg.rve_default_options(0)
    opt.tol_stag, opt.tol_newton, opt.cg_rtol, opt.pcg_rtol = 1e-10, 1e-11, 1e-12, 1e-12
    opt.max_stag, opt.max_newton, opt.max_cg, opt.max_pcg = 200, 50, 20000, 20000

    def handle(params=None, ell=None):
        h = pkg.rve_create(3, cfg.n, cfg.L, 0, J)
        pkg.rve_set_options(h, opt)
        pkg.rve_set_phases(h, cfg.phase, params or cfg.params, cfg.ell if ell is None else ell)
        pkg.rve_set_load_path(h, cfg.strain_ctrl, cfg.target)
        return h

    h = handle()
    torch.cuda.synchronize()
    t0 = time.time()
    Jv = pkg.rve_adjoint_forward(h, args.adj_every)
    t1 = time.time()
    gp, ge, gs, info = pkg.rve_adjoint_backward(h, 1.0, len(cfg.params), J, V)
    t2 = time.time()
    D = float(pkg.rve_homogenized_stress(h)[0])
    pkg.rve_free(h)
    names = ["sigma_y", "H", "eps_C", "eps_R"]
    grads = {"matrix": dict(zip(names, gp[0].tolist())),
             "particle": {"kappa_C": gp[1][2], "kappa_R": gp[1][3]},
             "ell": ge.tolist(), "stiff_sum": float(gs.sum()), "stiff_absmax": float(np.abs(gs).max())}
    fd = {}
    hrel = 1e-6
    for item in [x for x in args.adj_fd.split(",") if x]:
        def J_of(sign):
            params = [dict(p) for p in cfg.params]
            ell = cfg.ell.copy()
            if item.startswith("ell"):
                j = int(item[3:])
                ell[j] *= 1 + sign * hrel
            else:
                q, k = item.split(":")
                params[int(q)][k] *= 1 + sign * hrel
            hh = handle(params, ell)
            for _ in range(cfg.target.shape[0]):
                pkg.rve_step_increment(hh)
            v = float(pkg.rve_homogenized_stress(hh)[0])
            pkg.rve_free(hh)
            return v
        if item.startswith("ell"):
            j = int(item[3:])
            ref, scale = ge[j], float(cfg.ell[j].max())
        else:
            q, k = item.split(":")
            ref, scale = gp[int(q)][names.index(k)], cfg.params[int(q)][k]
        fdv = (J_of(1) - J_of(-1)) / (2 * hrel * scale)
        fd[item] = {"adjoint": float(ref), "central_difference": fdv, "rel_err": abs(ref - fdv) / abs(fdv)}
    return {"metric": "adjoint gradient of the final <sigma>_11, 96^3 two-variable RVE (FP64)",
            "value": t2 - t0, "unit": "s (forward with checkpoints + reverse sweep)",
            "higher_is_better": False, "n_gpus": 1, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg.name, "grid": list(cfg.n), "spheres": 30,
                       "radius_vox": round(cfg.meta["radius"], 3), "vf": round(cfg.meta["vf_voxel"], 4),
                       "increments": cfg.target.shape[0], "checkpoint_every": args.adj_every,
                       "tolerances": {"stag": opt.tol_stag, "newton": opt.tol_newton, "cg": opt.cg_rtol,
                                      "pcg": opt.pcg_rtol}},
           "J": Jv, "J_after_backward": D, "forward_s": t1 - t0, "backward_s": t2 - t1, "info": info,
           "gradients": grads, "finite_differences": fd}


def run_curve(args):
    """Time to curve: the whole load path of the 256^3 workload (40 increments
    of 1e-3) in the mixed form, each increment through the cut-back step
    (halving on a Newton or staggered budget failure), timed on the device
    from the first increment to the last."""
    import torch
    import paper_2103_04770_gb300 as pkg

    torch.cuda.init()
    stream = torch.cuda.current_stream()
    cfg = workload(args.n, args.grid)
    V = int(np.prod(cfg.n))
    prec = pkg.RVE_MIXED if args.precision == "mixed" else pkg.RVE_FP64
    r = pkg.RVE(cfg, precision=prec, stream=stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    t0 = time.perf_counter()
    curve, vi, status = [], 0.0, "ok"
    n_incr = cfg.target.shape[0] if args.curve_incr <= 0 else min(args.curve_incr, cfg.target.shape[0])
    for i in range(n_incr):
        info = r.step_adaptive(max_cuts=7, raise_on_error=False)
        if info["status"] != pkg.RVE_OK:
            status = pkg.rve_status_string(info["status"])
            break
        vi += info["voxel_iterations"]
        curve.append([round(info["eps"][0], 6), round(info["sigma"][0], 4), round(info["D_max"], 4),
                      info["substeps"], int(info["cg_iters"]), int(info["pcg_iters"])])
        # progress on stderr, so that a run stopped early still leaves its curve
        print(json.dumps({"increment": i + 1, "elapsed_s": round(time.perf_counter() - t0, 3),
                          "point": curve[-1]}), file=sys.stderr, flush=True)
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    s = e0.elapsed_time(e1) * 1e-3
    r.close()
    peak = max(c[1] for c in curve) if curve else None
    return {"metric": "time to curve, 256^3 sphere RVE, %d increments of 1e-3" % n_incr, "value": s, "unit": "s",
            "higher_is_better": False, "n_gpus": 1, "dtype": "f32+f64" if prec == pkg.RVE_MIXED else "f64",
            "data": "synthetic", "config": workload_config(cfg, args.precision), "status": status,
            "increments_done": len(curve), "wall_s": wall, "voxel_iterations": vi,
            "voxel_iterations_per_s": vi / s if s > 0 else None, "peak_S11": peak,
            "curve_columns": ["E11", "S11", "D_max", "substeps", "cg", "pcg"], "curve": curve}


def run_formcurve(args):
    """The sphere RVE's load path (radius 10 voxels, 25 % spheres, l = 4
    voxels, uniaxial E11 in steps of 1e-3) run twice, independently, through
    the cut-back step: once in the mixed form, once in the FP64 form.  At every
    increment the mixed form's Sigma11 is compared with the FP64 form's,
    relative to the FP64 curve's max |Sigma11|; both forms' device times are
    reported (time to curve of each)."""
    import torch
    import paper_2103_04770_gb300 as pkg

    torch.cuda.init()
    stream = torch.cuda.current_stream()
    cfg = workload(args.n, args.grid)
    n_incr = cfg.target.shape[0] if args.curve_incr <= 0 else min(args.curve_incr, cfg.target.shape[0])
    runs = {}
    for name, prec in (("mixed", pkg.RVE_MIXED), ("fp64", pkg.RVE_FP64)):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        curve, status = [], "ok"
        with pkg.RVE(cfg, precision=prec, stream=stream) as r:
            torch.cuda.synchronize()
            e0.record(stream)
            for i in range(n_incr):
                info = r.step_adaptive(max_cuts=7, raise_on_error=False)
                if info["status"] != pkg.RVE_OK:
                    status = "increment %d: %s (%s budget)" % (
                        i + 1, pkg.rve_status_string(info["status"]), FAIL_STAGES.get(info["fail_stage"], "?"))
                    break
                curve.append([round(info["eps"][0], 6), float(info["sigma"][0]), float(info["D_max"]),
                              info["substeps"], int(info["cg_iters"]), int(info["pcg_iters"])])
                print(json.dumps({"form": name, "increment": i + 1, "point": curve[-1]}), file=sys.stderr,
                      flush=True)
            e1.record(stream)
            torch.cuda.synchronize()
        runs[name] = {"curve": curve, "status": status, "device_s": e0.elapsed_time(e1) * 1e-3}
    m, f = runs["mixed"]["curve"], runs["fp64"]["curve"]
    k = min(len(m), len(f))
    smax = max((abs(p[1]) for p in f), default=0.0)
    errs = [abs(m[i][1] - f[i][1]) / smax for i in range(k)] if smax > 0 else []
    return {"metric": "max |Sigma11_mixed - Sigma11_fp64| / max |Sigma11_fp64| over the load path",
            "value": max(errs) if errs else None, "unit": "relative", "higher_is_better": False,
            "n_gpus": 1, "dtype": "f32+f64 vs f64", "data": "synthetic",
            "config": workload_config(cfg, "mixed vs fp64"), "increments_compared": k,
            "within_1e-4": bool(errs) and max(errs) <= 1e-4, "per_increment_rel_err": errs,
            "time_to_curve_s": {n: runs[n]["device_s"] for n in runs},
            "status": {n: runs[n]["status"] for n in runs},
            "curve_columns": ["E11", "S11", "D_max", "substeps", "cg", "pcg"],
            "curves": {n: runs[n]["curve"] for n in runs}}


FAIL_STAGES = {0: "none", 1: "Newton", 2: "CG", 3: "PCG", 4: "staggered", 5: "numeric"}


def run_objectivity(args):
    """Mesh objectivity of the 2D single-particle cell: the FP64 GPU form
    runs the load path (uniaxial E11 in steps of 1e-3) at 128^2, 256^2 and
    512^2 with the length fixed in physical units (l = L/16), each increment
    through the cut-back step (on the finer grids Newton needs sub-steps where
    plasticity spreads from the particle), until the end of the path or the
    first increment that cannot be converged.  Past the peak of the 512^2 curve, the softening branches of the
    coarser grids are compared with it: the largest |Sigma11(E) - Sigma11_512(E)|
    over the common increments, relative to the 512^2 peak."""
    import torch
    import rve_inputs as I
    import paper_2103_04770_gb300 as pkg

    torch.cuda.init()
    curves = {}
    for N in args.obj_grids:
        cfg = I.config_mesh_objectivity(N, n_incr=args.obj_incr)
        opt = pkg.rve_default_options(0)
        opt.max_stag = 1000
        opt.max_cg = args.obj_max_cg
        t0 = time.perf_counter()
        pts, status = [], "end of path"
        with pkg.RVE(cfg, precision=0, options=opt) as r:
            for i in range(cfg.target.shape[0]):
                info = r.step_adaptive(max_cuts=7, raise_on_error=False)
                if info["status"] != pkg.RVE_OK:
                    status = "increment %d: %s (%s budget)" % (
                        i + 1, pkg.rve_status_string(info["status"]), FAIL_STAGES.get(info["fail_stage"], "?"))
                    break
                pts.append([round(info["eps"][0], 6), info["sigma"][0], info["D_max"], info["staggered_iters"],
                            info["substeps"]])
                print(json.dumps({"N": N, "increment": i + 1, "S11": info["sigma"][0], "D_max": info["D_max"],
                                  "stag": info["staggered_iters"], "substeps": info["substeps"],
                                  "newton": info["newton_iters"], "cg": info["cg_iters"],
                                  "pcg": info["pcg_iters"]}), file=sys.stderr, flush=True)
        curves[N] = {"curve": pts, "status": status, "seconds": round(time.perf_counter() - t0, 1)}
    ref_N = max(curves)
    ref = np.array([p[1] for p in curves[ref_N]["curve"]])
    ipk = int(np.argmax(ref))
    out = {}
    for N, c in curves.items():
        if N == ref_N:
            continue
        s = np.array([p[1] for p in c["curve"]])
        m = min(len(s), len(ref))
        post = range(ipk, m)
        dev = max((abs(s[i] - ref[i]) for i in post), default=None)
        out[str(N)] = {"increments_compared_past_peak": len(post),
                       "max_rel_dev_past_peak": None if dev is None else dev / ref[ipk],
                       "within_3_percent": None if dev is None else bool(dev / ref[ipk] <= 0.03)}
    return {"metric": "mesh objectivity of the softening branch, 2D single particle, l = L/16",
            "value": max((v["max_rel_dev_past_peak"] for v in out.values()
                          if v["max_rel_dev_past_peak"] is not None), default=None),
            "unit": "max |Sigma11 - Sigma11_%d| / peak past the %d^2 peak" % (ref_N, ref_N),
            "higher_is_better": False, "n_gpus": 1, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "2d_disc_objectivity", "grids": list(curves), "ell": "L/16",
                       "load": "uniaxial E11 steps of 1e-3, Sigma22 = Sigma12 = 0, plane strain",
                       "options": "production FP64 (tol 1e-6), staggered budget 1000, CG budget %d per Newton step, "
                                  "cut-back step (max 7 halvings)" % args.obj_max_cg},
            "peak_increment_%d" % ref_N: ipk + 1, "comparison": out,
            "curve_columns": ["E11", "S11", "D_max", "staggered", "substeps"],
            "curves": {str(N): c for N, c in curves.items()}}


def _run_curve_cfg(pkg, cfg, precision, budget_s, max_cuts=6, tag=None):
    """The load path of cfg through the cut-back step, until its end, the
    first failure or the wall-clock budget; returns the curve and why it
    stopped."""
    opt = pkg.rve_default_options(precision)
    opt.max_stag = 200
    pts, status = [], "end of path"
    t0 = time.perf_counter()
    with pkg.RVE(cfg, precision=precision, options=opt) as r:
        for i in range(cfg.target.shape[0]):
            info = r.step_adaptive(max_cuts=max_cuts, raise_on_error=False)
            if info["status"] != pkg.RVE_OK:
                status = "increment %d: %s (%s budget)" % (
                    i + 1, pkg.rve_status_string(info["status"]), FAIL_STAGES.get(info["fail_stage"], "?"))
                break
            pts.append([round(info["eps"][0], 6), round(info["sigma"][0], 5), round(info["D_max"], 5),
                        info["substeps"]])
            print(json.dumps({"curve": tag or cfg.name, "increment": i + 1, "point": pts[-1]}), file=sys.stderr,
                  flush=True)
            if time.perf_counter() - t0 > budget_s:
                status = "wall-clock budget of %d s after increment %d" % (budget_s, i + 1)
                break
    return {"curve": pts, "status": status, "seconds": round(time.perf_counter() - t0, 1)}


def _curve_summary(c):
    """Peak stress, strain at the peak, and the strain at which the stress
    has fallen to 80 % of the peak (ductility; None if not reached)."""
    if not c["curve"]:
        return {}
    E = [p[0] for p in c["curve"]]
    S = [p[1] for p in c["curve"]]
    ip = int(np.argmax(S))
    e80 = next((E[i] for i in range(ip, len(S)) if S[i] <= 0.8 * S[ip]), None)
    return {"peak_S11": S[ip], "E11_at_peak": E[ip], "E11_at_80pct_past_peak": e80, "last_E11": E[-1],
            "max_D": max(p[2] for p in c["curve"])}


def run_studies2d(args):
    """The 2D studies of Section 4.1 with the paper's parameters: grid
    sensitivity of the local and non-local Lemaitre and GTN models on
    32^2 / 64^2 / 128^2 (Section 4.1.1), the matrix length l_M in {0.025, 0.05,
    0.075} L on 128^2 (Section 4.1.2), and the non-local plastic strain across
    the interface for l_M / l_I in {1, 5, 10, 20, 50} (one Helmholtz solve per
    ratio on the plastic strain field of the non-local Lemaitre run).  The
    paper's curves exist only as figures, so these runs report behaviour: the
    spread between resolutions of the non-local curves against the local ones,
    ductility against l_M, and how far abar reaches into the inclusion."""
    import torch
    import rve_inputs as I
    import paper_2103_04770_gb300 as pkg

    torch.cuda.init()
    out = {"grid_sensitivity": {}, "length_effect": {}, "interface_profile": {}}
    n_incr = int(round(args.study_emax / args.study_de))
    for model in args.study_models:
        for local in (False, True):
            key = "%s_%s" % (model, "local" if local else "nonlocal")
            curves = {}
            for N in (32, 64, 128):
                cfg = I.config_paper2d(N, model, local, n_incr=n_incr, dE=args.study_de)
                curves[N] = _run_curve_cfg(pkg, cfg, 0, args.study_budget_s, tag=cfg.name)
                curves[N]["summary"] = _curve_summary(curves[N])
            # largest stress difference to the 128^2 curve over the common increments
            ref = [p[1] for p in curves[128]["curve"]]
            spread = {}
            for N in (32, 64):
                s = [p[1] for p in curves[N]["curve"]]
                m = min(len(s), len(ref))
                spread[str(N)] = max((abs(s[i] - ref[i]) for i in range(m)), default=None)
            out["grid_sensitivity"][key] = {"curves": {str(N): c for N, c in curves.items()},
                                            "max_abs_dS11_vs_128": spread}
    for model in args.study_models:
        for lM in (0.025, 0.05, 0.075):
            cfg = I.config_paper2d(128, model, False, ell_M=lM, n_incr=n_incr, dE=args.study_de)
            c = _run_curve_cfg(pkg, cfg, 0, args.study_budget_s, tag=cfg.name + "_lM%.3f" % lM)
            c["summary"] = _curve_summary(c)
            out["length_effect"]["%s_lM_%.3f" % (model, lM)] = c
    # interface profiles: the plastic strain of the non-local Lemaitre run at
    # its last increment, regularised with l_I = l_M / ratio
    cfg = I.config_paper2d(128, "lemaitre", False, n_incr=n_incr, dE=args.study_de)
    N = 128
    V = N * N
    opt = pkg.rve_default_options(0)
    opt.max_stag = 200
    with pkg.RVE(cfg, precision=0, options=opt) as r:
        for i in range(cfg.target.shape[0]):
            info = r.step_adaptive(max_cuts=6, raise_on_error=False)
            if info["status"] != pkg.RVE_OK:
                break
            if info["eps"][0] >= args.study_profile_e:
                break
        ep = torch.empty(V, device="cuda", dtype=torch.float64)
        pkg.rve_get_field(r.h, 4, ep)
        E_at = info["eps"][0]
    phase = torch.as_tensor(cfg.phase.reshape(-1), device="cuda")
    alpha = ep * (phase == 0).to(torch.float64)
    lM = 0.05 * N
    line = N // 2
    inside = (cfg.phase.reshape(N, N)[line] == 1)
    for ratio in (1, 5, 10, 20, 50):
        h = pkg.rve_create(2, cfg.n, cfg.L, 0, 1)
        try:
            pkg.rve_set_phases(h, cfg.phase, cfg.params, np.array([[lM, lM / ratio]]))
            abar = torch.empty(V, device="cuda", dtype=torch.float64)
            it = pkg.rve_op_helmholtz_solve(h, 0, alpha, abar, 1e-12, 5000)
            prof = abar.cpu().numpy().reshape(N, N)[line]
            a_in = prof[inside]
            out["interface_profile"]["ratio_%d" % ratio] = {
                "pcg_iterations": it, "profile_along_x1": [round(float(x), 7) for x in prof],
                "max_abar_inside_over_max": float(a_in.max() / prof.max()) if prof.max() > 0 else None,
                "mean_abar_inside_over_mean_matrix": float(a_in.mean() / prof[~inside].mean())}
        finally:
            pkg.rve_free(h)
    out["interface_profile"]["E11"] = E_at
    return {"metric": "2D parameter studies of Section 4.1 (grid sensitivity, l_M effect, interface profiles)",
            "value": None, "unit": "curves", "n_gpus": 1, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "paper2d_studies", "models": args.study_models, "E11_max": args.study_emax,
                       "dE11": args.study_de, "steps": "cut-back steps, at most 6 halvings",
                       "budget_s_per_curve": args.study_budget_s,
                       "materials": "Section 4.1 parameters (rve_inputs PAPER2D_*)"},
            "results": out}


def run_topology3d(args):
    """Convergence for a fixed topology (Section 4.2): the 30-sphere, 20 %
    RVE generated on 32^3 and replicated to 64^3 and 96^3 voxels, non-local
    Lemaitre (the paper's 3D parameters), mixed form, uniaxial tension; the
    curves at the three resolutions and their largest stress differences."""
    import torch
    import rve_inputs as I
    import paper_2103_04770_gb300 as pkg

    torch.cuda.init()
    n_incr = int(round(args.study_emax / args.study_de))
    curves = {}
    for f in (1, 2, 3):
        cfg = I.config_fixed_topology(f, model=args.topology_model, n_incr=n_incr, dE=args.study_de)
        curves[cfg.n[0]] = _run_curve_cfg(pkg, cfg, 1, args.study_budget_s, tag=cfg.name)
        curves[cfg.n[0]]["summary"] = _curve_summary(curves[cfg.n[0]])
        curves[cfg.n[0]]["sha256_base"] = cfg.meta["sha256_base"][:16]
    ref = [p[1] for p in curves[96]["curve"]]
    diff = {}
    for N in (32, 64):
        s = [p[1] for p in curves[N]["curve"]]
        m = min(len(s), len(ref))
        diff[str(N)] = max((abs(s[i] - ref[i]) / max(ref) for i in range(m)), default=None)
    return {"metric": "fixed-topology refinement (Section 4.2): 32^3 geometry on 32^3 / 64^3 / 96^3",
            "value": diff.get("64"), "unit": "max |Sigma11 - Sigma11_96| / peak, 64^3 curve",
            "higher_is_better": False, "n_gpus": 1, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "fixed_topology_3d", "model": args.topology_model, "E11_max": args.study_emax,
                       "dE11": args.study_de, "spheres": 30, "vf": 0.2, "l_M": "0.05 L", "l_I": "0.001 L"},
            "max_rel_dS11_vs_96": diff, "curves": {str(N): c for N, c in curves.items()}}


def main():
    args = parse()
    rank, ws, dist = dist_init()
    if args.workload in ("studies2d", "topology3d") and args.impl == "ours":
        if rank == 0:
            print(json.dumps(run_studies2d(args) if args.workload == "studies2d" else run_topology3d(args)))
        return
    if args.workload == "objectivity" and args.impl == "ours":
        if rank == 0:
            print(json.dumps(run_objectivity(args)))
        return
    if args.workload == "formcurve" and args.impl == "ours":
        if rank == 0:
            print(json.dumps(run_formcurve(args)))
        return
    if args.curve and args.impl == "ours":
        if rank == 0:
            print(json.dumps(run_curve(args)))
        return
    if args.workload == "adjoint" and args.impl == "ours":
        if rank == 0:
            print(json.dumps(run_adjoint(args)))
        return
    if args.workload == "batch" and args.impl == "ours":
        out = run_batch(args, rank, ws, dist)
        if rank == 0:
            print(json.dumps(out))
        if dist is not None:
            dist.destroy_process_group()
        return
    if args.impl == "reference":
        out, _ = run_reference(args, rank, ws, dist)
        if rank == 0:
            print(json.dumps(out))
        if dist is not None:
            dist.destroy_process_group()
        return
    out, cfg = run_ours(args, rank, ws, dist)
    if rank == 0:
        if not args.no_cpu and ws == 1:
            th = cpu_threads()
            v, t = oracle_sample(cfg, args.cpu_iters, th)
            out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": th, "kind": "oracle",
                                   "sample": "first Newton iteration of increment 1 on the full %s workload: "
                                             "return map + residual + %d FP64 oracle CG iteration(s), all "
                                             "timed (%.1f s); FFTs on %d threads (scipy.fft), other numpy "
                                             "steps on one" % ("x".join(map(str, cfg.n)), args.cpu_iters, t, th),
                                   "host_threads": cpu_threads()}
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
