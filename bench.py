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
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--curve", action="store_true",
                    help="time the whole load path (cut-back steps) instead of the headline rate")
    ap.add_argument("--curve-incr", type=int, default=0, help="--curve: first K increments only (0: all)")
    ap.add_argument("--cpu-iters", type=int, default=1)
    ap.add_argument("--workload", default="spheres256", choices=["spheres256", "batch", "adjoint"],
                    help="batch: the 32-RVE {64,96,128}^3 two-variable workload; adjoint: gradients of "
                         "the final stress of the 96^3 two-variable RVE (each its own JSON line)")
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


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the mixed-form kernel class, from one ncu full capture on the 256x128x256
# sphere RVE (profiles/x1_cg_and_gamma_tma_passes_3d_spheres_256x128x256_mixed.md),
# per voxel of that grid: the traffic grows in proportion to the voxels, so a
# launch on V voxels moves V times this.  Valid for the kernels as captured.
DRAM_BYTES_PER_VOXEL = {
    "x1_inv_matvec": (830.541824e6 + 360.079360e6) / (256 * 128 * 256),   # k_xinv<EpiCG>
    "x1_fwd_tangent": (475.303936e6 + 364.743680e6) / (256 * 128 * 256),  # k_xfwd<ProTangent>
    "gamma_last_axis": (226.528512e6 + 161.263360e6) / (256 * 128 * 256),  # k_gamma_tma
}


# ------------------------------------------------------------------ ours
def run_ours(args, rank, ws, dist):
    import torch
    import paper_2103_04770_gb300 as pkg

    torch.cuda.init()
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()
    cfg = workload(args.n, args.grid)
    V = int(np.prod(cfg.n))
    prec = pkg.RVE_MIXED if args.precision == "mixed" else pkg.RVE_FP64

    # -------- device-resident timing
    r = pkg.RVE(cfg, precision=prec, stream=stream)
    for _ in range(args.warmup):
        r.step()
    pkg.rve_profile_reset(r.h)
    pkg.rve_profile(r.h, True)
    clocks = ClockSampler()
    if rank == 0:
        clocks.start(dev)
    barrier(dist)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = [r.step() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    ck = clocks.stop() if rank == 0 else None
    ms = e0.elapsed_time(e1)
    prof = pkg.rve_profile_read(r.h)
    pkg.rve_profile(r.h, False)
    vi = sum(i["voxel_iterations"] for i in infos)
    rate, ms_max = aggregate(dist, ms, vi)
    r.close()

    # -------- roofline of the dominant kernel class (live CUDA events)
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
    # DRAM bytes per launch scaled from the smaller capture (3D, mixed form
    # and the six-component kernels only)
    traffic = None
    if dom in DRAM_BYTES_PER_VOXEL and prec == pkg.RVE_MIXED and len(cfg.n) == 3:
        traffic = round(DRAM_BYTES_PER_VOXEL[dom] * V)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_source": peak_src,
                "traffic": traffic, "bytes_per_launch": dbytes / max(dlaunch, 1),
                "avg_launch_ms": dms / max(dlaunch, 1), "launches": dlaunch,
                "classes": {k: {"ms": round(v[0], 3), "launches": v[1],
                                "GBps": round(v[2] / (v[0] * 1e-3) / 1e9, 1) if v[0] > 0 else None}
                            for k, v in prof.items() if v[1] > 0}}
    gpu_launches = int(sum(v[1] for v in prof.values()))

    out = {"metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64" if prec == pkg.RVE_MIXED else "f64", "data": "synthetic",
           "config": workload_config(cfg, args.precision), "roofline": roofline,
           "gpu_launches": gpu_launches, "clocks": ck,
           "increments": [{"incr": i["increment"], "stag": i["staggered_iters"], "newton": i["newton_iters"],
                           "cg": i["cg_iters"], "pcg": i["pcg_iters"], "S11": i["sigma"][0],
                           "D_max": i["D_max"]} for i in infos]}

    # -------- end to end through the public API with host buffers
    if not args.no_e2e:
        r2 = pkg.RVE(cfg, precision=prec, stream=stream)
        for _ in range(args.warmup):
            r2.step()
        phase_host = np.ascontiguousarray(cfg.phase)
        barrier(dist)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pkg.rve_set_phases(r2.h, phase_host, cfg.params, cfg.ell)          # H2D of the microstructure
        pkg.rve_set_load_path(r2.h, cfg.strain_ctrl, cfg.target)
        vi2 = 0.0
        for _ in range(args.steps):
            inf = pkg.rve_step_increment(r2.h)                             # D2H step record
            s = pkg.rve_homogenized_stress(r2.h)                           # D2H result
            vi2 += inf["voxel_iterations"]
        torch.cuda.synchronize()
        t2 = time.perf_counter() - t0
        t2 = allreduce(dist, t2, "max")
        vi2 = allreduce(dist, vi2, "sum")
        r2.close()
        h2d = V + 6 * 8 * cfg.target.shape[0] + 64 * len(cfg.params) + 8 * cfg.ell.size
        d2h = 208 + 48
        out["e2e"] = {"value": vi2 / t2, "unit": UNIT, "h2d_bytes_per_step": h2d / args.steps,
                      "d2h_bytes_per_step": d2h, "includes": "rve_set_phases(host map) + "
                      "rve_set_load_path + steps + rve_homogenized_stress per step", "s": t2}

    # -------- plain FP64 GPU form on the same workload
    if not args.no_fp64 and prec == pkg.RVE_MIXED and args.fp64_steps > 0:
        r3 = pkg.RVE(cfg, precision=pkg.RVE_FP64, stream=stream)
        for _ in range(args.warmup):
            r3.step()
        barrier(dist)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        inf3 = [r3.step() for _ in range(args.fp64_steps)]
        f1.record(stream)
        torch.cuda.synchronize()
        ms3 = allreduce(dist, f0.elapsed_time(f1), "max")
        vi3 = allreduce(dist, sum(i["voxel_iterations"] for i in inf3), "sum")
        s64 = [i["sigma"][0] for i in inf3]
        r3.close()
        # homogenised-stress error of the mixed form against the FP64 form on
        # the same increments (the mixed run's increments warmup+1..)
        s_mixed = [i["sigma"][0] for i in infos[:args.fp64_steps]]
        err = max(abs(a - b) for a, b in zip(s_mixed, s64)) / max(abs(x) for x in s64)
        out["fp64_form"] = {"value": vi3 / (ms3 * 1e-3), "unit": UNIT, "steps": args.fp64_steps,
                            "ms_per_step": ms3 / args.fp64_steps,
                            "mixed_over_fp64": out["value"] / (vi3 / (ms3 * 1e-3)),
                            "sigma11_rel_err_mixed_vs_fp64": err}
    return out, cfg


# ------------------------------------------------------------------ oracle
def oracle_sample(cfg, iters):
    """Bounded sample of the same workload on the host with the FP64 oracle:
    the first increment's return map and residual, then `iters` mechanical
    CG iterations at full size.  Returns (voxel-iterations/s, seconds)."""
    from oracle import rve_oracle as O
    g = O.Grid(cfg.n, cfg.L)
    st = O.make_state(g, cfg.phase, O.phases_from_dicts(cfg.params), cfg.ell)
    ctrl_c = cfg.strain_ctrl.astype(float)
    mask = 1.0 - ctrl_c
    tm = O.to_mandel_target(cfg.target[0])
    eps = (st.eps + ctrl_c * tm).reshape(g.shape + (6,))
    rm = O.return_map(eps.reshape(g.V, 6), st.epsp, st.ep, st.abar, st.phase, st.phases)
    sig = rm["sigma"].reshape(g.shape + (6,))
    C = rm["C"].reshape(g.shape + (6, 6))
    res = -O.G_apply(sig - mask * tm, g, mask)
    t0 = time.perf_counter()
    O.cg(lambda x: O.G_apply(np.einsum("...ij,...j->...i", C, x), g, mask), res, 1e-30, iters)
    t = time.perf_counter() - t0
    return g.V * iters / t, t


def cpu_threads():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def run_reference(args, rank, ws, dist):
    """The oracle, as it stands, on the host cores: each step is one
    mechanical CG iteration of the oracle on the full workload."""
    cfg = workload(args.n, args.grid)
    if rank != 0:
        return None, cfg
    from oracle import rve_oracle as O
    g = O.Grid(cfg.n, cfg.L)
    st = O.make_state(g, cfg.phase, O.phases_from_dicts(cfg.params), cfg.ell)
    ctrl_c = cfg.strain_ctrl.astype(float)
    mask = 1.0 - ctrl_c
    tm = O.to_mandel_target(cfg.target[0])
    eps = (st.eps + ctrl_c * tm).reshape(g.shape + (6,))
    rm = O.return_map(eps.reshape(g.V, 6), st.epsp, st.ep, st.abar, st.phase, st.phases)
    sig = rm["sigma"].reshape(g.shape + (6,))
    C = rm["C"].reshape(g.shape + (6, 6))
    res = -O.G_apply(sig - mask * tm, g, mask)
    A = lambda x: O.G_apply(np.einsum("...ij,...j->...i", C, x), g, mask)  # noqa: E731
    for _ in range(args.warmup):
        O.cg(A, res, 1e-30, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.cg(A, res, 1e-30, 1)
    t = time.perf_counter() - t0
    v = g.V * args.steps / t
    sample = "one FP64 oracle CG iteration (G*(C_T:p) + update) per step on the full 256^3 workload"
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": workload_config(cfg, "fp64 (CPU oracle)"),
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
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


def main():
    args = parse()
    rank, ws, dist = dist_init()
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
            v, t = oracle_sample(cfg, args.cpu_iters)
            out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                   "sample": "%d FP64 oracle CG iteration(s) of the first increment on the "
                                             "full 256^3 workload (%.1f s; numpy FFT, single thread)"
                                             % (args.cpu_iters, t),
                                   "host_threads": cpu_threads()}
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
