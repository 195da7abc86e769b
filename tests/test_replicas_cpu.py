"""The multi-process path of bench.py on CPU (gloo, world size 2): a single
RVE does not shard, so N ranks run independent replicas and the job rate is
the ranks' work summed over the slowest rank's time; the reference arm runs
on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    r, w, dist = bench.dist_init()
    assert (r, w) == (rank, ws) and dist.get_backend() == "gloo"
    ms = [30.0, 50.0][rank]          # per-rank timed region
    work = [1.0e6, 3.0e6][rank]      # per-rank voxel-iterations
    bench.barrier(dist)
    rate, ms_max = bench.aggregate(dist, ms, work)
    out.put((rank, rate, ms_max))
    dist.destroy_process_group()


@pytest.mark.skipif(torch.cuda.is_available(), reason="CPU test of the gloo path")
def test_replica_aggregation_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, ms_max in res:
        assert ms_max == 50.0
        assert rate == pytest.approx(4.0e6 / 0.050)


@pytest.mark.skipif(torch.cuda.is_available(), reason="CPU test of the gloo path")
def test_reference_arm_under_two_ranks_prints_once():
    """torchrun with two ranks: rank 0 times the oracle and prints one JSON
    line with impl = reference; rank 1 exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--grid", "16,16,16", "--steps", "1", "--warmup", "1"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
