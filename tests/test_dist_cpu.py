"""The multi-process (replica) path of bench.py on CPU: world_size 2 over
gloo -- process-group set-up from the launcher's environment, barrier,
max-over-ranks timing, and per-rank query batches -- and the reference
arm's JSON line (the FP64 oracle on a small sample)."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_setup(None)
    assert (w, r) == (world, rank)
    bench.barrier(w)
    m = bench.max_over_ranks(w, float(10 * (rank + 1)))
    q = bench.rank_queries(5000, 16, rank)
    out.put((rank, m, q.tolist()))
    dist.destroy_process_group()


def test_two_rank_replicas_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(out.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [m for _, m, _ in res] == [20.0, 20.0]
    assert set(res[0][2]).isdisjoint(res[1][2]) or res[0][2] != res[1][2]


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--scale", "0.005", "--steps", "1", "--warmup", "1"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    assert line["impl"] == "reference"
    for k in ("metric", "value", "unit", "ms_per_step", "cpu_baseline", "e2e", "config"):
        assert k in line
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["value"] > 0


def test_all_cores_oracle_helper():
    """The CPU baseline's all-cores leg: the oracle run once per query
    column in spawned processes over a shared-memory copy of the graph,
    timed; the shared segments are released afterwards."""
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_1912_06525_gb300 import synth
    g = synth.erdos_renyi(3000, 0.003, seed=2)
    W = oracle.adjacency(g.n, g.rowptr, g.col, g.val)
    beta = 0.5 / oracle.lambda_max(W)
    before = set(os.listdir("/dev/shm"))
    qs = np.array([1, 7, 11])
    dt, Ka = bench.oracle_all_cores(g, beta, qs, 1e-10, 2)
    assert dt > 0 and Ka.shape == (g.n, 3)
    assert set(os.listdir("/dev/shm")) - before == set()
    # the vectors the workers kept are the oracle's own solves of those columns
    Kd = oracle.katz_direct(W, beta, qs)
    assert oracle.error_inf_rel(Ka, Kd).max() < 1e-8
    # top-20 agreement of a list with itself is 1; with a planted swap of a
    # clear winner for a poor candidate it drops
    ids, _ = oracle.linkpred_topk(W, Kd, qs, 20)
    assert bench.topk_agreement(g, Kd, qs, ids) == 1.0
    bad = ids.copy()
    order = np.argsort(Kd[:, 0])
    worst = [int(x) for x in order if x not in set(ids[0]) and x != qs[0]][0]
    bad[0, 0] = worst
    assert bench.topk_agreement(g, Kd, qs, bad) == 2 / 3
    info = bench.host_cpu()
    assert info["nproc"] >= 1 and info["model"]


def test_ncu_traffic_only_on_the_captured_workload(monkeypatch):
    """The bench line's roofline traffic (ncu DRAM bytes per launch) is
    given for the default n = 4M unit-weight run only; a variant such as
    BF16 dyadic weights, another damping or a smaller batch reports null."""
    sys.path.insert(0, ROOT)
    import bench

    def args_of(*argv):
        monkeypatch.setattr(sys, "argv", ["bench.py", *argv])
        return bench.parse()

    assert bench.traffic_measured_on(args_of())
    assert bench.traffic_measured_on(args_of("--steps", "20", "--warmup", "5", "--c", "0.9"))
    for variant in (["--weights", "dyadic"], ["--c", "0.5"], ["--paper-beta"],
                    ["--batch", "256"], ["--scale", "0.1"], ["--workload", "2"],
                    ["--method", "cg"], ["--cheb", "bf16"], ["--standin", "gowalla"],
                    ["--multi"], ["--rank", "64"]):
        assert not bench.traffic_measured_on(args_of(*variant)), variant
