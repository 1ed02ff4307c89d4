#!/usr/bin/env python
"""Benchmark: Katz queries/s at 1e-6 relative error on the n=4M modular graph.

One step = one batch of b=1,024 uniformly drawn query nodes answered by
LRC-Katz (``katz_query_batch``: RHS build, M11 solves, couplings, PCG on the
Schur complement with the rank-128 low-rank preconditioner, back-solve,
FP64 iterative refinement to the 1e-6 infinity-norm error bound) followed
by the top-20 link-prediction candidates of every query (``linkpred_topk``).

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Katz queries/sec at 1e-6 rel. error (n=4M); SpMM % of HBM roofline vs plain CG"
UNIT = "queries/s"

# ncu DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch
# of the dominant kernel, keyed by the source hash of the kernel files it was
# measured on (null once they change).  cheb_step: the five launches of one
# query step captured on the same graph recipe at n = 400,000, b = 323
# (12.23 GB of DRAM traffic against 9.48 GB algorithmic, 1.29x: two launches
# without x_{k-1} at 1.15x, three with it at 1.16-1.49x), the ratio applied
# to the full step's 59.3 GB algorithmic per launch (the same five-launch
# mix at n = 4,000,000, b = 1,024).
NCU_TRAFFIC = {("cheb_step", "4ee85f96c8132900"): 76.5e9}


def traffic_measured_on(args):
    """The NCU_TRAFFIC figures hold for the run they were captured on: the
    n = 4M graph's unit-weight pattern at the default damping, batch, rank,
    gathers and method.  Other runs report traffic as null."""
    return (not args.standin and not args.multi and args.workload == 3
            and args.weights == "unit" and args.scale == 1.0 and args.batch == 0
            and args.rank == 0 and args.c in (None, 0.9) and not args.paper_beta
            and args.method == "lrc" and args.gather == "auto" and args.cheb == "auto"
            and args.rhs_coupling == "auto")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=float, default=1.0, help="shrink the workload (tests only)")
    ap.add_argument("--rhs-coupling", default="auto", choices=["auto", "on", "off"],
                    help="store Z = beta M11^-1 W12 for the first Schur right-hand side")
    ap.add_argument("--c", type=float, default=None,
                    help="beta = c / lambda_max (default 0.9 on the n=4M graph, 0.5 on n=1M)")
    ap.add_argument("--paper-beta", action="store_true",
                    help="the paper's damping beta = 1 / (lambda_max + 1) instead of --c")
    ap.add_argument("--method", default="lrc", choices=["lrc", "cg"])
    ap.add_argument("--gather", default="auto",
                    choices=["auto", "register", "pipelined", "rowpipe", "chunked"],
                    help="kernel of the wide fused products (auto: the autotuner's choice)")
    ap.add_argument("--cheb", default="auto", choices=["auto", "f32", "bf16", "mixed"],
                    help="gathers of the large M11 block's Chebyshev steps: auto (the "
                         "library's choice), f32, bf16 (hi plane on every step after the "
                         "first), mixed (hi plane except a closing hi + lo step)")
    ap.add_argument("--batch", type=int, default=0,
                    help="override the query batch width b (small profiling cases)")
    ap.add_argument("--warm", action="store_true",
                    help="the learned warm start instead: train on 50,000 queries of the n=1M "
                         "graph (scaled by --scale), evaluate 4,096 held-out queries cold and warm")
    ap.add_argument("--workload", type=int, default=3, choices=[1, 2, 3],
                    help="3: n=4M modular graph (the metric's workload); 2: n=1M power law")
    ap.add_argument("--standin", default="", choices=[""] + sorted(__import__(
                        "paper_1912_06525_gb300.synth", fromlist=["TABLE1"]).TABLE1),
                    help="a Table 1 stand-in graph instead of the workload (1,000 queries, "
                         "unit weights, beta = 1/(lambda_max+1), r = 25 unless --rank)")
    ap.add_argument("--multi", action="store_true",
                    help="the many-graphs workload instead: 2,048 SBM graphs (n log-uniform in "
                         "[500, 50,000], scaled by --scale), beta = 0.95/lambda_max per graph, "
                         "8 queries per graph, per-graph LRC index (ranks 8-32) against CG")
    ap.add_argument("--rank", type=int, default=0,
                    help="rank r of the low-rank correction (0: the workload's, 128 or 64)")
    ap.add_argument("--weights", default="unit", choices=["unit", "dyadic"],
                    help="dyadic: the workload's pattern with symmetric weights k/64 in "
                         "[0.5, 2), stored and streamed as BF16 values")
    ap.add_argument("--rank-sweep", default="", metavar="STANDIN",
                    help="iterations and throughput against the rank r on a Table 1 stand-in: "
                         "Schur PCG iterations of one FP32 solve at a fixed relative residual "
                         "(1e-5), and mixed-precision queries/s at the 1e-6 bound")
    ap.add_argument("--sparse-katz", type=int, default=0, metavar="T",
                    help="also time Sparse-Katz (Algorithm 3) with T landmarks and s = 20")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cg", action="store_true")
    return ap.parse_args()


def values_label(g, stored):
    """What the index stores for the matrix values: unit-weight graphs keep
    the pattern only (every weight 1, exact in any type)."""
    if g.val is None or np.all(np.asarray(g.val) == 1.0):
        return "pattern only (unit weights)"
    return f"{stored} values"


def workload_desc(g, b, c, rank, scale, workload=3):
    if workload == 2:
        desc = (f"Chung-Lu power law n={g.n:,} (exponent 2.1, mean degree 16, cap 20,000), "
                f"{values_label(g, 'FP32')}, b={b} queries, r={rank}, top-1% hubs, "
                f"beta={c:.6g}/lambda_max, tol 1e-6 (inf-norm error bound)")
    else:
        desc = (f"modular SBM n={g.n:,} (512 lognormal communities, degree 20, 5% inter, "
                f"2,000 hubs x ~5,000 edges), {values_label(g, 'BF16')}, b={b} queries, "
                f"r={rank}, beta={c:.6g}/lambda_max, tol 1e-6 (inf-norm error bound)")
    return {
        "workload": desc,
        "n": g.n, "nnz": g.nnz, "global_batch": b, "rank": rank, "c": c, "scale": scale,
        "l2_flush": "inputs larger than L2 (graph 0.6 GB, FP32 n x b block 16 GB)",
    }


# ---------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev), "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------- helpers
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_queries(n, b, rank):
    """Query batch of one replica (ranks draw disjoint seeds)."""
    from paper_1912_06525_gb300 import synth
    return synth.queries(n, b, seed=synth.BASE_SEED + 300 + rank)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# dense TF32 tensor rate relative to BF16 (nominal 1.1 vs 2.25 PFLOP/s)
TF32_PER_BF16 = 1.1 / 2.25
# profiler tags whose algorithmic count is flops, not bytes
FLOP_TAGS = ("tc_gemm_tf32x3",)


def tf32_peak():
    """TF32 dense peak in TFLOP/s: the measured BF16 burst rate times the
    nominal TF32/BF16 ratio, else the fallback BF16 rate times that ratio."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["bf16_tflops"]) * TF32_PER_BF16, "measured bf16 x nominal tf32/bf16"
    return 1900.0 * TF32_PER_BF16, "fallback bf16 x nominal tf32/bf16"


def kernel_hash():
    h = hashlib.sha256()
    for f in ("kernels_vec.cu", "kernels.h", "common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1912_06525_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def host_cpu():
    """The host CPU as the oracle sees it: model (or architecture) and the
    logical cores present (the oracle itself runs on one)."""
    model = ""
    try:  # lscpu names Arm cores (Neoverse-V2 on Grace); /proc/cpuinfo does not
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if not model and key in ("model name", "cpu model", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    import platform
    return {"model": model or platform.machine(), "nproc": os.cpu_count()}


def oracle_sample(g, beta, c, q_sample, tol):
    """FP64 oracle CG (as it stands) on a few query columns; the stopping
    rule is set so the oracle meets the same error bound as the GPU."""
    import oracle
    W = oracle.adjacency(g.n, g.rowptr, g.col, g.val)
    B = beta * W[:, q_sample].toarray()
    ratio = (np.abs(B).max(axis=0) / np.sqrt((B * B).sum(axis=0))).min()
    rtol = tol * (1 - c) * ratio
    t = time.perf_counter()
    K, it = oracle.katz_cg(W, beta, q_sample, rtol=rtol, B=B)
    dt = time.perf_counter() - t
    return K, dt, it, rtol


# The oracle on several query columns at once: one process per column
# (spawned, so safe after CUDA is initialised), each running the oracle's
# CG unchanged on the graph shared read-only through shared memory.
_POOL_W = None


def _pool_attach(specs, n, beta, out_spec=None):
    global _POOL_W
    import scipy.sparse as sp
    from multiprocessing import shared_memory
    arrs, keep = [], []
    for name, shape, dtype in specs:
        m = shared_memory.SharedMemory(name=name)
        keep.append(m)
        arrs.append(np.ndarray(shape, dtype=dtype, buffer=m.buf))
    out = None
    if out_spec is not None:
        m = shared_memory.SharedMemory(name=out_spec[0])
        keep.append(m)
        out = np.ndarray(out_spec[1], dtype=out_spec[2], buffer=m.buf)
    _POOL_W = (sp.csr_matrix((arrs[2], arrs[1], arrs[0]), shape=(n, n)), beta, keep, out)


def _pool_ready(_):
    return _POOL_W is not None


def _pool_solve(args):
    import oracle
    q, rtol, slot = args
    W, beta, _, out = _POOL_W
    # column q of the symmetric W is its row q (an O(degree) slice)
    B = beta * W.getrow(q).toarray().reshape(-1, 1)
    X, it = oracle.katz_cg(W, beta, [q], rtol=rtol, B=B)
    if out is not None and slot >= 0:  # keep the Katz vector for the parity check
        out[:, slot] = X[:, 0]
    return int(it[0])


class OraclePool:
    """`workers` spawned processes, each holding the graph (shared
    read-only through shared memory) and running the oracle's CG on one
    query column per task.  Use as a context manager; solve() returns the
    wall time of one batch of columns solved at once."""

    def __init__(self, g, beta, workers, keep_columns=0):
        self.g, self.beta, self.workers = g, beta, workers
        self.keep = keep_columns  # > 0: solve() keeps up to this many Katz vectors
        self.shms, self.pool, self.columns = [], None, None

    def __enter__(self):
        import multiprocessing as mp
        from multiprocessing import shared_memory
        import oracle
        try:
            W = oracle.adjacency(self.g.n, self.g.rowptr, self.g.col, self.g.val)
            need = sum(a.nbytes for a in (W.indptr, W.indices, W.data))
            need += 8 * self.g.n * self.keep
            st = os.statvfs("/dev/shm")
            if st.f_bavail * st.f_frsize < 1.25 * need:  # a full tmpfs would SIGBUS the writer
                raise RuntimeError(f"/dev/shm has room for less than {need / 1e9:.1f} GB")
            specs = []
            for a in (W.indptr, W.indices, W.data):
                m = shared_memory.SharedMemory(create=True, size=max(1, a.nbytes))
                self.shms.append(m)
                np.ndarray(a.shape, dtype=a.dtype, buffer=m.buf)[:] = a
                specs.append((m.name, a.shape, a.dtype.str))
            out_spec = None
            if self.keep > 0:
                shape = (self.g.n, self.keep)
                m = shared_memory.SharedMemory(create=True, size=8 * self.g.n * self.keep)
                self.shms.append(m)
                self.columns = np.ndarray(shape, dtype=np.float64, buffer=m.buf)
                out_spec = (m.name, shape, np.dtype(np.float64).str)
            # bounded waits: a pool whose workers cannot start would respawn
            # them forever; __exit__ terminates it
            self.pool = mp.get_context("spawn").Pool(
                self.workers, initializer=_pool_attach,
                initargs=(specs, self.g.n, self.beta, out_spec))
            ready = self.pool.map_async(_pool_ready, range(self.workers),
                                        chunksize=1).get(timeout=90)
            if not all(ready):
                raise RuntimeError("oracle workers did not attach the graph")
        except BaseException:
            self.__exit__(None, None, None)
            raise
        return self

    def solve(self, q_sample, rtol):
        """Wall time of the columns q_sample solved at once; with
        keep_columns, column j of self.columns then holds k_{q_sample[j]}."""
        t = time.perf_counter()
        self.pool.map_async(_pool_solve,
                            [(int(q), rtol, j if j < self.keep else -1)
                             for j, q in enumerate(q_sample)],
                            chunksize=1).get(timeout=180)
        return time.perf_counter() - t

    def __exit__(self, *exc):
        if self.pool is not None:
            self.pool.terminate()
            self.pool.join()
            self.pool = None
        self.columns = None
        for m in self.shms:
            m.close()
            m.unlink()
        self.shms = []
        return False


def oracle_all_cores(g, beta, q_sample, rtol, workers):
    """Wall time of the oracle's CG on len(q_sample) columns solved by
    `workers` spawned processes at once (one column each), and the Katz
    vectors they returned (n x len(q_sample))."""
    with OraclePool(g, beta, workers, keep_columns=len(q_sample)) as pool:
        dt = pool.solve(q_sample, rtol)
        return dt, np.array(pool.columns)


def topk_agreement(g, Kref, q_sample, ids_gpu, k=20, band_rel=2e-6):
    """Share of the sampled queries whose GPU top-k list equals the oracle's
    up to exact ties: every oracle candidate scoring more than band_rel *
    ||k_q||_inf above the oracle's k-th score is in the GPU list, and every
    GPU candidate scores within that band of the k-th score or above
    (candidates, q and its neighbours excluded, follow the oracle's
    link-prediction reading of Section 3.3)."""
    import oracle
    W = oracle.adjacency(g.n, g.rowptr, g.col, g.val)
    rid, rsc = oracle.linkpred_topk(W, Kref, q_sample, k)
    ok = 0
    for j, q in enumerate(q_sample):
        band = band_rel * np.abs(Kref[:, j]).max()
        must = set(rid[j][rsc[j] > rsc[j][-1] + band].tolist())
        got = set(int(x) for x in ids_gpu[j])
        excl = set(W.indices[W.indptr[q]:W.indptr[q + 1]].tolist()) | {int(q)}
        cand_ok = all(x >= 0 and x not in excl and Kref[x, j] >= rsc[j][-1] - band
                      for x in got)
        ok += int(must <= got and cand_ok and len(got) == k)
    return ok / max(1, len(q_sample))


# ---------------------------------------------------------------- reference
def run_reference(args, world, rank):
    if rank != 0:
        return
    from paper_1912_06525_gb300 import synth
    import oracle
    g, q, c, r = synth.workload(3, args.scale)
    c = 0.9 if args.c is None else args.c
    W = oracle.adjacency(g.n, g.rowptr, g.col, g.val)
    lam = oracle.lambda_max(W)
    if args.paper_beta:
        c = lam / (lam + 1.0)
    beta = c / lam
    # the stopping rule of one column, as in oracle_sample
    _, dt1, _, rtol = oracle_sample(g, beta, c, q[:1], 1e-6)
    workers = max(1, min(os.cpu_count() or 1, 32))
    times, per_step, sample = [], 1, "1 query of the batch per step on one core"
    try:
        if workers < 2:
            raise RuntimeError("one core")
        with OraclePool(g, beta, workers) as pool:
            for st in range(args.warmup + args.steps):
                j0 = (st * workers) % max(1, len(q) - workers)
                dt = pool.solve(q[j0:j0 + workers], rtol)
                if st >= args.warmup:
                    times.append(dt)
        per_step = workers
        sample = (f"{workers} queries of the batch per step, solved at once, one per process "
                  f"on {workers} cores (1 core: 1 query in {dt1:.1f} s)")
    except Exception:
        times = []
        for st in range(args.warmup + args.steps):
            qs = q[st % len(q): st % len(q) + 1]
            _, dt, it, rtol = oracle_sample(g, beta, c, qs, 1e-6)
            if st >= args.warmup:
                times.append(dt)
    ms = 1000 * float(np.mean(times))
    value = per_step * 1000.0 / ms
    cfg = workload_desc(g, len(q), c, r, args.scale)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": cfg,
           "cpu_baseline": {"kind": "oracle", "cores": per_step, "value": value, "unit": UNIT,
                            "host": host_cpu(),
                            "sample": sample + ", FP64 CG (SciPy CSR) to the same 1e-6 "
                                               "error bound"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- ours
def run_multi(args, world, rank, local):
    """Many graphs of uneven size at once: per-graph LRC (katz_multi_query_lrc)
    timed against the CUDA-graph-replayed CG of the same batch."""
    import torch
    import __graft_entry__
    from paper_1912_06525_gb300 import katz, synth

    __graft_entry__.build()
    torch.cuda.set_device(local)
    count = max(8, int(round(2048 * args.scale)))
    graphs = synth.multi_sbm(count, 500, 50_000, seed=synth.BASE_SEED + 5)
    lams = [katz.katz_lambda_max(g, steps=64) for g in graphs]
    betas = [0.95 / l for l in lams]
    t0 = time.perf_counter()
    m = katz.katz_index_build_many(graphs, betas, value_dtype=katz.KATZ_UNIT,
                                   rank=args.rank or 32, block_max=64)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    n2, ranks, _ = katz.katz_multi_get_info(m)
    qpg = 8
    rng = np.random.default_rng(synth.BASE_SEED + 6 + rank)
    q = np.concatenate([rng.choice(g.n, size=qpg, replace=False) for g in graphs]).astype(np.int32)
    n = sum(g.n for g in graphs)
    nnz = sum(g.nnz for g in graphs)
    qd = torch.from_numpy(q).cuda()
    K = torch.empty((n, qpg), dtype=torch.float32, device="cuda")
    res = {}
    for name, fn in (("lrc", katz.katz_multi_query_lrc), ("cg", katz.katz_multi_query)):
        for _ in range(args.warmup):
            fn(m, qd, qpg, K, tol=1e-6)
        torch.cuda.synchronize()
        barrier(world)
        stream = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        katz.katz_profile_enable(name == "lrc")
        l0 = katz.katz_launch_count()
        e0.record(stream)
        for _ in range(args.steps):
            st, it, rel = fn(m, qd, qpg, K, tol=1e-6)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        ms = max_over_ranks(world, e0.elapsed_time(e1) / args.steps)
        prof = {t: katz.katz_profile_read(t) for t in
                ("spmm_f32", "cheb_step", "ff_residual", "block_solve_f32", "gemm_f32",
                 "tc_gemm")} if name == "lrc" else {}
        katz.katz_profile_enable(False)
        res[name] = {"queries_per_s": world * count * qpg / (ms / 1000), "ms_per_batch": ms,
                     "mean_inner_iters": float(np.mean(it)),
                     "refine_steps": st["refine_steps"], "max_rel_res": st["max_rel_res"],
                     "status": st["status"], "launches": katz.katz_launch_count() - l0,
                     "kernels": {t: {"launches": v["launches"], "ms_per_batch": v["ms"] / args.steps}
                                 for t, v in prof.items() if v["launches"]}}
    if rank == 0:
        out = {"metric": "Katz queries/sec at 1e-6 rel. error, many graphs at once", "unit": UNIT,
               "value": res["lrc"]["queries_per_s"], "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": res["lrc"]["ms_per_batch"],
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f32 (f64-class refinement)", "data": "synthetic",
               "config": {"workload": f"{count} SBM graphs, n log-uniform in [500, 50,000] "
                                      f"(sum n = {n:,}, nnz = {nnz:,}), 4-64 communities, mean "
                                      f"degree 8-32, beta = 0.95/lambda_max per graph, {qpg} "
                                      f"queries per graph, per-graph LRC (ranks "
                                      f"{int(ranks.min())}-{int(ranks.max())}, separator "
                                      f"{int(n2.sum()):,} hubs), tol 1e-6",
                          "graphs": count, "n": n, "nnz": nnz, "index_build_s": build_s},
               "lrc": res["lrc"], "cg": res["cg"]}
        print(json.dumps(out), flush=True)


def run_small(args, world, rank, local):
    """n = 2,000 SBM, FP64 weights, r = 16, 16 queries, LRC and CG to a
    relative residual of 1e-10: latency-bound, so the line reports the time
    per batch (not a roofline fraction)."""
    import torch
    import __graft_entry__
    import oracle
    from paper_1912_06525_gb300 import katz, synth

    __graft_entry__.build()
    torch.cuda.set_device(local)
    g, q, c, r = synth.workload(1)
    lam = katz.katz_lambda_max(g, steps=200)
    beta = c / lam
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F64, rank=r, block_max=64)
    qd = torch.from_numpy(q).cuda()
    K = torch.empty((g.n, len(q)), dtype=torch.float64, device="cuda")
    res = {}
    for name, fn in (("lrc", katz.katz_query_batch), ("cg", katz.cg_query_batch)):
        kw = dict(out_dtype=katz.KATZ_F64, tol=1e-10, tol_kind=katz.KATZ_TOL_RESIDUAL)
        for _ in range(args.warmup):
            fn(idx, qd, K, **kw)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            st, it, rel = fn(idx, qd, K, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(world, e0.elapsed_time(e1) / args.steps)
        W = oracle.adjacency(g.n, g.rowptr, g.col, g.val)
        err = float(oracle.error_inf_rel(K.cpu().numpy(), oracle.katz_direct(W, beta, q)).max())
        res[name] = {"ms_per_batch": ms, "queries_per_s": world * len(q) / (ms / 1000),
                     "mean_iters": float(np.mean(it)), "max_rel_res": st["max_rel_res"],
                     "max_err_vs_oracle": err, "status": st["status"]}
    if rank == 0:
        print(json.dumps({"metric": "Katz query batch latency at rel. residual 1e-10 (n=2,000)",
                          "unit": "ms", "value": res["lrc"]["ms_per_batch"], "n_gpus": world,
                          "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": res["lrc"]["ms_per_batch"], "higher_is_better": False,
                          "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic",
                          "config": {"workload": "SBM n=2,000, 8 communities, mean degree 10, "
                                                 "10% inter, FP64 weights, beta=0.5/lambda_max, "
                                                 "r=16, 16 queries, rel. residual 1e-10",
                                     "n": g.n, "nnz": g.nnz, "global_batch": len(q)},
                          "lrc": res["lrc"], "cg": res["cg"]}), flush=True)


def run_warm(args, world, rank, local):
    """Learned warm start on the n = 1M power-law graph: the network is
    trained on the method's own Katz vectors of 50,000 queries (scaled by
    --scale), then 4,096 held-out queries run cold and warm at 1e-6."""
    import torch
    import __graft_entry__
    from paper_1912_06525_gb300 import katz, synth

    __graft_entry__.build()
    torch.cuda.set_device(local)
    g, _, c, r = synth.workload(4, args.scale)
    lam = katz.katz_lambda_max(g, steps=96)
    beta = c / lam
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F32, rank=r, n_hubs=g.n // 100,
                                block_max=64, split=False)
    rng = np.random.default_rng(synth.BASE_SEED + 44)
    n_train = max(1024, int(50_000 * min(1.0, args.scale)))
    perm = rng.permutation(g.n).astype(np.int32)
    train, test = perm[:n_train], np.sort(perm[n_train:n_train + 4096])
    t0 = time.perf_counter()
    tr = katz.katz_warmstart_train(idx, train, hidden=256, epochs=20, batch=256, lr=1e-3)
    train_s = time.perf_counter() - t0
    b = 1024
    katz.katz_autotune(idx, b)
    res = {}
    for name, fn, warm in (("cold", katz.katz_query_batch, 0),
                           ("warm", katz.katz_query_batch, 1),
                           ("cg_cold", katz.cg_query_batch, 0),
                           ("cg_warm", katz.cg_query_batch, 1)):
        its, ms, fb, ref, gam = [], 0.0, 0, [], []
        for j0 in range(0, len(test), b):
            qd = torch.from_numpy(test[j0:j0 + b]).cuda()
            Kb = torch.empty((g.n, len(qd)), dtype=torch.float32, device="cuda")
            fn(idx, qd, Kb, tol=1e-6, warm_start=warm)  # untimed
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(torch.cuda.current_stream())
            st, it, rel = fn(idx, qd, Kb, tol=1e-6, warm_start=warm)
            e1.record(torch.cuda.current_stream())
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            its.extend(it.tolist())
            fb += int(st["ms"][5])
            ref.append(st["refine_steps"])
            gam.append(st["ms"][6])
        res[name] = {"queries_per_s": len(test) / (ms / 1000), "ms": ms,
                     ("mean_pcg_iters" if fn is katz.katz_query_batch else "mean_cg_iters"):
                         float(np.mean(its)),
                     "warm_fallbacks": fb, "refine_steps": ref,
                     **({"mean_gamma": float(np.mean(gam))}
                        if fn is katz.cg_query_batch and warm else {})}
    if rank == 0:
        print(json.dumps({"metric": "Katz queries/sec at 1e-6 rel. error, warm vs cold start",
                          "unit": UNIT, "value": res["warm"]["queries_per_s"], "n_gpus": world,
                          "steps": 1, "warmup": 1, "ms_per_step": res["warm"]["ms"],
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                          "dtype": "f32 (bf16 network)", "data": "synthetic",
                          "config": {"workload": f"Chung-Lu n={g.n:,} (exponent 2.1, mean degree "
                                                 f"16), r={r}, network 32-256-{r} (GELU), "
                                                 f"{n_train:,} training queries, 4,096 held out",
                                     "n": g.n, "train_s": train_s,
                                     "train_loss": [tr["initial_loss"], tr["final_loss"]]},
                          "cold": res["cold"], "warm": res["warm"],
                          "cg_cold": res["cg_cold"], "cg_warm": res["cg_warm"]}), flush=True)


def run_rank_sweep(args, world, rank, local):
    """Iterations and throughput against the rank r of the correction
    (the analogue of the paper's Figs. 3-4) on a Table 1 stand-in, in the
    paper's setting (beta = 1/(lambda_max + 1), top-1% hubs): for each r the
    mean Schur PCG iterations of one FP32 solve stopped at relative residual
    1e-5 (a fixed inner tolerance, so the count reflects the preconditioner),
    plain CG's iterations at the same tolerance, the mixed-precision
    queries/s at the 1e-6 bound, and the index's device bytes."""
    import torch
    import __graft_entry__
    from paper_1912_06525_gb300 import katz, synth

    __graft_entry__.build()
    torch.cuda.set_device(local)
    g = synth.table1_standin(args.rank_sweep, args.scale)
    q = synth.queries(g.n, min(1000, g.n), seed=synth.BASE_SEED + 55)
    lam = katz.katz_lambda_max(g, steps=96)
    beta = 1.0 / (lam + 1.0)
    qd = torch.from_numpy(q).cuda()
    K = torch.empty((g.n, len(q)), dtype=torch.float32, device="cuda")
    rows, cg_it = [], None
    for r in (0, 5, 10, 15, 20, 25, 50, 100):
        idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_UNIT, rank=r,
                                    n_hubs=g.n // 100, block_max=64, split=False)
        katz.katz_autotune(idx, len(q))
        st, it, _ = katz.katz_query_batch(idx, qd, K, tol=1e-5, tol_kind=katz.KATZ_TOL_RESIDUAL,
                                          precision=katz.KATZ_PREC_F32)
        if cg_it is None:
            _, itc, _ = katz.cg_query_batch(idx, qd, K, tol=1e-5,
                                            tol_kind=katz.KATZ_TOL_RESIDUAL,
                                            precision=katz.KATZ_PREC_F32)
            cg_it = float(np.mean(itc))
        for _ in range(2):
            katz.katz_query_batch(idx, qd, K, tol=1e-6)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(torch.cuda.current_stream())
        for _ in range(3):
            stm, itm, _ = katz.katz_query_batch(idx, qd, K, tol=1e-6)
        e1.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        info = idx.info()
        rows.append({"rank": info["rank"], "pcg_iters_fixed_tol": float(np.mean(it)),
                     "queries_per_s": len(q) / (ms / 1000), "mixed_iters": float(np.mean(itm)),
                     "refine_steps": stm["refine_steps"], "sigma_1": info["lambda_max_R"],
                     "index_device_bytes": info["device_bytes"]})
        del idx
    if rank == 0:
        n0, d0, l0 = synth.TABLE1[args.rank_sweep]
        print(json.dumps({"metric": "Schur PCG iterations against the rank r (fixed inner "
                                    "tolerance 1e-5)", "unit": "iterations",
                          "value": rows[-1]["pcg_iters_fixed_tol"], "n_gpus": world,
                          "higher_is_better": False, "data": "synthetic",
                          "config": {"workload": f"stand-in for {args.rank_sweep} (n={g.n:,}, "
                                                 f"nnz={g.nnz:,}, lambda_max={lam:.1f}), "
                                                 f"beta=1/(lambda_max+1), top-1% hubs, "
                                                 f"{len(q)} queries"},
                          "cg_iters_fixed_tol": cg_it, "sweep": rows}), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl != "reference" and args.workload == 1:
        run_small(args, world, rank, local)
        return
    if args.impl != "reference" and args.warm:
        run_warm(args, world, rank, local)
        return
    if args.impl != "reference" and args.rank_sweep:
        run_rank_sweep(args, world, rank, local)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.multi:
        run_multi(args, world, rank, local)
        return
    import torch
    import __graft_entry__
    from paper_1912_06525_gb300 import katz, synth

    __graft_entry__.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    if args.standin:  # Section 4's setting on a Table 1 stand-in
        g = synth.table1_standin(args.standin, args.scale)
        q = synth.queries(g.n, min(1000, g.n), seed=synth.BASE_SEED + 55)
        c, rank_r = 0.5, 25
        args.paper_beta = True
    else:
        g, q, c, rank_r = synth.workload(args.workload, args.scale)
        c = args.c if args.c is not None else (0.9 if args.workload == 3 else 0.5)
        if args.weights == "dyadic":
            g = synth.with_dyadic_weights(g, synth.BASE_SEED + 9)
    if args.rank > 0:
        rank_r = args.rank
    if args.batch > 0:
        q = synth.queries(g.n, args.batch, seed=synth.BASE_SEED + 77)
    b = len(q)
    if world > 1:  # replicas: each rank answers its own batch
        q = rank_queries(g.n, b, rank)
    t0 = time.perf_counter()
    lam = katz.katz_lambda_max(g, steps=96)
    if args.paper_beta:  # Section 4: beta = 1 / (||W||_2 + 1)
        c = lam / (lam + 1.0)
    beta = c / lam
    rc = {"auto": 0, "on": 1, "off": -1}[args.rhs_coupling]
    if args.standin:  # unit weights; top-1% hubs, the rest kept whole
        idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_UNIT, rank=rank_r,
                                    n_hubs=g.n // 100, block_max=64, split=False,
                                    rhs_coupling=rc)
    elif args.workload == 3:
        n_hubs = int(g.meta["hubs"].shape[0])
        idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_BF16, rank=rank_r,
                                    n_hubs=n_hubs, block_max=64, split=False, rhs_coupling=rc)
    else:  # power law: top-1% hubs; the rest keeps a giant component, kept whole
        idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F32, rank=rank_r,
                                    n_hubs=g.n // 100, block_max=64, split=False,
                                    rhs_coupling=rc)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    info = idx.info()

    tune = katz.katz_autotune(idx, b)  # SpMM launch shape for this b (untimed)
    qd = torch.from_numpy(q).to(dev)
    K = torch.empty((g.n, b), dtype=torch.float32, device=dev)
    ids = torch.empty((b, 20), dtype=torch.int32, device=dev)
    sc = torch.empty((b, 20), dtype=torch.float64, device=dev)
    qfn = katz.katz_query_batch if args.method == "lrc" else katz.cg_query_batch
    gk = {"auto": katz.KATZ_GATHER_AUTO, "register": katz.KATZ_GATHER_REGISTER,
          "pipelined": katz.KATZ_GATHER_PIPELINED, "rowpipe": katz.KATZ_GATHER_ROWPIPE,
          "chunked": katz.KATZ_GATHER_CHUNKED}[args.gather]
    last = {}

    cg_mode = {"auto": katz.KATZ_CHEB_AUTO, "f32": katz.KATZ_CHEB_F32,
               "bf16": katz.KATZ_CHEB_BF16, "mixed": katz.KATZ_CHEB_MIXED}[args.cheb]
    qkw = {"cheb_gather": cg_mode} if args.method == "lrc" else {}

    def step(qq, KK, ii, ss):
        st, it, rel = qfn(idx, qq, KK, out_dtype=katz.KATZ_F32, tol=1e-6, gather_kernel=gk, **qkw)
        katz.linkpred_topk(idx, qq, KK, katz.KATZ_F32, 20, ii, ss)
        last.update(st=st, it=it, rel=rel)

    for _ in range(args.warmup):
        step(qd, K, ids, sc)
    torch.cuda.synchronize()

    clocks = Clocks(local if world == 1 else local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    l0 = katz.katz_launch_count()
    katz.katz_profile_enable(True)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    for _ in range(args.steps):
        step(qd, K, ids, sc)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier(world)
    launches = katz.katz_launch_count() - l0
    prof = {t: katz.katz_profile_read(t) for t in
            ("spmm_f32", "spmm_f64", "cheb_step", "cheb_step_bf16g", "ff_residual", "ff_out",
             "block_solve_f32", "gemm_f32", "tc_gemm", "tc_gemm_tf32x3", "topk")}
    katz.katz_profile_enable(False)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(world, ms)
    value = world * b / (ms / 1000.0)
    lrc_stats = dict(last["st"])
    lrc_iters = float(np.mean(last["it"]))

    # ---- plain CG on the same batch (the comparison method), timed like the
    # LRC arm: warm-up calls, then CUDA events on the stream over several
    # batches (the same queries, the same 1e-6 error bound)
    cg = None
    if not args.no_cg:
        cg_warm, cg_steps = max(1, min(args.warmup, 3)), max(1, min(args.steps, 5))
        for _ in range(cg_warm):
            katz.cg_query_batch(idx, qd, K, out_dtype=katz.KATZ_F32, tol=1e-6, gather_kernel=gk)
        torch.cuda.synchronize()
        katz.katz_profile_enable(True)
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(cg_steps):
            st_cg, it_cg, rel_cg = katz.cg_query_batch(idx, qd, K, out_dtype=katz.KATZ_F32,
                                                       tol=1e-6, gather_kernel=gk)
        c1.record(stream)
        torch.cuda.synchronize()
        cg_ms = max_over_ranks(world, c0.elapsed_time(c1) / cg_steps)
        pc = katz.katz_profile_read("spmm_f32")
        katz.katz_profile_enable(False)
        hbm, _ = peaks()
        cg = {"queries_per_s": world * b / (cg_ms / 1000), "ms_per_batch": cg_ms,
              "steps": cg_steps, "warmup": cg_warm, "timing": "CUDA events over the steps",
              "mean_iters": float(np.mean(it_cg)), "refine_steps": st_cg["refine_steps"],
              "max_rel_res": st_cg["max_rel_res"], "status": st_cg["status"],
              "lrc_speedup": cg_ms / ms,
              "spmm_f32_gbs": pc["bytes"] / (pc["ms"] / 1e3) / 1e9 if pc["ms"] else None,
              "spmm_f32_frac": (pc["bytes"] / (pc["ms"] / 1e3) / 1e9) / hbm if pc["ms"] else None}
        # restore the LRC answer for the parity sample below
        step(qd, K, ids, sc)

    # ---- Sparse-Katz re-ranking (Algorithm 3): 1 + T solves per query
    sk = None
    if args.sparse_katz > 0:
        T = args.sparse_katz
        sid = torch.empty((b, 20), dtype=torch.int32, device=dev)
        srho = torch.empty((b, 20), dtype=torch.float64, device=dev)
        sland = torch.empty((b, T), dtype=torch.int32, device=dev)
        katz.sparse_katz_topk(idx, qd, 20, T, sid, srho, sland)
        torch.cuda.synchronize()
        e2 = torch.cuda.Event(enable_timing=True)
        e3 = torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        st_sk = katz.sparse_katz_topk(idx, qd, 20, T, sid, srho, sland)
        e3.record(stream)
        torch.cuda.synchronize()
        sk_ms = e2.elapsed_time(e3)
        sk = {"queries_per_s": b / (sk_ms / 1000), "ms_per_batch": sk_ms, "s": 20, "T": T,
              "distinct_landmarks": st_sk["distinct_landmarks"],
              "solves_per_query": 1 + st_sk["distinct_landmarks"] / b, "status": st_sk["status"],
              "max_rel_res": st_sk["max_rel_res"]}

    # ---- end to end through the C-ABI from host queries to host top-k lists:
    # the queries are copied in from pinned host memory, the Katz block stays
    # in device memory, and the link predictions (ids and scores) come back
    e2e = None
    if not args.no_e2e:
        qh = torch.from_numpy(q).pin_memory()
        idh = torch.empty((b, 20), dtype=torch.int32).pin_memory()
        sch = torch.empty((b, 20), dtype=torch.float64).pin_memory()
        n_e2e = max(1, min(args.steps, 3))
        step(qh, K, idh, sch)
        torch.cuda.synchronize()
        barrier(world)
        t = time.perf_counter()
        for _ in range(n_e2e):
            step(qh, K, idh, sch)
        torch.cuda.synchronize()
        barrier(world)
        e2e_ms = max_over_ranks(world, 1000 * (time.perf_counter() - t) / n_e2e)
        e2e = {"value": world * b / (e2e_ms / 1000), "unit": UNIT,
               "h2d_bytes_per_step": int(q.nbytes),
               "d2h_bytes_per_step": int(b * 20 * (4 + 8))}

    # ---- roofline of the dominant kernel; the Chebyshev step's launches
    # (FP32 or hi-plane gathers, the same algorithmic bytes) count as one kernel
    hbm, src = peaks()
    ch = [prof[t] for t in ("cheb_step", "cheb_step_bf16g")]
    prof_dom = {t: v for t, v in prof.items() if not t.startswith("cheb_step")}
    prof_dom["cheb_step"] = {k: sum(v[k] for v in ch) for k in ("launches", "ms", "bytes")}
    shares = {t: p["ms"] for t, p in prof_dom.items() if p["launches"]}
    tot = sum(shares.values()) or 1.0
    dom = max(shares, key=shares.get) if shares else "spmm_f32"
    p = prof_dom[dom]
    ach = p["bytes"] / (p["ms"] / 1e3) / 1e9 if p["ms"] else 0.0
    if dom in FLOP_TAGS:
        tpk, tsrc = tf32_peak()
        ach = p["bytes"] / (p["ms"] / 1e3) / 1e12 if p["ms"] else 0.0
        roof = {"kernel": dom, "bound": "tensor", "achieved": ach, "peak": tpk, "unit": "TFLOP/s",
                "frac": ach / tpk, "peak_source": tsrc, "traffic": None}
    else:
        roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "peak_source": f"{src} (hbm_gbs)",
                "traffic": (NCU_TRAFFIC.get((dom, kernel_hash())) if traffic_measured_on(args)
                            else None), "traffic_unit": "bytes per launch"}
    roof.update({"launches_per_step": p["launches"] / args.steps,
                 "alg_units_per_launch": p["bytes"] / max(1, p["launches"]),
                 "share_of_step": p["ms"] / (ms * args.steps)})
    kernels = {t: {"launches": v["launches"], "ms_per_step": v["ms"] / args.steps,
                   ("tflops" if t in FLOP_TAGS else "gbs"):
                       v["bytes"] / (v["ms"] / 1e3) / (1e12 if t in FLOP_TAGS else 1e9)
                       if v["ms"] else None}
               for t, v in prof.items() if v["launches"]}

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N=1), and
    # parity of the GPU answers on every column the oracle solved: max
    # infinity-norm relative error and top-20 agreement up to exact ties
    cpu = None
    parity = None
    if world == 1 and rank == 0 and not args.no_cpu_baseline:
        ns = 2
        qs = q[:ns]
        Kref, dt, it, rtol = oracle_sample(g, beta, c, qs, 1e-6)
        cols, refs = list(range(ns)), [Kref]
        cpu = {"value": ns / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
               "sample": f"{ns} of the {b} queries, FP64 CG (SciPy CSR, 1 thread) to the same "
                         f"1e-6 error bound (rtol {rtol:.2e}), {dt:.1f} s"}
        # all host cores: one column per process, as many columns as cores
        workers = max(1, min(os.cpu_count() or 1, 32))
        if workers > 1:
            try:
                qa = q[ns:ns + workers]
                dta, Ka = oracle_all_cores(g, beta, qa, rtol, workers)
                cols += list(range(ns, ns + len(qa)))
                refs.append(Ka)
                cpu.update({"value": len(qa) / dta, "cores": workers,
                            "value_1core": ns / dt,
                            "sample": f"{len(qa)} of the {b} queries solved at once, one per "
                                      f"process on {workers} cores, FP64 CG (SciPy CSR) to the "
                                      f"same 1e-6 error bound (rtol {rtol:.2e}), {dta:.1f} s; "
                                      f"1 core: {ns} queries in {dt:.1f} s"})
            except Exception as e:  # keep the single-core number
                cpu["all_cores_error"] = str(e)[:200]
        import oracle
        Kref = np.concatenate(refs, axis=1)
        Kg = K[:, cols].double().cpu().numpy()
        err = oracle.error_inf_rel(Kg, Kref)
        parity = {"columns": len(cols), "max_err_vs_oracle": float(err.max()),
                  "topk_agree": topk_agreement(g, Kref, q[cols], ids[cols].cpu().numpy()),
                  "oracle_bound": "FP64 CG to the same 1e-6 error bound (its own error is "
                                  "at most that bound)"}

    if rank == 0:
        cfg = workload_desc(g, b, c, rank_r, args.scale, args.workload)
        if args.standin:
            n0, d0, l0 = synth.TABLE1[args.standin]
            cfg["workload"] = (f"stand-in for {args.standin} (Table 1: n={n0:,}, average degree "
                               f"{d0}, ||G||_2={l0}): Chung-Lu n={g.n:,}, nnz={g.nnz:,}, "
                               f"lambda_max={lam:.1f}, unit weights, b={b} queries, r={rank_r}, "
                               f"top-1% hubs, beta=1/(lambda_max+1), tol 1e-6")
        cfg.update({"method": args.method, "parallelism": "replicas" if world > 1 else "single",
                    "spmm_autotune": tune, "gather_kernel": args.gather,
                    "cheb_gather": args.cheb,
                    "n2": info["n2"], "n1": info["n1"], "index_build_s": build_s,
                    "index_device_bytes": info["device_bytes"],
                    "rhs_coupling": bool(info["rhs_coupling"]),
                    "sigma_1": info["lambda_max_R"],
                    "lambda_max": lam, "beta": beta,
                    "beta_rule": "1/(lambda_max+1)" if args.paper_beta else "c/lambda_max"})
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": ("f32 (" + values_label(g, "bf16" if args.workload == 3 else "f32") +
                         ", float-float f64-class residual refinement)"),
               "data": "synthetic",
               "config": cfg, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": int(launches), "clocks": clk,
               "lrc": {"mean_iters": lrc_iters, **{k: lrc_stats[k] for k in
                                                   ("refine_steps", "max_rel_res", "status")}},
               "cg": cg, "sparse_katz": sk, "kernels": kernels,
               "max_err_vs_oracle": parity["max_err_vs_oracle"] if parity else None,
               "topk_agree": parity["topk_agree"] if parity else None,
               "parity": parity}
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
