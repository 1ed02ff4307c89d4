"""CUDA path against the FP64 oracle, through the C-ABI.

Tolerances: Katz vectors must match to max relative error <= 1e-6 in the
infinity norm (the accuracy target of the query path); the FP64-only
sparse product matches to 1e-12; FP32 products to 2e-6 (a few FP32 ulps
of the row sums).  Integer outputs (partition) must be bit-identical.
"""
import numpy as np
import pytest

import oracle as O
from paper_1912_06525_gb300 import katz, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def W_of(g):
    return O.adjacency(g.n, g.rowptr, g.col, g.val)


def hub_graph(seed=1, weighted=False):
    """Chung-Lu graph plus a 900-leaf star: exercises the split-row kernel
    (rows above 384 entries) and gives a hub-dominated spectrum."""
    a = synth.chung_lu(2500, 2.1, 6.0, 400.0, seed=seed)
    s = synth.star(900)
    g = synth.disjoint_union([a, s])
    r = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    m = r < g.col
    u = np.concatenate([r[m], [0, 2500]])
    v = np.concatenate([g.col[m], [2500, 5]])  # connect the star to the rest
    wf = synth.dyadic_weights(seed + 7) if weighted else None
    return synth.edges_to_graph(g.n, u, v, {"kind": "hub"}, wf)


def run(fn, idx, g, q, dtype=katz.KATZ_F64, **kw):
    K = torch.zeros((g.n, len(q)), dtype=torch.float64 if dtype == katz.KATZ_F64 else torch.float32,
                    device="cuda")
    stats, iters, rel = fn(idx, torch.from_numpy(q).cuda(), K, out_dtype=dtype, **kw)
    return K.double().cpu().numpy(), stats, iters, rel


# ------------------------------------------------------------------ a0
@pytest.mark.parametrize("maker", [lambda: synth.workload(1)[0], lambda: hub_graph(2),
                                   lambda: synth.star(50)])
def test_lambda_max(maker):
    g = maker()
    lam = katz.katz_lambda_max(g, steps=200)
    assert lam == pytest.approx(O.lambda_max(W_of(g)), rel=1e-9)


@pytest.mark.parametrize("maker", [
    lambda: synth.sbm_bernoulli([300] * 6, 0.05, 0.004, seed=21),
    lambda: hub_graph(5, weighted=True),
    lambda: synth.disjoint_union([synth.erdos_renyi(400, 0.03, seed=4), synth.star(60),
                                  synth.path(9)]),
])
def test_lambda_upper_bound_is_rigorous(maker):
    """A few Lanczos steps leave the Ritz value visibly below lambda_max;
    the Collatz-Wielandt bound stays above it at every step count (it holds
    for any positive vector), and is tight once the Ritz vector converges.
    The index build certifies beta with the upper bound: a beta chosen from
    the underestimate (beta * lambda_max > 1) is refused, and the index
    reports both sides."""
    g = maker()
    lam = O.lambda_max(W_of(g))
    lo2, up2 = katz.katz_lambda_bounds(g, steps=2)
    assert lo2 < lam * (1 - 1e-3), "two steps should underestimate visibly"
    for steps in (2, 3, 5, 12, 200):
        lo, up = katz.katz_lambda_bounds(g, steps=steps)
        assert lo <= lam * (1 + 1e-12) and up >= lam, (steps, lo, up, lam)
    assert up <= lam * (1 + 1e-6)
    beta_bad = 0.999 / lo2
    if beta_bad * lam >= 1:
        with pytest.raises(katz.KatzError) as e:
            katz.katz_index_build(g, beta_bad, value_dtype=katz.KATZ_F64, build_lrc=False)
        assert e.value.code == katz.KATZ_ENOTSPD
    idx = katz.katz_index_build(g, 0.9 / lam, value_dtype=katz.KATZ_F64, build_lrc=False)
    info = idx.info()
    assert info["lambda_max_W"] <= lam * (1 + 1e-12) <= info["lambda_upper"] * (1 + 1e-12)
    assert info["lambda_upper"] <= lam * (1 + 1e-6)


# ------------------------------------------------------- sparse product
@pytest.mark.parametrize("b", [1, 3, 16, 257])
@pytest.mark.parametrize("vdt", [katz.KATZ_F64, katz.KATZ_F32, katz.KATZ_BF16])
def test_apply_M(b, vdt):
    g = hub_graph(3, weighted=True)
    W = W_of(g)
    beta = 0.5 / O.lambda_max(W)
    idx = katz.katz_index_build(g, beta, value_dtype=vdt, build_lrc=False)
    rng = np.random.default_rng(b)
    X = rng.normal(size=(g.n, b))
    ref = O.apply_M(W, beta, X)
    for dt, tdt, tol in [(katz.KATZ_F64, torch.float64, 1e-12), (katz.KATZ_F32, torch.float32, 2e-6)]:
        Xd = torch.from_numpy(X).to(tdt).cuda()
        Y = torch.empty_like(Xd)
        katz.katz_apply_M(idx, Xd, Y, b, dt)
        got = Y.double().cpu().numpy()
        scale = np.abs(X).max() * (1 + beta * np.abs(W).sum(axis=1).max())
        assert np.abs(got - ref).max() <= tol * scale


# ------------------------------------------------------------ CG queries
@pytest.mark.parametrize("prec", [katz.KATZ_PREC_MIXED, katz.KATZ_PREC_F64])
def test_cg_workload1(prec):
    g, q, c, r = synth.workload(1)
    W = W_of(g)
    beta = c / O.lambda_max(W)
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F64, build_lrc=False)
    ref = O.katz_direct(W, beta, q)
    K, st, it, rel = run(katz.cg_query_batch, idx, g, q, tol=1e-10,
                         tol_kind=katz.KATZ_TOL_RESIDUAL, precision=prec)
    assert st["status"] == "KATZ_OK"
    assert rel.max() <= 1e-10
    assert O.error_inf_rel(K, ref).max() <= 1e-8
    K2, st2, _, _ = run(katz.cg_query_batch, idx, g, q, tol=1e-6)
    assert O.error_inf_rel(K2, ref).max() <= 1e-6


def test_cg_iterations_match_oracle_cg():
    """Same method, same stopping rule: FP64 GPU CG and FP64 oracle CG take
    the same number of iterations (up to one for rounding at the boundary)."""
    g, q, c, r = synth.workload(1)
    W = W_of(g)
    beta = c / O.lambda_max(W)
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F64, build_lrc=False)
    K, st, it, rel = run(katz.cg_query_batch, idx, g, q, tol=1e-9,
                         tol_kind=katz.KATZ_TOL_RESIDUAL, precision=katz.KATZ_PREC_F64)
    _, it_ref = O.katz_cg(W, beta, q, rtol=1e-9 * 0.3)
    assert np.abs(it - it_ref).max() <= 1


# ----------------------------------------------------------- LRC queries
@pytest.mark.parametrize("hubs,bmax,split", [(0, 64, True), (20, 32, True), (40, 16, False)])
def test_lrc_workload1(hubs, bmax, split):
    g, q, c, r = synth.workload(1)
    W = W_of(g)
    beta = c / O.lambda_max(W)
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F64, rank=r, n_hubs=hubs,
                                block_max=bmax, split=split)
    ref = O.katz_direct(W, beta, q)
    K, st, it, rel = run(katz.katz_query_batch, idx, g, q, tol=1e-10,
                         tol_kind=katz.KATZ_TOL_RESIDUAL)
    assert st["status"] == "KATZ_OK", st
    assert rel.max() <= 1e-10
    assert O.error_inf_rel(K, ref).max() <= 1e-8
    # the partition is the oracle's, node for node
    perm, bp, n1, n2 = katz.katz_index_get_partition(idx)
    p = O.partition(g.n, g.rowptr, g.col, hubs, bmax, split)
    assert perm.tolist() == p["perm"].tolist() and bp.tolist() == p["block_ptr"].tolist()


@pytest.mark.parametrize("vdt", [katz.KATZ_F64, katz.KATZ_F32, katz.KATZ_BF16])
@pytest.mark.parametrize("prec", [katz.KATZ_PREC_MIXED, katz.KATZ_PREC_F64])
def test_lrc_weighted_hub_graph(vdt, prec):
    g = hub_graph(4, weighted=True)
    W = W_of(g)
    beta = 0.9 / O.lambda_max(W)
    idx = katz.katz_index_build(g, beta, value_dtype=vdt, rank=12, n_hubs=25, block_max=32)
    q = synth.queries(g.n, 19, seed=9)
    q[0] = 2500  # the star's hub
    ref = O.katz_direct(W, beta, q)
    for fn in (katz.katz_query_batch, katz.cg_query_batch):
        K, st, it, rel = run(fn, idx, g, q, tol=1e-6, precision=prec)
        assert st["status"] == "KATZ_OK", (fn.__name__, st)
        assert O.error_inf_rel(K, ref).max() <= 1e-6, fn.__name__


def test_ritz_values_match_oracle():
    g = hub_graph(5)
    W = W_of(g)
    beta = 0.9 / O.lambda_max(W)
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F64, rank=10, n_hubs=30,
                                block_max=16)
    sig = katz.katz_index_get_sigma(idx)
    p = O.partition(g.n, g.rowptr, g.col, 30, 16, True)
    ref = O.lrc_build(W, beta, p, 10, block_max=16)
    dense = np.sort(np.linalg.eigvalsh(ref["R"]))[::-1][:10]
    np.testing.assert_allclose(sig, dense, rtol=1e-8, atol=1e-12)
    assert (sig >= 0).all() and (sig < 1).all()


def test_lrc_needs_fewer_iterations_at_hard_damping():
    """Reported, and checked loosely: on a hub-dominated graph at
    beta = 1/(lambda+1) (Section 4's hardest case) the preconditioned Schur
    solve needs fewer iterations than CG on M."""
    g = hub_graph(6)
    W = W_of(g)
    lam = O.lambda_max(W)
    beta = 1.0 / (lam + 1.0)
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F32, rank=16, n_hubs=40,
                                block_max=32)
    q = synth.queries(g.n, 32, seed=3)
    _, st_l, it_l, _ = run(katz.katz_query_batch, idx, g, q, tol=1e-6)
    _, st_c, it_c, _ = run(katz.cg_query_batch, idx, g, q, tol=1e-6)
    assert it_l.mean() < it_c.mean()


@pytest.mark.parametrize("b", [1, 5, 130])
def test_lrc_ragged_batches(b):
    g = hub_graph(7)
    W = W_of(g)
    beta = 0.7 / O.lambda_max(W)
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_UNIT, rank=8, n_hubs=20,
                                block_max=64)
    q = synth.queries(g.n, b, seed=b)
    ref = O.katz_direct(W, beta, q)
    K, st, _, _ = run(katz.katz_query_batch, idx, g, q, dtype=katz.KATZ_F32, tol=1e-6)
    assert O.error_inf_rel(K, ref).max() <= 1e-6


def test_isolated_and_degenerate_queries():
    g = synth.disjoint_union([synth.path(1), synth.single_edge(), synth.complete(6)])
    W = W_of(g)
    beta = 0.5 / O.lambda_max(W)
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_UNIT, rank=2, block_max=4)
    q = np.array([0, 1, 2, 3, 8], dtype=np.int32)
    ref = O.katz_direct(W, beta, q)
    for fn in (katz.katz_query_batch, katz.cg_query_batch):
        K, st, _, _ = run(fn, idx, g, q, tol=1e-8)
        assert np.all(K[:, 0] == 0)
        assert O.error_inf_rel(K, ref).max() <= 1e-8


def test_host_buffers_end_to_end():
    g, q, c, r = synth.workload(1)
    W = W_of(g)
    beta = c / O.lambda_max(W)
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F64, rank=r, block_max=64)
    K = np.zeros((g.n, len(q)), dtype=np.float32)
    katz.katz_query_batch(idx, q, K, out_dtype=katz.KATZ_F32, tol=1e-6)
    assert O.error_inf_rel(K.astype(np.float64), O.katz_direct(W, beta, q)).max() <= 1e-6


# --------------------------------------------------------- link prediction
def test_linkpred_topk_matches_oracle():
    g = hub_graph(8)
    W = W_of(g)
    beta = 0.8 / O.lambda_max(W)
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F32, build_lrc=False)
    q = synth.queries(g.n, 24, seed=8)
    Kref = np.ascontiguousarray(O.katz_direct(W, beta, q))
    Kd = torch.from_numpy(Kref).cuda()
    ids = torch.empty((len(q), 20), dtype=torch.int32, device="cuda")
    sc = torch.empty((len(q), 20), dtype=torch.float64, device="cuda")
    katz.linkpred_topk(idx, torch.from_numpy(q).cuda(), Kd, katz.KATZ_F64, 20, ids, sc)
    rid, rsc = O.linkpred_topk(W, Kref, q, 20)
    # the same FP64 scores go in, and the order is a strict total order
    np.testing.assert_array_equal(ids.cpu().numpy(), rid)
    np.testing.assert_array_equal(sc.cpu().numpy(), rsc)


def test_linkpred_topk_on_gpu_solution_up_to_ties():
    g, q, c, r = synth.workload(1)
    W = W_of(g)
    beta = c / O.lambda_max(W)
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F64, rank=r, block_max=64)
    K, _, _, _ = run(katz.katz_query_batch, idx, g, q, dtype=katz.KATZ_F32, tol=1e-6)
    Kd = torch.from_numpy(K.astype(np.float32)).cuda()
    ids = torch.empty((len(q), 20), dtype=torch.int32, device="cuda")
    sc = torch.empty((len(q), 20), dtype=torch.float64, device="cuda")
    katz.linkpred_topk(idx, torch.from_numpy(q).cuda(), Kd, katz.KATZ_F32, 20, ids, sc)
    Kref = O.katz_direct(W, beta, q)
    rid, rsc = O.linkpred_topk(W, Kref, q, 20)
    ids = ids.cpu().numpy()
    for j in range(len(q)):
        band = 2e-6 * np.abs(Kref[:, j]).max()
        must = set(rid[j][rsc[j] > rsc[j][-1] + band].tolist())
        assert must <= set(ids[j].tolist())
        cand = set(np.nonzero(Kref[:, j] >= rsc[j][-1] - band)[0].tolist())
        assert set(ids[j].tolist()) <= cand


# ---------------------------------------------------------------- errors
def test_damping_bound_and_bad_queries():
    g = synth.complete(8)
    with pytest.raises(katz.KatzError) as e:
        katz.katz_index_build(g, 1.2 / 7.0, value_dtype=katz.KATZ_UNIT, build_lrc=False)
    assert e.value.code == katz.KATZ_ENOTSPD
    idx = katz.katz_index_build(g, 0.5 / 7.0, value_dtype=katz.KATZ_UNIT, build_lrc=False)
    K = torch.zeros((8, 1), dtype=torch.float32, device="cuda")
    with pytest.raises(katz.KatzError) as e:
        katz.cg_query_batch(idx, np.array([8], dtype=np.int32), K)
    assert e.value.code == katz.KATZ_EINVAL
    with pytest.raises(katz.KatzError) as e:
        katz.katz_query_batch(idx, np.array([1], dtype=np.int32), K)  # no LRC part
    assert e.value.code == katz.KATZ_EINVAL
    # an empty batch is rejected on the host, before any launch
    K0 = np.zeros((8, 1), dtype=np.float32)
    with pytest.raises(katz.KatzError) as e:
        katz.cg_query_batch(idx, np.zeros(0, dtype=np.int32), K0)
    assert e.value.code == katz.KATZ_EINVAL


def test_rank_extremes():
    """r = 0: the preconditioner is M22^{-1} alone; r = n2: S~^{-1} = S^{-1}
    (Theorem 1 with every eigenpair kept), one Schur PCG iteration in exact
    arithmetic; the FP32 solve applies W^ through BF16 tensor-core products
    (~1e-2 relative), so a few iterations, and fewer than with r = 0."""
    g = hub_graph(9)
    W = W_of(g)
    beta = 0.9 / O.lambda_max(W)
    n_hubs = 40
    q = synth.queries(g.n, 40, seed=10)
    ref = O.katz_direct(W, beta, q)
    iters = {}
    for r in (0, n_hubs):
        idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F32, rank=r, n_hubs=n_hubs,
                                    block_max=32, split=False)
        info = katz.katz_index_get_info(idx)
        assert info["n2"] == n_hubs and info["rank"] == r
        # a tolerance well inside FP32 so that the counts reflect the
        # preconditioner, not FP32 stagnation
        K, st, it, rel = run(katz.katz_query_batch, idx, g, q, tol=1e-4,
                             precision=katz.KATZ_PREC_F32)
        assert O.error_inf_rel(K, ref).max() <= 1e-3
        iters[r] = it
        K, st, it, rel = run(katz.katz_query_batch, idx, g, q, tol=1e-6)
        assert st["status"] == "KATZ_OK"
        assert O.error_inf_rel(K, ref).max() <= 1e-6
    assert iters[n_hubs].max() <= 4, iters[n_hubs]
    assert iters[n_hubs].mean() < iters[0].mean(), (iters[n_hubs].mean(), iters[0].mean())
