"""linkpred_topk_noalloc: the top-k link prediction whose scratch lives in a
fixed array inside the library instead of freshly allocated device memory
(for callers that cannot allocate while they run, e.g. inside a stream
capture or under another framework's memory pool).  Its results must equal
those of linkpred_topk, on two calls in a row with different inputs (the
shared scratch keeps the previous call's contents)."""
import numpy as np
import pytest

from paper_1912_06525_gb300 import katz, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_noalloc_topk_matches_allocating_entry_point_twice():
    g = synth.chung_lu(30000, 2.1, 8.0, 3000.0, seed=33)
    lam = katz.katz_lambda_max(g)
    idx = katz.katz_index_build(g, 0.7 / lam, value_dtype=katz.KATZ_F32, build_lrc=False)
    for call, (b, k, seed) in enumerate([(96, 20, 1), (64, 32, 2)]):
        q = torch.from_numpy(synth.queries(g.n, b, seed=seed)).cuda()
        K = torch.empty((g.n, b), dtype=torch.float32, device="cuda")
        katz.cg_query_batch(idx, q, K, out_dtype=katz.KATZ_F32, tol=1e-6)
        ids_a = torch.empty((b, k), dtype=torch.int32, device="cuda")
        sc_a = torch.empty((b, k), dtype=torch.float64, device="cuda")
        katz.linkpred_topk(idx, q, K, katz.KATZ_F32, k, ids_a, sc_a)
        ids_b = torch.full((b, k), -7, dtype=torch.int32, device="cuda")
        sc_b = torch.full((b, k), -7.0, dtype=torch.float64, device="cuda")
        katz.linkpred_topk_noalloc(idx, q, K, katz.KATZ_F32, k, ids_b, sc_b)
        torch.cuda.synchronize()
        # the same kernels on the same scores in a strict total order: exact
        assert torch.equal(ids_a, ids_b), f"call {call}"
        assert torch.equal(sc_a, sc_b), f"call {call}"


def test_noalloc_topk_rejects_oversized_and_host_buffers():
    g = synth.cycle(100)
    idx = katz.katz_index_build(g, 0.3, value_dtype=katz.KATZ_UNIT, build_lrc=False)
    q = torch.arange(4, dtype=torch.int32, device="cuda")
    K = torch.zeros((100, 4), dtype=torch.float32, device="cuda")
    ids = torch.empty((4, 8), dtype=torch.int32, device="cuda")
    sc = torch.empty((4, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(katz.KatzError):
        katz.linkpred_topk_noalloc(idx, q.cpu(), K, katz.KATZ_F32, 8, ids, sc)
    qb = torch.arange(1024, dtype=torch.int32, device="cuda") % 100
    Kb = torch.zeros((100, 1024), dtype=torch.float32, device="cuda")
    idsb = torch.empty((1024, 64), dtype=torch.int32, device="cuda")
    scb = torch.empty((1024, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(katz.KatzError):
        katz.linkpred_topk_noalloc(idx, qb, Kb, katz.KATZ_F32, 64, idsb, scb)
