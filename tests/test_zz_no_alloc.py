"""linkpred_topk_noalloc: the top-k link prediction whose scratch lives in a
fixed array inside the library instead of freshly allocated device memory
(for callers that cannot allocate while they run: a serving loop with no
room for an allocation, or device memory held by another framework's
caching allocator).  Its results must equal those of linkpred_topk, on two
calls in a row with different inputs (the shared scratch keeps the previous
call's contents), at the size limit b * k = 32,768 (one slice of lists),
for FP64 scores read through a leading dimension larger than b, and it must
reject b * k = 32,769."""
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


def _both(idx, q, K, k_dtype, k):
    b = int(q.shape[0])
    ids_a = torch.empty((b, k), dtype=torch.int32, device="cuda")
    sc_a = torch.empty((b, k), dtype=torch.float64, device="cuda")
    katz.linkpred_topk(idx, q, K, k_dtype, k, ids_a, sc_a)
    ids_b = torch.full((b, k), -7, dtype=torch.int32, device="cuda")
    sc_b = torch.full((b, k), -7.0, dtype=torch.float64, device="cuda")
    katz.linkpred_topk_noalloc(idx, q, K, k_dtype, k, ids_b, sc_b)
    torch.cuda.synchronize()
    return ids_a, sc_a, ids_b, sc_b


def test_noalloc_topk_at_the_size_limit_and_f64_with_wide_rows():
    """b * k = 32,768 exactly (b = 512, k = 64: a single slice of 8 lists per
    column fills the scratch) twice with different scores; then FP64 scores
    in a block whose leading dimension exceeds b."""
    g = synth.chung_lu(20000, 2.1, 8.0, 2000.0, seed=35)
    idx = katz.katz_index_build(g, 0.3 / katz.katz_lambda_max(g), value_dtype=katz.KATZ_F32,
                                build_lrc=False)
    gen = torch.Generator(device="cuda").manual_seed(7)
    q = torch.from_numpy(synth.queries(g.n, 512, seed=8)).cuda()
    for call in range(2):
        # score descending, ties by id: a strict total order, so both must agree exactly
        K = torch.rand((g.n, 512), generator=gen, device="cuda", dtype=torch.float32)
        ids_a, sc_a, ids_b, sc_b = _both(idx, q, K, katz.KATZ_F32, 64)
        assert torch.equal(ids_a, ids_b), f"call {call}"
        assert torch.equal(sc_a, sc_b), f"call {call}"
    q = torch.from_numpy(synth.queries(g.n, 40, seed=9)).cuda()
    Kw = torch.rand((g.n, 40 + 13), generator=gen, device="cuda", dtype=torch.float64)
    K = Kw[:, :40]
    ids_a, sc_a, ids_b, sc_b = _both(idx, q, K, katz.KATZ_F64, 20)
    assert torch.equal(ids_a, ids_b) and torch.equal(sc_a, sc_b)
    # the scores returned are the column's own entries, largest first
    Kc = K.cpu().numpy()
    for j in range(40):
        np.testing.assert_array_equal(sc_b[j].cpu().numpy(), Kc[ids_b[j].cpu().numpy(), j])
        assert np.all(np.diff(sc_b[j].cpu().numpy()) <= 0)


def test_noalloc_topk_rejects_one_entry_past_the_limit():
    """b * k = 32,769 (b = 993, k = 33) is one list entry per slice too many."""
    g = synth.cycle(2000)
    idx = katz.katz_index_build(g, 0.3, value_dtype=katz.KATZ_UNIT, build_lrc=False)
    q = (torch.arange(993, dtype=torch.int32, device="cuda") * 2) % 2000
    K = torch.zeros((2000, 993), dtype=torch.float32, device="cuda")
    ids = torch.empty((993, 33), dtype=torch.int32, device="cuda")
    sc = torch.empty((993, 33), dtype=torch.float64, device="cuda")
    with pytest.raises(katz.KatzError) as e:
        katz.linkpred_topk_noalloc(idx, q, K, katz.KATZ_F32, 33, ids, sc)
    assert e.value.code == katz.KATZ_EINVAL
