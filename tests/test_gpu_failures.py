"""Failure detection without a GPU fault: iteration and refinement caps end
a call with KATZ_ENOCONV and filled outputs; a device allocation made to
fail on the host (katz_fault_inject_alloc) ends the call with KATZ_ENOMEM,
releases what it allocated, and leaves the library usable."""
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


def small():
    g = synth.chung_lu(3000, 2.2, 8.0, 300.0, seed=12)
    W = O.adjacency(g.n, g.rowptr, g.col, g.val)
    return g, W, 0.9 / O.lambda_max(W)


def test_caps_return_enoconv_with_filled_outputs():
    g, W, beta = small()
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F32, rank=8, n_hubs=30,
                                block_max=32, split=False)
    q = synth.queries(g.n, 16, seed=3)
    qd = torch.from_numpy(q).cuda()
    K = torch.full((g.n, len(q)), float("nan"), dtype=torch.float64, device="cuda")
    st, it, rel = katz.cg_query_batch(idx, qd, K, out_dtype=katz.KATZ_F64, tol=1e-10,
                                      tol_kind=katz.KATZ_TOL_RESIDUAL, max_iter=2, max_refine=1)
    assert st["status"] == "KATZ_ENOCONV"
    assert torch.isfinite(K).all().item()
    assert (rel > 1e-10).any() and np.isfinite(rel).all()
    st, it, rel = katz.katz_query_batch(idx, qd, K, out_dtype=katz.KATZ_F64, tol=1e-14,
                                        tol_kind=katz.KATZ_TOL_RESIDUAL, max_refine=1)
    assert st["status"] == "KATZ_ENOCONV"
    assert torch.isfinite(K).all().item()
    # the capped answer is still a (coarse) solution
    assert O.error_inf_rel(K.cpu().numpy(), O.katz_direct(W, beta, q)).max() < 1e-2


@pytest.mark.parametrize("after", [0, 3, 40])
def test_injected_allocation_failure_is_enomem_and_recoverable(after):
    g, W, beta = small()
    try:
        katz.katz_fault_inject_alloc(after)
        with pytest.raises(katz.KatzError) as e:
            katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F32, rank=8, n_hubs=30,
                                  block_max=32, split=False)
        assert e.value.code == katz.KATZ_ENOMEM
        assert "injected" in katz.katz_last_error()
    finally:
        katz.katz_fault_inject_alloc(-1)
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F32, rank=8, n_hubs=30,
                                block_max=32, split=False)
    q = synth.queries(g.n, 8, seed=4)
    qd = torch.from_numpy(q).cuda()
    K = torch.zeros((g.n, len(q)), dtype=torch.float64, device="cuda")
    # a failure inside a query (its scratch), then the same query again
    try:
        katz.katz_fault_inject_alloc(0)
        with pytest.raises(katz.KatzError) as e:
            katz.katz_query_batch(idx, qd, K, out_dtype=katz.KATZ_F64, tol=1e-6)
        assert e.value.code == katz.KATZ_ENOMEM
    finally:
        katz.katz_fault_inject_alloc(-1)
    st, it, rel = katz.katz_query_batch(idx, qd, K, out_dtype=katz.KATZ_F64, tol=1e-6)
    assert st["status"] == "KATZ_OK"
    assert O.error_inf_rel(K.cpu().numpy(), O.katz_direct(W, beta, q)).max() <= 1e-6
