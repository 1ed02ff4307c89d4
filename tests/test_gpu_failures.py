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


def test_bounded_pipeline_wait_reports_timeout_and_library_recovers():
    """A wait that nothing completes: with the test switch on, the tcgen05
    GEMM's producer issues no TMA copy, so the MMA issuer's bounded wait on
    the first stage runs out (nothing is in flight), the kernel frees its
    tensor memory and the call returns KATZ_ECUDA.  With the switch off the
    same call then succeeds and matches an FP32 product of the BF16
    operands."""
    gen = torch.Generator(device="cuda").manual_seed(3)
    A = torch.randn((128, 64), generator=gen, device="cuda").to(torch.bfloat16)
    B = torch.randn((96, 64), generator=gen, device="cuda").to(torch.bfloat16)
    C = torch.zeros((128, 96), dtype=torch.float32, device="cuda")
    try:
        katz.katz_test_stall_copies(True)
        with pytest.raises(katz.KatzError) as e:
            katz.katz_gemm_bf16(A, B, C)
        assert e.value.code == katz.KATZ_ECUDA
    finally:
        katz.katz_test_stall_copies(False)
    katz.katz_gemm_bf16(A, B, C)
    torch.cuda.synchronize()
    ref = A.float() @ B.float().T
    assert torch.allclose(C, ref, rtol=1e-5, atol=1e-4)
