"""The refinement residual reported for each column is the residual of the
K that is returned: on a modular graph with a small separator and a wide
batch (the case where an earlier way of forming the first pass's norms
cancelled and stopped early), for both kernels of the fused products, the
reported ||b - M k||_2 / ||b||_2 matches an FP64 evaluation of the returned
columns and the infinity-norm error bound holds against the oracle."""
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


@pytest.fixture(scope="module")
def setup():
    g, _, c, r = synth.workload(3, 0.02)
    W = O.adjacency(g.n, g.rowptr, g.col, g.val)
    beta = c / O.lambda_max(W)
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_BF16, rank=r,
                                n_hubs=int(g.meta["hubs"].shape[0]), block_max=64, split=False)
    return g, W, beta, idx


@pytest.mark.parametrize("kern", [katz.KATZ_GATHER_REGISTER, katz.KATZ_GATHER_PIPELINED])
@pytest.mark.parametrize("b", [256, 512])
def test_reported_residual_is_that_of_the_returned_solution(setup, kern, b):
    g, W, beta, idx = setup
    q = synth.queries(g.n, b, seed=synth.BASE_SEED + 77)
    K = torch.zeros((g.n, b), dtype=torch.float64, device="cuda")
    st, it, rel = katz.katz_query_batch(idx, torch.from_numpy(q).cuda(), K,
                                        out_dtype=katz.KATZ_F64, tol=1e-6, gather_kernel=kern)
    assert st["status"] == "KATZ_OK"
    assert np.all(np.isfinite(rel)) and rel.max() > 0
    cols = [0, 1, b // 2, b - 1]
    Kh = K.cpu().numpy()[:, cols]
    B = beta * W[:, q[cols]].toarray()
    R = B - (Kh - beta * (W @ Kh))
    true = np.linalg.norm(R, axis=0) / np.linalg.norm(B, axis=0)
    np.testing.assert_allclose(rel[cols], true, rtol=1e-3, atol=1e-15)
    Kref, _ = O.katz_cg(W, beta, q[cols], rtol=1e-12)
    assert O.error_inf_rel(Kh, Kref).max() <= 1e-6


@pytest.fixture(scope="module")
def heavy():
    """The power-law recipe at n = 50,000 (degree cap 10,000): hundreds of
    rows above 384 entries, each split into 512-entry segments by the
    residual kernels."""
    g, _, c, r = synth.workload(2, 0.05)
    deg = np.diff(g.rowptr)
    assert (deg > 384).sum() > 50 and deg.max() > 2000
    W = O.adjacency(g.n, g.rowptr, g.col, g.val)
    beta = c / O.lambda_max(W)
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F32, rank=r, n_hubs=g.n // 100,
                                block_max=64, split=False)
    return g, W, beta, idx, deg


@pytest.mark.parametrize("fn", ["lrc", "cg"])
def test_split_heavy_row_residual(heavy, fn):
    g, W, beta, idx, deg = heavy
    b = 256
    q = synth.queries(g.n, b, seed=synth.BASE_SEED + 78)
    q[:4] = np.argsort(-deg)[:4]  # the heaviest rows as queries too
    f = katz.katz_query_batch if fn == "lrc" else katz.cg_query_batch
    K = torch.zeros((g.n, b), dtype=torch.float64, device="cuda")
    st, it, rel = f(idx, torch.from_numpy(q).cuda(), K, out_dtype=katz.KATZ_F64, tol=1e-6)
    assert st["status"] == "KATZ_OK"
    cols = [0, 1, 100, b - 1]
    Kh = K.cpu().numpy()[:, cols]
    B = beta * W[:, q[cols]].toarray()
    R = B - (Kh - beta * (W @ Kh))
    true = np.linalg.norm(R, axis=0) / np.linalg.norm(B, axis=0)
    np.testing.assert_allclose(rel[cols], true, rtol=1e-3, atol=1e-15)
    Kref, _ = O.katz_cg(W, beta, q[cols], rtol=1e-12)
    assert O.error_inf_rel(Kh, Kref).max() <= 1e-6
