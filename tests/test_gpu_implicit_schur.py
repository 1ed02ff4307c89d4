"""Separators too large for a stored Schur complement (Section 3.2, Step 4;
Lemma 1): above n2_max the index keeps S implicit and every PCG iteration
applies S P = M22 P - M12^T M11^{-1} (M12 P) with one M11 solve; the
Lanczos correction (Eqs. 8-14) runs on T = M12^T M11^{-1} M12 applied the
same way.  The answers must meet the 1e-6 bound against the FP64 oracle,
and on a graph small enough for both forms the implicit index must give
the explicit one's Ritz values (the same operator) and answers."""
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


def _answers(idx, g, q, fn=katz.katz_query_batch, precision=katz.KATZ_PREC_MIXED):
    K = torch.zeros((g.n, len(q)), dtype=torch.float64, device="cuda")
    st, it, rel = fn(idx, torch.from_numpy(q).cuda(), K, out_dtype=katz.KATZ_F64, tol=1e-6,
                     precision=precision)
    assert st["status"] == "KATZ_OK", st
    return K.cpu().numpy(), st


def test_separator_of_20000_nodes_is_applied_implicitly():
    """n = 60,000 power-law graph with its 20,000 highest-degree nodes as
    separator (above the default n2_max of 16,384); the remainder falls
    into small blocks with dense inverses."""
    g = synth.chung_lu(60000, 2.1, 8.0, 2000.0, seed=41)
    W = O.adjacency(g.n, g.rowptr, g.col, g.val)
    lam = katz.katz_lambda_max(g, steps=96)
    beta = 0.9 / lam
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F32, rank=32, n_hubs=20000,
                                block_max=32, split=True)
    info = idx.info()
    assert info["n2"] == 20000 and info["schur_implicit"] == 1
    q = synth.queries(g.n, 24, seed=42)
    q[0] = int(np.argmax(np.diff(g.rowptr)))  # the largest hub (a separator node)
    Kref, _ = O.katz_cg(W, beta, q, rtol=1e-13)
    K, st = _answers(idx, g, q)
    assert O.error_inf_rel(K, Kref).max() <= 1e-6
    # the FP64 path through the same implicit operator
    K64, _ = _answers(idx, g, q[:4], precision=katz.KATZ_PREC_F64)
    assert O.error_inf_rel(K64, Kref[:, :4]).max() <= 1e-6


def test_implicit_and_explicit_schur_agree_with_a_chebyshev_block():
    """A graph whose non-separator part keeps a large component (solved by
    Chebyshev steps): n2_max below the separator forces the implicit form;
    its Ritz values and answers match the explicit index and the oracle."""
    g = synth.chung_lu(12000, 2.1, 12.0, 800.0, seed=43)
    W = O.adjacency(g.n, g.rowptr, g.col, g.val)
    beta = 0.9 / O.lambda_max(W)
    kw = dict(value_dtype=katz.KATZ_F32, rank=24, n_hubs=600, block_max=32, split=False)
    exp = katz.katz_index_build(g, beta, **kw)
    imp = katz.katz_index_build(g, beta, n2_max=256, **kw)
    assert exp.info()["schur_implicit"] == 0 and imp.info()["schur_implicit"] == 1
    assert imp.info()["n_large_blocks"] >= 1
    np.testing.assert_allclose(katz.katz_index_get_sigma(imp), katz.katz_index_get_sigma(exp),
                               rtol=1e-8, atol=1e-10)
    q = synth.queries(g.n, 40, seed=44)
    Kref, _ = O.katz_cg(W, beta, q, rtol=1e-13)
    for idx in (exp, imp):
        K, st = _answers(idx, g, q)
        assert O.error_inf_rel(K, Kref).max() <= 1e-6
        K, st = _answers(idx, g, q[:8], fn=katz.cg_query_batch)
        assert O.error_inf_rel(K, Kref[:, :8]).max() <= 1e-6
