"""The SpMM autotuner (launch-shape search) keeps results correct."""
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


def test_autotune_then_query_matches_oracle():
    g = synth.chung_lu(20000, 2.1, 8.0, 2000.0, seed=21)
    W = O.adjacency(g.n, g.rowptr, g.col, g.val)
    beta = 0.8 / O.lambda_max(W)
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F32, rank=16, n_hubs=200,
                                block_max=64)
    q = synth.queries(g.n, 48, seed=2)
    res = katz.katz_autotune(idx, len(q))
    assert res["col_tile"] in (0, 128, 256, 512, 1024)
    assert res["ms_best"] <= res["ms_default"] + 1e-9
    K = torch.zeros((g.n, len(q)), dtype=torch.float64, device="cuda")
    for fn in (katz.katz_query_batch, katz.cg_query_batch):
        fn(idx, torch.from_numpy(q).cuda(), K, out_dtype=katz.KATZ_F64, tol=1e-6)
        Kref = O.katz_cg(W, beta, q, rtol=1e-13)[0]
        assert O.error_inf_rel(K.cpu().numpy(), Kref).max() <= 1e-6
