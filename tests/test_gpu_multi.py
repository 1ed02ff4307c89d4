"""Many independent graphs of uneven size answered in one batched solve
(block-diagonal system, per-(graph, query) CG scalars, CUDA-graph replay):
every (graph, query) Katz vector matches the FP64 oracle of that graph
alone to 1e-6 (infinity-norm relative error)."""
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


@pytest.mark.parametrize("count,c,qpg", [(24, 0.95, 8), (7, 0.5, 3)])
def test_multi_graph_batch_matches_oracle(count, c, qpg):
    graphs = synth.multi_sbm(count, 60, 3000, seed=55 + count)
    Ws = [O.adjacency(g.n, g.rowptr, g.col, g.val) for g in graphs]
    betas = [c / O.lambda_max(W) for W in Ws]
    m = katz.katz_multi_build(graphs, betas, value_dtype=katz.KATZ_UNIT)
    rng = np.random.default_rng(1)
    q = np.concatenate([rng.choice(g.n, size=qpg, replace=False) for g in graphs]).astype(np.int32)
    n = sum(g.n for g in graphs)
    K = torch.zeros((n, qpg), dtype=torch.float64, device="cuda")
    stats, iters, rel = katz.katz_multi_query(m, torch.from_numpy(q).cuda(), qpg, K,
                                              out_dtype=katz.KATZ_F64, tol=1e-6)
    assert stats["status"] == "KATZ_OK", stats
    Kh = K.cpu().numpy()
    off = 0
    for gi, (g, W, beta) in enumerate(zip(graphs, Ws, betas)):
        qs = q[gi * qpg:(gi + 1) * qpg]
        ref = O.katz_direct(W, beta, qs)
        assert O.error_inf_rel(Kh[off:off + g.n], ref).max() <= 1e-6, gi
        off += g.n
    assert stats["graph_replays"] >= 1
