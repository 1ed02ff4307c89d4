"""Full-size parity in the benchmark's launch configuration.

The whole n x b block is solved on the GPU exactly as bench.py does (index
options, autotuned SpMM shape, mixed precision, 1e-6 infinity-norm error
bound); the FP64 oracle then solves a sample of the columns one by one (CG
to the same guaranteed bound, run tighter) and every sampled column must
match to 1e-6 relative error in the infinity norm."""
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


def sampled_parity(g, q, beta, K, cols):
    W = O.adjacency(g.n, g.rowptr, g.col, g.val)
    Kref, _ = O.katz_cg(W, beta, q[cols], rtol=1e-12)
    err = O.error_inf_rel(K[:, cols], Kref)
    assert err.max() <= 1e-6, err


def test_power_law_1m_full_batch():
    g, q, c, r = synth.workload(2)
    lam = katz.katz_lambda_max(g, steps=96)
    beta = c / lam
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F32, rank=r, n_hubs=g.n // 100,
                                block_max=64, split=False)
    katz.katz_autotune(idx, len(q))
    qd = torch.from_numpy(q).cuda()
    K = torch.empty((g.n, len(q)), dtype=torch.float32, device="cuda")
    for fn in (katz.katz_query_batch, katz.cg_query_batch):
        st, it, rel = fn(idx, qd, K, out_dtype=katz.KATZ_F32, tol=1e-6)
        assert st["status"] == "KATZ_OK"
        Kh = K.double().cpu().numpy()
        sampled_parity(g, q, beta, Kh, [0, 37, 128, len(q) - 1])


def test_modular_hubs_quarter_scale():
    g, q, c, r = synth.workload(3, 0.25)
    lam = katz.katz_lambda_max(g, steps=96)
    beta = 0.9 / lam
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_BF16, rank=r,
                                n_hubs=int(g.meta["hubs"].shape[0]), block_max=64, split=False)
    qd = torch.from_numpy(q).cuda()
    K = torch.empty((g.n, len(q)), dtype=torch.float32, device="cuda")
    st, it, rel = katz.katz_query_batch(idx, qd, K, out_dtype=katz.KATZ_F32, tol=1e-6)
    assert st["status"] == "KATZ_OK"
    sampled_parity(g, q, beta, K.double().cpu().numpy(), [1, len(q) // 2])
