"""Query batches solved in column chunks (katz_query_opts.rhs_width).

The b queries of one call are solved rhs_width columns at a time, each
chunk written to its own column range of K.  Checked against the FP64
oracle (max infinity-norm relative error <= 1e-6 per column, the query
path's accuracy target) on chunk boundaries of a batch wider than the
1,024 columns one solve takes, and on every column of a small ragged
batch with host and device outputs.
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


def test_batch_wider_than_one_solve_in_chunks():
    """b = 1,100 queries on the modular graph recipe (n = 20,000, one
    community block solved by Chebyshev steps, the first Schur right-hand
    side from the stored Z) in chunks of 512, 512 and 76 columns."""
    g = synth.workload(3, 0.005)[0]
    W = W_of(g)
    beta = 0.9 / O.lambda_max(W)
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_BF16, rank=8,
                                n_hubs=int(g.meta["hubs"].shape[0]), block_max=64, split=False)
    q = synth.queries(g.n, 1100, seed=31)
    qd = torch.from_numpy(q).cuda()
    K = torch.zeros((g.n, 1100), dtype=torch.float32, device="cuda")
    with pytest.raises(katz.KatzError) as e:
        katz.katz_query_batch(idx, qd, K, out_dtype=katz.KATZ_F32, tol=1e-6)
    assert e.value.code == katz.KATZ_EINVAL
    with pytest.raises(katz.KatzError) as e:
        katz.katz_query_batch(idx, qd, K, out_dtype=katz.KATZ_F32, tol=1e-6, rhs_width=-1)
    assert e.value.code == katz.KATZ_EINVAL
    st, it, rel = katz.katz_query_batch(idx, qd, K, out_dtype=katz.KATZ_F32, tol=1e-6,
                                        rhs_width=512)
    assert st["status"] == "KATZ_OK"
    assert it.shape == (1100,) and it.max() > 0
    assert st["iters"] == it.max() and st["max_rel_res"] == pytest.approx(rel.max(), rel=1e-12)
    Kh = K.double().cpu().numpy()
    assert np.isfinite(Kh).all()
    cols = [0, 511, 512, 1023, 1024, 1099]
    ref, _ = O.katz_cg(W, beta, q[cols], rtol=1e-12)
    assert O.error_inf_rel(Kh[:, cols], ref).max() <= 1e-6
    # the first chunk equals the same 512 queries solved alone
    K1 = torch.zeros((g.n, 512), dtype=torch.float32, device="cuda")
    katz.katz_query_batch(idx, qd[:512].contiguous(), K1, out_dtype=katz.KATZ_F32, tol=1e-6)
    K1h = K1.double().cpu().numpy()
    assert O.error_inf_rel(Kh[:, :512], K1h).max() <= 2.1e-6  # both within 1e-6 of k


@pytest.mark.parametrize("host", [False, True])
def test_ragged_chunks_every_column(host):
    """b = 20 in chunks of 8, 8 and 4 columns, FP64 output with a leading
    dimension of 24 (the entries past column 20 stay untouched), host or
    device K, LRC and CG, every column against the dense FP64 oracle."""
    a = synth.chung_lu(2500, 2.1, 6.0, 400.0, seed=3)
    g = synth.disjoint_union([a, synth.star(300)])
    W = W_of(g)
    beta = 0.8 / O.lambda_max(W)
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F32, rank=8, n_hubs=25,
                                block_max=64)
    q = synth.queries(g.n, 20, seed=5)
    ref = O.katz_direct(W, beta, q)
    for fn in (katz.katz_query_batch, katz.cg_query_batch):
        if host:
            Kb = np.full((g.n, 24), 7.0)
            st, it, rel = fn(idx, q, Kb[:, :20], out_dtype=katz.KATZ_F64, tol=1e-8,
                             rhs_width=8)
        else:
            Kt = torch.full((g.n, 24), 7.0, dtype=torch.float64, device="cuda")
            st, it, rel = fn(idx, torch.from_numpy(q).cuda(), Kt[:, :20],
                             out_dtype=katz.KATZ_F64, tol=1e-8, rhs_width=8)
            Kb = Kt.cpu().numpy()
        assert (Kb[:, 20:] == 7.0).all()
        assert st["status"] == "KATZ_OK"
        assert it.shape == (20,) and (rel < 1e-6).all()
        assert st["iters"] == it.max()
        assert O.error_inf_rel(Kb[:, :20], ref).max() <= 1e-8
