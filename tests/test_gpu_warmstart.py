"""Learned warm start: the GPU network's forward/backward against the FP64
oracle (same BF16-rounded weights), and the warm-started LRC query against
the FP64 oracle Katz vectors, with the iteration counts reported."""
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


def bf16(x):
    return torch.from_numpy(x).float().to(torch.bfloat16).double().numpy()


def test_mlp_gradients_match_oracle():
    """Tolerance: FP32 accumulation over <= 256 terms of O(1) products
    (relative ~1e-5) against the FP64 oracle, on identical BF16 weights."""
    rng = np.random.default_rng(0)
    m, din, dh, dout = 37, 32, 256, 24
    X = rng.normal(size=(m, din))
    T = rng.normal(size=(m, dout))
    W1 = bf16(rng.normal(size=(dh, din)) / np.sqrt(din))
    b1 = rng.normal(size=dh) * 0.1
    W2 = bf16(rng.normal(size=(dout, dh)) / np.sqrt(dh))
    b2 = rng.normal(size=dout) * 0.1
    Xf = X.astype(np.float32).astype(np.float64)
    Tf = T.astype(np.float32).astype(np.float64)
    b1f = b1.astype(np.float32).astype(np.float64)
    b2f = b2.astype(np.float32).astype(np.float64)
    loss, (dW1, db1, dW2, db2) = O.mlp_loss_grad(Xf, Tf, W1, b1f, W2, b2f)
    params = np.concatenate([W1.ravel(), b1f, W2.ravel(), b2f]).astype(np.float32)
    P = torch.from_numpy(params).cuda()
    G = torch.zeros_like(P)
    gl = katz.katz_mlp_loss_grad(torch.from_numpy(Xf.astype(np.float32)).cuda(),
                                 torch.from_numpy(Tf.astype(np.float32)).cuda(), P, G, din, dh, dout)
    assert gl == pytest.approx(loss, rel=1e-5)
    g = G.cpu().numpy().astype(np.float64)
    ref = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2])
    assert np.abs(g - ref).max() <= 1e-5 * np.abs(ref).max() + 1e-7


def test_warm_started_queries_match_oracle_and_report_iterations():
    a = synth.chung_lu(6000, 2.1, 6.0, 600.0, seed=71)
    g = a
    W = O.adjacency(g.n, g.rowptr, g.col, g.val)
    lam = O.lambda_max(W)
    beta = 1.0 / (lam + 1.0)
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F32, rank=16, n_hubs=60,
                                block_max=32)
    rng = np.random.default_rng(3)
    perm = rng.permutation(g.n).astype(np.int32)
    train, test = perm[:1500], np.sort(perm[1500:1564])
    st = katz.katz_warmstart_train(idx, train, hidden=256, epochs=30, batch=128, lr=2e-3)
    assert st["final_loss"] < st["initial_loss"]
    K = torch.zeros((g.n, len(test)), dtype=torch.float64, device="cuda")
    qd = torch.from_numpy(test).cuda()
    _, it_cold, _ = katz.katz_query_batch(idx, qd, K, out_dtype=katz.KATZ_F64, tol=1e-6)
    st_w, it_warm, _ = katz.katz_query_batch(idx, qd, K, out_dtype=katz.KATZ_F64, tol=1e-6,
                                             warm_start=1)
    ref = O.katz_direct(W, beta, test)
    assert O.error_inf_rel(K.cpu().numpy(), ref).max() <= 1e-6
    print(f"mean Schur PCG iterations: cold {it_cold.mean():.2f}, warm {it_warm.mean():.2f}, "
          f"fallbacks {st_w['ms'][5]:.0f}/{len(test)}, train loss {st['initial_loss']:.3e} -> "
          f"{st['final_loss']:.3e}")
    assert it_warm.mean() <= it_cold.mean() + 1.0


def test_warm_started_cg_matches_oracle_and_reports_its_gain():
    """CG on M started from the network's guess (K2 = W_r c_hat on the
    separator, K1 = M11^{-1} B1 + beta M11^{-1} W12 W_r c_hat elsewhere):
    the answers meet the 1e-6 bound against the oracle like the cold start,
    each column's guess is scaled to its energy-optimal multiple (columns
    scaled to zero are counted), and the CG iterations cold and warm are
    printed.  A graph
    whose hubs carry much of each Katz vector, so that the separator part
    matters."""
    g = synth.chung_lu(8000, 2.1, 6.0, 800.0, seed=72)
    W = O.adjacency(g.n, g.rowptr, g.col, g.val)
    beta = 0.9 / O.lambda_max(W)
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F32, rank=24, n_hubs=80,
                                block_max=32, split=False)
    rng = np.random.default_rng(4)
    perm = rng.permutation(g.n).astype(np.int32)
    train, test = perm[:3000], np.sort(perm[3000:3128])
    st = katz.katz_warmstart_train(idx, train, hidden=256, epochs=30, batch=128, lr=2e-3)
    assert st["final_loss"] < st["initial_loss"]
    qd = torch.from_numpy(test).cuda()
    ref = O.katz_direct(W, beta, test)
    res = {}
    for warm in (0, 1):
        K = torch.zeros((g.n, len(test)), dtype=torch.float64, device="cuda")
        s, it, rel = katz.cg_query_batch(idx, qd, K, out_dtype=katz.KATZ_F64, tol=1e-6,
                                         warm_start=warm)
        assert s["status"] == "KATZ_OK"
        assert O.error_inf_rel(K.cpu().numpy(), ref).max() <= 1e-6, warm
        res[warm] = (it.mean(), s["ms"][5], s["refine_steps"], s["ms"][6])
    print(f"mean CG iterations: cold {res[0][0]:.2f}, warm {res[1][0]:.2f} (zero-scaled "
          f"{res[1][1]:.0f}/{len(test)}, mean scale {res[1][3]:.3f}, refinement steps "
          f"{res[0][2]} / {res[1][2]})")
    assert 0 <= res[1][1] <= len(test)
