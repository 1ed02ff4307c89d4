"""Pins for the oracle's LRC-Katz parts: partition (Section 3.2, Steps
2-3), Lemma 1, the exact inverse of Eq. 13, Theorem 1, the Lanczos step of
Algorithm 1, PCG of Algorithm 2, and the warm-start network's gradients."""
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

import oracle as O
from paper_1912_06525_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def W_of(g):
    return O.adjacency(g.n, g.rowptr, g.col, g.val)


def random_partition(W, rng, sep_frac):
    """Any separator set and any grouping of the remaining components into
    blocks gives an invertible M11 (Lemma 1 holds for every such split)."""
    n = W.shape[0]
    sep = rng.random(n) < sep_frac
    rest = np.nonzero(~sep)[0]
    _, lab = connected_components(W[rest][:, rest], directed=False)
    groups = {}
    for node, l in zip(rest, lab):
        groups.setdefault(l, []).append(node)
    comps = list(groups.values())
    rng.shuffle(comps)
    blocks = []  # merge neighbouring components at random into one block
    for c in comps:
        if blocks and rng.random() < 0.3:
            blocks[-1] = blocks[-1] + list(c)
        else:
            blocks.append(list(c))
    blocks = [list(rng.permutation(b)) for b in blocks]
    perm = np.array([v for b in blocks for v in b] + list(rng.permutation(np.nonzero(sep)[0])),
                    dtype=np.int64)
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    bp = np.concatenate([[0], np.cumsum([len(b) for b in blocks])]).astype(np.int64)
    return {"perm": perm, "iperm": iperm, "block_ptr": bp, "n1": int(bp[-1]),
            "n2": n - int(bp[-1])}


# ---------------------------------------------------------------- partition
def test_partition_golden_path7():
    g = synth.path(7)
    p = O.partition(g.n, g.rowptr, g.col, n_hubs=0, block_max=3, split=True)
    want = {}
    for line in open(os.path.join(GOLDEN, "partition_path7.txt")):
        if line.strip() and not line.startswith("#"):
            k, *v = line.split()
            want[k] = [int(x) for x in v]
    assert p["perm"].tolist() == want["perm"]
    assert p["block_ptr"].tolist() == want["block_ptr"]
    assert p["n1"] == want["n1"][0] and p["n2"] == want["n2"][0]


def test_partition_star_hub():
    g = synth.star(5)
    p = O.partition(g.n, g.rowptr, g.col, n_hubs=1, block_max=4)
    assert p["perm"].tolist() == [1, 2, 3, 4, 5, 0]
    assert p["block_ptr"].tolist() == [0, 1, 2, 3, 4, 5]


@pytest.mark.parametrize("split,hubs,bmax", [(True, 0, 16), (True, 10, 32), (False, 20, 8)])
def test_partition_properties(split, hubs, bmax):
    g = synth.chung_lu(600, 2.1, 6.0, 120.0, seed=7)
    W = W_of(g)
    p = O.partition(g.n, g.rowptr, g.col, hubs, bmax, split)
    O.check_partition(W, p)
    sizes = np.diff(p["block_ptr"])
    if split:
        assert sizes.max() <= bmax
    assert (np.diff(sizes) >= 0).all()
    deg = g.degrees()
    top = np.lexsort((np.arange(g.n), -deg))[:hubs]
    assert set(top.tolist()) <= set(p["perm"][p["n1"]:].tolist())


# ------------------------------------------------------------------ Lemma 1
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lemma1_any_partition_gives_direct_solution(seed):
    rng = np.random.default_rng(seed)
    g = synth.sbm_bernoulli([25, 25, 30], 0.15, 0.02, seed=seed + 40, weighted=True)
    W = W_of(g)
    b = 0.85 / O.lambda_max(W)
    part = random_partition(W, rng, 0.25)
    O.check_partition(W, part)
    idx = O.lrc_build(W, b, part, rank=4, block_max=10 ** 9)
    Q = [0, 26, 79]
    B = b * W[:, Q].toarray()
    res = O.lrc_query(idx, B, tol=1e-14)
    Kd = O.katz_direct(W, b, Q)
    assert O.error_inf_rel(res["K"], Kd).max() < 1e-11
    # Eq. 7: F equals B2 - M12^T M11^{-1} B1 written out densely
    n1 = part["n1"]
    Mp = (np.eye(g.n) - b * W.toarray())[part["perm"]][:, part["perm"]]
    Bp = B[part["perm"]]
    F = Bp[n1:] - Mp[:n1, n1:].T @ np.linalg.solve(Mp[:n1, :n1], Bp[:n1])
    np.testing.assert_allclose(res["F"], F, rtol=1e-10, atol=1e-15)


def test_lrc_with_project_partition_and_large_blocks():
    g = synth.chung_lu(400, 2.1, 5.0, 80.0, seed=3)
    W = W_of(g)
    b = 0.9 / O.lambda_max(W)
    Q = [1, 50, 399]
    for split, bmax in [(True, 8), (False, 8)]:
        res, idx = O.katz_lrc(W, b, Q, n_hubs=8, block_max=bmax, rank=6, split=split)
        assert O.error_inf_rel(res["K"], O.katz_direct(W, b, Q)).max() < 1e-11


# ----------------------------------------- Eq. 13, Theorem 1 and Lanczos
def _idx(seed=0, rank=5, hubs=6):
    g = synth.chung_lu(300, 2.1, 6.0, 60.0, seed=seed)
    W = W_of(g)
    b = 0.9 / O.lambda_max(W)
    part = O.partition(g.n, g.rowptr, g.col, hubs, 6, True)
    return W, b, O.lrc_build(W, b, part, rank, block_max=6)


def test_full_rank_correction_is_exact_inverse():
    """With all n2 eigenpairs, S~^{-1} = S^{-1} (Eq. 13) and PCG converges
    in one iteration."""
    W, b, idx0 = _idx(rank=10 ** 6)
    n2 = idx0["n2"]
    # Lanczos stops on an invariant subspace; eigenvalue 0 of R (separator
    # nodes without M11 neighbours) contributes D = 0, so every nonzero
    # sigma must be present.
    sig_all = np.sort(np.linalg.eigvalsh(idx0["R"]))[::-1]
    nz = sig_all[sig_all > 1e-10]
    np.testing.assert_allclose(idx0["sigma"][: len(nz)], nz, rtol=1e-9)
    St = idx0["M22inv"] + idx0["Wr"] @ np.diag(idx0["D"]) @ idx0["Wr"].T
    np.testing.assert_allclose(St @ idx0["S"], np.eye(n2), atol=1e-9)
    B = b * W[:, [3, 9]].toarray()
    res = O.lrc_query(idx0, B, tol=1e-9)
    assert (res["iters"] <= 1).all() and res["iters"].max() == 1


def test_rank_zero_is_plain_M22_preconditioner():
    W, b, idx = _idx(rank=0)
    assert idx["Wr"].shape[1] == 0
    B = b * W[:, [4]].toarray()
    res = O.lrc_query(idx, B, tol=1e-13)
    assert O.error_inf_rel(res["K"], O.katz_direct(W, b, [4])).max() < 1e-11


@pytest.mark.parametrize("rank", [1, 4, 9])
def test_theorem1_spectrum(rank):
    """eig(S S~^{-1}) = {1 (rank times)} U {1 - sigma_i, i > rank}
    with sigma the eigenvalues of R (Theorem 1)."""
    W, b, idx = _idx(seed=1, rank=rank)
    sig_all = np.sort(np.linalg.eigvalsh(idx["R"]))[::-1]
    want = np.sort(np.concatenate([np.ones(rank), 1 - sig_all[rank:]]))
    got = O.schur_precond_spectrum(idx)
    np.testing.assert_allclose(got, want, atol=1e-9)


def test_ritz_values_match_dense_eigenvalues_and_bounds():
    W, b, idx = _idx(seed=2, rank=8)
    sig_all = np.sort(np.linalg.eigvalsh(idx["R"]))[::-1]
    np.testing.assert_allclose(idx["sigma"], sig_all[:8], rtol=1e-9, atol=1e-12)
    assert (sig_all >= -1e-12).all() and (sig_all < 1).all()
    # W_r^T M22 W_r = I (W_r = L^{-T} U_r with orthonormal U_r)
    G = idx["Wr"].T @ idx["M22"] @ idx["Wr"]
    np.testing.assert_allclose(G, np.eye(8), atol=1e-9)
    # S = L (I - R) L^T (the identity before Eq. 11)
    L = idx["L"]
    np.testing.assert_allclose(L @ (np.eye(idx["n2"]) - idx["R"]) @ L.T, idx["S"], atol=1e-10)


def test_pcg_fewer_iterations_with_more_rank():
    W, b, i1 = _idx(seed=3, rank=1)
    _, _, i8 = _idx(seed=3, rank=12)
    B = b * W[:, [0, 5, 8, 13]].toarray()
    it1 = O.lrc_query(i1, B, tol=1e-10)["iters"]
    it8 = O.lrc_query(i8, B, tol=1e-10)["iters"]
    assert it8.sum() <= it1.sum()


# ------------------------------------------------------------ warm-start MLP
# Phi(1) and phi(1) of the standard normal distribution (printed tables;
# phi(1) = exp(-1/2) / sqrt(2 pi)).
PHI1 = 0.8413447460685429
DPHI1 = 0.24197072451914337


def test_gelu_against_normal_table_values():
    """GELU(x) = x Phi(x): GELU(0) = 0, GELU(1) = Phi(1), GELU(-1) =
    -(1 - Phi(1)), the odd part GELU(x) - GELU(-x) = x, GELU(x) -> x for
    large x; its derivative Phi(x) + x phi(x) is 1/2 at 0 and
    Phi(1) + phi(1) at 1."""
    from oracle import katz_oracle
    assert O.gelu(np.array(0.0)) == 0.0
    assert O.gelu(np.array(1.0)) == pytest.approx(PHI1, rel=1e-15)
    assert O.gelu(np.array(-1.0)) == pytest.approx(-(1.0 - PHI1), rel=1e-14)
    x = np.array([-3.0, -0.5, 0.7, 2.5, 9.0])
    np.testing.assert_allclose(O.gelu(x) - O.gelu(-x), x, rtol=1e-14)
    assert O.gelu(np.array(12.0)) == pytest.approx(12.0, rel=1e-15)
    assert katz_oracle._gelu_grad(np.array(0.0)) == pytest.approx(0.5, rel=1e-15)
    assert katz_oracle._gelu_grad(np.array(1.0)) == pytest.approx(PHI1 + DPHI1, rel=1e-14)


def test_mlp_forward_written_out():
    """A 2 -> 2 -> 1 network by hand: with W1 = [[1, 0], [0, -1]], b1 = 0
    and x = (1, 1) the hidden pre-activations are (1, -1), so the hidden
    layer is (Phi(1), -(1 - Phi(1))); W2 = [[1, 2]], b2 = 1/2 gives
    y = Phi(1) - 2 (1 - Phi(1)) + 1/2.  A second row x = (0, 0) gives
    y = b2 (GELU(0) = 0)."""
    X = np.array([[1.0, 1.0], [0.0, 0.0]])
    W1 = np.array([[1.0, 0.0], [0.0, -1.0]])
    b1 = np.zeros(2)
    W2 = np.array([[1.0, 2.0]])
    b2 = np.array([0.5])
    Y, Hp, H = O.mlp_forward(X, W1, b1, W2, b2)
    np.testing.assert_array_equal(Hp, [[1.0, -1.0], [0.0, 0.0]])
    np.testing.assert_allclose(H[0], [PHI1, -(1.0 - PHI1)], rtol=1e-14)
    assert Y.shape == (2, 1)
    assert Y[0, 0] == pytest.approx(PHI1 - 2.0 * (1.0 - PHI1) + 0.5, rel=1e-14)
    assert Y[1, 0] == 0.5
    # loss of the target row t = y - 1 (error 1 on one row, 0 on the other)
    # is mean(||e||^2) / 2 = 1/4, and dL/db2 = mean(e) = 1/2
    T = Y - np.array([[1.0], [0.0]])
    loss, (_, _, _, db2) = O.mlp_loss_grad(X, T, W1, b1, W2, b2)
    assert loss == pytest.approx(0.25, rel=1e-14)
    np.testing.assert_allclose(db2, [0.5], rtol=1e-14)


def test_mlp_gradients_finite_differences():
    rng = np.random.default_rng(0)
    X = rng.normal(size=(7, 5))
    T = rng.normal(size=(7, 3))
    W1 = rng.normal(size=(6, 5)) * 0.5
    b1 = rng.normal(size=6) * 0.1
    W2 = rng.normal(size=(3, 6)) * 0.5
    b2 = rng.normal(size=3) * 0.1
    params = [W1, b1, W2, b2]
    loss, grads = O.mlp_loss_grad(X, T, *params)
    h = 1e-6
    for p, g in zip(params, grads):
        it = np.nditer(p, flags=["multi_index"])
        for _ in it:
            i = it.multi_index
            old = p[i]
            p[i] = old + h
            lp, _ = O.mlp_loss_grad(X, T, *params)
            p[i] = old - h
            lm, _ = O.mlp_loss_grad(X, T, *params)
            p[i] = old
            assert g[i] == pytest.approx((lp - lm) / (2 * h), rel=1e-6, abs=1e-8)


def test_adamw_first_step_closed_form():
    """From zero moments, bias correction makes the first step
    -lr * g/(|g|+eps) - lr*wd*p."""
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -0.01, 0.0])
    p1, m, v = O.adamw_step(p, g, np.zeros(3), np.zeros(3), 1, lr=0.1, wd=0.01)
    want = p - 0.1 * (g / (np.abs(g) + 1e-8) + 0.01 * p)
    np.testing.assert_allclose(p1, want, rtol=1e-12)


def test_adamw_steps_two_and_three_by_hand():
    """Steps t = 2, 3 where the bias corrections 1 - b^t differ from the
    first step's.  With b1 = 1/2, b2 = 3/4, lr = 1, eps = wd = 0 and the
    scalar gradients 2, -2, 1 from p = 0, written out by hand:
      t=1: m = 1,     v = 1,      m^ = 2,    v^ = 4,      p = -1
      t=2: m = -1/2,  v = 7/4,    m^ = -2/3, v^ = 4,      p = -1 + 1/3
      t=3: m = 1/4,   v = 25/16,  m^ = 2/7,  v^ = 100/37, p = -2/3 - sqrt(37)/35
    and a constant gradient, for which every bias-corrected step is the
    same -lr * g/(|g| + eps) - lr*wd*p whatever t is."""
    p, m, v = np.zeros(1), np.zeros(1), np.zeros(1)
    want = [-1.0, -2.0 / 3.0, -2.0 / 3.0 - np.sqrt(37.0) / 35.0]
    for t, (g, w) in enumerate(zip((2.0, -2.0, 1.0), want), start=1):
        p, m, v = O.adamw_step(p, np.array([g]), m, v, t, lr=1.0, b1=0.5, b2=0.75, eps=0.0)
        np.testing.assert_allclose(p, [w], rtol=1e-14)
    np.testing.assert_allclose(m, [0.25], rtol=1e-14)
    np.testing.assert_allclose(v, [25.0 / 16.0], rtol=1e-14)
    g = np.array([0.3, -0.02, 1e-3])
    p, m, v = np.array([1.0, -2.0, 0.5]), np.zeros(3), np.zeros(3)
    for t in range(1, 4):
        want = p - 0.05 * (g / (np.abs(g) + 1e-8) + 0.01 * p)
        p, m, v = O.adamw_step(p, g, m, v, t, lr=0.05, wd=0.01)
        np.testing.assert_allclose(p, want, rtol=1e-12)


def test_union_with_folded_damping_is_block_diagonal():
    """Disjoint graphs with each graph's damping folded into its weights
    (W~ = beta_g W_g on graph g's block, index beta = 1): the union's Katz
    column of a node is that graph's own Katz vector (zero on the other
    graphs), and with each graph's own hubs as separator the union's Schur
    complement and R (Eq. 11) are block diagonal, block g equal to the S_g
    and R_g of graph g built alone (Lemma 1 on a block-diagonal M)."""
    gs = [synth.erdos_renyi(45, 0.12, seed=s, weighted=s % 2 == 0) for s in (1, 2, 3)]
    Ws = [W_of(g) for g in gs]
    betas = [c / O.lambda_max(W) for c, W in zip((0.6, 0.8, 0.95), Ws)]
    Wt = sp.block_diag([b * W for b, W in zip(betas, Ws)]).tocsr()
    offs = np.concatenate([[0], np.cumsum([g.n for g in gs])])
    for gi, g in enumerate(gs):
        Ku = O.katz_direct(Wt, 1.0, [offs[gi] + 5])[:, 0]
        Kg = O.katz_direct(Ws[gi], betas[gi], [5])[:, 0]
        np.testing.assert_allclose(Ku[offs[gi]:offs[gi + 1]], Kg, rtol=1e-12, atol=1e-15)
        assert np.abs(np.delete(Ku, np.arange(offs[gi], offs[gi + 1]))).max() == 0.0
    # per-graph partitions (each graph's 4 highest degrees) joined graph-major
    parts = [O.partition(g.n, g.rowptr, g.col, 4, 64, False) for g in gs]
    blocks, seps, bptr = [], [], [0]
    for gi, p in enumerate(parts):
        bp = p["block_ptr"]
        for k in range(len(bp) - 1):
            blocks.append(offs[gi] + p["perm"][bp[k]:bp[k + 1]])
            bptr.append(bptr[-1] + bp[k + 1] - bp[k])
        seps.append(offs[gi] + p["perm"][p["n1"]:])
    perm = np.concatenate(blocks + seps).astype(np.int64)
    n1 = int(sum(p["n1"] for p in parts))
    part_u = {"perm": perm, "block_ptr": np.array(bptr), "n1": n1, "n2": len(perm) - n1}
    U = O.lrc_build(Wt, 1.0, part_u, 2)
    s0 = 0
    for gi, (g, p) in enumerate(zip(gs, parts)):
        ref = O.lrc_build(Ws[gi], betas[gi], p, 2)
        s1 = s0 + ref["n2"]
        np.testing.assert_allclose(U["S"][s0:s1, s0:s1], ref["S"], rtol=1e-11, atol=1e-14)
        np.testing.assert_allclose(U["R"][s0:s1, s0:s1], ref["R"], rtol=1e-10, atol=1e-13)
        off = np.delete(U["S"][s0:s1], np.arange(s0, s1), axis=1)
        assert np.abs(off).max() == 0.0
        s0 = s1


def test_packed_columns_give_every_graph_block():
    """One M11 solve of width max_g n2_g, with separator node l of EVERY
    graph in column l, yields each graph's block of T = M12^T M11^{-1} M12
    (Lemma 1): the graphs' right-hand sides occupy disjoint rows of the
    block-diagonal M11, so they never mix.  Dense FP64 on the union."""
    gs = [synth.erdos_renyi(n, 0.1, seed=n) for n in (30, 45, 60)]
    Ws = [W_of(g) for g in gs]
    betas = [0.9 / O.lambda_max(W) for W in Ws]
    Wt = sp.block_diag([b * W for b, W in zip(betas, Ws)]).tocsr()
    offs = np.concatenate([[0], np.cumsum([g.n for g in gs])])
    hubs = [offs[gi] + np.argsort(-np.diff(g.rowptr), kind="stable")[:h]
            for gi, (g, h) in enumerate(zip(gs, (3, 5, 4)))]
    sep = np.concatenate(hubs)
    rest = np.setdiff1d(np.arange(offs[-1]), sep)
    M = np.eye(offs[-1]) - Wt.toarray()
    M11, M12 = M[np.ix_(rest, rest)], M[np.ix_(rest, sep)]
    T = M12.T @ np.linalg.solve(M11, M12)          # the whole n2 x n2 at once
    width = max(len(h) for h in hubs)
    E = np.zeros((len(sep), width))
    gstart = np.concatenate([[0], np.cumsum([len(h) for h in hubs])])
    for gi in range(len(gs)):
        for l in range(len(hubs[gi])):
            E[gstart[gi] + l, l] = 1.0
    Tp = M12.T @ np.linalg.solve(M11, M12 @ E)      # one packed solve
    for gi in range(len(gs)):
        a, b = gstart[gi], gstart[gi + 1]
        np.testing.assert_allclose(Tp[a:b, :b - a], T[a:b, a:b], rtol=1e-12, atol=1e-14)
        if b - a < width:  # columns past this graph's separator stay empty on its rows
            assert np.abs(Tp[a:b, b - a:]).max() == 0.0
