"""Pins of the oracle's Sparse-Katz (Algorithm 3, Section 3.3, Fig. 2)
against routes that do not go through it: the dense inverse of M with
SciPy's Pearson routine and Python sorting on tiny graphs (brute force),
the star graph's closed-form Katz matrix, the two-landmark case where the
Pearson correlation is the sign of a product, and the one-landmark case
that leaves the Katz order unchanged."""
import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_1912_06525_gb300 import synth


def W_of(g):
    return O.adjacency(g.n, g.rowptr, g.col, g.val)


def test_pearson_against_library_and_its_invariances():
    rng = np.random.default_rng(3)
    for T in (2, 3, 9, 40):
        x, y = rng.normal(size=T), rng.normal(size=T)
        assert O.pearson(x, y) == pytest.approx(stats.pearsonr(x, y)[0], abs=1e-13)
        # invariant under positive affine maps, odd under negation
        assert O.pearson(3 * x + 7, 0.5 * y - 2) == pytest.approx(O.pearson(x, y), abs=1e-13)
        assert O.pearson(-x, y) == pytest.approx(-O.pearson(x, y), abs=1e-13)
        assert O.pearson(x, 2 * x + 1) == pytest.approx(1.0, abs=1e-14)
    assert O.pearson(np.ones(5), rng.normal(size=5)) == 0.0
    assert O.pearson(np.array([2.0]), np.array([7.0])) == 0.0


def brute_force(W, beta, q, s, T):
    """Dense K = (I - beta W)^{-1} - I, Python sorting, SciPy Pearson."""
    n = W.shape[0]
    K = np.linalg.inv(np.eye(n) - beta * W.toarray()) - np.eye(n)
    nb = set(W.indices[W.indptr[q]:W.indptr[q + 1]].tolist())
    cand = sorted((j for j in range(n) if j != q and j not in nb), key=lambda j: (-K[j, q], j))[:s]
    land = sorted((j for j in range(n) if j != q), key=lambda j: (-K[j, q], j))[:T]
    rho = []
    for c in cand:
        x, y = K[q, land], K[c, land]
        rho.append(0.0 if np.ptp(x) == 0 or np.ptp(y) == 0 else stats.pearsonr(x, y)[0])
    order = sorted(range(len(cand)), key=lambda i: (-rho[i], i))
    return [cand[i] for i in order], [rho[i] for i in order], land


@pytest.mark.parametrize("seed,s,T", [(1, 5, 3), (2, 8, 9), (3, 20, 6), (4, 3, 25)])
def test_sparse_katz_brute_force(seed, s, T):
    g = synth.erdos_renyi(45, 0.12, seed=seed, weighted=seed % 2 == 0)
    W = W_of(g)
    beta = 0.8 / O.lambda_max(W)
    Q = [0, 7, 19, 44]
    ids, rho, land, cand = O.sparse_katz(W, beta, Q, s, T)
    for j, q in enumerate(Q):
        bi, br, bl = brute_force(W, beta, q, s, T)
        assert land[j].tolist() == bl
        m = len(bi)
        assert ids[j, :m].tolist() == bi and (ids[j, m:] == -1).all()
        np.testing.assert_allclose(rho[j, :m], br, atol=1e-10, rtol=0)
        # the re-ranking permutes the Katz-ordered candidate list
        assert sorted(ids[j, :m].tolist()) == sorted(cand[j, :m].tolist())


@pytest.mark.parametrize("m,s,T", [(6, 3, 4), (12, 8, 9)])
def test_sparse_katz_star_closed_form(m, s, T):
    """Star with hub 0: for leaves i, c and any landmark leaf t (c = t
    included) K[c, t] = beta^2/d and K[c, 0] = beta/d (d = 1 - m beta^2), so
    row c of K_T equals row q of K_T for every candidate leaf c: rho = 1 and
    the Katz order (tied leaves by id) stays."""
    W = W_of(synth.star(m))
    beta = 0.6 / np.sqrt(m)
    d = 1 - m * beta * beta
    K = np.full((m + 1, m + 1), beta * beta / d)  # leaf-leaf, self included
    K[0, 1:] = K[1:, 0] = beta / d
    K[0, 0] = m * beta * beta / d

    def closed_form(W_, b_, cols):
        return K[:, np.asarray(cols)]

    ids, rho, land, _ = O.sparse_katz(W, beta, [1], s, T, solve=closed_form)
    assert land[0].tolist() == [0] + list(range(2, T + 1))
    assert ids[0].tolist() == list(range(2, s + 2))
    np.testing.assert_allclose(rho[0], 1.0, atol=1e-12)


def test_sparse_katz_two_landmarks_sign_rule():
    """With T = 2 the Pearson correlation of two 2-vectors is the sign of
    (x1 - x2)(y1 - y2): rho_c = sign((K[q,t1] - K[q,t2]) (K[c,t1] - K[c,t2]))."""
    g = synth.erdos_renyi(40, 0.1, seed=9, weighted=True)
    W = W_of(g)
    beta = 0.9 / O.lambda_max(W)
    K = O.katz_matrix(W, beta)
    for q in (3, 11, 30):
        ids, rho, land, _ = O.sparse_katz(W, beta, [q], 10, 2)
        t1, t2 = land[0]
        for c, r in zip(ids[0], rho[0]):
            if c < 0:
                continue
            assert r == pytest.approx(np.sign((K[q, t1] - K[q, t2]) * (K[c, t1] - K[c, t2])), abs=1e-13)


def test_sparse_katz_one_landmark_keeps_katz_order():
    g = synth.erdos_renyi(50, 0.08, seed=5)
    W = W_of(g)
    beta = 0.7 / O.lambda_max(W)
    Q = [2, 9]
    ids, rho, _, cand = O.sparse_katz(W, beta, Q, 12, 1)
    lp, _ = O.linkpred_topk(W, O.katz_direct(W, beta, Q), Q, 12)
    assert (rho == 0).all()
    assert ids.tolist() == lp.tolist() == cand.tolist()


def test_sparse_katz_golden_star_fixture():
    """The hand derivation in tests/golden/sparse_katz_star.txt, with the
    closed-form Katz columns (exact ties) fed to the oracle."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "sparse_katz_star.txt")
    fx = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            key, *vals = line.split()
            fx[key] = vals
    m = int(fx["graph"][1])
    W = W_of(synth.star(m))
    beta = 0.5 / np.sqrt(m)
    d = 1 - m * beta * beta
    K = np.full((m + 1, m + 1), beta * beta / d)
    K[0, 1:] = K[1:, 0] = beta / d
    K[0, 0] = m * beta * beta / d
    ids, rho, land, cand = O.sparse_katz(W, beta, [int(fx["query"][0])], int(fx["s"][0]),
                                         int(fx["T"][0]), solve=lambda W_, b_, c: K[:, c])
    assert land[0].tolist() == [int(v) for v in fx["landmarks"]]
    assert cand[0].tolist() == [int(v) for v in fx["candidates"]]
    assert ids[0].tolist() == [int(v) for v in fx["ids"]]
    np.testing.assert_allclose(rho[0], [float(v) for v in fx["rho"]], atol=1e-12)
