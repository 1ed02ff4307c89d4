"""Pins for the oracle's Katz definitions (Section 3.1, Eqs. 1-3).

Each check ties the oracle to something other than itself: closed forms
derived by hand, the walk-count series, the spectral form of the
eigen-decomposition, invariants of K, or brute force.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1912_06525_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def W_of(g):
    return O.adjacency(g.n, g.rowptr, g.col, g.val)


# ------------------------------------------------------------ closed forms
@pytest.mark.parametrize("b", [0.1, 0.5, 0.9])
def test_single_edge_closed_form(b):
    W = W_of(synth.single_edge())
    K = O.katz_matrix(W, b)
    assert K[0, 1] == pytest.approx(b / (1 - b * b), rel=1e-13)
    assert K[0, 0] == pytest.approx(b * b / (1 - b * b), rel=1e-13)
    Kd = O.katz_direct(W, b, [0, 1])
    np.testing.assert_allclose(Kd, K, rtol=1e-12, atol=0)


@pytest.mark.parametrize("m", [1, 3, 10])
def test_star_closed_form(m):
    W = W_of(synth.star(m))
    b = 0.7 / np.sqrt(m)  # beta * lambda_max = 0.7
    d = 1 - m * b * b
    K = O.katz_direct(W, b, np.arange(m + 1))
    assert K[0, 0] == pytest.approx(m * b * b / d, rel=1e-12)
    for leaf in range(1, m + 1):
        assert K[leaf, 0] == pytest.approx(b / d, rel=1e-12)
        assert K[leaf, leaf] == pytest.approx(b * b / d, rel=1e-12)
        for other in range(1, m + 1):
            if other != leaf:
                assert K[other, leaf] == pytest.approx(b * b / d, rel=1e-12)


@pytest.mark.parametrize("n", [2, 5, 12])
def test_complete_graph_closed_form(n):
    W = W_of(synth.complete(n))
    b = 0.6 / (n - 1)
    K = O.katz_matrix(W, b)
    kij = b / ((1 + b) * (1 + b - n * b))
    kii = (1 / (1 + b)) * (1 + b / (1 + b - n * b)) - 1
    off = K[~np.eye(n, dtype=bool)]
    np.testing.assert_allclose(off, kij, rtol=1e-12)
    np.testing.assert_allclose(np.diag(K), kii, rtol=1e-11)


def test_apply_M_written_out_on_a_weighted_path():
    """M X = X - beta W X (Eq. 3) on the path 0 -(2)- 1 -(1/2)- 2 at
    beta = 1/4, so M = [[1, -1/2, 0], [-1/2, 1, -1/8], [0, -1/8, 1]]; the
    products below are worked out by hand (all exact in binary)."""
    rowptr = np.array([0, 1, 3, 4])
    col = np.array([1, 0, 2, 1])
    val = np.array([2.0, 2.0, 0.5, 0.5])
    W = O.adjacency(3, rowptr, col, val)
    X = np.array([[1.0, 0.0], [2.0, 1.0], [4.0, -8.0]])
    Y = O.apply_M(W, 0.25, X)
    np.testing.assert_array_equal(Y, [[0.0, -0.5], [1.0, 2.0], [3.75, -8.125]])


@pytest.mark.parametrize("n", [3, 8, 13])
def test_cycle_spectral_form(n):
    """C_n is circulant: eigenvalues 2 cos(2 pi k / n), Fourier vectors."""
    W = W_of(synth.cycle(n))
    b = 0.45
    K = O.katz_direct(W, b, np.arange(n))
    k = np.arange(n)
    lam = 2 * np.cos(2 * np.pi * k / n)
    for i in range(n):
        for j in range(n):
            ref = np.mean((1 / (1 - b * lam) - 1) * np.cos(2 * np.pi * k * (i - j) / n))
            assert K[i, j] == pytest.approx(ref, rel=1e-11, abs=1e-14)


@pytest.mark.parametrize("n", [4, 9])
def test_path_spectral_form(n):
    """P_n: eigenvalues 2 cos(pi k/(n+1)), vectors sqrt(2/(n+1)) sin(pi j k/(n+1))."""
    W = W_of(synth.path(n))
    b = 0.4
    k = np.arange(1, n + 1)
    lam = 2 * np.cos(np.pi * k / (n + 1))
    V = np.sqrt(2 / (n + 1)) * np.sin(np.pi * np.outer(np.arange(1, n + 1), k) / (n + 1))
    Kref = V @ np.diag(1 / (1 - b * lam) - 1) @ V.T
    np.testing.assert_allclose(O.katz_matrix(W, b), Kref, rtol=1e-11, atol=1e-14)


def test_golden_closed_forms_file_is_consistent():
    """The hand-derived table in tests/golden agrees with the oracle."""
    lines = [l.split(None, 3) for l in open(os.path.join(GOLDEN, "closed_forms.txt"))
             if l.strip() and not l.startswith("#")]
    b, m, n = 0.15, 4, 6
    env = {"b": b, "m": m, "n": n}
    mats = {"single_edge": O.katz_matrix(W_of(synth.single_edge()), b),
            "star": O.katz_matrix(W_of(synth.star(m)), b),
            "complete": O.katz_matrix(W_of(synth.complete(n)), b)}
    where = {"K01": (0, 1), "K00": (0, 0), "K0_leaf": (0, 1), "Kleaf_leaf": (1, 1),
             "Kleaf_other": (1, 2), "Kij": (0, 1), "Kii": (0, 0)}
    for g, _, entry, formula in lines:
        val = eval(formula.replace("^", "**"), {}, env)
        assert mats[g][where[entry]] == pytest.approx(val, rel=1e-12)


# ---------------------------------------------------------- lambda_max
def test_lambda_max_closed_forms():
    assert O.lambda_max(W_of(synth.complete(7))) == pytest.approx(6.0, rel=1e-12)
    assert O.lambda_max(W_of(synth.star(9))) == pytest.approx(3.0, rel=1e-12)
    assert O.lambda_max(W_of(synth.cycle(10))) == pytest.approx(2.0, rel=1e-12)
    assert O.lambda_max(W_of(synth.path(6))) == pytest.approx(2 * np.cos(np.pi / 7), rel=1e-12)


def test_lambda_max_sparse_route_matches_dense():
    g = synth.erdos_renyi(3500, 0.003, seed=3)
    W = W_of(g)
    dense = float(np.linalg.eigvalsh(W.toarray())[-1])
    assert O.lambda_max(W) == pytest.approx(dense, rel=1e-10)


# ------------------------------------------------ series and other routes
@pytest.mark.parametrize("c", [0.3, 0.8])
def test_series_matches_direct_within_tail_bound(c):
    g = synth.erdos_renyi(60, 0.1, seed=5, weighted=True)
    W = W_of(g)
    lam = O.lambda_max(W)
    b = c / lam
    L = 60
    for q in [0, 7, 33]:
        s = O.katz_series(W, b, q, L)
        k = O.katz_direct(W, b, [q])[:, 0]
        bound = (b * lam) ** (L + 1) / (1 - b * lam)
        assert np.linalg.norm(s - k) <= bound * 1.0001 + 1e-14
        assert np.linalg.norm(s - k) < 1e-3 * np.linalg.norm(k) + bound


def test_walk_counts_are_powers_of_W():
    """(W^l)_{ij} counts walks: on the path 0-1-2 there are 2 walks of length
    2 from 1 back to 1 and 1 from 0 to 2; K's series coefficients follow."""
    W = W_of(synth.path(3))
    b = 1e-3
    s = O.katz_series(W, b, 1, 2)
    assert s[1] == pytest.approx(2 * b ** 2, rel=1e-12)
    assert s[0] == pytest.approx(b, rel=1e-9)
    s0 = O.katz_series(W, b, 0, 2)
    assert s0[2] == pytest.approx(b ** 2, rel=1e-12)


def test_dense_inverse_direct_and_cg_agree():
    g = synth.sbm_bernoulli([30, 30, 40], 0.2, 0.02, seed=11, weighted=True)
    W = W_of(g)
    b = 0.9 / O.lambda_max(W)
    Q = [0, 31, 99]
    Kinv = O.katz_matrix(W, b)[:, Q]
    Kd = O.katz_direct(W, b, Q)
    Kc, it = O.katz_cg(W, b, Q, rtol=1e-14)
    np.testing.assert_allclose(Kd, Kinv, rtol=1e-10, atol=1e-14)
    assert O.error_inf_rel(Kc, Kd).max() < 1e-11
    assert (it > 0).all()


# ----------------------------------------------------------- invariants
def test_symmetry_nonnegativity_support_and_lower_bound():
    g = synth.disjoint_union([synth.erdos_renyi(40, 0.1, seed=2, weighted=True),
                              synth.cycle(7), synth.path(1)])
    W = W_of(g)
    b = 0.8 / O.lambda_max(W)
    K = O.katz_direct(W, b, np.arange(g.n))
    np.testing.assert_allclose(K, K.T, rtol=1e-11, atol=1e-15)
    assert (K >= -1e-15).all()
    from scipy.sparse.csgraph import connected_components
    _, comp = connected_components(W, directed=False)
    same = comp[:, None] == comp[None, :]
    iso = g.n - 1
    deg = g.degrees()
    live = (deg[:, None] > 0) & (deg[None, :] > 0)
    assert (K[same & live] > 0).all()
    assert np.all(np.abs(K[~same]) < 1e-15)
    assert np.all(K[:, iso] == 0)
    assert (K >= b * W.toarray() - 1e-15).all()


def test_monotone_in_beta():
    W = W_of(synth.erdos_renyi(50, 0.12, seed=9))
    lam = O.lambda_max(W)
    K1 = O.katz_direct(W, 0.3 / lam, [3, 17])
    K2 = O.katz_direct(W, 0.6 / lam, [3, 17])
    assert (K2 >= K1 - 1e-15).all()


def test_damping_bound_violation_is_detected():
    W = W_of(synth.complete(6))
    with pytest.raises(np.linalg.LinAlgError):
        O.katz_direct(W, 1.05 / 5.0, [0])
    with pytest.raises(ValueError):
        O.katz_cg(W, 1.5 / 5.0, [0, 1, 2])


def test_error_metric():
    ref = np.array([[1.0, 0.0], [-4.0, 0.0]])
    got = np.array([[1.0, 0.0], [-4.0004, 0.0]])
    np.testing.assert_allclose(O.error_inf_rel(got, ref), [1e-4, 0.0], rtol=1e-9)


# ---------------------------------------------------------- link prediction
def test_linkpred_topk_brute_force_and_ties():
    g = synth.star(6)
    W = W_of(g)
    b = 0.3 / np.sqrt(6)
    d = 1 - 6 * b * b
    # exact closed-form columns (Eq. 2 for the star): leaves tie exactly
    K = np.zeros((7, 2))
    K[0, 0], K[1:, 0] = b / d, b * b / d
    K[0, 1], K[1:, 1] = 6 * b * b / d, b / d
    ids, sc = O.linkpred_topk(W, K, [1, 0], 3)
    # leaf 1: candidates are the other leaves (hub is a neighbour), all tied
    assert ids[0].tolist() == [2, 3, 4]
    # hub: every node is a neighbour -> no candidates
    assert ids[1].tolist() == [-1, -1, -1]
    g2 = synth.erdos_renyi(30, 0.15, seed=4, weighted=True)
    W2 = W_of(g2)
    K2 = O.katz_direct(W2, 0.5 / O.lambda_max(W2), [5])
    ids2, sc2 = O.linkpred_topk(W2, K2, [5], 5)
    nb = set(W2.indices[W2.indptr[5]:W2.indptr[6]].tolist()) | {5}
    brute = sorted([(-K2[j, 0], j) for j in range(30) if j not in nb])[:5]
    assert ids2[0].tolist() == [j for _, j in brute]


# --------------------------------------------------------------- SplitMix64
def test_splitmix64_published_vector():
    """SplitMix64 from seed 0: the widely published first outputs."""
    assert O.splitmix64(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                  0x06C45D188009454F]
    u = O.splitmix64_uniform(0, 1)[0]
    assert u == (0xE220A8397B1DCDAF >> 11) / 2.0 ** 53 - 0.5
