"""Pins, on the FP64 oracle's pieces, of two regroupings the query path
uses (host only):

* the first Schur right-hand side of a query from the coupling
  Z = beta M11^{-1} W12: F = B2 - M12^T M11^{-1} B1 (Eq. 7) equals
  B2 + Z^T B1 because M11 is symmetric, and Z^T B1 is a sum over the
  deg(q) rows of Z that the sparse B1 = beta W e_q touches;
* refinement corrections whose Y1 = M11^{-1} R1 is replaced by the first
  Chebyshev iterate R1 / theta (theta the centre of M11's spectrum) still
  converge to the Katz vectors: the error of Y1 only enters the Schur
  right-hand side, so with the back-substitution K1 = M11^{-1}(R1 - M12 K2)
  solved exactly the residual after such a correction is confined to the
  separator rows, and every pass measures the true residual."""
import numpy as np
import scipy.sparse as sp

import oracle as O
from paper_1912_06525_gb300 import synth


def _graph():
    g = synth.modular_hubs(3000, 12, np.log(250.0), 0.5, 12.0, 0.05, 20, 150, seed=5)
    return O.adjacency(g.n, g.rowptr, g.col, g.val), g


def _index(W, beta):
    part = O.partition(W.shape[0], W.indptr, W.indices, 20, 64, False)
    return O.lrc_build(W, beta, part, rank=8, block_max=64), part


def test_first_schur_rhs_from_the_stored_coupling():
    W, g = _graph()
    beta = 0.9 / O.lambda_max(W)
    idx, part = _index(W, beta)
    n1 = idx["n1"]
    assert n1 > 0 and idx["n2"] > 0
    # M11 symmetric, so (M11^{-1} M12)^T = M12^T M11^{-1}
    assert abs(idx["M11"] - idx["M11"].T).max() == 0
    Z = -idx["m11"].solve(idx["M12"])           # beta M11^{-1} W12 (M12 = -beta W12)
    Wp = idx["Wp"]
    assert np.allclose(Z, beta * idx["m11"].solve(Wp[:n1, n1:].toarray()), rtol=0, atol=1e-15)
    rng = np.random.default_rng(3)
    Q = rng.choice(g.n, size=24, replace=False)
    Q[0] = int(part["perm"][n1])              # a separator node
    B = beta * W[:, Q].toarray()
    ref = O.lrc_query(idx, B)
    Bp = B[part["perm"]]
    B1, B2 = Bp[:n1], Bp[n1:]
    # gather form: column j sums the rows of Z at the nonzeros of B1[:, j]
    F = B2.copy()
    for j in range(len(Q)):
        rows = np.nonzero(B1[:, j])[0]
        assert len(rows) <= W[:, Q[j]].nnz
        F[:, j] += Z[rows].T @ B1[rows, j]
    scale = np.abs(ref["F"]).max()
    assert np.abs(F - ref["F"]).max() <= 1e-13 * scale
    # and the dense product with the other sign convention
    assert np.abs(B2 + Z.T @ B1 - ref["F"]).max() <= 1e-13 * scale


def _correction(idx, R, theta, one_step_y1):
    """D ~ M^{-1} R by one LRC pass (Lemma 1, Eqs. 6-7) in index order, with
    the exact Y1 or with Y1 = R1 / theta; S K2 = F solved directly."""
    n1 = idx["n1"]
    R1, R2 = R[:n1], R[n1:]
    Y1 = R1 / theta if one_step_y1 else idx["m11"].solve(R1)
    F = R2 - idx["M12"].T @ Y1
    K2 = np.linalg.solve(idx["S"], F)
    K1 = idx["m11"].solve(R1 - idx["M12"] @ K2)
    return np.vstack([K1, K2])


def test_corrections_with_a_one_step_y1_still_converge():
    W, g = _graph()
    beta = 0.9 / O.lambda_max(W)
    idx, part = _index(W, beta)
    n1 = idx["n1"]
    ev = np.linalg.eigvalsh(idx["Wp"][:n1, :n1].toarray())
    theta = 1.0 - 0.5 * beta * (ev[-1] + ev[0])  # centre of M11's spectrum
    Q = np.random.default_rng(9).choice(g.n, size=8, replace=False)
    B = (beta * W[:, Q].toarray())[part["perm"]]
    Mp = sp.eye(g.n, format="csr") - beta * idx["Wp"]
    ref = O.katz_direct(W, beta, Q)[part["perm"]]
    for one_step in (False, True):
        K = np.zeros_like(B)
        norms = []
        for it in range(40):
            R = B - Mp @ K
            norms.append(np.linalg.norm(R, axis=0).max())
            if it > 0:  # the M11 rows were solved exactly by the last correction
                assert np.abs(R[:n1]).max() <= 1e-14 * np.abs(B).max()
            if norms[-1] <= 1e-14 * np.linalg.norm(B, axis=0).max():
                break
            K = K + _correction(idx, R, theta, one_step)
        # each pass shrinks the residual (exact Y1: in one pass to rounding)
        assert all(b < 0.5 * a for a, b in zip(norms, norms[1:]) if a > 1e-13)
        assert np.abs(K - ref).max() <= 1e-12 * np.abs(ref).max()
        if one_step:
            # the inexact Y1 leaves a separator residual for one more pass
            assert len(norms) == 3 and norms[1] > 1e-6 * norms[0]
