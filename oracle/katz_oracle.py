"""FP64 oracle: Katz vectors, the LRC-Katz index and query, link prediction.

Test infrastructure only (see the package docstring).  All arithmetic is
float64.  Notation follows the paper with its damping factor written beta
(the paper's alpha) and the adjacency matrix W (the paper's G):

    K   = sum_{l>=1} beta^l W^l = (I - beta W)^{-1} - I          (Eqs. 1-2)
    M k_q = beta g_q,   M = I - beta W,   g_q = W e_q            (Eq. 3)

Graphs are passed as symmetric CSR triples (n, rowptr, col, val) with
``val`` None for unit weights.
"""
from __future__ import annotations

from collections import deque
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

__all__ = [
    "adjacency", "lambda_max", "katz_matrix", "katz_series", "katz_direct",
    "katz_cg", "apply_M", "partition", "check_partition", "splitmix64", "splitmix64_uniform",
    "lrc_build", "lrc_query", "katz_lrc", "schur_precond_spectrum",
    "linkpred_topk", "top_nodes", "pearson", "sparse_katz", "error_inf_rel", "gelu",
    "mlp_forward", "mlp_loss_grad", "adamw_step",
]


# ---------------------------------------------------------------- basics
def adjacency(n, rowptr, col, val=None) -> sp.csr_matrix:
    """W as a SciPy CSR matrix in float64 (Section 3.1)."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    v = np.ones(col.shape[0]) if val is None else np.asarray(val, dtype=np.float64)
    return sp.csr_matrix((v, col, rowptr), shape=(n, n))


def lambda_max(W: sp.csr_matrix) -> float:
    """Largest eigenvalue of the symmetric W, which equals ||W||_2 for a
    non-negative symmetric matrix; the damping bound is beta < 1/||W||_2
    (Section 3.1, after Eq. 2).  Dense ``eigvalsh`` for small n, ARPACK
    Lanczos otherwise (a library eigen-routine used as one step)."""
    n = W.shape[0]
    if n <= 3000:
        return float(np.linalg.eigvalsh(W.toarray())[-1])
    val = spla.eigsh(W, k=1, which="LA", tol=1e-14, maxiter=100000,
                     v0=np.ones(n), return_eigenvectors=False)
    return float(val[0])


def apply_M(W: sp.csr_matrix, beta: float, X: np.ndarray) -> np.ndarray:
    """M X = X - beta W X, with M = I - beta W (Eq. 3)."""
    return X - beta * (W @ X)


def katz_matrix(W: sp.csr_matrix, beta: float) -> np.ndarray:
    """Dense Katz matrix K = (I - beta W)^{-1} - I (Eq. 2); tiny n only."""
    n = W.shape[0]
    M = np.eye(n) - beta * W.toarray()
    return np.linalg.inv(M) - np.eye(n)


def katz_series(W: sp.csr_matrix, beta: float, q: int, terms: int) -> np.ndarray:
    """Truncated walk-count series sum_{l=1}^{terms} beta^l W^l e_q (Eq. 1,
    with (W^l)_{ij} counting walks of length l, Eq. 2)."""
    n = W.shape[0]
    v = np.zeros(n)
    v[q] = 1.0
    out = np.zeros(n)
    for _ in range(terms):
        v = beta * (W @ v)
        out += v
    return out


def katz_direct(W: sp.csr_matrix, beta: float, Q) -> np.ndarray:
    """Columns q of K by a dense Cholesky solve of M k_q = beta g_q (Eq. 3).

    M is SPD when beta * lambda_max < 1, so the Cholesky factor exists; a
    failure raises ``numpy.linalg.LinAlgError``.  Returns n x b
    (column j = k_{Q[j]})."""
    n = W.shape[0]
    Wd = W.toarray()
    M = np.eye(n) - beta * Wd
    L = np.linalg.cholesky(M)
    B = beta * Wd[:, np.asarray(Q)]
    return sla.cho_solve((L, True), B)


def katz_cg(W: sp.csr_matrix, beta: float, Q, rtol: float = 1e-13,
            maxit: int = 100000, B: np.ndarray | None = None):
    """Plain conjugate gradients on M k = beta g_q, zero start, one column
    per query, each column stopped when ||r||_2 <= rtol ||b||_2 (the
    comparison method of Sections 1 and 4).  Returns (K n x b, iterations
    per column).  A column whose p^T M p <= 0 raises ValueError (M not
    positive definite)."""
    if B is None:
        B = beta * W[:, np.asarray(Q)].toarray()
    B = np.asarray(B, dtype=np.float64)
    n, b = B.shape
    X = np.zeros((n, b))
    R = B.copy()
    P = R.copy()
    rr = np.einsum("ij,ij->j", R, R)
    bnorm = np.sqrt(np.einsum("ij,ij->j", B, B))
    active = np.sqrt(rr) > rtol * bnorm
    iters = np.zeros(b, dtype=np.int64)
    for _ in range(maxit):
        if not active.any():
            break
        a = np.nonzero(active)[0]
        Pa = P[:, a]
        Qa = apply_M(W, beta, Pa)
        pq = np.einsum("ij,ij->j", Pa, Qa)
        if np.any(pq <= 0):
            raise ValueError("p^T M p <= 0: M is not positive definite")
        alpha = rr[a] / pq
        X[:, a] += alpha * Pa
        R[:, a] -= alpha * Qa
        rr_new = np.einsum("ij,ij->j", R[:, a], R[:, a])
        P[:, a] = R[:, a] + (rr_new / rr[a]) * Pa
        rr[a] = rr_new
        iters[a] += 1
        active[a] = np.sqrt(rr_new) > rtol * bnorm[a]
    return X, iters


def error_inf_rel(K: np.ndarray, Kref: np.ndarray) -> np.ndarray:
    """Per-column max |K - Kref| / max |Kref| (the infinity-norm relative
    error; 0 for an all-zero reference column with K exact)."""
    num = np.abs(K - Kref).max(axis=0)
    den = np.abs(Kref).max(axis=0)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)


# --------------------------------------------------------------- partition
def _bfs_order(start, rowptr, col, allowed):
    """FIFO breadth-first order from ``start`` over nodes with allowed[v]
    True; neighbours are visited in CSR order.  Returns (order, level)."""
    order = [start]
    level = {start: 0}
    dq = deque([start])
    while dq:
        u = dq.popleft()
        lu = level[u]
        for v in col[rowptr[u]:rowptr[u + 1]]:
            v = int(v)
            if allowed[v] and v not in level:
                level[v] = lu + 1
                order.append(v)
                dq.append(v)
    return order, level


def partition(n, rowptr, col, n_hubs: int, block_max: int, split: bool = True):
    """Vertex-separator partition and reordering (Section 3.2, Steps 2-3).

    The paper uses a multi-way minimum-vertex-separator partitioner with a
    cap on the separator (METIS); that tool is not used here.  This is the
    project's own reading, stated exactly so that two implementations agree
    node for node:

    1. Hubs: the ``n_hubs`` nodes of largest degree (ties: smaller id)
       go to the separator.
    2. Connected components of the remaining graph are blocks.  If
       ``split`` is true, any block with more than ``block_max`` nodes is
       split: BFS from its smallest-id node; the last node in that BFS order
       roots a second BFS whose level sets L_0..L_d are formed; the first
       level k with 2*(|L_0|+..+|L_k|) >= |block| joins the separator; the
       rest is split into components again, recursively.
    3. Order: blocks by (size, smallest id) ascending, nodes inside a block
       by id; then the separator by id.

    Returns dict(perm, iperm, block_ptr, n1, n2): perm[new] = old node.
    """
    rowptr = np.asarray(rowptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    deg = np.diff(rowptr)
    sep = np.zeros(n, dtype=bool)
    if n_hubs > 0:
        order = np.lexsort((np.arange(n), -deg))
        sep[order[:n_hubs]] = True

    def components(nodes_allowed):
        seen = np.zeros(n, dtype=bool)
        comps = []
        for s in np.nonzero(nodes_allowed)[0]:
            if seen[s]:
                continue
            order, _ = _bfs_order(int(s), rowptr, col, nodes_allowed)
            seen[order] = True
            comps.append(sorted(order))
        return comps

    pending = components(~sep)
    blocks = []
    while pending:
        c = pending.pop()
        if not split or len(c) <= block_max:
            blocks.append(c)
            continue
        allowed = np.zeros(n, dtype=bool)
        allowed[c] = True
        o1, _ = _bfs_order(c[0], rowptr, col, allowed)
        root = o1[-1]
        o2, lev = _bfs_order(root, rowptr, col, allowed)
        depth = max(lev.values())
        counts = np.bincount(np.array([lev[v] for v in o2]), minlength=depth + 1)
        cum = np.cumsum(counts)
        k = int(np.nonzero(2 * cum >= len(c))[0][0])
        cut = [v for v in o2 if lev[v] == k]
        sep[cut] = True
        allowed[cut] = False
        pending.extend(components(allowed))
    blocks.sort(key=lambda b: (len(b), b[0]))
    sep_nodes = list(np.nonzero(sep)[0])
    perm = np.array([v for b in blocks for v in b] + sep_nodes, dtype=np.int64)
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    block_ptr = np.concatenate([[0], np.cumsum([len(b) for b in blocks])]).astype(np.int64)
    n1 = int(block_ptr[-1])
    return {"perm": perm, "iperm": iperm, "block_ptr": block_ptr,
            "n1": n1, "n2": n - n1}


def check_partition(W: sp.csr_matrix, part) -> None:
    """Assert the defining property of Steps 2-3: after reordering, M11 is
    block diagonal (no edge joins two different blocks) and perm is a
    permutation."""
    n = W.shape[0]
    perm, bp, n1 = part["perm"], part["block_ptr"], part["n1"]
    assert np.array_equal(np.sort(perm), np.arange(n))
    blk = np.full(n, -1, dtype=np.int64)
    for i in range(len(bp) - 1):
        blk[perm[bp[i]:bp[i + 1]]] = i
    C = W.tocoo()
    a, b = blk[C.row], blk[C.col]
    bad = (a >= 0) & (b >= 0) & (a != b)
    assert not bad.any(), "edge between two M11 blocks"


# --------------------------------------------------- counter-based generator
def splitmix64(seed: int, count: int) -> list[int]:
    """Raw SplitMix64 outputs (Steele, Lea and Flood, 2014):
    state_i = seed + (i+1)*0x9E3779B97F4A7C15, then the published mix
    (xor-shift 30, multiply 0xBF58476D1CE4E5B9, xor-shift 27, multiply
    0x94D049BB133111EB, xor-shift 31)."""
    mask = (1 << 64) - 1
    out = []
    for i in range(count):
        z = (seed + (i + 1) * 0x9E3779B97F4A7C15) & mask
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        out.append(z ^ (z >> 31))
    return out


def splitmix64_uniform(seed: int, count: int) -> np.ndarray:
    """Uniform doubles in [-0.5, 0.5): the top 53 bits of each SplitMix64
    output as a fraction, minus one half.  Used for the Lanczos start vector
    l(0) of Algorithm 1 (a "normalized random vector")."""
    return np.array([(z >> 11) * (1.0 / 9007199254740992.0) - 0.5
                     for z in splitmix64(seed, count)])


# ------------------------------------------------------------ LRC-Katz index
class _M11Solver:
    """Applies M11^{-1} block by block (Lemma 1 needs M11 invertible).

    Blocks up to ``block_max`` nodes: dense Cholesky M11,i = L1 L1^T and the
    explicit inverse (Step 4; Algorithm 1, the L1 line).  Larger blocks
    (kept whole when splitting is off) are factorised by SciPy's sparse LU.
    """

    def __init__(self, M11: sp.csr_matrix, block_ptr, block_max):
        self.bp = np.asarray(block_ptr)
        self.inv = []
        M11 = M11.tocsr()
        for i in range(len(self.bp) - 1):
            a, b = int(self.bp[i]), int(self.bp[i + 1])
            Mi = M11[a:b, a:b]
            if b - a <= block_max:
                L1 = np.linalg.cholesky(Mi.toarray())
                L1inv = sla.solve_triangular(L1, np.eye(b - a), lower=True)
                self.inv.append(("dense", L1inv.T @ L1inv))
            else:
                self.inv.append(("lu", spla.splu(Mi.tocsc())))

    def solve(self, X: np.ndarray) -> np.ndarray:
        Y = np.empty_like(X)
        for i, (kind, F) in enumerate(self.inv):
            a, b = int(self.bp[i]), int(self.bp[i + 1])
            Y[a:b] = F @ X[a:b] if kind == "dense" else F.solve(X[a:b])
        return Y


def _lanczos_top(apply_R, n2: int, rank: int, steps: int, v0: np.ndarray,
                 res_tol: float = 1e-8):
    """Lanczos on the symmetric operator R with full reorthogonalisation
    (Algorithm 1, the Lanczos line, with R applied as a matrix-vector
    product).  At least ``steps`` steps; then extended until the top
    ``rank`` Ritz pairs have residual estimates beta_m |y_m,i| <=
    res_tol * max(1, |theta_i|), or the Krylov space is exhausted.  Returns
    the ``rank`` largest Ritz values (descending) and their Ritz vectors."""
    cap = n2
    V = np.zeros((n2, cap + 1))
    alpha = np.zeros(cap)
    beta = np.zeros(cap)
    V[:, 0] = v0 / np.linalg.norm(v0)
    k = 0
    check = min(steps, cap)
    for j in range(cap):
        w = apply_R(V[:, j])
        alpha[j] = V[:, j] @ w
        w -= V[:, : j + 1] @ (V[:, : j + 1].T @ w)
        w -= V[:, : j + 1] @ (V[:, : j + 1].T @ w)
        beta[j] = np.linalg.norm(w)
        k = j + 1
        if beta[j] <= 1e-14 * max(1.0, abs(alpha[j])):
            break
        if k >= check:
            T = np.diag(alpha[:k]) + np.diag(beta[: k - 1], 1) + np.diag(beta[: k - 1], -1)
            theta, Y = np.linalg.eigh(T)
            top = np.argsort(-theta)[:rank]
            if np.all(beta[j] * np.abs(Y[-1, top]) <= res_tol * np.maximum(1.0, np.abs(theta[top]))):
                break
            check = k + max(10, k // 2)
        V[:, j + 1] = w / beta[j]
    T = np.diag(alpha[:k]) + np.diag(beta[: k - 1], 1) + np.diag(beta[: k - 1], -1)
    theta, Y = np.linalg.eigh(T)
    idx = np.argsort(-theta)[:rank]
    return theta[idx], V[:, :k] @ Y[:, idx]


def lrc_build(W: sp.csr_matrix, beta: float, part: dict, rank: int,
              lanczos_steps: int | None = None, seed: int = 20191212,
              block_max: int = 128):
    """Algorithm 1 (Preprocess) in float64.

    Builds, in the partition's order: M11^{-1} (blockwise), M12, M22, its
    Cholesky factor L (M22 = L L^T), the Schur complement
    S = M22 - M12^T M11^{-1} M12 (Lemma 1), and the top ``rank`` eigenpairs
    (sigma_i, u_i) of R = L^{-1} M12^T M11^{-1} M12 L^{-T} (Eq. 11) by Lanczos
    from a normalised SplitMix64 start vector.  The preconditioner data are
    W_r = L^{-T} U_r and D = diag(sigma/(1-sigma)), so that
    S~^{-1} = M22^{-1} + W_r D W_r^T (Eq. 14, with
    (I - Sigma~)^{-1} - I = diag(sigma_i/(1-sigma_i)) on the kept ranks).
    """
    n = W.shape[0]
    perm, n1 = part["perm"], part["n1"]
    n2 = n - n1
    Wp = W[perm][:, perm].tocsr()
    M = (sp.eye(n, format="csr") - beta * Wp).tocsr()
    M11 = M[:n1, :n1]
    M12 = M[:n1, n1:].toarray() if n2 else np.zeros((n1, 0))
    M22 = M[n1:, n1:].toarray()
    m11 = _M11Solver(M11, part["block_ptr"], block_max)
    T = M12.T @ m11.solve(M12) if n1 and n2 else np.zeros((n2, n2))
    S = M22 - T
    L = np.linalg.cholesky(M22) if n2 else np.zeros((0, 0))
    r = min(rank, n2)
    if n2:
        Linv = sla.solve_triangular(L, np.eye(n2), lower=True)
        R = Linv @ T @ Linv.T
        R = 0.5 * (R + R.T)
        steps = lanczos_steps or max(2 * r, r + 20)
        v0 = splitmix64_uniform(seed, n2)
        sigma, U = _lanczos_top(lambda v: R @ v, n2, r, steps, v0)
        Wr = Linv.T @ U
        M22inv = Linv.T @ Linv
    else:
        sigma, Wr, M22inv, R = np.zeros(0), np.zeros((0, 0)), np.zeros((0, 0)), np.zeros((0, 0))
    return {"n": n, "n1": n1, "n2": n2, "beta": beta, "part": part, "Wp": Wp,
            "M11": M11, "m11": m11, "M12": M12, "M22": M22, "L": L, "S": S,
            "R": R, "sigma": sigma, "Wr": Wr, "D": sigma / (1.0 - sigma),
            "M22inv": M22inv}


def _precond(idx, Rv):
    """z = S~^{-1} r = M22^{-1} r + W_r D W_r^T r (Eq. 14)."""
    return idx["M22inv"] @ Rv + idx["Wr"] @ (idx["D"][:, None] * (idx["Wr"].T @ Rv))


def lrc_query(idx: dict, B: np.ndarray, tol: float = 1e-13, maxit: int = 10000,
              K2_0: np.ndarray | None = None):
    """Algorithm 2 (LRC-Katz) for right-hand sides B given in node order.

    1. Permute B and split it into B1 (first n1 rows) and B2 (Lemma 1).
    2. F = B2 - M12^T M11^{-1} B1 (Eq. 7).
    3. Solve S K2 = F by preconditioned CG with S~^{-1} (Eq. 14) as the
       preconditioner (Hestenes-Stiefel PCG; the garbled listing of
       Algorithm 2 is read as standard PCG), zero start unless K2_0 is given,
       per column until ||F - S K2||_2 <= tol ||F||_2.
    4. K1 = M11^{-1} (B1 - M12 K2) (Eq. 6), merge and undo the permutation.

    Returns dict(K (node order), F, K2, K1, iters)."""
    n, n1, n2 = idx["n"], idx["n1"], idx["n2"]
    perm = idx["part"]["perm"]
    Bp = np.asarray(B, dtype=np.float64)[perm]
    b = Bp.shape[1]
    B1, B2 = Bp[:n1], Bp[n1:]
    Y1 = idx["m11"].solve(B1) if n1 else np.zeros((0, b))
    F = B2 - idx["M12"].T @ Y1
    S = idx["S"]
    K2 = np.zeros((n2, b)) if K2_0 is None else np.array(K2_0, dtype=np.float64)
    iters = np.zeros(b, dtype=np.int64)
    if n2:
        Rr = F - S @ K2
        Z = _precond(idx, Rr)
        P = Z.copy()
        rz = np.einsum("ij,ij->j", Rr, Z)
        fn = np.sqrt(np.einsum("ij,ij->j", F, F))
        active = np.sqrt(np.einsum("ij,ij->j", Rr, Rr)) > tol * fn
        for _ in range(maxit):
            if not active.any():
                break
            a = np.nonzero(active)[0]
            SP = S @ P[:, a]
            pSp = np.einsum("ij,ij->j", P[:, a], SP)
            al = rz[a] / pSp
            K2[:, a] += al * P[:, a]
            Rr[:, a] -= al * SP
            Za = _precond(idx, Rr[:, a])
            rz_new = np.einsum("ij,ij->j", Rr[:, a], Za)
            P[:, a] = Za + (rz_new / rz[a]) * P[:, a]
            rz[a] = rz_new
            iters[a] += 1
            active[a] = np.sqrt(np.einsum("ij,ij->j", Rr[:, a], Rr[:, a])) > tol * fn[a]
    K1 = idx["m11"].solve(B1 - idx["M12"] @ K2) if n1 else np.zeros((0, b))
    Kp = np.vstack([K1, K2])
    K = np.empty_like(Kp)
    K[perm] = Kp
    return {"K": K, "F": F, "K2": K2, "K1": K1, "Y1": Y1, "iters": iters}


def katz_lrc(W: sp.csr_matrix, beta: float, Q, n_hubs: int, block_max: int,
             rank: int, split: bool = True, tol: float = 1e-13):
    """k_q for every q in Q by LRC-Katz (Algorithms 1 and 2) end to end."""
    part = partition(W.shape[0], W.indptr, W.indices, n_hubs, block_max, split)
    idx = lrc_build(W, beta, part, rank, block_max=block_max)
    B = beta * W[:, np.asarray(Q)].toarray()
    return lrc_query(idx, B, tol=tol), idx


def schur_precond_spectrum(idx: dict) -> np.ndarray:
    """Eigenvalues of S S~^{-1} (ascending), the quantity of Theorem 1."""
    if idx["n2"] == 0:
        return np.zeros(0)
    Sinv_t = idx["M22inv"] + idx["Wr"] @ np.diag(idx["D"]) @ idx["Wr"].T
    ev = np.linalg.eigvals(idx["S"] @ Sinv_t)
    return np.sort(ev.real)


# -------------------------------------------------------- link prediction
def linkpred_topk(W: sp.csr_matrix, K: np.ndarray, Q, k: int):
    """Katz link prediction (Section 3.3): for query column j, rank every
    node except Q[j] and its current neighbours by K[:, j] descending, ties
    by node id ascending, and return the first k (ids b x k, scores b x k).
    Fewer than k candidates leave id -1 and score 0."""
    n = W.shape[0]
    Q = np.asarray(Q)
    ids = np.full((len(Q), k), -1, dtype=np.int64)
    sc = np.zeros((len(Q), k))
    for j, q in enumerate(Q):
        mask = np.ones(n, dtype=bool)
        mask[q] = False
        mask[W.indices[W.indptr[q]:W.indptr[q + 1]]] = False
        cand = np.nonzero(mask)[0]
        order = np.lexsort((cand, -K[cand, j]))[:k]
        ids[j, : len(order)] = cand[order]
        sc[j, : len(order)] = K[cand[order], j]
    return ids, sc


def top_nodes(scores: np.ndarray, k: int, exclude=()) -> np.ndarray:
    """The k nodes of highest score, score descending and node id ascending
    on ties, leaving out the nodes in ``exclude`` (fewer than k if too few
    remain): the Top-s and Top-T selections of Algorithm 3 (Section 3.3)."""
    keep = np.ones(scores.shape[0], dtype=bool)
    keep[np.asarray(list(exclude), dtype=np.int64)] = False
    cand = np.nonzero(keep)[0]
    return cand[np.lexsort((cand, -scores[cand]))[:k]]


def pearson(x: np.ndarray, y: np.ndarray) -> float:
    """Pearson correlation of two equal-length vectors (the row-wise
    correlation of Algorithm 3, Section 3.3): the centred inner product over
    the product of the centred norms.  Either vector constant
    (zero spread; every vector of length 1) gives 0, no linear
    association."""
    xc = x - x.mean()
    yc = y - y.mean()
    sxx = float(xc @ xc)
    syy = float(yc @ yc)
    if sxx == 0.0 or syy == 0.0:
        return 0.0
    return float(xc @ yc) / np.sqrt(sxx * syy)


def sparse_katz(W: sp.csr_matrix, beta: float, Q, s: int, T: int, solve=None):
    """Sparse-Katz re-ranking of the link-prediction list (Algorithm 3,
    Section 3.3, Fig. 2), in the algorithm's order:

    1. k_q, the Katz vector of the query (Eq. 3);
    2. the Top-s list: the s best link candidates of k_q (q and its current
       neighbours left out, as in ``linkpred_topk``);
    3. the T landmark nodes t: the T highest scores of k_q over every node
       but q (neighbours included), and their Katz vectors k_t, the columns
       of the n x T matrix K_T;
    4. for every candidate j, rho_j = Pearson correlation of row q and row j
       of K_T (the T-vectors (k_t[q])_t and (k_t[j])_t);
    5. the Top-s list re-ordered by rho descending, ties kept in Katz order.

    ``solve(W, beta, ids)`` returns Katz columns (default: dense Cholesky for
    n <= 3000, else CG to 1e-13).  Returns (ids b x s, rho b x s, landmarks
    b x T, Katz-ordered candidates b x s); missing candidates are id -1 with
    rho 0 at the end of the row."""
    if solve is None:
        solve = (katz_direct if W.shape[0] <= 3000
                 else (lambda W_, b_, ids: katz_cg(W_, b_, ids)[0]))
    Q = np.asarray(Q)
    b = len(Q)
    Kq = solve(W, beta, Q)
    ids = np.full((b, s), -1, dtype=np.int64)
    rho = np.zeros((b, s))
    land = np.zeros((b, T), dtype=np.int64)
    cand_k = np.full((b, s), -1, dtype=np.int64)
    for j, q in enumerate(Q):
        nbrs = W.indices[W.indptr[q]:W.indptr[q + 1]]
        cand = top_nodes(Kq[:, j], s, exclude=[q, *nbrs.tolist()])
        lm = top_nodes(Kq[:, j], T, exclude=[q])
        land[j, : len(lm)] = lm
        cand_k[j, : len(cand)] = cand
        KT = solve(W, beta, lm)
        r = np.array([pearson(KT[q, :], KT[c, :]) for c in cand])
        order = sorted(range(len(cand)), key=lambda i: (-r[i], i))
        ids[j, : len(cand)] = cand[order]
        rho[j, : len(cand)] = r[order]
    return ids, rho, land, cand_k


# ---------------------------------------------------- warm-start network
def gelu(x):
    """Exact GELU x * Phi(x) with the erf form of Phi."""
    from scipy.special import erf
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def _gelu_grad(x):
    return 0.5 * (1.0 + _erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def _erf(x):
    from scipy.special import erf
    return erf(x)


def mlp_forward(X, W1, b1, W2, b2):
    """Two-layer network y = W2 GELU(W1 x + b1) + b2, rows of X are inputs.
    Returns (Y, H_pre, H)."""
    Hp = X @ W1.T + b1
    H = gelu(Hp)
    return H @ W2.T + b2, Hp, H


def mlp_loss_grad(X, T, W1, b1, W2, b2):
    """Mean squared error L = mean over rows of ||y - t||^2 / 2 and its
    gradients (dW1, db1, dW2, db2) by the chain rule."""
    Y, Hp, H = mlp_forward(X, W1, b1, W2, b2)
    m = X.shape[0]
    E = Y - T
    loss = 0.5 * float(np.sum(E * E)) / m
    dY = E / m
    dW2 = dY.T @ H
    db2 = dY.sum(axis=0)
    dH = dY @ W2
    dHp = dH * _gelu_grad(Hp)
    dW1 = dHp.T @ X
    db1 = dHp.sum(axis=0)
    return loss, (dW1, db1, dW2, db2)


def adamw_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8, wd=0.0):
    """One AdamW update (Loshchilov and Hutter): decoupled weight decay,
    bias-corrected first and second moments.  Returns (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    p = p - lr * (mh / (np.sqrt(vh) + eps) + wd * p)
    return p, m, v
