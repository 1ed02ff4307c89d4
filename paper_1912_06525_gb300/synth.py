"""Seeded synthetic graphs and query sets.

This module only draws inputs: undirected graphs in symmetric CSR form and
query node sets.  It holds none of the Katz arithmetic, so both the CUDA path
and the FP64 oracle can be fed from it.

The graph shapes stand in for the large real-world networks of Section 4
(Table 1), which are not available here:

* ``sbm_bernoulli``   - stochastic block model with exact Bernoulli(p) pairs.
* ``sbm_degree``      - block model drawn by edge counts (large graphs).
* ``chung_lu``        - power-law expected-degree graph (erased variant).
* ``modular_hubs``    - lognormal-sized SBM communities plus hub nodes.
* ``multi_sbm``       - many independent SBM graphs of uneven size.
* ``table1_standin``  - Chung-Lu graphs with the size, average degree and
  spectral norm of the six networks of Table 1.
* ``path/cycle/star/complete/single_edge`` - tiny graphs with closed forms.

Every generator drops self-loops and duplicate edges; weights default to 1.
All random draws come from ``numpy.random.default_rng(seed)`` (PCG64), which
gives identical streams on x86 and Arm.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math
import numpy as np

BASE_SEED = 20191212


@dataclass
class Graph:
    """Symmetric CSR adjacency W of an undirected graph (no self-loops).

    ``rowptr`` int64[n+1], ``col`` int32[nnz] (sorted within each row),
    ``val`` float64[nnz] or None for unit weights.  ``meta`` carries the
    generator's parameters (community labels, hub ids, ...).
    """
    n: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def values(self) -> np.ndarray:
        """Edge weights as float64 (ones for an unweighted graph)."""
        if self.val is None:
            return np.ones(self.nnz, dtype=np.float64)
        return self.val

    def degrees(self) -> np.ndarray:
        return np.diff(self.rowptr)


def edges_to_graph(n: int, u: np.ndarray, v: np.ndarray, meta=None,
                   weight_fn=None) -> Graph:
    """Build symmetric CSR from an undirected edge list.

    Self-loops are dropped and duplicate (unordered) pairs merged.  If
    ``weight_fn`` is given it maps the deduplicated (lo, hi) pair arrays to
    one weight per undirected edge, so both directions carry the same value.
    """
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    lo = np.minimum(u, v)
    hi = np.maximum(u, v)
    key = np.sort(lo * n + hi)
    if key.shape[0]:
        key = key[np.concatenate([[True], key[1:] != key[:-1]])]
    lo = key // n
    hi = key - lo * n
    w = None if weight_fn is None else np.asarray(weight_fn(lo, hi), dtype=np.float64)
    rows = np.concatenate([lo, hi])
    cols = np.concatenate([hi, lo])
    k2 = rows * n + cols
    order = np.argsort(k2, kind="stable")
    rows = rows[order]
    cols = cols[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    val = None
    if w is not None:
        val = np.concatenate([w, w])[order]
    return Graph(n=n, rowptr=rowptr, col=cols.astype(np.int32), val=val,
                 meta=dict(meta or {}))


def dyadic_weights(seed: int):
    """Weight function giving values k/64 in [0.5, 2), exact in BF16/FP32."""
    def fn(lo, hi):
        rng = np.random.default_rng(seed)
        return rng.integers(32, 128, size=lo.shape[0]) / 64.0
    return fn


def with_dyadic_weights(g: Graph, seed: int) -> Graph:
    """The same pattern with symmetric weights k/64 in [0.5, 2) (exact in
    BF16): each undirected edge's weight is a hash of (min, max, seed), so
    both stored directions carry the same value."""
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.rowptr))
    cols = g.col.astype(np.int64)
    lo, hi = np.minimum(rows, cols), np.maximum(rows, cols)
    z = (lo * 0x9E3779B1 + hi * 0x85EBCA77 + seed * 0xC2B2AE3D) & 0xFFFFFFFF
    z ^= z >> 15
    z = (z * 0x2C1B3C6D) & 0xFFFFFFFF
    z ^= z >> 12
    w = (32 + (z % 96)) / 64.0
    return Graph(n=g.n, rowptr=g.rowptr, col=g.col, val=w.astype(np.float64),
                 meta=dict(g.meta, weights="dyadic"))


# ----------------------------------------------------------------- tiny graphs
def single_edge() -> Graph:
    return edges_to_graph(2, np.array([0]), np.array([1]), {"kind": "single_edge"})


def path(n: int) -> Graph:
    i = np.arange(n - 1)
    return edges_to_graph(n, i, i + 1, {"kind": "path"})


def cycle(n: int) -> Graph:
    i = np.arange(n)
    return edges_to_graph(n, i, (i + 1) % n, {"kind": "cycle"})


def star(m: int) -> Graph:
    """Node 0 joined to leaves 1..m."""
    return edges_to_graph(m + 1, np.zeros(m, dtype=np.int64), np.arange(1, m + 1),
                          {"kind": "star"})


def complete(n: int) -> Graph:
    iu, ju = np.triu_indices(n, 1)
    return edges_to_graph(n, iu, ju, {"kind": "complete"})


def erdos_renyi(n: int, p: float, seed: int, weighted: bool = False) -> Graph:
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, 1)
    m = rng.random(iu.shape[0]) < p
    wf = dyadic_weights(seed + 1) if weighted else None
    return edges_to_graph(n, iu[m], ju[m], {"kind": "er", "p": p}, wf)


def disjoint_union(graphs: list[Graph]) -> Graph:
    """Block-diagonal union (node ids offset in order)."""
    us, vs, ws = [], [], []
    off = 0
    weighted = any(g.val is not None for g in graphs)
    for g in graphs:
        r = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.rowptr))
        c = g.col.astype(np.int64)
        m = r < c
        us.append(r[m] + off)
        vs.append(c[m] + off)
        ws.append(g.values()[m])
        off += g.n
    u = np.concatenate(us)
    v = np.concatenate(vs)
    wfn = None
    if weighted:
        wmap = dict(zip((np.minimum(u, v) * off + np.maximum(u, v)).tolist(),
                        np.concatenate(ws).tolist()))
        wfn = lambda lo, hi: np.array([wmap[int(a) * off + int(b)] for a, b in zip(lo, hi)])
    return edges_to_graph(off, u, v, {"kind": "union"}, wfn)


# ------------------------------------------------------ stochastic block models
def sbm_bernoulli(sizes, p_in: float, p_out: float, seed: int,
                  weighted: bool = False) -> Graph:
    """Exact SBM: every pair is an edge independently with p_in or p_out."""
    sizes = np.asarray(sizes, dtype=np.int64)
    n = int(sizes.sum())
    lab = np.repeat(np.arange(sizes.shape[0]), sizes)
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, 1)
    p = np.where(lab[iu] == lab[ju], p_in, p_out)
    m = rng.random(iu.shape[0]) < p
    wf = dyadic_weights(seed + 1) if weighted else None
    return edges_to_graph(n, iu[m], ju[m],
                          {"kind": "sbm", "labels": lab, "p_in": p_in, "p_out": p_out}, wf)


def _community_edges(rng, offsets, sizes, deg):
    """Uniform random pairs inside each community; about deg*size/2 each."""
    counts = rng.poisson(sizes * deg / 2.0)
    total = int(counts.sum())
    comm = np.repeat(np.arange(sizes.shape[0]), counts)
    s = sizes[comm]
    a = offsets[comm] + (rng.random(total) * s).astype(np.int64)
    b = offsets[comm] + (rng.random(total) * s).astype(np.int64)
    return a, b


def _inter_edges(rng, n, lab, m):
    """m uniform pairs whose endpoints lie in different communities."""
    a = rng.integers(0, n, size=int(m * 1.2) + 16)
    b = rng.integers(0, n, size=a.shape[0])
    keep = lab[a] != lab[b]
    return a[keep][:m], b[keep][:m]


def sbm_degree(sizes, mean_deg: float, inter_frac: float, seed: int) -> Graph:
    """Block model drawn by edge counts: intra degree (1-f)d, inter degree f*d."""
    rng = np.random.default_rng(seed)
    sizes = np.asarray(sizes, dtype=np.int64)
    n = int(sizes.sum())
    offsets = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    lab = np.repeat(np.arange(sizes.shape[0]), sizes)
    a1, b1 = _community_edges(rng, offsets, sizes, mean_deg * (1 - inter_frac))
    a2, b2 = _inter_edges(rng, n, lab, int(round(n * mean_deg * inter_frac / 2)))
    return edges_to_graph(n, np.concatenate([a1, a2]), np.concatenate([b1, b2]),
                          {"kind": "sbm_degree", "labels": lab})


def chung_lu(n: int, gamma: float, mean_deg: float, max_deg: float, seed: int) -> Graph:
    """Power-law expected-degree graph.

    Expected degrees w_i = c * (i+i0)^(-1/(gamma-1)) (a discrete power law
    with exponent gamma), capped at ``max_deg`` and rescaled to ``mean_deg``.
    Edges: m = sum(w)/2 endpoint pairs drawn independently with probability
    proportional to w, then self-loops and repeats erased.  Node ids are
    shuffled so that degree is not correlated with id.
    """
    rng = np.random.default_rng(seed)
    w = _chung_lu_weights(n, gamma, mean_deg, max_deg)
    perm = rng.permutation(n)
    wn = np.empty(n)
    wn[perm] = w
    m = int(round(wn.sum() / 2))
    cdf = np.cumsum(wn)
    cdf /= cdf[-1]
    a = np.searchsorted(cdf, rng.random(m), side="right")
    b = np.searchsorted(cdf, rng.random(m), side="right")
    a = np.minimum(a, n - 1)
    b = np.minimum(b, n - 1)
    return edges_to_graph(n, a, b, {"kind": "chung_lu", "gamma": gamma,
                                     "expected_degree": wn})


# Section 4, Table 1: (nodes, average degree, ||G||_2) of the six networks
# of the runtime and iteration experiments.
TABLE1 = {
    "dblp_lcc": (93_156, 3.82, 39.5753),
    "arxiv_lcc": (86_376, 11.98, 99.3319),
    "email_enron": (36_692, 10.02, 111.2871),
    "gowalla": (196_591, 9.67, 169.3612),
    "flickr": (513_969, 12.41, 663.3587),
    "hollywood_2009": (1_139_905, 99.13, 2247.5591),
}


def _chung_lu_weights(n: int, gamma: float, mean_deg: float, max_deg: float) -> np.ndarray:
    i = np.arange(n, dtype=np.float64)
    w = (i + 1.0) ** (-1.0 / (gamma - 1.0))
    for _ in range(50):  # scale to the mean under the cap (fixed point)
        w = w * (mean_deg / np.minimum(w, max_deg).mean())
        w = np.minimum(w, max_deg)
    return w


def table1_standin(name: str, scale: float = 1.0, seed: int = BASE_SEED) -> Graph:
    """Stand-in for one network of Table 1: a Chung-Lu graph (exponent
    2.1) with the table's node count (times ``scale``) and average degree,
    whose degree cap is chosen so that the expected-degree estimate of the
    largest eigenvalue, max(sum w^2 / sum w, sqrt(max w)) (Chung, Lu and
    Vu), equals the table's ||G||_2, measured on the realised degrees (the
    erased edge draw loses repeated hub edges, so the aim is raised and the
    graph redrawn, up to four times, until the realised estimate is within
    3%).  The eigenvalue itself is not computed here."""
    n0, deg, lam = TABLE1[name]
    n = max(1000, int(round(n0 * scale)))
    deg = min(deg, (n - 1) / 4.0)
    lo, hi = deg * 1.01, n / 2.0

    def est(cap):
        w = _chung_lu_weights(n, 2.1, deg, cap)
        return max(float((w * w).sum() / w.sum()), float(np.sqrt(w.max())))

    def cap_for(target):
        a, b = lo, hi
        for _ in range(60):  # est() grows with the cap
            mid = math.sqrt(a * b)
            if est(mid) < target:
                a = mid
            else:
                b = mid
        return math.sqrt(a * b)

    # the erased draw loses repeated edges, most at the hubs; aim the
    # expected estimate higher until the realised degrees meet the target
    aim = lam
    for _ in range(4):
        g = chung_lu(n, 2.1, deg, cap_for(aim), seed + sum(map(ord, name)))
        d = np.diff(g.rowptr).astype(np.float64)
        got = max(float((d * d).sum() / d.sum()), float(np.sqrt(d.max())))
        if abs(got - lam) <= 0.03 * lam:
            break
        aim *= lam / got
    g.meta.update({"kind": "table1_standin", "network": name, "target_norm": lam,
                   "target_mean_degree": deg})
    return g


def modular_hubs(n: int, n_comm: int, mu_log: float, sigma_log: float,
                 mean_deg: float, inter_frac: float, n_hubs: int, hub_deg: int,
                 seed: int) -> Graph:
    """Lognormal-sized SBM communities plus hub nodes.

    Community sizes ~ lognormal(mu, sigma), renormalised to sum to n.  Each
    node has about (1-f)d intra-community and f*d inter-community
    neighbours.  ``n_hubs`` existing nodes are each joined to ``hub_deg``
    extra uniform random targets.
    """
    rng = np.random.default_rng(seed)
    raw = rng.lognormal(mu_log, sigma_log, size=n_comm)
    sizes = np.floor(raw / raw.sum() * n).astype(np.int64)
    sizes = np.maximum(sizes, 2)
    diff = n - int(sizes.sum())
    order = np.argsort(-raw)
    j = 0
    while diff != 0:
        step = 1 if diff > 0 else -1
        k = order[j % n_comm]
        if sizes[k] + step >= 2:
            sizes[k] += step
            diff -= step
        j += 1
    offsets = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    lab = np.repeat(np.arange(n_comm), sizes)
    a1, b1 = _community_edges(rng, offsets, sizes, mean_deg * (1 - inter_frac))
    a2, b2 = _inter_edges(rng, n, lab, int(round(n * mean_deg * inter_frac / 2)))
    hubs = rng.choice(n, size=n_hubs, replace=False)
    a3 = np.repeat(hubs.astype(np.int64), hub_deg)
    b3 = rng.integers(0, n, size=a3.shape[0])
    return edges_to_graph(n, np.concatenate([a1, a2, a3]), np.concatenate([b1, b2, b3]),
                          {"kind": "modular_hubs", "labels": lab, "hubs": hubs,
                           "sizes": sizes})


def multi_sbm(count: int, n_lo: int, n_hi: int, seed: int,
              comm_lo: int = 4, comm_hi: int = 64, deg_lo: float = 8.0,
              deg_hi: float = 32.0, inter_frac: float = 0.10) -> list[Graph]:
    """Many independent SBM graphs with log-uniform node counts."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count)).astype(np.int64)
    out = []
    for g in range(count):
        n = int(ns[g])
        k = int(rng.integers(comm_lo, comm_hi + 1))
        k = max(1, min(k, n // 4))
        d = float(rng.uniform(deg_lo, deg_hi))
        base = n // k
        sizes = np.full(k, base, dtype=np.int64)
        sizes[: n - base * k] += 1
        gg = sbm_degree(sizes, d, inter_frac, int(rng.integers(0, 2**62)))
        gg.meta.update({"graph_index": g, "mean_deg_target": d})
        out.append(gg)
    return out


def queries(n: int, b: int, seed: int) -> np.ndarray:
    """b distinct query nodes, uniform without replacement (int32)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=b, replace=False)).astype(np.int32)


# ------------------------------------------------- the five workload shapes
def workload(config: int, scale: float = 1.0):
    """(graph, query ids, c, rank) for workload ``config`` (1-4).

    1: SBM n=2,000, 8 communities, mean degree 10, 10% inter; c=0.5, r=16.
    2: Chung-Lu n=1M, exponent 2.1, mean degree 16, cap 20,000; c=0.5, r=64.
    3: lognormal-SBM n=4M, 512 communities, degree 20, 5% inter, 2,000 hubs
       of about 5,000 extra edges; c in {0.1, 0.5, 0.9}; r=128.
    4: the graph of 2 (learned warm start).
    ``scale`` < 1 shrinks n (and b) for quick tests, keeping the recipe.
    """
    seed = BASE_SEED + config
    if config == 1:
        n = max(16, int(2000 * scale))
        k = 8
        s = n // k
        sizes = [s] * k
        sizes[-1] += n - s * k
        p_in = 9.0 / (s - 1)
        p_out = 1.0 / (n - s)
        g = sbm_bernoulli(sizes, p_in, p_out, seed)
        return g, queries(g.n, min(16, g.n), seed + 100), 0.5, 16
    if config in (2, 4):
        n = max(1000, int(1_000_000 * scale))
        g = chung_lu(n, 2.1, 16.0, min(20000.0, n / 5), 2 + BASE_SEED)
        b = 256 if scale >= 1 else max(8, int(256 * scale ** 0.5))
        return g, queries(g.n, min(b, g.n), seed + 100), 0.5, 64
    if config == 3:
        n = max(20000, int(4_000_000 * scale))
        n_comm = max(4, int(512 * scale))
        n_hubs = max(8, int(2000 * scale))
        hub_deg = max(50, int(5000 * min(1.0, scale * 8)))
        g = modular_hubs(n, n_comm, math.log(7800 * n / 4_000_000), 0.5, 20.0,
                         0.05, n_hubs, hub_deg, seed)
        b = 1024 if scale >= 1 else max(8, int(1024 * scale ** 0.5))
        return g, queries(g.n, min(b, g.n), seed + 100), 0.9, 128
    raise ValueError(f"unknown workload {config}")
