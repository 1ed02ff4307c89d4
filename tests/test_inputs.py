"""The Table 1 stand-in graphs (Section 4) have the table's node count and
average degree, and a largest eigenvalue near the table's ||G||_2."""
import numpy as np
import pytest

import oracle as O
from paper_1912_06525_gb300 import synth


@pytest.mark.parametrize("name", ["dblp_lcc", "email_enron", "arxiv_lcc"])
def test_table1_standins_match_the_table(name):
    n0, deg, lam = synth.TABLE1[name]
    g = synth.table1_standin(name)
    assert g.n == n0
    assert abs(g.nnz / g.n - deg) <= 0.03 * deg
    # symmetric, no self-loops
    W = O.adjacency(g.n, g.rowptr, g.col, g.val)
    assert (W != W.T).nnz == 0 and W.diagonal().sum() == 0
    assert abs(O.lambda_max(W) - lam) <= 0.1 * lam


def test_table1_standin_is_seeded():
    a = synth.table1_standin("email_enron", 0.1)
    b = synth.table1_standin("email_enron", 0.1)
    assert np.array_equal(a.rowptr, b.rowptr) and np.array_equal(a.col, b.col)


def test_many_graph_recipe():
    """multi_sbm: node counts log-uniform in [n_lo, n_hi], symmetric block
    models; where communities are large enough to hold the target degree
    (size >= 4 x the intra-community degree), the mean degree is within 25%
    of the drawn target and about 10% of the edges run between communities
    (smaller communities cannot hold it: repeated pairs are erased)."""
    gs = synth.multi_sbm(40, 200, 4000, seed=3)
    ns = np.array([g.n for g in gs])
    assert ns.min() >= 200 and ns.max() <= 4000
    # log-uniform: the geometric midpoint splits the counts roughly in half
    assert 0.2 < (ns < np.sqrt(200 * 4000)).mean() < 0.8
    checked = 0
    for g in gs:
        W = O.adjacency(g.n, g.rowptr, g.col, g.val)
        assert (W != W.T).nnz == 0 and W.diagonal().sum() == 0
        lab = np.asarray(g.meta["labels"])
        k = len(set(lab.tolist()))
        target = g.meta["mean_deg_target"]
        if g.n / k < 4 * 0.9 * target:
            continue
        checked += 1
        assert abs(g.nnz / g.n - target) <= 0.25 * target, (g.nnz / g.n, target)
        r = np.repeat(np.arange(g.n), np.diff(g.rowptr))
        inter = (lab[r] != lab[g.col]).mean()
        assert 0.05 <= inter <= 0.15, inter
    assert checked >= 5


def test_dyadic_weights_on_a_pattern_are_symmetric_and_exact_in_bf16():
    """The weighted variant of a workload keeps its pattern and gives both
    stored directions of an edge the same weight k/64 in [0.5, 2), a value
    BF16 holds exactly (8 significant bits)."""
    import numpy as np
    from paper_1912_06525_gb300 import synth
    g = synth.sbm_bernoulli([60] * 5, 0.2, 0.02, seed=4)
    gw = synth.with_dyadic_weights(g, 9)
    assert np.array_equal(gw.rowptr, g.rowptr) and np.array_equal(gw.col, g.col)
    W = O.adjacency(gw.n, gw.rowptr, gw.col, gw.val)
    assert abs(W - W.T).max() == 0.0
    k = gw.val * 64
    assert np.all(k == np.round(k)) and k.min() >= 32 and k.max() < 128
    # k/64 with k < 256 needs at most 8 significant bits
    assert np.all(np.frexp(gw.val)[0] * 256 == np.round(np.frexp(gw.val)[0] * 256))
