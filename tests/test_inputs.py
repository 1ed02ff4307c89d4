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
