"""The first Schur right-hand side of a query from the stored coupling
Z = beta M11^{-1} W12 (Eq. 7 with M12^T M11^{-1} = -Z^T, M11 symmetric):
F = B2 + Z^T B1 gathered from the rows of Z that the sparse B1 = beta W e_q
touches, instead of an M11 solve of the whole block.  Both paths are checked
against the FP64 oracle, on unit, FP32 and BF16 weights, with queries whose
neighbour lists span several shared-memory stages (the 900-leaf star centre),
queries next to separator nodes only, and an index saved and loaded again."""
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


def graph(weighted, seed=11):
    a = synth.chung_lu(3000, 2.2, 8.0, 300.0, seed=seed)
    s = synth.star(900)
    iso = synth.path(1)
    g = synth.disjoint_union([a, s, iso, iso])
    r = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    m = r < g.col
    u = np.concatenate([r[m], [0, 3000]])
    v = np.concatenate([g.col[m], [3000, 7]])
    wf = synth.dyadic_weights(seed + 3) if weighted else None
    return synth.edges_to_graph(g.n, u, v, {"kind": "rhs-coupling"}, wf)


def queries(g, idx, b, seed):
    """Random nodes plus the star centre (900 neighbours), a separator node
    and, where there is one, a node whose neighbours are all separator nodes."""
    perm, _, n1, n2 = katz.katz_index_get_partition(idx)
    sep = set(int(x) for x in perm[n1:])
    q = list(synth.queries(g.n, b - 3, seed=seed))
    q.append(3000)
    q.append(int(perm[n1]))
    deg = np.diff(g.rowptr)
    only_sep = [i for i in range(g.n) if deg[i] > 0 and i not in sep
                and all(int(c) in sep for c in g.col[g.rowptr[i]:g.rowptr[i + 1]])]
    q.append(only_sep[0] if only_sep else 1)
    return np.asarray(list(dict.fromkeys(int(x) for x in q)), dtype=np.int32)


@pytest.mark.parametrize("vdt,weighted", [(katz.KATZ_UNIT, False), (katz.KATZ_F32, True),
                                          (katz.KATZ_BF16, True)])
def test_first_schur_rhs_from_z_matches_oracle(vdt, weighted):
    g = graph(weighted)
    W = O.adjacency(g.n, g.rowptr, g.col, g.val)
    beta = 0.85 / O.lambda_max(W)
    out = {}
    for rc in (-1, 1):
        idx = katz.katz_index_build(g, beta, value_dtype=vdt, rank=16, n_hubs=30, block_max=32,
                                    split=False, rhs_coupling=rc)
        info = katz.katz_index_get_info(idx)
        assert info["rhs_coupling"] == (1 if rc > 0 else 0)
        assert info["n_large_blocks"] >= 1 and info["n2"] >= 30
        q = queries(g, idx, 160, seed=4)
        K = torch.zeros((g.n, len(q)), dtype=torch.float64, device="cuda")
        st, it, rel = katz.katz_query_batch(idx, torch.from_numpy(q).cuda(), K,
                                            out_dtype=katz.KATZ_F64, tol=1e-6)
        assert st["status"] == "KATZ_OK"
        assert st["ms"][7] == (1.0 if rc > 0 else 0.0)
        ref = O.katz_direct(W, beta, q)
        assert O.error_inf_rel(K.cpu().numpy(), ref).max() <= 1e-6
        out[rc] = K.cpu().numpy()
    # both first passes land within the bound of the same solution
    assert np.abs(out[1] - out[-1]).max() <= 4e-6 * np.abs(out[-1]).max()


def test_rhs_coupling_auto_rules():
    """Automatic: stored where M11 has a block solved iteratively; never for
    all-dense M11 blocks (split components) unless forced."""
    g = graph(False)
    W = O.adjacency(g.n, g.rowptr, g.col, g.val)
    beta = 0.8 / O.lambda_max(W)
    whole = katz.katz_index_build(g, beta, rank=8, n_hubs=30, block_max=32, split=False)
    assert katz.katz_index_get_info(whole)["rhs_coupling"] == 1
    parts = katz.katz_index_build(g, beta, rank=8, n_hubs=30, block_max=128, split=True)
    info = katz.katz_index_get_info(parts)
    assert info["n_large_blocks"] == 0 and info["rhs_coupling"] == 0
    forced = katz.katz_index_build(g, beta, rank=8, n_hubs=30, block_max=128, split=True,
                                   rhs_coupling=1)
    assert katz.katz_index_get_info(forced)["rhs_coupling"] == 1
    q = queries(g, forced, 64, seed=9)
    ref = O.katz_direct(W, beta, q)
    K = torch.zeros((g.n, len(q)), dtype=torch.float64, device="cuda")
    st, _, _ = katz.katz_query_batch(forced, torch.from_numpy(q).cuda(), K,
                                     out_dtype=katz.KATZ_F64, tol=1e-6)
    assert st["status"] == "KATZ_OK" and st["ms"][7] == 1.0
    assert O.error_inf_rel(K.cpu().numpy(), ref).max() <= 1e-6


def test_stored_z_survives_save_and_load(tmp_path):
    g = graph(True)
    W = O.adjacency(g.n, g.rowptr, g.col, g.val)
    beta = 0.85 / O.lambda_max(W)
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F32, rank=16, n_hubs=30,
                                block_max=32, split=False, rhs_coupling=1)
    path = tmp_path / "z.katzidx"
    katz.katz_index_save(idx, path)
    back = katz.katz_index_load(path)
    assert katz.katz_index_get_info(back)["rhs_coupling"] == 1
    q = queries(g, back, 96, seed=12)
    ref = O.katz_direct(W, beta, q)
    K = torch.zeros((g.n, len(q)), dtype=torch.float64, device="cuda")
    st, _, _ = katz.katz_query_batch(back, torch.from_numpy(q).cuda(), K,
                                     out_dtype=katz.KATZ_F64, tol=1e-6)
    assert st["status"] == "KATZ_OK" and st["ms"][7] == 1.0
    assert O.error_inf_rel(K.cpu().numpy(), ref).max() <= 1e-6
