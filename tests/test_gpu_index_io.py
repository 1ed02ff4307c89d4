"""Index persistence: an index written by katz_index_save and read back by
katz_index_load answers queries as the original did (the stored artefact
of Algorithm 1, Section 3.2), and the loaded copy matches the FP64 oracle.

Tolerances: the loaded index holds the same bytes, so its Katz vectors
agree with the original's to the run-to-run spread of the FP64 atomic
reductions (1e-9 of the column maximum, far below the 1e-6 query bound);
integer outputs (partition, info) must be identical."""
import gc

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


def graph(weighted, seed=5):
    a = synth.chung_lu(5000, 2.2, 8.0, 400.0, seed=seed)
    s = synth.star(700)
    g = synth.disjoint_union([a, s])
    r = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    m = r < g.col
    u = np.concatenate([r[m], [0, 5000]])
    v = np.concatenate([g.col[m], [5000, 9]])
    wf = synth.dyadic_weights(seed + 1) if weighted else None
    return synth.edges_to_graph(g.n, u, v, {"kind": "io"}, wf)


def solve(fn, idx, g, q, **kw):
    K = torch.zeros((g.n, len(q)), dtype=torch.float64, device="cuda")
    st, it, rel = fn(idx, torch.from_numpy(q).cuda(), K, out_dtype=katz.KATZ_F64, tol=1e-6, **kw)
    assert st["status"] == "KATZ_OK"
    return K.cpu().numpy(), it


def close(A, B):
    return np.abs(A - B).max(axis=0) <= 1e-9 * np.abs(A).max(axis=0)


@pytest.mark.parametrize("vdt,weighted,split,coupling", [
    (katz.KATZ_F32, True, False, 1),
    (katz.KATZ_BF16, True, True, -1),
    (katz.KATZ_UNIT, False, False, 0),
])
def test_loaded_index_answers_like_the_saved_one(tmp_path, vdt, weighted, split, coupling):
    g = graph(weighted)
    W = O.adjacency(g.n, g.rowptr, g.col, g.val)
    beta = 0.85 / O.lambda_max(W)
    idx = katz.katz_index_build(g, beta, value_dtype=vdt, rank=16, n_hubs=40, block_max=32,
                                split=split, coupling_gemm=coupling)
    q = synth.queries(g.n, 97, seed=8)
    katz.katz_autotune(idx, len(q))
    K0, _ = solve(katz.katz_query_batch, idx, g, q)
    C0, _ = solve(katz.cg_query_batch, idx, g, q)
    # device_bytes also counts the query scratch, which is not stored
    info0 = {k: v for k, v in katz.katz_index_get_info(idx).items() if k != "device_bytes"}
    perm0, bp0, _, _ = katz.katz_index_get_partition(idx)
    sig0 = katz.katz_index_get_sigma(idx)
    path = tmp_path / "index.katzidx"
    katz.katz_index_save(idx, path)
    del idx
    gc.collect()

    idx2 = katz.katz_index_load(path)
    info1 = katz.katz_index_get_info(idx2)
    assert {k: v for k, v in info1.items() if k != "device_bytes"} == info0
    assert 0 < info1["device_bytes"]
    perm1, bp1, _, _ = katz.katz_index_get_partition(idx2)
    assert perm1.tolist() == perm0.tolist() and bp1.tolist() == bp0.tolist()
    assert katz.katz_index_get_sigma(idx2).tolist() == sig0.tolist()
    K1, _ = solve(katz.katz_query_batch, idx2, g, q)
    C1, _ = solve(katz.cg_query_batch, idx2, g, q)
    assert close(K0, K1).all() and close(C0, C1).all()
    cols = [0, 48, 96]
    ref = O.katz_direct(W, beta, q[cols])
    assert O.error_inf_rel(K1[:, cols], ref).max() <= 1e-6


def test_cg_only_index_roundtrip(tmp_path):
    g = graph(True, seed=6)
    W = O.adjacency(g.n, g.rowptr, g.col, g.val)
    beta = 0.5 / O.lambda_max(W)
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F64, build_lrc=False)
    q = synth.queries(g.n, 33, seed=2)
    C0, _ = solve(katz.cg_query_batch, idx, g, q)
    path = tmp_path / "cg.katzidx"
    katz.katz_index_save(idx, path)
    idx2 = katz.katz_index_load(path)
    C1, _ = solve(katz.cg_query_batch, idx2, g, q)
    assert close(C0, C1).all()
    assert O.error_inf_rel(C1[:, :4], O.katz_direct(W, beta, q[:4])).max() <= 1e-6


def test_warm_start_network_survives_the_roundtrip(tmp_path):
    g = synth.chung_lu(4000, 2.1, 6.0, 400.0, seed=72)
    W = O.adjacency(g.n, g.rowptr, g.col, g.val)
    beta = 1.0 / (O.lambda_max(W) + 1.0)
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F32, rank=16, n_hubs=40,
                                block_max=32)
    rng = np.random.default_rng(4)
    perm = rng.permutation(g.n).astype(np.int32)
    katz.katz_warmstart_train(idx, perm[:800], hidden=128, epochs=5, batch=128, lr=2e-3)
    test = np.sort(perm[800:864])
    K0, it0 = solve(katz.katz_query_batch, idx, g, test, warm_start=1)
    path = tmp_path / "warm.katzidx"
    katz.katz_index_save(idx, path)
    idx2 = katz.katz_index_load(path)
    K1, it1 = solve(katz.katz_query_batch, idx2, g, test, warm_start=1)
    assert close(K0, K1).all()
    assert np.abs(it0.astype(int) - it1.astype(int)).max() <= 1
    # the loaded index (features, Lanczos basis) can be trained again
    st = katz.katz_warmstart_train(idx2, perm[:800], hidden=128, epochs=1, batch=128, lr=2e-3)
    assert np.isfinite(st["final_loss"])


def test_corrupt_payload_is_rejected(tmp_path):
    g = graph(False, seed=7)
    W = O.adjacency(g.n, g.rowptr, g.col, g.val)
    idx = katz.katz_index_build(g, 0.5 / O.lambda_max(W), value_dtype=katz.KATZ_F32, rank=8,
                                n_hubs=20, block_max=32)
    path = tmp_path / "bad.katzidx"
    katz.katz_index_save(idx, path)
    data = bytearray(path.read_bytes())
    data[len(data) * 3 // 5] ^= 0x10
    path.write_bytes(bytes(data))
    with pytest.raises(katz.KatzError) as e:
        katz.katz_index_load(path)
    assert e.value.code == katz.KATZ_EINVAL
    path.write_bytes(bytes(data[: len(data) // 2]))
    with pytest.raises(katz.KatzError) as e:
        katz.katz_index_load(path)
    assert e.value.code == katz.KATZ_EINVAL
