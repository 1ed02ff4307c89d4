"""Parity of both kernels of the wide fused products -- the register kernels
and the pipelined (TMA bulk-copy) ones, forced through the query option --
against the FP64 oracle.  Widths b >= 61 (padded width >= 64) let the
pipelined kernels take the large-block Chebyshev steps and the refinement
residual; the graphs have a large component kept whole (split=False), a
900-entry hub row that wraps the shared-memory ring many times, isolated
nodes (rows without entries), and unit, FP32 and BF16 (dyadic, exact)
weights."""
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
    g = synth.disjoint_union([a, s, iso, iso, iso])
    r = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    m = r < g.col
    u = np.concatenate([r[m], [0, 3000]])
    v = np.concatenate([g.col[m], [3000, 7]])  # connect the star to the rest
    wf = synth.dyadic_weights(seed + 3) if weighted else None
    return synth.edges_to_graph(g.n, u, v, {"kind": "pipe"}, wf)


@pytest.mark.parametrize("vdt", [katz.KATZ_UNIT, katz.KATZ_F32, katz.KATZ_BF16])
@pytest.mark.parametrize("b", [61, 333, 1024])
def test_pipelined_paths_match_oracle(vdt, b):
    g = graph(weighted=vdt != katz.KATZ_UNIT)
    W = O.adjacency(g.n, g.rowptr, g.col, g.val)
    beta = 0.85 / O.lambda_max(W)
    idx = katz.katz_index_build(g, beta, value_dtype=vdt, rank=16, n_hubs=30, block_max=32,
                                split=False)
    q = synth.queries(g.n, b, seed=b)
    q[0] = 3000           # the star's hub (900 entries)
    q[1] = g.n - 1        # an isolated node: its column is zero
    ref = O.katz_direct(W, beta, q)
    for kern in (katz.KATZ_GATHER_REGISTER, katz.KATZ_GATHER_PIPELINED,
                 katz.KATZ_GATHER_CHUNKED):
        for fn in (katz.katz_query_batch, katz.cg_query_batch):
            K = torch.zeros((g.n, b), dtype=torch.float64, device="cuda")
            st, it, rel = fn(idx, torch.from_numpy(q).cuda(), K, out_dtype=katz.KATZ_F64, tol=1e-6,
                             gather_kernel=kern)
            assert st["status"] == "KATZ_OK", (fn.__name__, kern, st)
            Kh = K.cpu().numpy()
            assert np.all(Kh[:, 1] == 0)
            err = O.error_inf_rel(Kh, ref)
            assert err.max() <= 1e-6, (fn.__name__, kern, err.max())


@pytest.mark.parametrize("vdt", [katz.KATZ_UNIT, katz.KATZ_BF16])
@pytest.mark.parametrize("b", [5, 333, 1024])
def test_chebyshev_gather_precisions_match_oracle(vdt, b):
    """The large M11 block's Chebyshev steps with FP32 iterates (AUTO, F32;
    the register kernel with strided rows or contiguous row runs per CTA,
    and the row-pipelined one),
    with split BF16 iterates gathered as hi + lo on a solve's last step
    (MIXED), and with hi-plane gathers on every step (BF16): the refined
    answers all meet the 1e-6 bound; 128-column tiles of 16-byte lane
    accesses (b = 5) and 256-column tiles of 32-byte ones, ragged tails,
    unit and BF16 weights."""
    g = graph(weighted=vdt != katz.KATZ_UNIT, seed=13)
    W = O.adjacency(g.n, g.rowptr, g.col, g.val)
    beta = 0.9 / O.lambda_max(W)
    idx = katz.katz_index_build(g, beta, value_dtype=vdt, rank=16, n_hubs=30, block_max=32,
                                split=False)
    assert idx.info()["n_large_blocks"] >= 1
    q = synth.queries(g.n, b, seed=b + 1)
    q[0] = 3000
    ref = O.katz_direct(W, beta, q)
    for mode, kern in ((katz.KATZ_CHEB_AUTO, katz.KATZ_GATHER_REGISTER),
                       (katz.KATZ_CHEB_F32, katz.KATZ_GATHER_REGISTER),
                       (katz.KATZ_CHEB_BF16, katz.KATZ_GATHER_REGISTER),
                       (katz.KATZ_CHEB_MIXED, katz.KATZ_GATHER_REGISTER),
                       (katz.KATZ_CHEB_AUTO, katz.KATZ_GATHER_ROWPIPE),
                       (katz.KATZ_CHEB_F32, katz.KATZ_GATHER_ROWPIPE),
                       (katz.KATZ_CHEB_AUTO, katz.KATZ_GATHER_CHUNKED),
                       (katz.KATZ_CHEB_F32, katz.KATZ_GATHER_CHUNKED),
                       (katz.KATZ_CHEB_BF16, katz.KATZ_GATHER_CHUNKED)):
        K = torch.zeros((g.n, b), dtype=torch.float32, device="cuda")
        st, it, rel = katz.katz_query_batch(idx, torch.from_numpy(q).cuda(), K, tol=1e-6,
                                            gather_kernel=kern, cheb_gather=mode)
        assert st["status"] == "KATZ_OK", (mode, st)
        err = O.error_inf_rel(K.double().cpu().numpy(), ref)
        assert err.max() <= 1e-6, (mode, err.max())


def test_autotune_reports_kernel_choice():
    g = graph(weighted=False)
    beta = 0.85 / katz.katz_lambda_max(g, steps=96)
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_UNIT, rank=16, n_hubs=30,
                                block_max=32, split=False)
    res = katz.katz_autotune(idx, 256)
    assert isinstance(res["cheb_pipe"], bool)
    assert res["cheb_ctas_per_sm"] in (8, 16, 32, 64, 128)
    assert res["cheb_row_chunk"] in (0, 32, 64, 128, 256)
    assert res["residual_row_chunk"] in (0, 32, 64, 128, 256)
    assert res["residual_ctas_per_sm"] in (8, 16, 32, 64, 128)
    q = synth.queries(g.n, 256, seed=5)
    K = torch.zeros((g.n, 256), dtype=torch.float32, device="cuda")
    st, _, _ = katz.katz_query_batch(idx, torch.from_numpy(q).cuda(), K, tol=1e-6)
    assert st["status"] == "KATZ_OK"


@pytest.mark.parametrize("coupling", [-1, 1])
def test_coupling_product_paths_match_oracle(coupling):
    """Back-substitution by a second M11 solve (coupling_gemm=-1) or by the
    stored beta M11^{-1} W12 on the tensor cores (coupling_gemm=1); the first
    Schur right-hand side by an M11 solve (rhs_coupling=-1), which the
    tensor-core back-substitution needs (Y1)."""
    g = graph(weighted=True)
    W = O.adjacency(g.n, g.rowptr, g.col, g.val)
    beta = 0.85 / O.lambda_max(W)
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F32, rank=16, n_hubs=30,
                                block_max=32, split=False, coupling_gemm=coupling,
                                rhs_coupling=-1)
    q = synth.queries(g.n, 200, seed=4)
    ref = O.katz_direct(W, beta, q)
    for prec in (katz.KATZ_PREC_MIXED, katz.KATZ_PREC_F32):
        K = torch.zeros((g.n, len(q)), dtype=torch.float64, device="cuda")
        st, it, rel = katz.katz_query_batch(idx, torch.from_numpy(q).cuda(), K,
                                            out_dtype=katz.KATZ_F64, tol=1e-6, precision=prec)
        assert st["status"] == "KATZ_OK"
        bound = 1e-6 if prec == katz.KATZ_PREC_MIXED else 1e-4
        assert O.error_inf_rel(K.cpu().numpy(), ref).max() <= bound


def test_large_separator_tensor_core_schur_products_match_oracle():
    """A separator of 4,200 hubs (>= 4,096) puts S P and M22^{-1} R of the
    FP32 Schur PCG on the tensor cores (three-TF32 products)."""
    g = synth.chung_lu(60000, 2.1, 10.0, 3000.0, seed=31)
    W = O.adjacency(g.n, g.rowptr, g.col, g.val)
    beta = 0.9 / O.lambda_max(W)
    idx = katz.katz_index_build(g, beta, value_dtype=katz.KATZ_F32, rank=32, n_hubs=4200,
                                block_max=64, split=False)
    assert katz.katz_index_get_info(idx)["n2"] == 4200
    q = synth.queries(g.n, 128, seed=6)
    cols = [0, 1, 64, 127]
    Kref, _ = O.katz_cg(W, beta, q[cols], rtol=1e-12)
    for fn in (katz.katz_query_batch, katz.cg_query_batch):
        K = torch.zeros((g.n, len(q)), dtype=torch.float64, device="cuda")
        st, it, rel = fn(idx, torch.from_numpy(q).cuda(), K, out_dtype=katz.KATZ_F64, tol=1e-6)
        assert st["status"] == "KATZ_OK", (fn.__name__, st)
        assert O.error_inf_rel(K.cpu().numpy()[:, cols], Kref).max() <= 1e-6, fn.__name__
