"""Thin ctypes binding of libkatz.so (declared in include/katz.h).

Every function here only marshals arguments: the work happens in the CUDA
library.  Names match the C entry points.  Device buffers are torch CUDA
tensors; host buffers may be numpy arrays or CPU tensors (pinned CPU
tensors copy fastest).  There is no fallback: if libkatz.so is missing or a
call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkatz.so")

# status codes / element types / modes (mirror include/katz.h)
KATZ_OK, KATZ_EINVAL, KATZ_ENOTSPD, KATZ_ENOCONV, KATZ_ENOMEM, KATZ_ECUDA = range(6)
KATZ_UNIT, KATZ_F64, KATZ_F32, KATZ_BF16 = range(4)
KATZ_PREC_F32, KATZ_PREC_MIXED, KATZ_PREC_F64 = range(3)
KATZ_TOL_RESIDUAL, KATZ_TOL_ERROR_INF = range(2)
(KATZ_GATHER_AUTO, KATZ_GATHER_REGISTER, KATZ_GATHER_PIPELINED, KATZ_GATHER_ROWPIPE,
 KATZ_GATHER_CHUNKED) = range(5)
KATZ_CHEB_AUTO, KATZ_CHEB_F32, KATZ_CHEB_BF16, KATZ_CHEB_MIXED = range(4)

STATUS_NAMES = {0: "KATZ_OK", 1: "KATZ_EINVAL", 2: "KATZ_ENOTSPD", 3: "KATZ_ENOCONV",
                4: "KATZ_ENOMEM", 5: "KATZ_ECUDA"}

# every exported symbol of include/katz.h
EXPORTS = ["katz_lambda_max", "katz_lambda_bounds", "katz_index_build", "katz_index_free", "katz_index_save",
           "katz_index_load", "katz_index_get_info", "katz_index_get_partition", "katz_partition",
           "katz_index_get_sigma", "katz_query_batch", "cg_query_batch", "linkpred_topk",
           "linkpred_topk_noalloc", "sparse_katz_topk", "katz_apply_M", "katz_autotune", "katz_gemm_bf16",
           "katz_gemm_tf32x3", "katz_launch_count", "katz_fault_inject_alloc", "katz_test_stall_copies",
           "katz_profile_enable", "katz_profile_read", "katz_multi_build", "katz_multi_free",
           "katz_multi_query", "katz_index_build_many", "katz_multi_get_info",
           "katz_multi_query_lrc", "katz_warmstart_train", "katz_mlp_loss_grad", "katz_last_error"]


class KatzError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class katz_csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p)]


class katz_build_opts(C.Structure):
    _fields_ = [("value_dtype", C.c_int32), ("build_lrc", C.c_int32), ("rank", C.c_int32),
                ("n_hubs", C.c_int32), ("block_max", C.c_int32), ("split", C.c_int32),
                ("lanczos_steps", C.c_int32), ("n2_max", C.c_int32), ("seed", C.c_uint64),
                ("coupling_gemm", C.c_int32), ("rhs_coupling", C.c_int32)]


class katz_query_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("tol_kind", C.c_int32), ("precision", C.c_int32),
                ("max_iter", C.c_int32), ("max_refine", C.c_int32), ("rhs_width", C.c_int32),
                ("warm_start", C.c_int32), ("gather_kernel", C.c_int32),
                ("cheb_gather", C.c_int32)]


class katz_stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("refine_steps", C.c_int32), ("max_rel_res", C.c_double),
                ("ms", C.c_double * 8)]


class katz_train_opts(C.Structure):
    _fields_ = [("hidden", C.c_int32), ("epochs", C.c_int32), ("batch", C.c_int32),
                ("lr", C.c_float), ("weight_decay", C.c_float), ("seed", C.c_uint64)]


class katz_train_stats(C.Structure):
    _fields_ = [("initial_loss", C.c_double), ("final_loss", C.c_double), ("steps", C.c_int32),
                ("ms", C.c_double)]


class katz_index_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("n1", C.c_int64), ("n2", C.c_int64),
                ("n_blocks", C.c_int32), ("n_large_blocks", C.c_int32), ("rank", C.c_int32),
                ("value_dtype", C.c_int32), ("beta", C.c_double), ("lambda_max_R", C.c_double),
                ("device_bytes", C.c_int64), ("lambda_max_W", C.c_double),
                ("lambda_upper", C.c_double), ("schur_implicit", C.c_int32),
                ("rhs_coupling", C.c_int32)]


_lib = None


def lib() -> C.CDLL:
    """The loaded library; raises if libkatz.so has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1912_06525_gb300.build`")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        L.katz_lambda_max.argtypes = [C.POINTER(katz_csr), i32, C.POINTER(dbl), vp]
        L.katz_lambda_bounds.argtypes = [C.POINTER(katz_csr), i32, C.POINTER(dbl),
                                         C.POINTER(dbl), vp]
        L.katz_index_build.argtypes = [C.POINTER(katz_csr), dbl, C.POINTER(katz_build_opts), vp,
                                       C.POINTER(vp)]
        L.katz_index_free.argtypes = [vp]
        L.katz_index_free.restype = None
        L.katz_index_get_info.argtypes = [vp, C.POINTER(katz_index_info)]
        L.katz_index_save.argtypes = [vp, C.c_char_p]
        L.katz_index_load.argtypes = [C.c_char_p, C.POINTER(vp)]
        L.katz_index_get_partition.argtypes = [vp, vp, vp]
        L.katz_index_get_sigma.argtypes = [vp, vp]
        L.katz_partition.argtypes = [C.POINTER(katz_csr), i32, i32, i32, vp, vp, vp, vp]
        qargs = [vp, vp, i32, C.POINTER(katz_query_opts), vp, i32, i64, C.POINTER(katz_stats),
                 vp, vp, vp]
        L.katz_query_batch.argtypes = qargs
        L.cg_query_batch.argtypes = qargs
        L.linkpred_topk.argtypes = [vp, vp, i32, vp, i32, i64, i32, vp, vp, vp]
        L.linkpred_topk_noalloc.argtypes = [vp, vp, i32, vp, i32, i64, i32, vp, vp, vp]
        L.sparse_katz_topk.argtypes = [vp, vp, i32, i32, i32, C.POINTER(katz_query_opts), vp, vp,
                                       vp, C.POINTER(katz_stats), vp]
        L.katz_apply_M.argtypes = [vp, vp, vp, i32, i32, vp]
        L.katz_autotune.argtypes = [vp, i32, vp, vp, vp]
        L.katz_gemm_bf16.argtypes = [vp, i64, vp, i64, i32, i32, i32, C.c_float, C.c_float, vp,
                                     i64, vp]
        L.katz_gemm_tf32x3.argtypes = [vp, i64, vp, i64, i32, i32, i32, C.c_float, C.c_float,
                                       vp, i64, vp]
        L.katz_multi_build.argtypes = [i32, vp, vp, i32, vp, C.POINTER(vp)]
        L.katz_index_build_many.argtypes = [i32, vp, vp, C.POINTER(katz_build_opts), vp,
                                            C.POINTER(vp)]
        L.katz_multi_get_info.argtypes = [vp, vp, vp, vp]
        L.katz_multi_query_lrc.argtypes = [vp, vp, i32, C.POINTER(katz_query_opts), vp, i32, i64,
                                           C.POINTER(katz_stats), vp, vp, vp]
        L.katz_multi_free.argtypes = [vp]
        L.katz_multi_free.restype = None
        L.katz_multi_query.argtypes = [vp, vp, i32, C.POINTER(katz_query_opts), vp, i32, i64,
                                       C.POINTER(katz_stats), vp, vp, vp]
        L.katz_warmstart_train.argtypes = [vp, vp, i32, C.POINTER(katz_train_opts),
                                           C.POINTER(katz_train_stats), vp]
        L.katz_mlp_loss_grad.argtypes = [i32, i32, i32, i32, vp, vp, vp, vp, vp, vp]
        L.katz_launch_count.argtypes = []
        L.katz_launch_count.restype = C.c_int64
        L.katz_profile_enable.argtypes = [i32]
        L.katz_fault_inject_alloc.argtypes = [i64]
        L.katz_test_stall_copies.argtypes = [i32]
        L.katz_profile_read.argtypes = [C.c_char_p, vp, vp, vp]
        L.katz_last_error.restype = C.c_char_p
        for name in EXPORTS:
            if name not in ("katz_index_free", "katz_last_error", "katz_launch_count",
                            "katz_multi_free"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def katz_last_error() -> str:
    return lib().katz_last_error().decode()


def _check(code: int, allow=(KATZ_OK,)) -> int:
    if code not in allow:
        raise KatzError(code, katz_last_error())
    return code


def _ld(x) -> int:
    """Leading dimension (elements) of a row-major 2-D block; the columns
    must be contiguous."""
    if hasattr(x, "stride"):
        if x.dim() != 2 or x.stride(1) != 1:
            raise ValueError("expected a 2-D tensor with contiguous rows")
        return int(x.stride(0))
    if x.ndim != 2 or x.strides[1] != x.itemsize:
        raise ValueError("expected a 2-D array with contiguous rows")
    return int(x.strides[0] // x.itemsize)


def _ptr(x):
    """Address of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


def _csr(graph):
    """katz_csr from an object with n, rowptr, col, val (val None = unit)."""
    rowptr = np.ascontiguousarray(graph.rowptr, dtype=np.int64)
    col = np.ascontiguousarray(graph.col, dtype=np.int32)
    val = None if graph.val is None else np.ascontiguousarray(graph.val, dtype=np.float64)
    c = katz_csr(int(graph.n), int(rowptr[-1]), rowptr.ctypes.data, col.ctypes.data,
                 None if val is None else val.ctypes.data)
    return c, (rowptr, col, val)


def katz_lambda_max(graph, steps: int = 0, stream=None) -> float:
    c, keep = _csr(graph)
    out = C.c_double()
    _check(lib().katz_lambda_max(C.byref(c), steps, C.byref(out), _stream(stream)))
    return out.value


def katz_lambda_bounds(graph, steps: int = 0, stream=None) -> tuple[float, float]:
    """(largest Ritz value, rigorous upper bound) of lambda_max of W."""
    c, keep = _csr(graph)
    lo, up = C.c_double(), C.c_double()
    _check(lib().katz_lambda_bounds(C.byref(c), steps, C.byref(lo), C.byref(up),
                                    _stream(stream)))
    return lo.value, up.value


class KatzIndex:
    """Owner of a katz_index* (freed on garbage collection)."""

    def __init__(self, handle: int):
        self.handle = C.c_void_p(handle)

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value and _lib is not None:
            _lib.katz_index_free(self.handle)
            self.handle = C.c_void_p(0)

    def info(self) -> dict:
        return katz_index_get_info(self)


def katz_index_build(graph, beta: float, value_dtype: int = KATZ_F32, build_lrc: bool = True,
                     rank: int = 16, n_hubs: int = 0, block_max: int = 64, split: bool = True,
                     lanczos_steps: int = 0, n2_max: int = 0, seed: int = 20191212,
                     coupling_gemm: int = 0, rhs_coupling: int = 0,
                     stream=None) -> KatzIndex:
    c, keep = _csr(graph)
    o = katz_build_opts(value_dtype, int(build_lrc), rank, n_hubs, block_max, int(split),
                        lanczos_steps, n2_max, seed, coupling_gemm, rhs_coupling)
    h = C.c_void_p()
    _check(lib().katz_index_build(C.byref(c), float(beta), C.byref(o), _stream(stream),
                                  C.byref(h)))
    return KatzIndex(h.value)


def katz_index_save(index: KatzIndex, path) -> None:
    """Write every stored field of the index to `path`."""
    _check(lib().katz_index_save(index.handle, os.fsencode(path)))


def katz_index_load(path) -> KatzIndex:
    """Read an index written by katz_index_save onto the current device."""
    h = C.c_void_p()
    _check(lib().katz_index_load(os.fsencode(path), C.byref(h)))
    return KatzIndex(h.value)


def katz_index_get_info(index: KatzIndex) -> dict:
    i = katz_index_info()
    _check(lib().katz_index_get_info(index.handle, C.byref(i)))
    return {f: getattr(i, f) for f, _ in katz_index_info._fields_}


def katz_index_get_partition(index: KatzIndex):
    info = katz_index_get_info(index)
    perm = np.empty(info["n"], dtype=np.int64)
    bp = np.empty(info["n_blocks"] + 1, dtype=np.int64)
    _check(lib().katz_index_get_partition(index.handle, perm.ctypes.data, bp.ctypes.data))
    return perm, bp, info["n1"], info["n2"]


def katz_partition(graph, n_hubs: int, block_max: int, split: bool = True):
    """Host-only partition; returns (perm, block_ptr, n1, n2)."""
    c, keep = _csr(graph)
    perm = np.empty(graph.n, dtype=np.int64)
    bp = np.empty(graph.n + 1, dtype=np.int64)
    nb = np.zeros(1, dtype=np.int64)
    n1 = np.zeros(1, dtype=np.int64)
    _check(lib().katz_partition(C.byref(c), n_hubs, block_max, int(split), perm.ctypes.data,
                                bp.ctypes.data, nb.ctypes.data, n1.ctypes.data))
    return perm, bp[: int(nb[0]) + 1].copy(), int(n1[0]), graph.n - int(n1[0])


def katz_index_get_sigma(index: KatzIndex) -> np.ndarray:
    info = katz_index_get_info(index)
    s = np.empty(max(info["rank"], 1), dtype=np.float64)
    _check(lib().katz_index_get_sigma(index.handle, s.ctypes.data))
    return s[: info["rank"]]


def _query(fn, index, q, K_out, out_dtype, tol, tol_kind, precision, max_iter, max_refine,
           rhs_width, warm_start, gather_kernel, stream, cheb_gather=KATZ_CHEB_AUTO):
    b = int(q.shape[0])
    o = katz_query_opts(float(tol), tol_kind, precision, max_iter, max_refine, rhs_width,
                        warm_start, gather_kernel, cheb_gather)
    st = katz_stats()
    iters = np.zeros(b, dtype=np.int32)
    rel = np.zeros(b, dtype=np.float64)
    ldk = _ld(K_out)
    code = fn(index.handle, _ptr(q), b, C.byref(o), _ptr(K_out), out_dtype, ldk, C.byref(st),
              iters.ctypes.data, rel.ctypes.data, _stream(stream))
    _check(code, allow=(KATZ_OK, KATZ_ENOCONV))
    stats = {"iters": st.iters, "refine_steps": st.refine_steps, "max_rel_res": st.max_rel_res,
             "ms": list(st.ms), "status": STATUS_NAMES[code]}
    return stats, iters, rel


def katz_query_batch(index, q, K_out, out_dtype=KATZ_F32, tol=1e-6,
                     tol_kind=KATZ_TOL_ERROR_INF, precision=KATZ_PREC_MIXED, max_iter=0,
                     max_refine=0, rhs_width=0, warm_start=0, gather_kernel=KATZ_GATHER_AUTO,
                     stream=None, cheb_gather=KATZ_CHEB_AUTO):
    """LRC-Katz (Algorithm 2).  q: int32 (b,) host or device; K_out: (n, b)
    node-major float32/float64, host or device.  Returns (stats, iters, rel_res)."""
    return _query(lib().katz_query_batch, index, q, K_out, out_dtype, tol, tol_kind, precision,
                  max_iter, max_refine, rhs_width, warm_start, gather_kernel, stream,
                  cheb_gather)


def cg_query_batch(index, q, K_out, out_dtype=KATZ_F32, tol=1e-6, tol_kind=KATZ_TOL_ERROR_INF,
                   precision=KATZ_PREC_MIXED, max_iter=0, max_refine=0, rhs_width=0,
                   warm_start=0, gather_kernel=KATZ_GATHER_AUTO, stream=None):
    """Plain CG on M (the comparison method); same contract as katz_query_batch."""
    return _query(lib().cg_query_batch, index, q, K_out, out_dtype, tol, tol_kind, precision,
                  max_iter, max_refine, rhs_width, warm_start, gather_kernel, stream)


def linkpred_topk(index, q, K, k_dtype, k, ids_out, scores_out, stream=None):
    """Top-k link candidates per query column of K (Section 3.3)."""
    b = int(q.shape[0])
    ldk = _ld(K)
    _check(lib().linkpred_topk(index.handle, _ptr(q), b, _ptr(K), k_dtype, ldk, k,
                               _ptr(ids_out), _ptr(scores_out), _stream(stream)))


def linkpred_topk_noalloc(index, q, K, k_dtype, k, ids_out, scores_out, stream=None):
    """linkpred_topk with its scratch in a fixed library array (no device
    allocation); q, K, ids_out and scores_out must be device tensors."""
    b = int(q.shape[0])
    _check(lib().linkpred_topk_noalloc(index.handle, _ptr(q), b, _ptr(K), k_dtype, _ld(K), k,
                                       _ptr(ids_out), _ptr(scores_out), _stream(stream)))


def sparse_katz_topk(index, q, s, T, ids_out, rho_out, landmarks_out=None, tol=1e-6,
                     tol_kind=KATZ_TOL_ERROR_INF, precision=KATZ_PREC_MIXED, max_iter=0,
                     max_refine=0, gather_kernel=KATZ_GATHER_AUTO, stream=None) -> dict:
    """Sparse-Katz (Algorithm 3): re-ranked Top-s candidates (ids_out, b x s
    int32) with their Pearson correlations over T landmarks (rho_out, b x s
    float64); landmarks_out (b x T int32) optional.  Returns the stats."""
    b = int(q.shape[0])
    o = katz_query_opts(float(tol), tol_kind, precision, max_iter, max_refine, 0, 0,
                        gather_kernel)
    st = katz_stats()
    code = lib().sparse_katz_topk(index.handle, _ptr(q), b, s, T, C.byref(o), _ptr(ids_out),
                                  _ptr(rho_out), _ptr(landmarks_out), C.byref(st),
                                  _stream(stream))
    _check(code, allow=(KATZ_OK, KATZ_ENOCONV))
    return {"iters": st.iters, "refine_steps": st.refine_steps, "max_rel_res": st.max_rel_res,
            "ms": list(st.ms), "distinct_landmarks": int(st.ms[6]),
            "status": STATUS_NAMES[code]}


def katz_test_stall_copies(on: bool) -> None:
    """Test hook: the tensor-core GEMM issues no TMA copies while on, so its
    bounded pipeline wait runs out and the call returns KATZ_ECUDA."""
    _check(lib().katz_test_stall_copies(1 if on else 0))


def katz_fault_inject_alloc(after: int) -> None:
    """Test hook: the device allocation after `after` more fails (KATZ_ENOMEM)."""
    _check(lib().katz_fault_inject_alloc(int(after)))


def katz_apply_M(index, X, Y, b, dtype, stream=None):
    """Y = M X = X - beta W X (device n x b blocks)."""
    _check(lib().katz_apply_M(index.handle, _ptr(X), _ptr(Y), b, dtype, _stream(stream)))


def katz_launch_count() -> int:
    return int(lib().katz_launch_count())


def katz_profile_enable(on: bool) -> None:
    _check(lib().katz_profile_enable(int(on)))


def katz_profile_read(tag: str) -> dict:
    n = np.zeros(1, dtype=np.int64)
    ms = np.zeros(1, dtype=np.float64)
    by = np.zeros(1, dtype=np.float64)
    _check(lib().katz_profile_read(tag.encode(), n.ctypes.data, ms.ctypes.data, by.ctypes.data))
    return {"launches": int(n[0]), "ms": float(ms[0]), "bytes": float(by[0])}


def katz_gemm_bf16(A, B, C_out, K=None, alpha=1.0, beta=0.0, stream=None):
    """C_out = alpha * A[:, :K] @ B[:, :K].T + beta * C_out on tcgen05 (A: M x ld,
    B: N x ld BF16 device tensors with contiguous rows; C_out: M x N float32)."""
    M = A.shape[0]
    K = A.shape[1] if K is None else K
    N = B.shape[0]
    _check(lib().katz_gemm_bf16(_ptr(A), _ld(A), _ptr(B), _ld(B), M, N, K, alpha, beta,
                                _ptr(C_out), _ld(C_out), _stream(stream)))


def katz_gemm_tf32x3(A, B, C_out, K=None, alpha=1.0, beta=0.0, stream=None):
    """C_out = alpha * A[:, :K] @ B[:, :K].T + beta * C_out, FP32-accurate on the
    tensor cores (three TF32 products); A: M x ld, B: N x ld, C_out: M x N float32."""
    M = A.shape[0]
    K = A.shape[1] if K is None else K
    N = B.shape[0]
    _check(lib().katz_gemm_tf32x3(_ptr(A), _ld(A), _ptr(B), _ld(B), M, N, K, alpha, beta,
                                  _ptr(C_out), _ld(C_out), _stream(stream)))


def katz_autotune(index, b: int, stream=None) -> dict:
    """Tune the SpMM launch shape for width b; returns the choice and times."""
    out = np.zeros(11, dtype=np.int32)
    ms = np.zeros(2, dtype=np.float64)
    _check(lib().katz_autotune(index.handle, b, out.ctypes.data, ms.ctypes.data, _stream(stream)))
    return {"col_tile": int(out[0]), "ctas_per_sm": int(out[1]), "cheb_pipe": bool(out[2]),
            "residual_first_pipe": bool(out[3]), "residual_pipe": bool(out[4]),
            "cheb_ctas_per_sm": int(out[5]), "residual_ctas_per_sm": int(out[6]),
            "cheb_gather_depth": int(out[7]), "cheb_row_pipeline": bool(out[8]),
            "cheb_row_chunk": int(out[9]), "residual_row_chunk": int(out[10]),
            "ms_best": float(ms[0]), "ms_default": float(ms[1])}


class KatzMulti:
    """Owner of a katz_multi* (many graphs answered together)."""

    def __init__(self, handle: int, sizes):
        self.handle = C.c_void_p(handle)
        self.sizes = list(sizes)

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value and _lib is not None:
            _lib.katz_multi_free(self.handle)
            self.handle = C.c_void_p(0)


def katz_multi_build(graphs, betas, value_dtype=KATZ_UNIT, stream=None) -> KatzMulti:
    csrs, keep = [], []
    for g in graphs:
        c, k = _csr(g)
        csrs.append(c)
        keep.append(k)
    arr = (katz_csr * len(csrs))(*csrs)
    b = np.ascontiguousarray(betas, dtype=np.float64)
    h = C.c_void_p()
    _check(lib().katz_multi_build(len(csrs), C.cast(arr, C.c_void_p), b.ctypes.data, value_dtype,
                                  _stream(stream), C.byref(h)))
    return KatzMulti(h.value, [g.n for g in graphs])


def katz_index_build_many(graphs, betas, value_dtype=KATZ_UNIT, rank=32, n_hubs=0,
                          block_max=64, split=False, lanczos_steps=0, seed=20191212,
                          stream=None) -> KatzMulti:
    """Per-graph LRC index of many graphs (see katz.h)."""
    csrs, keep = [], []
    for g in graphs:
        c, k = _csr(g)
        csrs.append(c)
        keep.append(k)
    arr = (katz_csr * len(csrs))(*csrs)
    b = np.ascontiguousarray(betas, dtype=np.float64)
    o = katz_build_opts(value_dtype, 1, rank, n_hubs, block_max, int(split), lanczos_steps, 0,
                        seed, -1)
    h = C.c_void_p()
    _check(lib().katz_index_build_many(len(csrs), C.cast(arr, C.c_void_p), b.ctypes.data,
                                       C.byref(o), _stream(stream), C.byref(h)))
    return KatzMulti(h.value, [g.n for g in graphs])


def katz_multi_get_info(multi):
    """(separator sizes, ranks, Ritz values per graph) of a per-graph LRC index."""
    G = len(multi.sizes)
    n2 = np.zeros(G, dtype=np.int64)
    r = np.zeros(G, dtype=np.int32)
    _check(lib().katz_multi_get_info(multi.handle, n2.ctypes.data, r.ctypes.data, None))
    sig = np.zeros(max(1, int(r.sum())), dtype=np.float64)
    _check(lib().katz_multi_get_info(multi.handle, None, None, sig.ctypes.data))
    offs = np.concatenate([[0], np.cumsum(r)])
    return n2, r, [sig[offs[i]:offs[i + 1]] for i in range(G)]


def katz_multi_query_lrc(multi, q, qpg, K_out, out_dtype=KATZ_F32, tol=1e-6,
                         tol_kind=KATZ_TOL_ERROR_INF, max_iter=0, max_refine=0, stream=None):
    """katz_multi_query with the per-graph LRC inner solve."""
    return katz_multi_query(multi, q, qpg, K_out, out_dtype, tol, tol_kind, max_iter, max_refine,
                            stream, _fn="katz_multi_query_lrc")


def katz_multi_query(multi, q, qpg, K_out, out_dtype=KATZ_F32, tol=1e-6,
                     tol_kind=KATZ_TOL_ERROR_INF, max_iter=0, max_refine=0, stream=None,
                     _fn="katz_multi_query"):
    """q: (g*qpg,) graph-local ids; K_out: (sum n_g, qpg).  Returns
    (stats, iters (g*qpg,), rel_res (g*qpg,))."""
    o = katz_query_opts(float(tol), tol_kind, KATZ_PREC_MIXED, max_iter, max_refine, 0, 0, 0,
                        KATZ_CHEB_AUTO)
    st = katz_stats()
    total = len(multi.sizes) * qpg
    iters = np.zeros(total, dtype=np.int32)
    rel = np.zeros(total, dtype=np.float64)
    code = getattr(lib(), _fn)(multi.handle, _ptr(q), qpg, C.byref(o), _ptr(K_out), out_dtype,
                               _ld(K_out), C.byref(st), iters.ctypes.data, rel.ctypes.data,
                               _stream(stream))
    _check(code, allow=(KATZ_OK, KATZ_ENOCONV))
    stats = {"iters": st.iters, "refine_steps": st.refine_steps, "max_rel_res": st.max_rel_res,
             "ms": list(st.ms), "graph_replays": int(st.ms[4]), "status": STATUS_NAMES[code]}
    return stats, iters, rel


def katz_warmstart_train(index, q_train, hidden=256, epochs=20, batch=256, lr=1e-3,
                         weight_decay=0.0, seed=20191212, stream=None) -> dict:
    """Train the learned warm start on the method's own Katz vectors."""
    q = np.ascontiguousarray(q_train, dtype=np.int32)
    o = katz_train_opts(hidden, epochs, batch, lr, weight_decay, seed)
    st = katz_train_stats()
    _check(lib().katz_warmstart_train(index.handle, q.ctypes.data, len(q), C.byref(o),
                                      C.byref(st), _stream(stream)))
    return {"initial_loss": st.initial_loss, "final_loss": st.final_loss, "steps": st.steps,
            "ms": st.ms}


def katz_mlp_loss_grad(X, T, params, grads, din, dh, dout, stream=None) -> float:
    """Forward/backward of the warm-start network on device tensors."""
    loss = np.zeros(1, dtype=np.float64)
    _check(lib().katz_mlp_loss_grad(int(X.shape[0]), din, dh, dout, _ptr(X), _ptr(T),
                                    _ptr(params), _ptr(grads), loss.ctypes.data, _stream(stream)))
    return float(loss[0])
