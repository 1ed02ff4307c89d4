"""C-ABI checks that need no GPU: the library loads, exports every entry
point declared in include/katz.h, validates inputs on the host, and its
host-side partitioner agrees node for node with the oracle's reading of
Section 3.2, Steps 2-3."""
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1912_06525_gb300 import katz, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    return katz.lib()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "katz.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int64_t|int|void|const char\*)\s+(\w+)\s*\(", txt, flags=re.M)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(L, name), name
    assert sorted(katz.EXPORTS) == names


def test_host_validation_rejects_bad_csr(L):
    g = synth.path(4)
    bad = synth.Graph(n=4, rowptr=g.rowptr, col=g.col.copy(), val=None)
    bad.col[0] = 7  # out of range
    with pytest.raises(katz.KatzError) as e:
        katz.katz_partition(bad, 0, 4)
    assert e.value.code == katz.KATZ_EINVAL
    asym = synth.Graph(n=3, rowptr=np.array([0, 1, 1, 1]), col=np.array([1], dtype=np.int32))
    with pytest.raises(katz.KatzError) as e:
        katz.katz_partition(asym, 0, 4)
    assert e.value.code == katz.KATZ_EINVAL
    loop = synth.Graph(n=2, rowptr=np.array([0, 1, 1]), col=np.array([0], dtype=np.int32))
    with pytest.raises(katz.KatzError):
        katz.katz_partition(loop, 0, 4)


def _same(g, hubs, bmax, split):
    perm, bp, n1, n2 = katz.katz_partition(g, hubs, bmax, split)
    ref = O.partition(g.n, g.rowptr, g.col, hubs, bmax, split)
    assert perm.tolist() == ref["perm"].tolist()
    assert bp.tolist() == ref["block_ptr"].tolist()
    assert (n1, n2) == (ref["n1"], ref["n2"])


def test_partition_bit_exact_small_cases(L):
    _same(synth.path(7), 0, 3, True)
    _same(synth.star(5), 1, 4, True)
    _same(synth.cycle(30), 0, 4, True)
    _same(synth.complete(9), 2, 3, True)
    _same(synth.path(1), 0, 4, True)


@pytest.mark.parametrize("split,hubs,bmax", [(True, 0, 16), (True, 25, 32), (False, 40, 8),
                                             (True, 5, 1)])
def test_partition_bit_exact_random_graphs(L, split, hubs, bmax):
    _same(synth.chung_lu(1500, 2.1, 6.0, 300.0, seed=11), hubs, bmax, split)
    _same(synth.sbm_bernoulli([50] * 6, 0.1, 0.005, seed=3), hubs, bmax, split)


def test_partition_bit_exact_workload1(L):
    g, q, c, r = synth.workload(1)
    _same(g, 0, 64, True)
    _same(g, 20, 32, True)


def _index_file_header(version=1, mark=0x01020304):
    return b"KATZIDX\0" + np.array([version, mark], dtype="<u4").tobytes()


def test_index_load_rejects_bad_files_on_the_host(L, tmp_path):
    """katz_index_load validates the file before touching device memory:
    missing, foreign, other-version and truncated files are KATZ_EINVAL."""
    cases = {
        "missing": None,
        "foreign": b"PK\x03\x04" + bytes(60),
        "version": _index_file_header(version=99) + bytes(16),
        "byteorder": _index_file_header(mark=0x04030201) + bytes(16),
        "truncated": _index_file_header() + bytes(5),
        "empty": b"",
    }
    for name, data in cases.items():
        path = tmp_path / f"{name}.katzidx"
        if data is not None:
            path.write_bytes(data)
        with pytest.raises(katz.KatzError) as e:
            katz.katz_index_load(path)
        assert e.value.code == katz.KATZ_EINVAL, name
    msg = katz.katz_last_error()
    assert "truncated" in msg or "magic" in msg


def test_injected_allocation_failure_on_the_host(L):
    """katz_fault_inject_alloc(0): the first device allocation of the build
    fails before any CUDA call is made, so the build unwinds with
    KATZ_ENOMEM on a machine without a GPU; the hook then switches off."""
    g = synth.path(6)
    try:
        katz.katz_fault_inject_alloc(0)
        with pytest.raises(katz.KatzError) as e:
            katz.katz_index_build(g, 0.2, value_dtype=katz.KATZ_UNIT, build_lrc=False)
        assert e.value.code == katz.KATZ_ENOMEM
        assert "injected" in katz.katz_last_error()
    finally:
        katz.katz_fault_inject_alloc(-1)


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), 0.0, -1.0])
def test_host_validation_rejects_bad_weights(L, bad):
    """Weights must be positive and finite (NaN, infinity, zero and
    negative values are rejected on the host with KATZ_EINVAL)."""
    g = synth.path(5)
    val = np.ones(len(g.col))
    # the edge 1-2 in both directions
    for i, j in ((1, 2), (2, 1)):
        k = g.rowptr[i] + int(np.nonzero(g.col[g.rowptr[i]:g.rowptr[i + 1]] == j)[0][0])
        val[k] = bad
    w = synth.Graph(n=g.n, rowptr=g.rowptr, col=g.col, val=val)
    with pytest.raises(katz.KatzError) as e:
        katz.katz_partition(w, 0, 4)
    assert e.value.code == katz.KATZ_EINVAL
