"""The Python binding mirrors include/katz.h: every struct of the header has
a ctypes twin with the same field names in the same order at the same
offsets, and every KATZ_* constant the binding defines has the header's
value.  Host-only (the header is parsed as text; nothing is loaded)."""
import ctypes as C
import os
import re

import pytest

from paper_1912_06525_gb300 import katz

HEADER = os.path.join(os.path.dirname(__file__), "..", "include", "katz.h")

_SIZES = {"int64_t": 8, "uint64_t": 8, "int32_t": 4, "uint32_t": 4, "double": 8, "float": 4}


def _header_text():
    with open(HEADER) as f:
        text = f.read()
    return re.sub(r"/\*.*?\*/", " ", text, flags=re.S)


def _structs():
    """{name: [(field, size, count)]} for every `typedef struct { ... } name;`."""
    out = {}
    for body, name in re.findall(r"typedef\s+struct\s*\{(.*?)\}\s*(\w+)\s*;", _header_text(),
                                 flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            m = re.match(r"(?:const\s+)?(\w+)\s*(\**)\s*(.*)$", decl)
            base, ptr, rest = m.group(1), m.group(2), m.group(3)
            for item in rest.split(","):
                item = item.strip()
                stars = ptr + ("*" if item.startswith("*") else "")
                item = item.lstrip("*").strip()
                am = re.match(r"(\w+)\s*(?:\[(\d+)\])?$", item)
                size = 8 if stars else _SIZES[base]
                fields.append((am.group(1), size, int(am.group(2) or 1)))
        out[name] = fields
    return out


def _c_layout(fields):
    """Offsets and total size under the natural alignment of each member."""
    off, offsets, align = 0, [], 1
    for _, size, count in fields:
        off = (off + size - 1) // size * size
        offsets.append(off)
        off += size * count
        align = max(align, size)
    return offsets, (off + align - 1) // align * align


def test_header_structs_were_found():
    names = set(_structs())
    for n in ("katz_csr", "katz_build_opts", "katz_query_opts", "katz_stats", "katz_index_info",
              "katz_train_opts", "katz_train_stats"):
        assert n in names, n


@pytest.mark.parametrize("name", ["katz_csr", "katz_build_opts", "katz_query_opts", "katz_stats",
                                  "katz_index_info", "katz_train_opts", "katz_train_stats"])
def test_binding_struct_matches_header(name):
    fields = _structs()[name]
    cls = getattr(katz, name)
    assert [f[0] for f in cls._fields_] == [f[0] for f in fields], name
    offsets, size = _c_layout(fields)
    for (fname, _), off in zip(cls._fields_, offsets):
        assert getattr(cls, fname).offset == off, (name, fname)
    assert C.sizeof(cls) == size, name


def test_binding_constants_match_header():
    defines = dict((k, int(v)) for k, v in
                   re.findall(r"#define\s+(KATZ_\w+)\s+(-?\d+)\b", _header_text()))
    checked = 0
    for k, v in defines.items():
        if hasattr(katz, k):
            assert getattr(katz, k) == v, k
            checked += 1
    # the query options' selectors are all mirrored
    for group in ("KATZ_GATHER_", "KATZ_CHEB_", "KATZ_PREC_", "KATZ_TOL_"):
        for k in defines:
            if k.startswith(group):
                assert hasattr(katz, k), k
    assert checked >= 15
