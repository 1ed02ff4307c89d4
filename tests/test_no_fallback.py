"""The product path has no CPU fallback (CPU checks, no GPU needed).

The binding raises when libkatz.so is missing instead of computing
anything itself, and neither the package nor the CUDA sources refer to the
oracle: only the tests, the smoke check and the benchmark's CPU-baseline
and reference legs may use it.
"""
import os
import re

import pytest

from paper_1912_06525_gb300 import katz, synth

PKG = os.path.dirname(os.path.abspath(katz.__file__))


def _package_files(exts):
    for root, dirs, files in os.walk(PKG):
        dirs[:] = [d for d in dirs if not d.startswith(("_", "."))]
        for f in files:
            if f.endswith(exts):
                yield os.path.join(root, f)


def test_binding_raises_without_the_library(monkeypatch, tmp_path):
    monkeypatch.setattr(katz, "_lib", None)
    monkeypatch.setattr(katz, "LIB_PATH", str(tmp_path / "libkatz.so"))
    with pytest.raises(RuntimeError, match="missing"):
        katz.lib()
    g = synth.single_edge()
    with pytest.raises(RuntimeError, match="missing"):
        katz.katz_lambda_max(g)


def test_package_never_imports_the_oracle():
    pat = re.compile(r"^\s*(import\s+oracle\b|from\s+oracle\b)", re.M)
    files = list(_package_files((".py",)))
    assert files
    for path in files:
        with open(path) as fh:
            assert not pat.search(fh.read()), f"{path} imports the oracle"


def test_cuda_sources_do_not_refer_to_the_oracle():
    files = list(_package_files((".cu", ".cuh", ".h")))
    assert len(files) >= 10
    for path in files:
        with open(path) as fh:
            src = fh.read()
        assert "oracle/" not in src and "katz_oracle" not in src, path
