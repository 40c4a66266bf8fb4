"""The product path and the oracle stay apart, and the product has no fallback.

- the package never imports the oracle, and the CUDA sources never include it;
- the oracle never imports the package nor includes the CUDA sources;
- loading the library fails loudly when it has not been built;
- without a GPU, a render problem cannot be set up at all (no host computation)."""
import ast
import os
import re
import sys

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2502_01826_gb300")
ORACLE = os.path.join(ROOT, "oracle")
sys.path.insert(0, ROOT)


def _py_imports(path):
    tree = ast.parse(open(path).read(), path)
    mods = []
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods += [a.name for a in node.names]
        elif isinstance(node, ast.ImportFrom):
            mods.append(node.module or "")
            mods += [a.name for a in node.names]
    return mods


def _files(top, exts):
    for d, _, names in os.walk(top):
        for n in names:
            if n.endswith(exts):
                yield os.path.join(d, n)


def test_package_never_imports_or_includes_the_oracle():
    for f in _files(PKG, (".py",)):
        assert not any(m == "oracle" or m.startswith("oracle.") for m in _py_imports(f)), f
    for f in _files(PKG, (".cu", ".cuh", ".h")):
        for inc in re.findall(r'#include\s+[<"]([^>"]+)[>"]', open(f).read()):
            assert "oracle" not in inc, (f, inc)


def test_oracle_never_imports_or_includes_the_package():
    for f in _files(ORACLE, (".py",)):
        assert not any("paper_2502_01826_gb300" in m for m in _py_imports(f)), f
    for f in _files(ORACLE, (".c", ".h", ".inc")):
        for inc in re.findall(r'#include\s+[<"]([^>"]+)[>"]', open(f).read()):
            assert "csrc" not in inc and "gsrf_internal" not in inc and "gsrf.h" != os.path.basename(inc), (f, inc)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_2502_01826_gb300 import _build, _lib
    monkeypatch.setattr(_build, "SO", str(tmp_path / "absent" / "libgsrf.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load()


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without a GPU")
def test_no_gpu_means_no_render():
    from paper_2502_01826_gb300 import _build
    from paper_2502_01826_gb300.render import Renderer, make_grid
    if not os.path.exists(_build.SO):
        pytest.skip("library not built here")
    with pytest.raises(Exception):
        Renderer(16, 1, make_grid(36, 9), 2.4e9)
