"""The product path has no CPU fallback: without the built CUDA library the binding raises at the
first call instead of computing anything, no module of the package imports the oracle, and the
oracle and the CUDA sources share no code."""
import ast
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2309_15676_gb300")


def test_missing_library_raises(monkeypatch, tmp_path):
    from paper_2309_15676_gb300 import _lib, api
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libmer.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(ImportError, match="CUDA library not built"):
        _lib.load()
    with pytest.raises(ImportError):
        api.Context(0)
    from paper_2309_15676_gb300 import synth
    with pytest.raises(ImportError):
        api.Volume(synth.volume_scene(n=4, views=1, width=4, height=4))


def test_package_does_not_import_the_oracle():
    offenders = []
    for name in sorted(os.listdir(PKG)):
        if not name.endswith(".py"):
            continue
        tree = ast.parse(open(os.path.join(PKG, name)).read())
        for node in ast.walk(tree):
            mods = []
            if isinstance(node, ast.Import):
                mods = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                mods = [node.module or ""]
            offenders += [(name, m) for m in mods if m.split(".")[0] == "oracle"]
    assert not offenders, offenders


def test_oracle_and_cuda_path_share_no_source():
    """The oracle's C includes only the C standard library, nothing in the CUDA sources mentions
    the oracle, and the oracle's Python imports nothing from the product package."""
    import re
    ORC = os.path.join(ROOT, "oracle")
    inc = re.findall(r'#include\s*[<"]([^>"]+)[>"]', open(os.path.join(ORC, "oracle.c")).read())
    assert set(inc) <= {"math.h", "stdint.h", "stdlib.h", "string.h", "stdio.h"}, inc
    csrc = os.path.join(PKG, "csrc")
    for name in os.listdir(csrc):
        assert "oracle" not in open(os.path.join(csrc, name), errors="replace").read().lower(), name
    for name in sorted(os.listdir(ORC)):
        if name.endswith(".py"):
            tree = ast.parse(open(os.path.join(ORC, name)).read())
            for node in ast.walk(tree):
                if isinstance(node, ast.ImportFrom) and node.module:
                    assert not node.module.startswith("paper_2309_15676_gb300"), (name, node.module)
                if isinstance(node, ast.Import):
                    assert not any(a.name.startswith("paper_2309_15676_gb300") for a in node.names), name
