"""The product path has no CPU fallback: without the built CUDA library the binding raises at the
first call instead of computing anything, and no module of the package imports the oracle."""
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
