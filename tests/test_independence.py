"""Structure checks (no GPU): the CUDA path and the oracle share no code and neither imports
the other; the product path has no CPU fallback and fails loudly without its library."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _sources(sub, exts):
    out = []
    for d, _, files in os.walk(os.path.join(ROOT, sub)):
        if "_build" in d or "__pycache__" in d:
            continue
        out += [os.path.join(d, f) for f in files if f.endswith(exts)]
    return out


def test_product_does_not_import_the_oracle():
    srcs = _sources("paper_2308_15407_gb300", (".py", ".cu", ".cpp", ".h")) + _sources("include", (".h",))
    assert srcs
    for path in srcs:
        text = open(path).read()
        assert not re.search(r"^\s*(from|import)\s+oracle\b", text, re.M), path
        assert "oracle/" not in text and "importlib" not in text, path


def test_oracle_does_not_import_the_product():
    srcs = _sources("oracle", (".py", ".c", ".h"))
    assert srcs
    for path in srcs:
        text = open(path).read()
        assert "paper_2308_15407_gb300" not in text and "libfdlb" not in text, path


def test_missing_library_raises(monkeypatch):
    from paper_2308_15407_gb300 import fdlb
    monkeypatch.setattr(fdlb, "_lib", None)
    monkeypatch.setattr(fdlb, "LIB_PATH", os.path.join(ROOT, "no_such_dir", "libfdlb.so"))
    with pytest.raises(RuntimeError, match="missing"):
        fdlb.load()
    with pytest.raises(RuntimeError):
        fdlb.workspace_bytes([fdlb.Params(nx=16, qx_half=4, qy=0, qz=0, kn=0.1, eta0=0.1)])
