"""The oracle and the CUDA path share no code: the package never imports the oracle, the
oracle never imports the package, and the CUDA sources include nothing from the oracle.
The product path has no CPU fallback: without the built library the binding raises."""
import ast
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1911_10487_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _imports(path):
    tree = ast.parse(open(path).read(), path)
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name.split(".")[0]
        elif isinstance(node, ast.ImportFrom):
            if node.level == 0 and node.module:
                yield node.module.split(".")[0]


def _py_files(d):
    for base, _, files in os.walk(d):
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(base, f)


def test_package_does_not_import_the_oracle():
    for f in _py_files(PKG):
        assert "oracle" not in set(_imports(f)), f


def test_oracle_does_not_import_the_package():
    for f in _py_files(ORACLE):
        assert "paper_1911_10487_gb300" not in set(_imports(f)), f


def test_cuda_sources_include_nothing_from_the_oracle():
    csrc = os.path.join(PKG, "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f)).read()
        assert "oracle" not in text.lower(), f


def test_missing_library_raises_instead_of_falling_back(monkeypatch):
    import paper_1911_10487_gb300._abi as abi
    monkeypatch.setattr(abi, "_lib", None)
    monkeypatch.setattr(abi, "_LIB_PATH", os.path.join(ROOT, "no_such_dir", "libflatlayer.so"))
    with pytest.raises(ImportError):
        abi.lib()
