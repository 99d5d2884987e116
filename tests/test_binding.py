"""The binding is marshalling only: it fails loudly without the CUDA library and never
reaches the oracle (CPU)."""
import ast
import os

import pytest

import paper_2312_07874_gb300 as E

PKG = os.path.dirname(os.path.abspath(E.__file__))


def test_missing_library_raises(monkeypatch):
    monkeypatch.setattr(E, "_lib", None)
    monkeypatch.setattr(E, "LIB_PATH", os.path.join(PKG, "no_such_libesd.so"))
    with pytest.raises(ImportError, match="not built"):
        E.lib()
    with pytest.raises(ImportError):
        E.esd_ref_info(3, 4)


def test_package_never_imports_the_oracle():
    """No module of the package imports oracle/ (or numpy-based method code from it)."""
    for name in os.listdir(PKG):
        if not name.endswith(".py"):
            continue
        tree = ast.parse(open(os.path.join(PKG, name)).read())
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                mods = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                mods = [node.module or ""]
            else:
                continue
            assert not any(m == "oracle" or m.startswith("oracle.") for m in mods), (name, mods)
