"""Host-side checks that need no GPU: the C-ABI library builds for sm_103a,
loads, and exports every entry point its header declares; host logic of the
binding; the product package does not reach into the oracle."""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _built_lib():
    from paper_2511_10073_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol():
    so = _built_lib()
    import ctypes
    lib = ctypes.CDLL(so)
    hdr = open(os.path.join(ROOT, "include", "pl.h")).read()
    names = sorted(set(re.findall(r"\b(pl_[a-z_0-9]+)\s*\(", hdr)))
    assert "pl_build_graph" in names and "pl_filter_init" in names and "pl_hpwl" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/pl.h but not exported"


def test_defaults_match_the_oracle_readings():
    _built_lib()
    import oracle
    import paper_2511_10073_gb300 as pl
    d = pl.params().as_dict()
    for k, v in oracle.DEFAULTS.items():
        got = d[k]
        if isinstance(v, tuple):
            assert tuple(got)[:len(v)] == tuple(type(got[0])(x) for x in v), k
        else:
            assert got == v, k


def test_params_override():
    _built_lib()
    import paper_2511_10073_gb300 as pl
    p = pl.params(nbx=12, tap_k=(2, 4, 8, 0), gamma=0.25)
    assert p.nbx == 12 and tuple(p.tap_k) == (2, 4, 8, 0) and p.gamma == 0.25
    assert p.nby == 32


def test_hpwl_workspace_size_host_only():
    _built_lib()
    import paper_2511_10073_gb300 as pl
    assert pl.pl_hpwl_workspace_size(0) >= 256
    assert pl.pl_hpwl_workspace_size(10_000_000) > pl.pl_hpwl_workspace_size(100)


def test_product_code_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2511_10073_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if not f.endswith(".py"):
                continue
            tree = ast.parse(open(os.path.join(dirpath, f)).read())
            for node in ast.walk(tree):
                if isinstance(node, ast.Import):
                    assert not any(a.name.split(".")[0] == "oracle" for a in node.names), f
                if isinstance(node, ast.ImportFrom):
                    assert (node.module or "").split(".")[0] != "oracle", f
    for dirpath, _, files in os.walk(os.path.join(pkg, "csrc")):
        for f in files:
            src = open(os.path.join(dirpath, f)).read()
            assert "orc_" not in src and "oracle" not in src.lower(), f


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_2511_10073_gb300 as pl
    monkeypatch.setattr(pl, "_lib", None)
    monkeypatch.setattr(pl, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="missing"):
        pl.lib()
