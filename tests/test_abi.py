"""The C-ABI library builds for sm_103a and exports every entry point that
include/mdnewton.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mdnewton.h")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mdn_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("mdn_create", "mdn_workspace_bytes", "mdn_load_system", "mdn_set_series", "mdn_newton",
              "mdn_get_series", "mdn_get_residual", "mdn_last_error", "mdn_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2301_12659_gb300 import build
    path = build.build()
    try:
        lib = ctypes.CDLL(path)
    except OSError as e:  # the CUDA runtime must be resolvable; it ships with the toolkit
        pytest.fail(f"cannot load {path}: {e}")
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_the_header():
    from paper_2301_12659_gb300 import mdnewton
    assert sorted(mdnewton.EXPORTS) == declared()
    for n in declared():
        assert callable(getattr(mdnewton, n))


def test_product_path_never_imports_the_oracle():
    """The oracle is test infrastructure: no product module imports or links it."""
    import ast
    pkg = os.path.join(ROOT, "paper_2301_12659_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            path = os.path.join(dirpath, f)
            if f.endswith(".py"):
                for node in ast.walk(ast.parse(open(path).read())):
                    if isinstance(node, ast.Import):
                        assert not any(a.name.split(".")[0] == "oracle" for a in node.names), path
                    if isinstance(node, ast.ImportFrom):
                        assert (node.module or "").split(".")[0] != "oracle", path
            elif f.endswith((".cu", ".cuh", ".h", ".cpp")):
                assert "mdoracle" not in open(path).read(), path


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """Without the built library the binding raises: there is no fallback."""
    from paper_2301_12659_gb300 import mdnewton
    monkeypatch.setattr(mdnewton, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        mdnewton.load(str(tmp_path / "libmdnewton-missing.so"))
