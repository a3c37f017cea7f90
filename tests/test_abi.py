"""CPU-side checks of the C-ABI boundary: the library builds, loads, and exports
every entry point that include/bc.h declares; the binding covers them all; the
product package never reaches the oracle."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bc_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1608_04472_gb300 import build
    return build.build()


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for required in ["bc_create", "bc_destroy", "bc_graph_load_csr", "bc_exact", "bc_adaptive_sources",
                     "bc_adaptive_pairs", "bc_uniform_sources", "bc_source_dependencies"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol(lib_path):
    from paper_1608_04472_gb300 import capi as mod
    assert sorted(mod.EXPORTED) == declared_functions()


def test_binding_constants_match_header():
    from paper_1608_04472_gb300 import capi as mod
    text = open(HEADER).read()
    defs = dict(re.findall(r"#define\s+(BC_[A-Z_]+)\s+(-?\d+)u?\b", text))
    names = ["BC_UNDIRECTED", "BC_VALIDATE", "BC_DIRECTED", "BC_NORMALIZE", "BC_STOPPED", "BC_CAPPED"]
    for name in names:
        assert name in defs, name
        assert getattr(mod, name) == int(defs[name]), name


def test_null_context_is_rejected(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.bc_set_batch_width.restype = ctypes.c_int32
    lib.bc_set_batch_width.argtypes = [ctypes.c_void_p, ctypes.c_int32]
    assert lib.bc_set_batch_width(None, 64) == -1
    lib.bc_last_error.restype = ctypes.c_char_p
    lib.bc_last_error.argtypes = [ctypes.c_void_p]
    assert lib.bc_last_error(None) == b"NULL context"


def test_product_package_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1608_04472_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "bc_oracle" not in src, f


def test_missing_library_fails_loudly(tmp_path):
    import subprocess
    import sys
    # copy the package without the .so and import it: must raise ImportError
    import shutil
    dst = tmp_path / "paper_1608_04472_gb300"
    shutil.copytree(os.path.join(ROOT, "paper_1608_04472_gb300"), dst,
                    ignore=shutil.ignore_patterns("*.so", "_build", "__pycache__"))
    code = "import paper_1608_04472_gb300 as p\ntry:\n    p.Context\nexcept ImportError:\n    print('LOUD')\n"
    r = subprocess.run([sys.executable, "-c", code], cwd=tmp_path, capture_output=True, text=True)
    assert "LOUD" in r.stdout, r.stdout + r.stderr
