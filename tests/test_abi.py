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


def _c_layout(text, name):
    """Field (name, offset, size) of `typedef struct name {...} name;` in the
    header, with natural alignment (every type here is 1, 4 or 8 bytes)."""
    import re
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), text, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    sizes = {"int32_t": 4, "uint32_t": 4, "int64_t": 8, "uint64_t": 8, "double": 8, "char": 1, "bc_graph": 8}
    out, off = [], 0
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        m = re.match(r"(?:const\s+)?(\w+)\s+(.*)", decl)
        base, names = m.group(1), m.group(2)
        for item in names.split(","):
            item = item.strip()
            ptr = item.startswith("*")
            nm = re.match(r"\**\s*(\w+)", item).group(1)
            dims = [int(d) for d in re.findall(r"\[(\d+)\]", item)]
            el = 8 if (ptr or base == "void") else sizes[base]
            count = 1
            for d in dims:
                count *= d
            off = (off + el - 1) // el * el
            out.append((nm, off, el * count))
            off += el * count
    return out


@pytest.mark.parametrize("name", ["bc_options", "bc_query_stats", "bc_query", "bc_tuning", "bc_stats"])
def test_binding_structs_match_the_header_layout(name):
    """Every struct the binding mirrors has the header's fields, in order, at
    the same offsets and sizes."""
    import ctypes
    from paper_1608_04472_gb300 import capi
    text = open(os.path.join(ROOT, "include", "bc.h")).read()
    declared = _c_layout(text, name)
    cls = getattr(capi, name)
    bound = [(f, getattr(cls, f).offset, getattr(cls, f).size) for f, _ in cls._fields_]
    assert bound == declared
    assert ctypes.sizeof(cls) >= declared[-1][1] + declared[-1][2]
