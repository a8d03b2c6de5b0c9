"""The C-ABI library loads on a CPU-only machine and exports every entry point that
include/bcpp.h declares (no compute calls: those need a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "bcpp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bcpp_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1406_4173_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    syms = declared_symbols()
    for s in ["bcpp_create", "bcpp_destroy", "bcpp_brandes", "bcpp_brandes_pp", "bcpp_brandes_batched",
              "bcpp_sssp", "bcpp_skeleton", "bcpp_csr_build", "bcpp_csr_validate", "bcpp_strerror"]:
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_exports(lib):
    from paper_1406_4173_gb300 import api
    assert set(api.EXPORTS) == set(declared_symbols())


def test_strerror_and_default_opts_without_gpu(lib):
    from paper_1406_4173_gb300 import api
    L = api.load_library()
    assert L.bcpp_strerror(0) == b"ok"
    assert b"2^64" in L.bcpp_strerror(5)
    o = api.c_opts()
    L.bcpp_default_opts(ctypes.byref(o))
    assert o.precision == 0 and o.halve_undirected == 1 and o.order_sources == 1


def test_struct_layouts_match_header(tmp_path):
    """ctypes mirrors of the C structs have the header's sizes and field offsets (gcc)."""
    import subprocess
    from paper_1406_4173_gb300 import api
    prog = tmp_path / "layout.c"
    checks = []
    for cname, pyt in [("bcpp_graph", api.c_graph), ("bcpp_opts", api.c_opts), ("bcpp_stats", api.c_stats)]:
        checks.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in pyt._fields_:
            checks.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    prog.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"bcpp.h\"\nint main(void){" +
                    "".join(checks) + "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    out = dict(line.split() for line in subprocess.check_output([str(exe)]).decode().splitlines())
    for cname, pyt in [("bcpp_graph", api.c_graph), ("bcpp_opts", api.c_opts), ("bcpp_stats", api.c_stats)]:
        assert int(out[cname]) == ctypes.sizeof(pyt), cname
        for f, _ in pyt._fields_:
            assert int(out[f"{cname}.{f}"]) == getattr(pyt, f).offset, (cname, f)


def test_product_path_has_no_oracle_import():
    pkg = os.path.join(ROOT, "paper_1406_4173_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "bc_oracle" not in text, f
