"""The C-ABI library builds, loads and exports every symbol include/qg.h declares.

No compute call is made here (no GPU needed); GPU behaviour is covered by the
``gpu``-marked parity tests.
"""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "qg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char)\s*\*?\s*(qg_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2508_06678_gb300._lib import LIB_PATH, load
    if not os.path.exists(LIB_PATH):
        from paper_2508_06678_gb300.build import build
        build()
    return load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("qg_create", "qg_set_state", "qg_get_state", "qg_step", "qg_sync", "qg_diagnostics",
                     "qg_destroy", "qg_sgs_apriori", "qg_last_error", "qg_version"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_declares_every_symbol():
    from paper_2508_06678_gb300._lib import SIGNATURES
    assert sorted(SIGNATURES) == declared_functions()


def test_struct_layouts_match_header(lib):
    import ctypes as C
    from paper_2508_06678_gb300._lib import qg_closure, qg_diag, qg_grid, qg_params
    assert C.sizeof(qg_grid) == 16
    assert C.sizeof(qg_closure) == 24
    assert C.sizeof(qg_params) == 48
    assert C.sizeof(qg_diag) == 56


def test_version_and_error_string(lib):
    assert lib.qg_version().decode().startswith("libqg")
    assert isinstance(lib.qg_last_error(), bytes)


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2508_06678_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f


def test_member_struct_layout(lib):
    import ctypes as C
    from paper_2508_06678_gb300._lib import qg_member
    assert C.sizeof(qg_member) == 120
