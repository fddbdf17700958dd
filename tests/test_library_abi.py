"""The C-ABI library loads and exports every symbol include/hpse.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hpse.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hpse_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1110_2316_gb300.build import build
    path = build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hpse_setup_mesh", "hpse_set_data", "hpse_apply_operator",
                     "hpse_apply_preconditioner", "hpse_pcg_solve", "hpse_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_python_binding_declares_every_symbol():
    from paper_1110_2316_gb300 import _lib
    assert set(declared_functions()) == set(_lib.SIGNATURES)


def test_host_only_calls(lib):
    from paper_1110_2316_gb300 import _lib
    L = _lib.load()
    assert L.hpse_status_string(0) == b"ok"
    assert L.hpse_status_string(2) == b"non-matching face"
    # invalid arguments are rejected on the host before touching a device
    assert L.hpse_setup_mesh(None, 0, None) == 1
    assert L.hpse_ndof(None) == -1
    assert L.hpse_set_block_threads(None, 0, 0, 4, 128) == 1
