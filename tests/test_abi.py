"""The C-ABI library loads and exports every function include/stag.h declares.

No compute call is made here (CPU-only test); argument checks that return
before any CUDA call are exercised.
"""
import ctypes
import os
import re

import pytest

from paper_1511_00088_gb300 import build as B
from paper_1511_00088_gb300 import stag

HEADER = os.path.join(B.INCLUDE, "stag.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(stag_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return stag.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["stag_create", "stag_destroy", "stag_links_upload", "stag_dslash_oe",
              "stag_dslash_eo", "stag_mdagm", "stag_cg_solve"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(B.LIB)
    missing = [n for n in declared_functions() if not hasattr(raw, n)]
    assert not missing, missing


def test_static_queries(lib):
    assert stag.stag_abi_version() == 1
    assert stag.stag_status_string(0) == "STAG_OK"
    assert stag.stag_status_string(-5) == "STAG_ERR_BREAKDOWN"


@pytest.mark.parametrize("dims", [(3, 4, 4, 4), (4, 4, 4, 0), (4, 4, 1, 4), (4, 6, 4, -2)])
def test_create_rejects_bad_dims_before_touching_cuda(lib, dims):
    st, h = stag.stag_create(dims, 1, None)
    assert st == stag.STAG_ERR_ARG and not h.value


def test_create_rejects_unknown_flags(lib):
    st, h = stag.stag_create((4, 4, 4, 4), 1 << 7, None)
    assert st == stag.STAG_ERR_ARG


@pytest.mark.parametrize("lang,std", [("c", "-std=c99"), ("c++", "-std=c++11")])
def test_header_is_plain_c_and_cxx(lang, std):
    """include/stag.h compiles on its own as C99 and as C++11 (no CUDA or
    torch types in the boundary)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    r = subprocess.run([cc, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-x", lang, HEADER],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
