"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every function
that include/emd.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_1812_02091_gb300 import _build

HEADER_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def declared_functions():
    names = set()
    for h in sorted(os.listdir(HEADER_DIR)):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(HEADER_DIR, h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[a-zA-Z_][\w\s\*]*?\b(emd_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("emd_db_create", "emd_db_destroy", "emd_query_batch", "emd_topk", "emd_last_error"):
        assert must in names


@pytest.mark.parametrize("name", declared_functions())
def test_symbol_exported(lib, name):
    assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_version_string(lib):
    lib.emd_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.emd_version()


def test_binding_names_match_header():
    import paper_1812_02091_gb300 as emd
    exported = set(emd.__all__)
    for name in declared_functions():
        assert name in exported, f"{name} has no Python binding"


def test_invalid_arguments_rejected_before_any_device_work(lib):
    """Argument checks run on the host: a missing embedding/cost pair is refused without
    touching a GPU."""
    import paper_1812_02091_gb300 as emd
    emd.load()
    out = ctypes.c_void_p()
    st = emd.load().emd_db_create(None, 10, 4, None, None, None, None, 1, None, ctypes.byref(out))
    assert st == 1
    assert "exactly one of emb and cost_matrix" in emd.emd_last_error()
