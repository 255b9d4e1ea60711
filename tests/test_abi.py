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


def test_option_struct_layout_and_host_checks(lib):
    """The binding's option struct lines up with the library's: the defaults the C code writes
    land in the fields of the same names (a shifted or missing field would misplace them), and
    out-of-range values of the Phase-1 form, the forward-sweep form and the SM-pair form are
    refused on the host before any device work."""
    import numpy as np
    import paper_1812_02091_gb300 as emd
    o = emd.emd_db_options_default()
    assert (o.device, o.rerank_margin, o.max_query_h, o.max_table_k, o.max_batch) == (0, 8, 2048, 64, 64)
    assert (o.prune_topk, o.lanes, o.batched, o.batch_columns, o.graphs, o.autotune) == (1, 1, 1, 16384, 1, 1)
    assert (o.fused_phase1, o.fwd_kernel, o.tc_pair) == (1, 0, 0)
    emb = np.eye(4, 2, dtype=np.float32)
    rp, col, val = np.array([0, 1], np.int64), np.array([0], np.int32), np.array([1.0], np.float32)
    for bad, text in ((dict(fused_phase1=3), "fused_phase1"), (dict(fwd_kernel=5), "fwd_kernel"),
                      (dict(tc_pair=3), "tc_pair"), (dict(tc_pair=-1), "tc_pair")):
        with pytest.raises(emd.EmdError) as err:
            emd.emd_db_create(emb, None, rp, col, val, emd.emd_db_options_default(**bad), v=4)
        assert text in str(err.value), err.value
