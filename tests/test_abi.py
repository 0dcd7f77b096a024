"""Host-side checks of the C ABI: the library loads, exports every entry point that
include/prdf.h declares, and rejects bad arguments before touching a device."""
import ctypes
import os
import re

import pytest

import __graft_entry__

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def prdf():
    __graft_entry__.build()
    from paper_2401_03256_gb300 import prdf as mod

    mod.load()
    return mod


def _declared():
    with open(os.path.join(ROOT, "include", "prdf.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w ]+?\**\s*\b(pr_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("pr_graph_create", "pr_apply_batch", "pr_static", "pr_naive_dynamic",
                     "pr_dynamic_frontier", "pr_get_ranks"):
        assert required in names


def test_library_exports_every_declared_symbol(prdf):
    lib = ctypes.CDLL(prdf.LIB_PATH)
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) == set(prdf.EXPORTED)


def test_params_default_are_the_papers(prdf):
    p = prdf.pr_params_default()
    assert p.alpha == 0.85 and p.tol == 1e-10 and p.max_iter == 500
    assert p.frontier_tol == p.tol / 1e5
    assert p.precision == prdf.PR_F64 and p.dead_end == prdf.PR_DEADEND_SELFLOOP


def test_struct_layouts(prdf):
    assert ctypes.sizeof(prdf.pr_params) == 3 * 8 + 6 * 4
    assert ctypes.sizeof(prdf.pr_stats) == 4 + 4 + 3 * 8 + 4 * 8


def test_bad_arguments_are_rejected_on_the_host(prdf):
    with pytest.raises(prdf.PrdfError) as e:
        prdf.pr_graph_create(0, [], [])
    assert e.value.status == prdf.PR_ERR_INVALID_ARG
    p = prdf.pr_params_default()
    p.alpha = 1.5
    with pytest.raises(prdf.PrdfError) as e:
        prdf.pr_graph_create(4, [0], [1], p)
    assert e.value.status == prdf.PR_ERR_INVALID_ARG
    p = prdf.pr_params_default()
    p.max_iter = 5000
    with pytest.raises(prdf.PrdfError) as e:
        prdf.pr_graph_create(4, [0], [1], p)
    assert e.value.status == prdf.PR_ERR_INVALID_ARG
    lib = prdf.load()
    assert lib.pr_apply_batch(None, 0, None, None, 0, None, None) == prdf.PR_ERR_INVALID_ARG
    assert lib.pr_static(None, None) == prdf.PR_ERR_INVALID_ARG
    assert lib.pr_status_string(prdf.PR_ERR_VERTEX_RANGE) == b"PR_ERR_VERTEX_RANGE"
