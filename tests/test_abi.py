"""The C ABI without a GPU: the library builds, loads, exports every function that
include/figaro.h declares, and rejects invalid databases and join trees on the host."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "figaro.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2204_00525_gb300 import binding, build_lib
    if not build_lib.is_current():
        build_lib.build()
    return binding.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(figaro_\w+)\s*\(", text, flags=re.M)))


def test_every_declared_function_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), f"{n} declared in figaro.h but not exported"


def test_error_strings(lib):
    assert lib.figaro_error_string(0) == b"FIGARO_OK"
    assert lib.figaro_error_string(2) == b"FIGARO_ERR_INVALID_TREE"
    assert lib.figaro_error_string(999) == b"FIGARO_ERR_UNKNOWN"


def _tree(binding, rels_np, parent, mem_host=True):
    """figaro_join_tree over numpy arrays (host pointers)."""
    keep = []
    n = len(rels_np)
    rels = (binding.figaro_relation * n)()
    for i, (attrs, keys, data) in enumerate(rels_np):
        a = (C.c_int32 * max(len(attrs), 1))(*attrs)
        cols = [np.ascontiguousarray(keys[:, k]) for k in range(len(attrs))]
        ptrs = (C.c_void_p * max(len(attrs), 1))(*[c.ctypes.data for c in cols])
        d = np.asfortranarray(data)
        keep += [a, ptrs, d] + cols
        rels[i] = binding.figaro_relation(data.shape[0], len(attrs), 0, a, ptrs, data.shape[1], 0,
                                          data.shape[0], d.ctypes.data if data.shape[1] else None)
    par = (C.c_int32 * n)(*parent)
    keep += [rels, par]
    return binding.figaro_join_tree(n, rels, par), keep


def _plan_status(binding, lib, rels_np, parent):
    tree, keep = _tree(binding, rels_np, parent)
    opt = binding.figaro_default_options()
    opt.mem = binding.FIGARO_MEM_HOST
    h = C.c_void_p()
    st = lib.figaro_plan(C.byref(tree), C.byref(opt), None, C.byref(h))
    assert not h.value
    return st, lib.figaro_last_error().decode()


def _rel(attrs, m=4, n=2, seed=0):
    rng = np.random.default_rng(seed)
    return (attrs, rng.integers(0, 3, size=(m, len(attrs))).astype(np.int64), rng.standard_normal((m, n)))


def test_host_validation(lib):
    from paper_2204_00525_gb300 import binding
    # two roots
    st, _ = _plan_status(binding, lib, [_rel([0]), _rel([0])], [-1, -1])
    assert st == 2
    # cycle (no root reachable for node 1 <-> 2)
    st, _ = _plan_status(binding, lib, [_rel([0]), _rel([0, 1]), _rel([1])], [-1, 2, 1])
    assert st == 2
    # attribute held by one relation only
    st, msg = _plan_status(binding, lib, [_rel([0, 5]), _rel([0])], [-1, 0])
    assert st == 2 and "one relation" in msg
    # not a join tree: attribute 1 in relations 1 and 2, but 2 hangs under 0 which lacks it
    st, msg = _plan_status(binding, lib, [_rel([0]), _rel([0, 1]), _rel([1, 0])], [-1, 0, 0])
    assert st == 2 and "not connected" in msg
    # bad sizes
    bad = ([0], np.zeros((0, 1), np.int64), np.zeros((0, 2)))
    st, _ = _plan_status(binding, lib, [bad, _rel([0])], [-1, 0])
    assert st == 1
    # no data columns at all
    st, _ = _plan_status(binding, lib, [_rel([0], n=0), _rel([0], n=0)], [-1, 0])
    assert st == 10


def test_null_arguments(lib):
    h = C.c_void_p()
    assert lib.figaro_plan(None, None, None, C.byref(h)) == 1
    assert lib.figaro_qr_r(None, None, 0) == 1
    assert lib.figaro_plan_destroy(None) == 0


def test_struct_layouts_match_header():
    from paper_2204_00525_gb300 import binding
    assert C.sizeof(binding.figaro_relation) == 56
    assert C.sizeof(binding.figaro_join_tree) == 24
    assert C.sizeof(binding.figaro_options) == 64
    assert C.sizeof(binding.figaro_plan_info) == 64


def test_option_values_are_checked_before_any_device_work(lib):
    """fuse_tails and autotune accept 0 or 1 only; the check comes before any CUDA call."""
    from paper_2204_00525_gb300 import binding
    for field, bad in (("fuse_tails", 2), ("autotune", -1), ("leaf", 7), ("precision", 5)):
        tree, keep = _tree(binding, [_rel([0]), _rel([0])], [-1, 0])
        opt = binding.figaro_default_options()
        opt.mem = binding.FIGARO_MEM_HOST
        setattr(opt, field, bad)
        h = C.c_void_p()
        assert lib.figaro_plan(C.byref(tree), C.byref(opt), None, C.byref(h)) == 1, field
        assert not h.value


def test_options_struct_matches_header_field_order():
    """The ctypes mirror of figaro_options lists the header's fields in the header's order."""
    import re
    from paper_2204_00525_gb300 import binding
    hdr = open(os.path.join(ROOT, "include", "figaro.h")).read()
    body = re.search(r"typedef struct figaro_options \{(.*?)\} figaro_options;", hdr, re.S).group(1)
    names = re.findall(r"int32_t\s+(\w+)(?:\[\d+\])?;", body)
    assert names == [f[0] for f in binding.figaro_options._fields_]
