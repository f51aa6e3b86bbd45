"""The C-ABI library loads without a GPU and exports every function that
include/shtb.h declares; the Python binding knows each of them.  No compute
call is made here (there may be no GPU)."""
import ctypes
import os
import re

import pytest

import paper_1110_4874_gb300 as sh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(inc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(shtb_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["shtb_plan_create", "shtb_plan_destroy", "shtb_synthesize", "shtb_adjoint",
                     "shtb_plan_stats", "shtb_strerror"]:
        assert required in names
    assert len(names) >= 20


def test_library_loads_and_exports_every_declared_symbol():
    lib = ctypes.CDLL(sh.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) == set(sh.SIGNATURES)
    for name in sh.SIGNATURES:
        assert callable(getattr(sh, name, None)), f"binding lacks {name}"


def test_strerror_and_opts_without_gpu():
    assert sh.strerror(sh.SHTB_EINVAL) == "invalid argument"
    opts = sh.PlanOpts()
    assert sh.lib().shtb_plan_opts_init(ctypes.byref(opts)) == 0
    assert opts.leaf_cols == 32 and opts.device == -1
    assert sh.lib().shtb_plan_opts_init(None) == sh.SHTB_EINVAL


def test_plan_create_argument_errors_need_no_gpu():
    h = ctypes.c_void_p()
    assert sh.lib().shtb_plan_create(0, 8, 0.0, None, ctypes.byref(h)) == sh.SHTB_EINVAL
    assert sh.lib().shtb_plan_create(8, -1, 0.0, None, ctypes.byref(h)) == sh.SHTB_EINVAL
    assert sh.lib().shtb_plan_create(8, 8, float("nan"), None, ctypes.byref(h)) == sh.SHTB_EINVAL
    assert sh.lib().shtb_plan_create(8, 8, 0.0, None, None) == sh.SHTB_EINVAL
    assert sh.lib().shtb_plan_destroy(None) == 0


def test_binding_struct_layouts_match_the_library():
    """The ctypes mirrors of the public structs have the library's sizes (a
    short mirror would let the library write past it)."""
    got = sh.shtb_struct_sizes()
    assert got == {"opts": ctypes.sizeof(sh.PlanOpts), "stats": ctypes.sizeof(sh.PlanStats),
                   "request": ctypes.sizeof(sh.Request), "batch_opts": ctypes.sizeof(sh.BatchOpts)}
