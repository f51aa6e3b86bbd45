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


def test_host_side_rejections_need_no_gpu():
    """Argument checks that fail before any device work: a spin other than 0
    or 2, host tensors handed to device calls, wrong dtypes and layouts, and
    NULL plans or files."""
    import torch
    opts = sh.shtb_plan_opts_init()
    assert opts.spin == 0 and opts.gpu_build == 0
    opts.spin = 1
    h = ctypes.c_void_p()
    assert sh.lib().shtb_plan_create(8, 16, 1e-10, ctypes.byref(opts), ctypes.byref(h)) == sh.SHTB_EINVAL
    cpu = torch.zeros((1, 10), dtype=torch.complex128)
    with pytest.raises(ValueError, match="CUDA"):
        sh.shtb_synthesize(None, cpu, torch.zeros((1, 12), dtype=torch.float64), 1)
    if torch.cuda.is_available():
        pytest.skip("the dtype and layout checks below are exercised by the GPU suite")
    for name in ("shtb_synthesize", "shtb_adjoint", "shtb_analyze", "shtb_synthesize_spin",
                 "shtb_adjoint_spin", "shtb_analyze_spin"):
        fn = getattr(sh.lib(), name)
        args = [None, None, None, 1] + ([None, 0] if "analyze" in name else []) + [None]
        assert fn(*args) == sh.SHTB_EINVAL, name
    assert sh.lib().shtb_plan_save(None, b"x") == sh.SHTB_EINVAL
    assert sh.lib().shtb_plan_load(None, None, ctypes.byref(h)) == sh.SHTB_EINVAL
    assert sh.lib().shtb_plan_load(b"/nonexistent/plan.bin", None, ctypes.byref(h)) == sh.SHTB_EIO
