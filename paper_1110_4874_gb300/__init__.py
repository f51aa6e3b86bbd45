"""GB300 (sm_103a) scalar spherical-harmonic synthesis on the HEALPix grid by
butterfly-compressed Legendre transforms (after Seljebotn, "Wavemoth",
arXiv 1110.4874).

This module is a thin ctypes binding of the C ABI in ``include/shtb.h``: the
functions named ``shtb_*`` marshal arguments (torch tensors -> device
pointers, the current CUDA stream) and call the library of the same name; all
arithmetic runs in the library's CUDA kernels.  There is no CPU fallback: if
the compiled library is missing, importing the binding's entry points raises.

Layouts (see include/shtb.h): a_lm complex128 [nmaps, (L+1)(L+2)/2], m-major
(index m(2L+1-m)/2 + l); maps float64 [nmaps, 12 nside^2] in RING order.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import synthetic  # noqa: F401  (seeded inputs; no transform arithmetic)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libshtb.so")

SHTB_OK = 0
SHTB_EINVAL = -1
SHTB_ENOMEM = -2
SHTB_ECUDA = -3
SHTB_EMISMATCH = -4
SHTB_ETIMEOUT = -5
SHTB_ENOTSUP = -6
SHTB_EIO = -7
SHTB_ECORRUPT = -8


class ShtbError(RuntimeError):
    """A non-zero return code of the C ABI."""

    def __init__(self, code: int, where: str, detail: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code}): {detail}")


class PlanOpts(ctypes.Structure):
    _fields_ = [("leaf_cols", ctypes.c_int), ("max_depth", ctypes.c_int),
                ("rho", ctypes.c_double), ("nthreads", ctypes.c_int), ("device", ctypes.c_int),
                ("cache_dir", ctypes.c_char_p), ("gpu_build", ctypes.c_int), ("spin", ctypes.c_int),
                ("residual_recurrence", ctypes.c_int)]


class PlanStats(ctypes.Structure):
    _fields_ = [("nside", ctypes.c_int), ("lmax", ctypes.c_int), ("eps", ctypes.c_double),
                ("nrings", ctypes.c_int), ("npix", ctypes.c_longlong), ("nalm", ctypes.c_longlong),
                ("compressed", ctypes.c_int), ("n_recurrence", ctypes.c_longlong),
                ("n_recurrence_exec", ctypes.c_longlong), ("n_dense", ctypes.c_longlong),
                ("n_rstored", ctypes.c_longlong), ("plan_device_bytes", ctypes.c_longlong),
                ("plan_read_bytes", ctypes.c_longlong), ("legendre_flops_per_map", ctypes.c_double),
                ("recurrence_flops", ctypes.c_double), ("phi_flops_per_map", ctypes.c_double),
                ("build_seconds", ctypes.c_double), ("kernel_launches", ctypes.c_longlong),
                ("n_ident", ctypes.c_longlong), ("depth_hist", ctypes.c_int * 16),
                ("from_cache", ctypes.c_int), ("spin", ctypes.c_int), ("n_rgen", ctypes.c_longlong)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "depth_hist"}
        d["depth_hist"] = list(self.depth_hist)
        return d


class Request(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("alm_dev", ctypes.c_void_p), ("map_dev", ctypes.c_void_p),
                ("nmaps", ctypes.c_int), ("dir", ctypes.c_int)]


class BatchOpts(ctypes.Structure):
    _fields_ = [("autotune", ctypes.c_int), ("warps_per_block", ctypes.c_int),
                ("group_width", ctypes.c_int), ("lpt", ctypes.c_int),
                ("spin_limit", ctypes.c_longlong), ("schedule", ctypes.c_int),
                ("streams", ctypes.c_int)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_DP = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); every symbol declared in include/shtb.h
SIGNATURES = {
    "shtb_plan_opts_init": (_I, [ctypes.POINTER(PlanOpts)]),
    "shtb_plan_create": (_I, [_I, _I, _D, ctypes.POINTER(PlanOpts), ctypes.POINTER(_P)]),
    "shtb_plan_destroy": (_I, [_P]),
    "shtb_plan_save": (_I, [_P, ctypes.c_char_p]),
    "shtb_plan_load": (_I, [ctypes.c_char_p, ctypes.POINTER(PlanOpts), ctypes.POINTER(_P)]),
    "shtb_plan_stats": (_I, [_P, ctypes.POINTER(PlanStats)]),
    "shtb_plan_reserve": (_I, [_P, _I]),
    "shtb_synthesize": (_I, [_P, _P, _P, _I, _P]),
    "shtb_adjoint": (_I, [_P, _P, _P, _I, _P]),
    "shtb_analyze": (_I, [_P, _P, _P, _I, _P, _I, _P]),
    "shtb_synthesize_spin": (_I, [_P, _P, _P, _I, _P]),
    "shtb_adjoint_spin": (_I, [_P, _P, _P, _I, _P]),
    "shtb_analyze_spin": (_I, [_P, _P, _P, _I, _P, _I, _P]),
    "shtb_synthesize_host": (_I, [_P, _P, _P, _I, _P]),
    "shtb_adjoint_host": (_I, [_P, _P, _P, _I, _P]),
    "shtb_strerror": (ctypes.c_char_p, [_I]),
    "shtb_last_error_message": (ctypes.c_char_p, []),
    "shtb_profile_enable": (_I, [_P, _I]),
    "shtb_profile_read": (_I, [_P, _DP, _I, ctypes.POINTER(_I)]),
    "shtb_measure_fp64_peak": (_I, [_I, _DP, _DP]),
    "shtb_test_legendre": (_I, [_P, _P, _P, _I, _P]),
    "shtb_test_butterfly": (_I, [_P, _P, _P, _I, _P]),
    "shtb_test_phi": (_I, [_P, _P, _P, _I, _P]),
    "shtb_test_phi_adjoint": (_I, [_P, _P, _P, _I, _P]),
    "shtb_test_legendre_adjoint": (_I, [_P, _P, _P, _I, _P]),
    "shtb_test_host_recurrence": (_I, [_I, _I, _I, _I, _DP]),
    "shtb_synthesize_noalloc": (_I, [_P, _P, _P, _I, _P]),
    "shtb_batch_opts_init": (_I, [ctypes.POINTER(BatchOpts)]),
    "shtb_batch_create": (_I, [ctypes.POINTER(Request), _I, ctypes.POINTER(BatchOpts),
                               ctypes.POINTER(_P)]),
    "shtb_batch_run": (_I, [_P, _P]),
    "shtb_batch_status": (_I, [_P, _P]),
    "shtb_batch_info": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), _DP]),
    "shtb_batch_destroy": (_I, [_P]),
    "shtb_batch_schedule": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "shtb_test_batch_stall": (_I, [_P, _I]),
    "shtb_test_host_id": (_I, [_I, _I, _DP, _D, ctypes.POINTER(_I), ctypes.POINTER(_I), _DP]),
    "shtb_test_gpu_id": (_I, [_I, _I, _DP, _D, ctypes.POINTER(_I), ctypes.POINTER(_I), _DP]),
    "shtb_test_host_butterfly": (_I, [_I, _I, _D, _I, _I, _I, _DP, _DP, _DP,
                                      ctypes.POINTER(ctypes.c_longlong)]),
    "shtb_test_host_spin_column": (_I, [_I, _I, _I, _I, _I, _DP]),
    "shtb_test_host_interp": (_I, [_I, _I, _D, _I, _I, _I, _DP, _DP, _DP,
                                   ctypes.POINTER(ctypes.c_longlong)]),
    "shtb_test_host_rec_blocks": (_I, [_I, _I, _D, _I, _I, _I, _DP, ctypes.POINTER(ctypes.c_longlong)]),
    "shtb_struct_sizes": (_I, [ctypes.POINTER(_I)] * 4),
}

_lib = None
_lock = threading.Lock()


def lib():
    """The loaded C library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"CUDA library {LIB_PATH} is missing; build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'` "
                    "(there is no CPU fallback)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def strerror(code: int) -> str:
    try:
        return lib().shtb_strerror(code).decode()
    except Exception:
        return "error"


def _check(rc: int, where: str):
    if rc != SHTB_OK:
        raise ShtbError(rc, where, lib().shtb_last_error_message().decode())


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream))


def _dptr(t, dtype, name):
    import torch
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------- C-ABI names
def shtb_plan_opts_init() -> PlanOpts:
    opts = PlanOpts()
    _check(lib().shtb_plan_opts_init(ctypes.byref(opts)), "shtb_plan_opts_init")
    return opts


def shtb_strerror(code: int) -> str:
    return strerror(code)


def shtb_last_error_message() -> str:
    return lib().shtb_last_error_message().decode()


def shtb_plan_create(nside: int, lmax: int, eps: float = 0.0, leaf_cols: int = 32,
                     max_depth: int = -1, rho: float = 0.0, nthreads: int = 0,
                     device: int = -1, cache_dir: str | None = None,
                     spin: int = 0, gpu_build: bool = False,
                     residual_recurrence: bool = False) -> ctypes.c_void_p:
    opts = shtb_plan_opts_init()
    opts.spin = spin
    opts.residual_recurrence = 1 if residual_recurrence else 0
    opts.gpu_build = 1 if gpu_build else 0
    opts.leaf_cols, opts.max_depth, opts.rho = leaf_cols, max_depth, rho
    opts.nthreads, opts.device = nthreads, device
    opts.cache_dir = os.fsencode(cache_dir) if cache_dir is not None else None
    h = ctypes.c_void_p()
    _check(lib().shtb_plan_create(nside, lmax, float(eps), ctypes.byref(opts), ctypes.byref(h)),
           "shtb_plan_create")
    return h


def shtb_plan_destroy(plan) -> None:
    _check(lib().shtb_plan_destroy(plan), "shtb_plan_destroy")


def shtb_plan_save(plan, path: str) -> None:
    _check(lib().shtb_plan_save(plan, os.fsencode(path)), "shtb_plan_save")


def shtb_plan_load(path: str, device: int = -1) -> ctypes.c_void_p:
    opts = shtb_plan_opts_init()
    opts.device = device
    h = ctypes.c_void_p()
    _check(lib().shtb_plan_load(os.fsencode(path), ctypes.byref(opts), ctypes.byref(h)), "shtb_plan_load")
    return h


def shtb_plan_stats(plan) -> dict:
    st = PlanStats()
    _check(lib().shtb_plan_stats(plan, ctypes.byref(st)), "shtb_plan_stats")
    return st.as_dict()


def shtb_plan_reserve(plan, nmaps: int) -> None:
    _check(lib().shtb_plan_reserve(plan, nmaps), "shtb_plan_reserve")


# Per call: the layouts of its input and output (see include/shtb.h) and the
# fields per transform unit (a polarised pair carries two of each).
_LAYOUTS = {
    "shtb_synthesize": ("alm", "map", 1),
    "shtb_synthesize_noalloc": ("alm", "map", 1),
    "shtb_adjoint": ("map", "alm", 1),
    "shtb_synthesize_spin": ("alm", "map", 2),
    "shtb_adjoint_spin": ("map", "alm", 2),
    "shtb_test_legendre": ("alm", "q", 1),
    "shtb_test_butterfly": ("alm", "qt", 1),
    "shtb_test_phi": ("q", "map", 1),
    "shtb_test_phi_adjoint": ("map", "q", 1),
    "shtb_test_legendre_adjoint": ("q", "alm", 1),
}


def _layout_elems(st, layout):
    """Elements (complex or real, as the layout's dtype) of one field."""
    L = st["lmax"]
    return {"alm": st["nalm"], "map": st["npix"], "q": st["nrings"] * (L + 1),
            "qt": 2 * 2 * st["nside"] * (L + 1)}[layout]


def _check_sizes(name, plan, tensors, nmaps):
    """Refuse tensors smaller than the call reads or writes: the kernels
    trust the sizes, so a short buffer would mean out-of-bounds device
    accesses.  tensors: (input, output) in the order of _LAYOUTS[name]."""
    if int(nmaps) < 1:
        return          # the library rejects it with SHTB_EINVAL
    st = shtb_plan_stats(plan)
    src_l, dst_l, fields = _LAYOUTS[name]
    for t, layout, what in zip(tensors, (src_l, dst_l), ("input", "output")):
        need = int(nmaps) * fields * _layout_elems(st, layout)
        if t.numel() < need:
            raise ValueError(f"{name}: {what} holds {t.numel()} elements, the call needs "
                             f"{need} ({nmaps} x {fields} x {layout} of nside={st['nside']}, "
                             f"lmax={st['lmax']})")


def _call_dev(name, plan, src, src_dtype, dst, dst_dtype, nmaps, stream):
    fn = getattr(lib(), name)
    ps, pd = _dptr(src, src_dtype, "input"), _dptr(dst, dst_dtype, "output")
    _check_sizes(name, plan, (src, dst), nmaps)
    _check(fn(plan, ps, pd, int(nmaps), _stream_handle(stream)), name)


def shtb_synthesize(plan, alm, maps, nmaps: int, stream=None) -> None:
    import torch
    _call_dev("shtb_synthesize", plan, alm, torch.complex128, maps, torch.float64, nmaps, stream)


def shtb_synthesize_noalloc(plan, alm, maps, nmaps: int, stream=None) -> None:
    """shtb_synthesize with its scratch in the library's static device array
    (no device allocation by the call; size-limited, see include/shtb.h)."""
    import torch
    _call_dev("shtb_synthesize_noalloc", plan, alm, torch.complex128, maps, torch.float64, nmaps,
              stream)


def shtb_adjoint(plan, maps, alm, nmaps: int, stream=None) -> None:
    import torch
    _call_dev("shtb_adjoint", plan, maps, torch.float64, alm, torch.complex128, nmaps, stream)


def shtb_synthesize_spin(plan, alm, maps, npairs: int, stream=None) -> None:
    """Polarised synthesis: alm complex128 [npairs][2][nalm] (E, B) -> maps
    float64 [npairs][2][npix] (Q, U), on a plan created with spin=2."""
    import torch
    _call_dev("shtb_synthesize_spin", plan, alm, torch.complex128, maps, torch.float64, npairs, stream)


def shtb_adjoint_spin(plan, maps, alm, npairs: int, stream=None) -> None:
    """Transpose of shtb_synthesize_spin: maps float64 [npairs][2][npix]
    (Q, U) -> alm complex128 [npairs][2][nalm] (E, B)."""
    import torch
    _call_dev("shtb_adjoint_spin", plan, maps, torch.float64, alm, torch.complex128, npairs, stream)


def shtb_analyze_spin(plan, maps, alm, npairs: int, ring_weight=None, niter: int = 0,
                      stream=None) -> None:
    """Polarised quadrature analysis (+ niter Jacobi steps): maps [npairs][2][npix]
    (Q, U) -> alm [npairs][2][nalm] (E, B); ring_weight as for shtb_analyze."""
    import torch
    w = None if ring_weight is None else _dptr(ring_weight, torch.float64, "ring_weight")
    pm, pa = _dptr(maps, torch.float64, "maps"), _dptr(alm, torch.complex128, "alm")
    _check_analysis_sizes("shtb_analyze_spin", plan, maps, alm, ring_weight, npairs, 2)
    _check(lib().shtb_analyze_spin(plan, pm, pa, int(npairs), w, int(niter),
                                   _stream_handle(stream)), "shtb_analyze_spin")


def shtb_analyze(plan, maps, alm, nmaps: int, ring_weight=None, niter: int = 0,
                 stream=None) -> None:
    """Quadrature analysis (+ niter Jacobi steps); ring_weight: None (equal
    area 4 pi / npix) or a contiguous float64 device tensor, one per ring."""
    import torch
    w = None if ring_weight is None else _dptr(ring_weight, torch.float64, "ring_weight")
    pm, pa = _dptr(maps, torch.float64, "maps"), _dptr(alm, torch.complex128, "alm")
    _check_analysis_sizes("shtb_analyze", plan, maps, alm, ring_weight, nmaps, 1)
    _check(lib().shtb_analyze(plan, pm, pa, int(nmaps), w, int(niter),
                              _stream_handle(stream)), "shtb_analyze")


def _check_analysis_sizes(name, plan, maps, alm, ring_weight, nmaps, fields):
    if int(nmaps) < 1:
        return
    st = shtb_plan_stats(plan)
    checks = [(maps, int(nmaps) * fields * st["npix"], "maps"),
              (alm, int(nmaps) * fields * st["nalm"], "alm")]
    if ring_weight is not None:
        checks.append((ring_weight, st["nrings"], "ring_weight"))
    for t, need, what in checks:
        if t.numel() < need:
            raise ValueError(f"{name}: {what} holds {t.numel()} elements, the call needs {need}")


def _hptr(t, dtype, name):
    if t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous host {dtype} tensor")
    return ctypes.c_void_p(t.data_ptr())


def shtb_synthesize_host(plan, alm_host, maps_host, nmaps: int, stream=None) -> None:
    import torch
    _check_sizes("shtb_synthesize", plan, (alm_host, maps_host), nmaps)
    _check(lib().shtb_synthesize_host(plan, _hptr(alm_host, torch.complex128, "alm"),
                                      _hptr(maps_host, torch.float64, "maps"), int(nmaps),
                                      _stream_handle(stream)), "shtb_synthesize_host")


def shtb_adjoint_host(plan, maps_host, alm_host, nmaps: int, stream=None) -> None:
    import torch
    _check_sizes("shtb_adjoint", plan, (maps_host, alm_host), nmaps)
    _check(lib().shtb_adjoint_host(plan, _hptr(maps_host, torch.float64, "maps"),
                                   _hptr(alm_host, torch.complex128, "alm"), int(nmaps),
                                   _stream_handle(stream)), "shtb_adjoint_host")


def shtb_profile_enable(plan, on: bool) -> None:
    _check(lib().shtb_profile_enable(plan, 1 if on else 0), "shtb_profile_enable")


STAGES = ("legendre_synth", "phi_synth", "phi_adjoint", "legendre_adjoint", "staging",
          "bf_residual", "bf_levels", "bf_combine")


def shtb_profile_read(plan) -> tuple[dict, int]:
    ms = (ctypes.c_double * len(STAGES))()
    n = ctypes.c_int()
    _check(lib().shtb_profile_read(plan, ms, len(STAGES), ctypes.byref(n)), "shtb_profile_read")
    return {k: ms[i] for i, k in enumerate(STAGES)}, n.value


def shtb_measure_fp64_peak(device: int = 0) -> tuple[float, float]:
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().shtb_measure_fp64_peak(device, ctypes.byref(a), ctypes.byref(b)),
           "shtb_measure_fp64_peak")
    return a.value, b.value


def shtb_test_legendre(plan, alm, q, nmaps: int, stream=None) -> None:
    import torch
    _call_dev("shtb_test_legendre", plan, alm, torch.complex128, q, torch.complex128, nmaps, stream)


def shtb_test_butterfly(plan, alm, qt, nmaps: int, stream=None) -> None:
    """Compressed Legendre stage: qt complex128 [nmaps, 2, 2 nside, lmax+1]."""
    import torch
    _call_dev("shtb_test_butterfly", plan, alm, torch.complex128, qt, torch.complex128, nmaps, stream)


def shtb_test_phi(plan, q, maps, nmaps: int, stream=None) -> None:
    import torch
    _call_dev("shtb_test_phi", plan, q, torch.complex128, maps, torch.float64, nmaps, stream)


def shtb_test_phi_adjoint(plan, maps, q, nmaps: int, stream=None) -> None:
    import torch
    _call_dev("shtb_test_phi_adjoint", plan, maps, torch.float64, q, torch.complex128, nmaps, stream)


def shtb_test_legendre_adjoint(plan, q, alm, nmaps: int, stream=None) -> None:
    import torch
    _call_dev("shtb_test_legendre_adjoint", plan, q, torch.complex128, alm, torch.complex128,
              nmaps, stream)


def shtb_test_host_recurrence(nside: int, lmax: int, m: int, r: int):
    import numpy as np
    out = np.zeros(lmax - m + 1)
    _check(lib().shtb_test_host_recurrence(nside, lmax, m, r, out.ctypes.data_as(_DP)),
           "shtb_test_host_recurrence")
    return out


def shtb_test_host_id(A, eps: float):
    """ID of a real matrix A (rows x n): returns (k, skel, T) with A ~= A[:, skel] @ T."""
    import numpy as np
    A = np.asfortranarray(np.asarray(A, dtype=np.float64))
    rows, n = A.shape
    k = ctypes.c_int()
    skel = np.zeros(max(n, 1), dtype=np.int32)
    T = np.zeros(max(n * n, 1))
    _check(lib().shtb_test_host_id(rows, n, A.ctypes.data_as(_DP), float(eps), ctypes.byref(k),
                                   skel.ctypes.data_as(ctypes.POINTER(_I)), T.ctypes.data_as(_DP)),
           "shtb_test_host_id")
    kk = k.value
    return kk, skel[:kk].copy(), T[:kk * n].reshape(kk, n).copy()


def shtb_test_gpu_id(A, eps: float):
    """shtb_test_host_id through the GPU plan builder's kernel."""
    import numpy as np
    A = np.asfortranarray(np.asarray(A, dtype=np.float64))
    rows, n = A.shape
    k = ctypes.c_int()
    skel = np.zeros(max(n, 1), dtype=np.int32)
    T = np.zeros(max(n * n, 1))
    _check(lib().shtb_test_gpu_id(rows, n, A.ctypes.data_as(_DP), float(eps), ctypes.byref(k),
                                  skel.ctypes.data_as(ctypes.POINTER(_I)), T.ctypes.data_as(_DP)),
           "shtb_test_gpu_id")
    kk = k.value
    return kk, skel[:kk].copy(), T[:kk * n].reshape(kk, n).copy()


def shtb_test_host_butterfly(nside: int, lmax: int, eps: float, m: int, t: int, a,
                             leaf_cols: int = 32):
    """Compressed and dense Lambda^T a for one (m, parity) on the host."""
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float64)
    Z = 2 * nside
    q = np.zeros(Z)
    qe = np.zeros(Z)
    info = (ctypes.c_longlong * 4)()
    _check(lib().shtb_test_host_butterfly(nside, lmax, float(eps), m, t, leaf_cols,
                                          a.ctypes.data_as(_DP), q.ctypes.data_as(_DP),
                                          qe.ctypes.data_as(_DP), info),
           "shtb_test_host_butterfly")
    return q, qe, {"depth": info[0], "n_dense": info[1], "n_r": info[2], "n_ident": info[3]}


def shtb_test_host_interp(nside: int, lmax: int, eps: float, m: int, t: int, a, leaf_cols: int = 32):
    """The interpolation variant of one (m, parity) chain on the host: q at
    the half-rings through the roots of P_{m+t+2n}^m and Eq. interpolation
    (dense), the direct product, and the stored-element counts of both
    routes under the plan's compression."""
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float64)
    Z = 2 * nside
    q = np.zeros(Z)
    qe = np.zeros(Z)
    info = (ctypes.c_longlong * 8)()
    _check(lib().shtb_test_host_interp(nside, lmax, float(eps), m, t, leaf_cols, a.ctypes.data_as(_DP),
                                       q.ctypes.data_as(_DP), qe.ctypes.data_as(_DP), info),
           "shtb_test_host_interp")
    keys = ("n", "roots_butterfly", "interp_butterfly", "interp_hierarchical", "rings_butterfly",
            "rings_dense", "two_step_dense", "rings_depth")
    return q, qe, dict(zip(keys, list(info)))


def shtb_test_host_rec_blocks(nside: int, lmax: int, eps: float, m: int, t: int, leaf_cols: int = 32):
    """Residual blocks of one (m, parity) chain regenerated on the host from
    the recurrence starts a residual_recurrence plan keeps, against the
    stored blocks: (largest error relative to the column's largest element,
    {blocks, elements, crop mismatches, depth})."""
    err = ctypes.c_double()
    info = (ctypes.c_longlong * 4)()
    _check(lib().shtb_test_host_rec_blocks(nside, lmax, float(eps), m, t, leaf_cols, ctypes.byref(err), info),
           "shtb_test_host_rec_blocks")
    return err.value, dict(zip(("blocks", "elements", "crop_mismatch", "depth"), list(info)))


def shtb_test_host_spin_column(nside: int, lmax: int, m: int, s: int, r: int):
    """s_lambda_lm (s = +-2) at half-ring r for l = m..lmax, as spin plans build it."""
    import numpy as np
    out = np.zeros(lmax - m + 1)
    _check(lib().shtb_test_host_spin_column(nside, lmax, m, s, r, out.ctypes.data_as(_DP)),
           "shtb_test_host_spin_column")
    return out


def shtb_struct_sizes() -> dict:
    """sizeof of the public structs in the compiled library."""
    v = [ctypes.c_int() for _ in range(4)]
    _check(lib().shtb_struct_sizes(*[ctypes.byref(x) for x in v]), "shtb_struct_sizes")
    return dict(zip(("opts", "stats", "request", "batch_opts"), (x.value for x in v)))


def shtb_batch_opts_init() -> BatchOpts:
    o = BatchOpts()
    _check(lib().shtb_batch_opts_init(ctypes.byref(o)), "shtb_batch_opts_init")
    return o


def shtb_batch_create(requests, autotune: bool = True, warps_per_block: int = 0,
                      group_width: int = 8, lpt: bool = True, spin_limit: int = 0,
                      schedule: int = 0, streams: int = 0):
    """requests: iterable of (plan, alm tensor [nmaps, nalm] complex128, maps tensor
    [nmaps, npix] float64), all on the current CUDA device."""
    import torch
    reqs = list(requests)
    arr = (Request * len(reqs))()
    for i, (plan, alm, maps) in enumerate(reqs):
        h = plan.handle if hasattr(plan, "handle") else plan
        arr[i].plan = h.value if hasattr(h, "value") else h
        arr[i].alm_dev = _dptr(alm, torch.complex128, "alm").value
        arr[i].map_dev = _dptr(maps, torch.float64, "maps").value
        arr[i].nmaps = int(alm.shape[0])
        _check_sizes("shtb_synthesize", arr[i].plan, (alm, maps), arr[i].nmaps)
        arr[i].dir = 0
    o = shtb_batch_opts_init()
    o.autotune, o.warps_per_block, o.group_width = int(autotune), warps_per_block, group_width
    o.lpt, o.spin_limit = int(lpt), spin_limit
    o.schedule, o.streams = schedule, streams
    h = ctypes.c_void_p()
    _check(lib().shtb_batch_create(arr, len(reqs), ctypes.byref(o), ctypes.byref(h)),
           "shtb_batch_create")
    return h


def shtb_batch_run(batch, stream=None) -> None:
    _check(lib().shtb_batch_run(batch, _stream_handle(stream)), "shtb_batch_run")


def shtb_batch_status(batch, stream=None) -> None:
    _check(lib().shtb_batch_status(batch, _stream_handle(stream)), "shtb_batch_status")


def shtb_batch_info(batch) -> dict:
    w, g, n, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(lib().shtb_batch_info(batch, ctypes.byref(w), ctypes.byref(g), ctypes.byref(n),
                                 ctypes.byref(t)), "shtb_batch_info")
    out = {"warps_per_block": w.value, "grid": g.value, "npacks": n.value, "tuned_ms": t.value}
    out.update(shtb_batch_schedule(batch))
    return out


def shtb_batch_schedule(batch) -> dict:
    s, n = ctypes.c_int(), ctypes.c_int()
    _check(lib().shtb_batch_schedule(batch, ctypes.byref(s), ctypes.byref(n)), "shtb_batch_schedule")
    return {"schedule": s.value, "streams": n.value}


def shtb_batch_destroy(batch) -> None:
    _check(lib().shtb_batch_destroy(batch), "shtb_batch_destroy")


def shtb_test_batch_stall(batch, on: bool) -> None:
    _check(lib().shtb_test_batch_stall(batch, int(on)), "shtb_test_batch_stall")


# ------------------------------------------------------------ convenience
class Plan:
    """A synthesis plan on one CUDA device (owns its device memory).

    eps <= 0 gives the uncompressed transform, eps > 0 the butterfly-compressed
    one.  Keyword options are those of shtb_plan_create: spin=2 for a
    polarised plan (synthesize_spin / adjoint_spin / analyze_spin),
    gpu_build=True to batch the plan's decompositions on the GPU,
    residual_recurrence=True to keep recurrence start values instead of the
    residual blocks (less plan memory, more FP64 work; no batches),
    cache_dir=... to keep plan files, and leaf_cols, max_depth, rho,
    nthreads, device."""

    def __init__(self, nside: int, lmax: int, eps: float = 0.0, **opts):
        import torch
        if "device" not in opts:
            opts["device"] = torch.cuda.current_device()
        self.nside, self.lmax, self.eps = nside, lmax, eps
        self.device = opts["device"]
        self._h = shtb_plan_create(nside, lmax, eps, **opts)
        st = shtb_plan_stats(self._h)
        self.npix, self.nalm, self.nrings = st["npix"], st["nalm"], st["nrings"]

    @property
    def handle(self):
        return self._h

    def stats(self) -> dict:
        return shtb_plan_stats(self._h)

    def reserve(self, nmaps: int) -> None:
        shtb_plan_reserve(self._h, nmaps)

    def synthesize(self, alm, out=None, stream=None):
        """alm complex128 [nmaps, nalm] (or [nalm]) on the plan's device -> maps float64."""
        import torch
        squeeze = alm.dim() == 1
        a = alm.reshape(-1, self.nalm).contiguous()
        nmaps = a.shape[0]
        if out is None:
            out = torch.empty((nmaps, self.npix), dtype=torch.float64, device=a.device)
        shtb_synthesize(self._h, a, out, nmaps, stream)
        return out[0] if squeeze else out

    def adjoint(self, maps, out=None, stream=None):
        """maps float64 [nmaps, npix] (or [npix]) -> Y^T f, complex128 [nmaps, nalm]."""
        import torch
        squeeze = maps.dim() == 1
        f = maps.reshape(-1, self.npix).contiguous()
        nmaps = f.shape[0]
        if out is None:
            out = torch.empty((nmaps, self.nalm), dtype=torch.complex128, device=f.device)
        shtb_adjoint(self._h, f, out, nmaps, stream)
        return out[0] if squeeze else out

    def synthesize_spin(self, alm, out=None, stream=None):
        """Polarised synthesis on a spin=2 plan: alm complex128 [npairs, 2, nalm]
        (or [2, nalm]), E then B -> maps float64 [npairs, 2, npix], Q then U."""
        import torch
        squeeze = alm.dim() == 2
        a = alm.reshape(-1, 2, self.nalm).contiguous()
        npairs = a.shape[0]
        if out is None:
            out = torch.empty((npairs, 2, self.npix), dtype=torch.float64, device=a.device)
        shtb_synthesize_spin(self._h, a, out, npairs, stream)
        return out[0] if squeeze else out

    def adjoint_spin(self, maps, out=None, stream=None):
        """Transpose of synthesize_spin: maps float64 [npairs, 2, npix] (or
        [2, npix]), Q then U -> complex128 [npairs, 2, nalm], E then B."""
        import torch
        squeeze = maps.dim() == 2
        f = maps.reshape(-1, 2, self.npix).contiguous()
        npairs = f.shape[0]
        if out is None:
            out = torch.empty((npairs, 2, self.nalm), dtype=torch.complex128, device=f.device)
        shtb_adjoint_spin(self._h, f, out, npairs, stream)
        return out[0] if squeeze else out

    def analyze_spin(self, maps, niter: int = 0, ring_weight=None, out=None, stream=None):
        """Polarised analysis on a spin=2 plan: maps [npairs, 2, npix] (or [2,
        npix]), Q then U -> complex128 [npairs, 2, nalm], E then B."""
        import torch
        squeeze = maps.dim() == 2
        f = maps.reshape(-1, 2, self.npix).contiguous()
        npairs = f.shape[0]
        if ring_weight is not None and ring_weight.numel() != self.nrings:
            raise ValueError(f"ring_weight needs one weight per ring ({self.nrings})")
        if out is None:
            out = torch.empty((npairs, 2, self.nalm), dtype=torch.complex128, device=f.device)
        shtb_analyze_spin(self._h, f, out, npairs, ring_weight, niter, stream)
        return out[0] if squeeze else out

    def analyze(self, maps, niter: int = 0, ring_weight=None, out=None, stream=None):
        """maps float64 [nmaps, npix] (or [npix]) -> a_lm complex128 by ring
        quadrature plus ``niter`` Jacobi refinement steps (shtb_analyze)."""
        import torch
        squeeze = maps.dim() == 1
        f = maps.reshape(-1, self.npix).contiguous()
        nmaps = f.shape[0]
        if ring_weight is not None and ring_weight.numel() != self.nrings:
            raise ValueError(f"ring_weight needs one weight per ring ({self.nrings})")
        if out is None:
            out = torch.empty((nmaps, self.nalm), dtype=torch.complex128, device=f.device)
        shtb_analyze(self._h, f, out, nmaps, ring_weight, niter, stream)
        return out[0] if squeeze else out

    def save(self, path: str) -> None:
        """Write the plan to a plan file (shtb_plan_save)."""
        shtb_plan_save(self._h, path)

    @classmethod
    def load(cls, path: str, device: int | None = None) -> "Plan":
        """A plan read from a plan file (shtb_plan_load) on `device`."""
        import torch
        self = cls.__new__(cls)
        self.device = torch.cuda.current_device() if device is None else device
        self._h = shtb_plan_load(path, self.device)
        st = shtb_plan_stats(self._h)
        self.nside, self.lmax, self.eps = st["nside"], st["lmax"], st["eps"]
        self.npix, self.nalm, self.nrings = st["npix"], st["nalm"], st["nrings"]
        return self

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            shtb_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd_function():
    import torch

    class Synthesis(torch.autograd.Function):
        """f = Y a with the hand-written adjoint kernel as its backward:
        grad_a = Y^T grad_f, the real-inner-product transpose, which is torch's
        convention for complex leaves (dL/dRe a + i dL/dIm a)."""

        @staticmethod
        def forward(ctx, alm, plan):
            ctx.plan = plan
            return plan.synthesize(alm)

        @staticmethod
        def backward(ctx, grad_maps):
            g = ctx.plan.adjoint(grad_maps.contiguous())
            return g, None

    class PolarisedSynthesis(torch.autograd.Function):
        """(Q, U) = Y_pol (a_E, a_B) with shtb_adjoint_spin as its backward."""

        @staticmethod
        def forward(ctx, alm, plan):
            ctx.plan = plan
            return plan.synthesize_spin(alm)

        @staticmethod
        def backward(ctx, grad_maps):
            return ctx.plan.adjoint_spin(grad_maps.contiguous()), None

    return Synthesis, PolarisedSynthesis


_synth_fn = None
_spin_fn = None


def synthesize(alm, plan: Plan):
    """Differentiable synthesis: maps = Y alm, backward through shtb_adjoint."""
    global _synth_fn, _spin_fn
    if _synth_fn is None:
        _synth_fn, _spin_fn = _autograd_function()
    return _synth_fn.apply(alm, plan)


def synthesize_spin(alm, plan: Plan):
    """Differentiable polarised synthesis on a spin=2 plan: alm [npairs, 2,
    nalm] (E, B) -> maps [npairs, 2, npix] (Q, U); backward through
    shtb_adjoint_spin."""
    global _synth_fn, _spin_fn
    if _spin_fn is None:
        _synth_fn, _spin_fn = _autograd_function()
    return _spin_fn.apply(alm, plan)
