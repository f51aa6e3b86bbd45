"""CPU FP64 oracle for scalar spherical-harmonic synthesis -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The product path (the CUDA
library and its Python binding) never imports, links or runs it, and it shares
no code with that path.

The arithmetic lives in ``sht_oracle.c`` (plain C, OpenMP over rings or m,
compensated FP64 sums); this module compiles it with gcc, loads it with ctypes
and wraps it for numpy arrays.  Every function cites the passage of Seljebotn,
"Wavemoth -- Fast spherical harmonic transforms by butterfly matrix
compression" (arXiv 1110.4874) that it follows:

* ``healpix_rings`` -- the HEALPix RING grid the paper works on (Sec. 2.2,
  the grid of Gorski et al. 2005).
* ``legendre`` -- the normalised associated Legendre functions of Eq. (Y-def),
  Condon-Shortley phase included, by the one-step recurrence.
* ``legendre_q`` -- q_m(z_k) of Eq. (legendre-transform).
* ``phi_synth`` -- the per-ring sum over m of Eq. (sh-baseline) with the ring
  longitudes of Eq. (phi), as a direct DFT.
* ``synthesize`` -- Eq. (shdef) at the pixels, i.e. the two stages above.
* ``phi_adjoint``, ``legendre_adjoint``, ``adjoint`` -- the transpose of the
  real-linear synthesis map under the plain real inner products (the Y^T of
  Eq. (datamodel)/(wiener)): (Y^T f)_l0 = sum_p f_p P_l^0(z_p) and
  (Y^T f)_lm = 2 sum_p f_p P_l^m(z_p) e^{-i m phi_p} for m >= 1.
* ``analyze`` -- spherical-harmonic analysis by the ring quadrature of Eq.
  (sh-forward-quadrature), optionally refined by Jacobi steps.
* ``spin_lambda``, ``spin_q``, ``spin_synthesize``, ``spin_adjoint``,
  ``spin_analyze`` --
  spin-weighted harmonics, the polarised (spin-2) synthesis of Q and U maps
  from E and B coefficients (the spin-weighted transforms of the paper's
  Discussion, Sec. 5) from the Wigner-d closed form, its transpose, and the
  quadrature analysis built on that transpose.

Parity of every function here is pinned by ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sht_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)
_LP = ctypes.POINTER(ctypes.c_longlong)


def build(force: bool = False) -> str:
    """Compile sht_oracle.c into a shared library (gcc, -O2, OpenMP).

    ``-ffp-contract=off`` keeps the compensated sums exact (no fused
    contractions behind the TwoSum steps)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_nalm.restype = ctypes.c_longlong
            lib.orc_nalm.argtypes = [ctypes.c_int]
            lib.orc_healpix_rings.argtypes = [ctypes.c_int, _DP, _DP, _DP, _DP, _IP, _IP, _LP]
            lib.orc_sin_from_cos.restype = None
            lib.orc_sin_from_cos.argtypes = [ctypes.c_int, _DP, _DP, _DP]
            lib.orc_legendre.restype = None
            lib.orc_legendre.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, _DP]
            lib.orc_legendre_q.argtypes = [ctypes.c_int, _DP, _DP, _DP, _DP, ctypes.c_int,
                                           ctypes.c_int, _DP, _DP, ctypes.c_int]
            lib.orc_phi_synth.argtypes = [ctypes.c_int, _IP, _IP, ctypes.c_int,
                                          ctypes.c_int, _DP, _DP, ctypes.c_int]
            lib.orc_synth.argtypes = [ctypes.c_int, _DP, _DP, _DP, _DP, _IP, _IP,
                                      ctypes.c_int, ctypes.c_int, _DP, _DP, ctypes.c_int]
            lib.orc_phi_adjoint.argtypes = [ctypes.c_int, _IP, _IP, ctypes.c_int,
                                            ctypes.c_int, _DP, _DP, ctypes.c_int]
            lib.orc_legendre_adjoint.argtypes = [ctypes.c_int, _DP, _DP, _DP, _DP,
                                                 ctypes.c_int, ctypes.c_int, _DP, _DP,
                                                 ctypes.c_int]
            lib.orc_adjoint.argtypes = [ctypes.c_int, _DP, _DP, _DP, _DP, _IP, _IP,
                                        ctypes.c_int, ctypes.c_int, _DP, _DP, ctypes.c_int]
            lib.orc_spin_lambda.restype = None
            lib.orc_spin_lambda.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_double, _DP]
            lib.orc_spin_q.argtypes = [ctypes.c_int, _DP, _DP, _DP, _DP, ctypes.c_int, ctypes.c_int,
                                       _DP, _DP, _DP, _DP, ctypes.c_int]
            lib.orc_spin_legendre_adjoint.argtypes = [ctypes.c_int, _DP, _DP, _DP, _DP, ctypes.c_int,
                                                      ctypes.c_int, _DP, _DP, _DP, _DP, ctypes.c_int]
            lib.orc_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(_DP)


def _ip(a):
    return a.ctypes.data_as(_IP)


def max_threads() -> int:
    """OpenMP threads the oracle uses when ``nthreads=0``."""
    return int(_load().orc_max_threads())


def nalm(lmax: int) -> int:
    """Number of stored (l, m >= 0) coefficients, (L+1)(L+2)/2."""
    return (lmax + 1) * (lmax + 2) // 2


class Rings:
    """An iso-latitude ring grid: z = cos(theta) and sin(theta) per ring, each
    as a double-double pair (hi + lo), pixels per ring J and the half-pixel
    flag s (phi_kj = pi (2j + s_k) / J_k).  If the low parts are omitted, z is
    taken as exact and sin(theta) = sqrt((1-z)(1+z)) is formed in
    double-double."""

    def __init__(self, z, sinth, J, s, zlo=None, sinlo=None):
        self.z = np.ascontiguousarray(z, dtype=np.float64)
        self.zlo = (np.zeros_like(self.z) if zlo is None
                    else np.ascontiguousarray(zlo, dtype=np.float64))
        if sinth is None or sinlo is None:
            st = np.empty_like(self.z)
            sl = np.empty_like(self.z)
            _load().orc_sin_from_cos(self.z.size, _dp(self.z), _dp(st), _dp(sl))
            self.sinth, self.sinlo = st, sl
        else:
            self.sinth = np.ascontiguousarray(sinth, dtype=np.float64)
            self.sinlo = np.ascontiguousarray(sinlo, dtype=np.float64)
        self.J = np.ascontiguousarray(J, dtype=np.int32)
        self.s = np.ascontiguousarray(s, dtype=np.int32)
        self.start = np.concatenate([[0], np.cumsum(self.J.astype(np.int64))])

    @property
    def nrings(self) -> int:
        return int(self.z.shape[0])

    @property
    def npix(self) -> int:
        return int(self.start[-1])

    def subset(self, idx) -> "Rings":
        idx = np.asarray(idx)
        return Rings(self.z[idx], self.sinth[idx], self.J[idx], self.s[idx],
                     self.zlo[idx], self.sinlo[idx])

    def phi(self, k: int) -> np.ndarray:
        """Longitudes of ring k (Eq. phi)."""
        j = np.arange(self.J[k])
        return np.pi * (2 * j + self.s[k]) / self.J[k]

    def _geo(self):
        return (_dp(self.z), _dp(self.zlo), _dp(self.sinth), _dp(self.sinlo))


def healpix_rings(nside: int) -> Rings:
    """The 4*nside-1 rings of the HEALPix grid, north to south."""
    if nside < 1:
        raise ValueError("nside must be >= 1")
    nr = 4 * nside - 1
    z, zl, st, sl = (np.empty(nr) for _ in range(4))
    J = np.empty(nr, dtype=np.int32)
    s = np.empty(nr, dtype=np.int32)
    start = np.empty(nr, dtype=np.int64)
    rc = _load().orc_healpix_rings(nside, _dp(z), _dp(zl), _dp(st), _dp(sl), _ip(J), _ip(s),
                                   start.ctypes.data_as(_LP))
    if rc != 0:
        raise ValueError("bad nside")
    return Rings(z, st, J, s, zl, sl)


def legendre(m: int, lmax: int, z: float, sinth: float | None = None,
             zlo: float = 0.0, sinlo: float | None = None) -> np.ndarray:
    """Ptilde_l^m(z) for l = m..lmax (Eq. Y-def, with (-1)^m).  Without
    sin(theta), it is formed from z in double-double."""
    if sinth is None or sinlo is None:
        zz = np.array([z], dtype=np.float64)
        st, sl = np.empty(1), np.empty(1)
        _load().orc_sin_from_cos(1, _dp(zz), _dp(st), _dp(sl))
        if sinth is None:
            sinth, sinlo = float(st[0]), float(sl[0])
        else:
            sinlo = 0.0
    out = np.zeros(max(lmax - m + 1, 0))
    if m <= lmax:
        _load().orc_legendre(int(m), int(lmax), float(z), float(zlo), float(sinth),
                             float(sinlo), _dp(out))
    return out


def _alm2d(alm, lmax):
    a = np.asarray(alm)
    if a.ndim == 1:
        a = a[None, :]
    if a.shape[-1] != nalm(lmax):
        raise ValueError("alm has the wrong length for lmax")
    return np.ascontiguousarray(a.astype(np.complex128)).view(np.float64), a.shape[0]


def legendre_q(rings: Rings, lmax: int, alm, nthreads: int = 0) -> np.ndarray:
    """q_m(z_k) for every ring and m = 0..lmax: complex [nmaps, nrings, lmax+1]."""
    a, nmaps = _alm2d(alm, lmax)
    q = np.zeros((nmaps, rings.nrings, lmax + 1), dtype=np.complex128)
    rc = _load().orc_legendre_q(rings.nrings, *rings._geo(), lmax,
                                nmaps, _dp(a), _dp(q.view(np.float64)), nthreads)
    assert rc == 0
    return q


def phi_synth(rings: Rings, lmax: int, q, nthreads: int = 0) -> np.ndarray:
    """Pixels from q_m(z_k): real [nmaps, npix]."""
    q = np.ascontiguousarray(np.asarray(q, dtype=np.complex128))
    if q.ndim == 2:
        q = q[None]
    nmaps = q.shape[0]
    assert q.shape[1:] == (rings.nrings, lmax + 1)
    out = np.zeros((nmaps, rings.npix))
    rc = _load().orc_phi_synth(rings.nrings, _ip(rings.J), _ip(rings.s), lmax, nmaps,
                               _dp(q.view(np.float64)), _dp(out), nthreads)
    assert rc == 0
    return out


def synthesize(rings: Rings, lmax: int, alm, nthreads: int = 0) -> np.ndarray:
    """f = Y a at every pixel of ``rings``: real [nmaps, npix] (Eq. shdef)."""
    a, nmaps = _alm2d(alm, lmax)
    out = np.zeros((nmaps, rings.npix))
    rc = _load().orc_synth(rings.nrings, *rings._geo(), _ip(rings.J),
                           _ip(rings.s), lmax, nmaps, _dp(a), _dp(out), nthreads)
    assert rc == 0
    return out


def phi_adjoint(rings: Rings, lmax: int, maps, nthreads: int = 0) -> np.ndarray:
    """F_m(k) = sum_j f_kj e^{-i m phi_kj}: complex [nmaps, nrings, lmax+1]."""
    f = np.ascontiguousarray(np.atleast_2d(np.asarray(maps, dtype=np.float64)))
    nmaps = f.shape[0]
    assert f.shape[1] == rings.npix
    F = np.zeros((nmaps, rings.nrings, lmax + 1), dtype=np.complex128)
    rc = _load().orc_phi_adjoint(rings.nrings, _ip(rings.J), _ip(rings.s), lmax, nmaps,
                                 _dp(f), _dp(F.view(np.float64)), nthreads)
    assert rc == 0
    return F


def legendre_adjoint(rings: Rings, lmax: int, F, nthreads: int = 0) -> np.ndarray:
    """a_lm = c_m sum_k Ptilde_l^m(z_k) F_m(k), c_0 = 1, c_m = 2: complex [nmaps, nalm]."""
    F = np.ascontiguousarray(np.asarray(F, dtype=np.complex128))
    if F.ndim == 2:
        F = F[None]
    nmaps = F.shape[0]
    alm = np.zeros((nmaps, nalm(lmax)), dtype=np.complex128)
    rc = _load().orc_legendre_adjoint(rings.nrings, *rings._geo(), lmax,
                                      nmaps, _dp(F.view(np.float64)),
                                      _dp(alm.view(np.float64)), nthreads)
    assert rc == 0
    return alm


def adjoint(rings: Rings, lmax: int, maps, nthreads: int = 0) -> np.ndarray:
    """Y^T f: complex [nmaps, nalm] (real-inner-product transpose of synthesize)."""
    f = np.ascontiguousarray(np.atleast_2d(np.asarray(maps, dtype=np.float64)))
    nmaps = f.shape[0]
    assert f.shape[1] == rings.npix
    alm = np.zeros((nmaps, nalm(lmax)), dtype=np.complex128)
    rc = _load().orc_adjoint(rings.nrings, *rings._geo(), _ip(rings.J),
                             _ip(rings.s), lmax, nmaps, _dp(f),
                             _dp(alm.view(np.float64)), nthreads)
    assert rc == 0
    return alm


def gauss_legendre_rings(nrings: int, nphi: int) -> tuple[Rings, np.ndarray]:
    """A Gauss-Legendre ring grid (the paper's methods apply to any
    iso-latitude grid, Sec. 1): nodes/weights from numpy's leggauss,
    nphi pixels per ring, phi_0 = 0.  Returns (rings, w_k)."""
    x, w = np.polynomial.legendre.leggauss(nrings)
    z = x[::-1].copy()
    w = w[::-1].copy()
    return Rings(z, None, np.full(nrings, nphi, np.int32), np.zeros(nrings, np.int32)), w


def _m_of_index(lmax: int) -> np.ndarray:
    """m of every stored coefficient (m-major layout, l = m..lmax)."""
    return np.repeat(np.arange(lmax + 1), np.arange(lmax + 1, 0, -1))


def analyze(rings: Rings, lmax: int, maps, ring_weight, niter: int = 0,
            nthreads: int = 0) -> np.ndarray:
    """Spherical-harmonic analysis by the quadrature rule of Eq.
    (sh-forward-quadrature): a_lm = sum_p w_p f_p conj(Y_lm(p)), with w_p
    the weight of pixel p's ring (``ring_weight[k]``, one per ring).

    conj(Y_lm(p)) = Ptilde_l^m(z_p) e^{-i m phi_p}, so the sum is the
    real-inner-product adjoint of ``adjoint`` applied to the weighted map,
    halved for m >= 1 (that adjoint carries the factor 2 of the -m terms).
    With ``niter`` > 0 the estimate is refined by Jacobi steps
    a <- a + A (f - Y a), A the quadrature rule above: the quadrature is
    not exact on HEALPix (Sec. 2.3), and each step removes part of the
    error.  Complex [nmaps, nalm]."""
    f = np.atleast_2d(np.asarray(maps, dtype=np.float64))
    w = np.repeat(np.asarray(ring_weight, dtype=np.float64), rings.J)
    h = np.where(_m_of_index(lmax) == 0, 1.0, 0.5)

    def quad(g):
        return adjoint(rings, lmax, g * w, nthreads) * h

    a = quad(f)
    for _ in range(niter):
        a = a + quad(f - synthesize(rings, lmax, a, nthreads))
    return a


def spin_lambda(s: int, m: int, lmax: int, z: float, sinth: float | None = None) -> np.ndarray:
    """s_lambda_lm(z) for l = 0..lmax (0 below l = max(|m|, |s|)):
    (-1)^s sqrt((2l+1)/4pi) d^l_{m,-s}(theta), the spin-s harmonic without
    its e^{i m phi} (Newman-Penrose convention; s = 0 gives Eq. Y-def).
    Any integer m in [-lmax, lmax]."""
    zz = np.array([z], dtype=np.float64)
    st, sl = np.empty(1), np.empty(1)
    _load().orc_sin_from_cos(1, _dp(zz), _dp(st), _dp(sl))
    if sinth is not None:
        st[0], sl[0] = sinth, 0.0
    out = np.zeros(lmax + 1)
    _load().orc_spin_lambda(int(s), int(m), int(lmax), float(z), 0.0, float(st[0]), float(sl[0]), _dp(out))
    return out


def spin_q(rings: Rings, lmax: int, alm_E, alm_B, nthreads: int = 0):
    """Polarised Legendre stage, HEALPix convention
    Q + iU = -sum (a_E + i a_B) 2Y and Q - iU = -sum (a_E - i a_B) (-2)Y:
    Q_m(z_k) = -sum_l [a_E F+ + i a_B F-] and U_m(z_k) = -sum_l [a_B F+ -
    i a_E F-], F+- = (2_lambda +- (-2)_lambda)/2.  Returns (qQ, qU), each
    complex [nmaps, nrings, lmax+1]; the maps follow from ``phi_synth``."""
    e, nmaps = _alm2d(alm_E, lmax)
    b, nb = _alm2d(alm_B, lmax)
    assert nb == nmaps
    qQ = np.zeros((nmaps, rings.nrings, lmax + 1), dtype=np.complex128)
    qU = np.zeros_like(qQ)
    rc = _load().orc_spin_q(rings.nrings, *rings._geo(), lmax, nmaps, _dp(e), _dp(b),
                            _dp(qQ.view(np.float64)), _dp(qU.view(np.float64)), nthreads)
    assert rc == 0
    return qQ, qU


def spin_synthesize(rings: Rings, lmax: int, alm_E, alm_B, nthreads: int = 0):
    """Q and U maps (real [nmaps, npix] each) of the E and B coefficients."""
    qQ, qU = spin_q(rings, lmax, alm_E, alm_B, nthreads)
    return phi_synth(rings, lmax, qQ, nthreads), phi_synth(rings, lmax, qU, nthreads)


def spin_adjoint(rings: Rings, lmax: int, Q, U, nthreads: int = 0):
    """Transpose of ``spin_synthesize`` under real inner products over the
    (Re, Im) pairs of a_E and a_B: returns (g_E, g_B), complex [nmaps, nalm],
    with <spin_synthesize(a_E, a_B), (Q, U)> = <a_E, g_E> + <a_B, g_B>.
    The ring sums are ``phi_adjoint``; the Legendre part is the transposed
    combine, g_E = c_m sum_k [-F+ G_Q - i F- G_U] and g_B = c_m sum_k
    [i F- G_Q - F+ G_U] (c_0 = 1, c_m = 2)."""
    GQ = phi_adjoint(rings, lmax, Q, nthreads)
    GU = phi_adjoint(rings, lmax, U, nthreads)
    nmaps = GQ.shape[0]
    gE = np.zeros((nmaps, nalm(lmax)), dtype=np.complex128)
    gB = np.zeros_like(gE)
    rc = _load().orc_spin_legendre_adjoint(rings.nrings, *rings._geo(), lmax, nmaps,
                                           _dp(GQ.view(np.float64)), _dp(GU.view(np.float64)),
                                           _dp(gE.view(np.float64)), _dp(gB.view(np.float64)), nthreads)
    assert rc == 0
    return gE, gB


def spin_analyze(rings: Rings, lmax: int, Q, U, ring_weight, niter: int = 0,
                 nthreads: int = 0):
    """Polarised analysis by the same quadrature rule as ``analyze`` (Eq.
    sh-forward-quadrature for the spin-2 harmonics): (a_E, a_B) = h_m *
    spin_adjoint(w Q, w U), h_0 = 1, h_m = 1/2, because the real-inner-product
    transpose carries the factor 2 of the -m terms; then ``niter`` Jacobi
    steps a <- a + A (f - Y a).  Returns (a_E, a_B), complex [nmaps, nalm]."""
    Q = np.atleast_2d(np.asarray(Q, dtype=np.float64))
    U = np.atleast_2d(np.asarray(U, dtype=np.float64))
    w = np.repeat(np.asarray(ring_weight, dtype=np.float64), rings.J)
    h = np.where(_m_of_index(lmax) == 0, 1.0, 0.5)

    def quad(q, u):
        gE, gB = spin_adjoint(rings, lmax, q * w, u * w, nthreads)
        return gE * h, gB * h

    aE, aB = quad(Q, U)
    for _ in range(niter):
        q, u = spin_synthesize(rings, lmax, aE, aB, nthreads)
        dE, dB = quad(Q - q, U - u)
        aE, aB = aE + dE, aB + dB
    return aE, aB
