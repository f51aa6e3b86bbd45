"""Pins of the CPU oracle against facts fixed by the paper and the mathematics.

Nothing here compares the oracle with itself: each test checks it against a
closed form, a library routine (scipy's spherical harmonics, numpy's
Gauss-Legendre nodes), a printed formula of the paper (the jump-two
coefficients of Eq. three-term), or an exact identity of the grid or of
linear algebra.  A dropped term, a wrong sign or index, a transposed operand
or a wrong factor in any oracle routine fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
from fractions import Fraction

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _alm_index(lmax, l, m):
    return m * (2 * lmax + 1 - m) // 2 + l


def _random_alm(lmax, nmaps, seed):
    rng = np.random.default_rng(seed)
    n = oracle.nalm(lmax)
    a = rng.standard_normal((nmaps, n)) + 1j * rng.standard_normal((nmaps, n))
    for l in range(lmax + 1):
        a[:, _alm_index(lmax, l, 0)] = a[:, _alm_index(lmax, l, 0)].real
    return a


# ------------------------------------------------------------ grid geometry
def _healpix_pix2ang(nside, p):
    """Pixel centre (z, phi) of RING pixel p from the pixel-index formulas of
    Gorski et al. 2005 (a per-pixel route, independent of the oracle's
    per-ring loop)."""
    npix = 12 * nside * nside
    ncap = 2 * nside * (nside - 1)
    if p < ncap:                                   # north polar cap
        i = (1 + math.isqrt(1 + 2 * p)) // 2
        j = p + 1 - 2 * i * (i - 1)
        return 1 - i * i / (3 * nside * nside), (j - 0.5) * (math.pi / 2) / i
    if p < npix - ncap:                            # equatorial belt
        q = p - ncap
        i = q // (4 * nside) + nside
        j = q % (4 * nside) + 1
        fodd = 1.0 if (i + nside) % 2 else 0.5
        return (4 * nside - 2 * i) / (3 * nside), (j - fodd) * math.pi / (2 * nside)
    q = npix - p - 1                               # south polar cap (mirror)
    i = (1 + math.isqrt(1 + 2 * q)) // 2
    j = 4 * i + 1 - (q + 1 - 2 * i * (i - 1))
    return -(1 - i * i / (3 * nside * nside)), (j - 0.5) * (math.pi / 2) / i


def _expand(rings):
    zs, phis = [], []
    for k in range(rings.nrings):
        zs.append(np.full(rings.J[k], rings.z[k]))
        phis.append(rings.phi(k))
    return np.concatenate(zs), np.concatenate(phis)


def test_healpix_nside1_golden():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "healpix_nside1_pixel_centres.txt"))
            if l.strip() and not l.startswith("#")]
    z, phi = _expand(oracle.healpix_rings(1))
    assert len(rows) == 12 == z.size
    for r in rows:
        p = int(r[0])
        assert z[p] == pytest.approx(int(r[1]) / int(r[2]), abs=1e-15)
        assert phi[p] == pytest.approx(math.pi * int(r[3]) / int(r[4]), abs=1e-15)


@pytest.mark.parametrize("nside", [1, 2, 3, 4, 7, 16, 33])
def test_healpix_rings_match_pixel_formulas(nside):
    rings = oracle.healpix_rings(nside)
    assert rings.nrings == 4 * nside - 1
    assert rings.npix == 12 * nside * nside
    z, phi = _expand(rings)
    for p in range(rings.npix):
        zp, php = _healpix_pix2ang(nside, p)
        assert z[p] == pytest.approx(zp, abs=1e-15)
        assert phi[p] == pytest.approx(php, abs=1e-13)
    # (z, sin theta) as double-double pairs lie on the unit circle
    zz = rings.z.astype(np.longdouble) + rings.zlo
    ss = rings.sinth.astype(np.longdouble) + rings.sinlo
    assert np.abs(zz * zz + ss * ss - 1).max() < 4 * np.finfo(np.longdouble).eps
    # and the low parts only refine the doubles
    assert np.all(np.abs(rings.zlo) <= np.spacing(np.abs(rings.z)))
    # rings are symmetric about the equator
    np.testing.assert_array_equal(rings.J, rings.J[::-1])
    np.testing.assert_allclose(rings.z, -rings.z[::-1], atol=0)


# ----------------------------------------------------- Legendre functions
def _closed_forms():
    out = []
    for line in open(os.path.join(GOLDEN, "legendre_closed_forms.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        l, m, sign, C, poly = line.split()
        out.append((int(l), int(m), int(sign), float(Fraction(C)), poly))
    return out


def test_legendre_closed_forms():
    forms = _closed_forms()
    assert len(forms) == 10
    for z in np.linspace(-0.999, 0.999, 37):
        s = math.sqrt((1 - z) * (1 + z))
        for l, m, sign, C, poly in forms:
            want = sign * math.sqrt(C / math.pi) * eval(poly, {"z": z, "s": s})
            got = oracle.legendre(m, 3, z)[l - m]
            assert got == pytest.approx(want, rel=1e-14, abs=1e-15), (l, m, z)


def test_legendre_matches_scipy():
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(7)
    for _ in range(40):
        m = int(rng.integers(0, 150))
        lmax = m + int(rng.integers(0, 150))
        z = float(rng.uniform(-0.99, 0.99))
        got = oracle.legendre(m, lmax, z)
        ls = np.arange(m, lmax + 1)
        want = sp.sph_harm_y(ls, m, math.acos(z), 0.0).real
        scale = max(np.abs(want).max(), 1e-300)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * scale)


def test_legendre_diagonal_log_closed_form():
    """|Ptilde_m^m| = sqrt((2m+1)/(4pi) (2m)!/(4^m m!^2)) sin^m(theta), in
    logarithms, far into the range where sin^m underflows in doubles."""
    nside = 2048
    rings = oracle.healpix_rings(nside)
    for k in [0, 1, 5, 40, 300, 2047]:
        z, st = rings.z[k], rings.sinth[k]
        for m in [1, 10, 100, 700, 1500, 4000]:
            v = oracle.legendre(m, m, z, st, rings.zlo[k], rings.sinlo[k])[0]
            logv = 0.5 * (math.log((2 * m + 1) / (4 * math.pi)) + math.lgamma(2 * m + 1)
                          - 2 * math.lgamma(m + 1) - m * math.log(4)) + m * math.log(st)
            if logv < math.log(1e-290):
                assert abs(v) < 1e-280
                continue
            assert math.log(abs(v)) == pytest.approx(logv, abs=1e-11)
            assert (v < 0) == (m % 2 == 1)     # Condon-Shortley sign


@pytest.mark.parametrize("lmax", [64, 1024, 4096])
def test_addition_theorem(lmax):
    """P_l^0(z)^2 + 2 sum_{m>=1} P_l^m(z)^2 = (2l+1)/(4 pi) for every l, at
    near-pole, mid and equatorial z (including the first HEALPix ring at
    Nside=2048, where most of the terms underflow).

    sin(theta) is formed from z in double-double, so (z, sin theta) lies on
    the unit circle to ~1e-32 and the identity must hold to a few ulp of the
    final double sums everywhere (a plain FP64 one-step recurrence misses it
    by 1.5e-11 at l = 4096 next to the pole and by 2.6e-13 at z = 0.5)."""
    cases = [(1 - 1 / (3 * 2048 ** 2), 1e-14), (1 - 1 / (3 * 64 ** 2), 1e-14), (0.0, 1e-14),
             (0.93, None), (0.5, None), (0.1, None), (-0.77, None)]
    for z, tol in cases:
        acc = np.zeros(lmax + 1)
        for m in range(lmax + 1):
            p = oracle.legendre(m, lmax, z)
            acc[m:] += (1.0 if m == 0 else 2.0) * p * p
        want = (2 * np.arange(lmax + 1) + 1) / (4 * math.pi)
        np.testing.assert_allclose(acc, want, rtol=tol if tol is not None else 2e-14)


def test_legendre_satisfies_paper_jump_two_recurrence():
    """The oracle's one-step values obey the paper's jump-two relation,
    Eq. (three-term): P_{l+2} = ((z^2 - d_l)/c_l) P_l - (c_{l-2}/c_l) P_{l-2},
    with c_l^m and d_l^m as printed in the appendix."""
    def c(l, m):
        return math.sqrt((l - m + 1) * (l - m + 2) * (l + m + 1) * (l + m + 2)
                         / ((2 * l + 1) * (2 * l + 3) ** 2 * (2 * l + 5)))

    def d(l, m):
        return (2 * l * (l + 1) - 2 * m * m - 1) / ((2 * l - 1) * (2 * l + 3))

    rng = np.random.default_rng(11)
    for _ in range(30):
        m = int(rng.integers(0, 300))
        lmax = m + 60
        z = float(rng.uniform(-0.95, 0.95))
        p = oracle.legendre(m, lmax, z)
        for l in range(m + 2, lmax - 1):
            lhs = p[l + 2 - m]
            rhs = (z * z - d(l, m)) / c(l, m) * p[l - m] - c(l - 2, m) / c(l, m) * p[l - 2 - m]
            assert lhs == pytest.approx(rhs, rel=1e-10, abs=1e-12)
        # self-starting chains: c_{m-2} = c_{m-1} = 0 would be the missing terms
        rhs = (z * z - d(m, m)) / c(m, m) * p[0]
        assert p[2] == pytest.approx(rhs, rel=1e-12, abs=1e-14)


# --------------------------------------------------------------- synthesis
def test_single_mode_inputs():
    """a_lm = 1 gives f = 2 P_l^m(z) cos(m phi); a_lm = i gives -2 P sin(m phi);
    m = 0 gives P_l^0(z) (Eq. shdef with a_{l,-m} = (-1)^m a*_lm)."""
    sp = pytest.importorskip("scipy.special")
    nside, lmax = 4, 9
    rings = oracle.healpix_rings(nside)
    z, phi = _expand(rings)
    th = np.arccos(z)
    for (l, m) in [(0, 0), (3, 0), (5, 2), (7, 7), (9, 4), (8, 1)]:
        for val in [1.0, 1j]:
            if m == 0 and val == 1j:
                continue
            a = np.zeros(oracle.nalm(lmax), complex)
            a[_alm_index(lmax, l, m)] = val
            f = oracle.synthesize(rings, lmax, a)[0]
            P = sp.sph_harm_y(l, m, th, 0.0).real
            if m == 0:
                want = P
            elif val == 1.0:
                want = 2 * P * np.cos(m * phi)
            else:
                want = -2 * P * np.sin(m * phi)
            np.testing.assert_allclose(f, want, atol=1e-14)


def test_synthesis_brute_force_vs_scipy():
    """Eq. (shdef) summed pixel by pixel with scipy's Y_lm over all m = -L..L."""
    sp = pytest.importorskip("scipy.special")
    nside, lmax = 4, 8
    rings = oracle.healpix_rings(nside)
    z, phi = _expand(rings)
    th = np.arccos(z)
    a = _random_alm(lmax, 2, 5)
    got = oracle.synthesize(rings, lmax, a)
    for b in range(2):
        want = np.zeros(z.size, complex)
        for l in range(lmax + 1):
            for m in range(-l, l + 1):
                alm = a[b, _alm_index(lmax, l, abs(m))]
                if m < 0:
                    alm = (-1) ** m * np.conj(alm)
                want += alm * sp.sph_harm_y(l, m, th, phi)
        assert np.abs(want.imag).max() < 1e-13
        np.testing.assert_allclose(got[b], want.real, atol=1e-13)


def test_mirror_parity():
    """Eq. (q-even-odd2): only-even (l-m) inputs are mirror-symmetric, only-odd
    inputs antisymmetric; the odd part vanishes on the equator."""
    nside, lmax = 8, 20
    rings = oracle.healpix_rings(nside)
    a = _random_alm(lmax, 1, 3)[0]
    par = np.array([(l - m) % 2 for m in range(lmax + 1) for l in range(m, lmax + 1)])
    for p, sign in [(0, 1.0), (1, -1.0)]:
        f = oracle.synthesize(rings, lmax, np.where(par == p, a, 0))[0]
        for k in range(2 * nside - 1):
            kk = rings.nrings - 1 - k
            np.testing.assert_allclose(f[rings.start[k]:rings.start[k + 1]],
                                       sign * f[rings.start[kk]:rings.start[kk + 1]], atol=1e-13)
        if p == 1:
            e = 2 * nside - 1
            assert np.abs(f[rings.start[e]:rings.start[e + 1]]).max() < 1e-14


def test_ring_phi_orthogonality():
    """On a HEALPix ring, sum_j e^{i(m-m')phi_j} = 0 for 0 < |m-m'| < J and
    J for m = m' (exact), so the Fourier-stage adjoint of a single-m q returns
    J q_m at m and 0 elsewhere (m + m' < J)."""
    nside, lmax = 8, 15
    rings = oracle.healpix_rings(nside)
    for k in [2, 7, 12]:
        one = rings.subset([k])
        J = int(one.J[0])
        for m0 in range(1, J // 2):
            if m0 > lmax:
                break
            q = np.zeros((1, 1, lmax + 1), complex)
            q[0, 0, m0] = 0.3 - 0.7j
            F = oracle.phi_adjoint(one, lmax, oracle.phi_synth(one, lmax, q))[0, 0]
            for m in range(1, lmax + 1):
                if m + m0 >= J or abs(m - m0) >= J:
                    continue
                want = J * q[0, 0, m0] if m == m0 else 0.0
                assert abs(F[m] - want) < 1e-12


def test_gauss_legendre_quadrature_orthogonality():
    """On a Gauss-Legendre ring grid (nodes/weights from numpy) with L+1 rings,
    2 pi sum_k w_k P_l^m(z_k) P_l'^m(z_k) = delta_ll' exactly for l, l' <= L."""
    lmax = 16
    rings, w = oracle.gauss_legendre_rings(lmax + 1, 2 * lmax + 1)
    for m in range(lmax + 1):
        P = np.array([oracle.legendre(m, lmax, z, s) for z, s in zip(rings.z, rings.sinth)])
        G = 2 * math.pi * (P.T * w) @ P
        np.testing.assert_allclose(G, np.eye(lmax - m + 1), atol=2e-14)


def test_gauss_legendre_discrete_analysis_roundtrip():
    """Quadrature weights times the adjoint invert synthesis exactly on a
    Gauss-Legendre grid with J >= 2L+1: Y^T(W Y a) = a for m = 0 (real part)
    and 2 a for m >= 1 (Eq. sh-forward-quadrature with the real-inner-product
    adjoint)."""
    lmax = 12
    rings, w = oracle.gauss_legendre_rings(lmax + 1, 2 * lmax + 3)
    a = _random_alm(lmax, 2, 9)
    f = oracle.synthesize(rings, lmax, a)
    wp = np.repeat(2 * math.pi * w / rings.J, rings.J)
    back = oracle.adjoint(rings, lmax, f * wp)
    want = a.copy()
    mcol = np.array([m for m in range(lmax + 1) for _ in range(m, lmax + 1)])
    want[:, mcol > 0] *= 2
    np.testing.assert_allclose(back, want, atol=2e-13)


def test_analysis_exact_on_gauss_legendre_grid():
    """oracle.analyze with the Gauss-Legendre weights (2 pi w_k / J per pixel)
    recovers a band-limited a_lm exactly: the quadrature of Eq.
    (sh-forward-quadrature) is exact there for l, l' <= L (L+1 rings,
    J >= 2L+1).  A wrong weight, a missing 1/2 for m >= 1 or a flipped phase
    sign each fail this."""
    lmax = 12
    rings, w = oracle.gauss_legendre_rings(lmax + 1, 2 * lmax + 1)
    a = _random_alm(lmax, 2, 31)
    f = oracle.synthesize(rings, lmax, a)
    back = oracle.analyze(rings, lmax, f, 2 * math.pi * w / rings.J)
    np.testing.assert_allclose(back, a, atol=5e-14)


def test_analysis_of_constant_map_on_healpix():
    """f = 1 on the HEALPix grid with the equal-area weight 4 pi / npix:
    a_00 = sqrt(4 pi) exactly (the weights sum to 4 pi and P_0^0 =
    1/sqrt(4 pi)), and every m = 1, 2, 3 coefficient vanishes because each
    ring's longitude sum of e^{-i m phi} is zero for 0 < m < J (J >= 4)."""
    nside, lmax = 8, 16
    rings = oracle.healpix_rings(nside)
    w = np.full(rings.nrings, 4 * math.pi / rings.npix)
    a = oracle.analyze(rings, lmax, np.ones((1, rings.npix)), w)[0]
    assert a[0] == pytest.approx(math.sqrt(4 * math.pi), rel=1e-14)
    mcol = np.array([m for m in range(lmax + 1) for _ in range(m, lmax + 1)])
    assert np.abs(a[(mcol >= 1) & (mcol <= 3)]).max() < 1e-15


def test_analysis_jacobi_refinement_converges_on_healpix():
    """The HEALPix quadrature is not exact, but for L <= 2 nside each Jacobi
    step a <- a + A (f - Y a) shrinks the error of a band-limited round trip
    by a roughly constant factor; after 16 steps it is at rounding level."""
    nside = 8
    rings = oracle.healpix_rings(nside)
    w = np.full(rings.nrings, 4 * math.pi / rings.npix)
    for lmax in (8, 16):
        a = _random_alm(lmax, 1, 40 + lmax)
        f = oracle.synthesize(rings, lmax, a)
        err = [np.abs(oracle.analyze(rings, lmax, f, w, niter=k) - a).max() / np.abs(a).max()
               for k in (0, 1, 2, 4, 8, 16)]
        assert err[0] > 1e-3                        # plain quadrature: visibly inexact
        assert all(e1 < 0.2 * e0 for e0, e1 in zip(err[:-1], err[1:]) if e0 > 1e-13)
        assert err[-1] < 1e-14


def test_adjoint_dot_product_identity():
    """<Y a, f> = <a, Y^T f> with real inner products over (Re, Im) a_lm."""
    nside, lmax = 8, 16
    rings = oracle.healpix_rings(nside)
    a = _random_alm(lmax, 3, 21)
    f = np.random.default_rng(22).standard_normal((3, rings.npix))
    lhs = np.sum(oracle.synthesize(rings, lmax, a) * f)
    at = oracle.adjoint(rings, lmax, f)
    rhs = np.sum(a.real * at.real + a.imag * at.imag)
    assert lhs == pytest.approx(rhs, rel=1e-13)
    # Im a_l0 is ignored by synthesis, so the adjoint's Im a_l0 is zero
    m0 = [_alm_index(lmax, l, 0) for l in range(lmax + 1)]
    assert np.all(at[:, m0].imag == 0)


def test_adjoint_is_explicit_transpose():
    """Dense Y from synthesising every real unit coefficient; Y^T applied to
    random maps must equal the oracle's adjoint."""
    nside, lmax = 2, 5
    rings = oracle.healpix_rings(nside)
    n = oracle.nalm(lmax)
    cols, which = [], []
    for i in range(n):
        for part in (1.0, 1j):
            e = np.zeros(n, complex)
            e[i] = part
            cols.append(oracle.synthesize(rings, lmax, e)[0])
            which.append((i, part))
    Y = np.array(cols).T                      # npix x 2n
    f = np.random.default_rng(4).standard_normal((2, rings.npix))
    yt = f @ Y                                # 2 x 2n
    at = oracle.adjoint(rings, lmax, f)
    for c, (i, part) in enumerate(which):
        got = at[:, i].real if part == 1.0 else at[:, i].imag
        np.testing.assert_allclose(got, yt[:, c], atol=1e-13)


def test_legendre_stage_matches_full_synthesis_on_ring_subset():
    """Evaluating a subset of rings gives exactly those rings of the full map."""
    nside, lmax = 8, 16
    rings = oracle.healpix_rings(nside)
    a = _random_alm(lmax, 2, 31)
    full = oracle.synthesize(rings, lmax, a)
    idx = [0, 5, 15, 16, 30]
    sub = rings.subset(idx)
    part = oracle.synthesize(sub, lmax, a)
    want = np.concatenate([full[:, rings.start[k]:rings.start[k + 1]] for k in idx], axis=1)
    np.testing.assert_array_equal(part, want)


# ------------------------------------------------------ spin-weighted (s = +-2)
def test_spin_zero_is_the_scalar_legendre_function():
    """At s = 0 the spin-weighted function is Eq. (Y-def) with the
    Condon-Shortley phase: the Wigner-d route equals the scalar recurrence."""
    for z in (0.97, 0.3, -0.55, 0.999):
        for m in (0, 1, 2, 7, 20):
            want = oracle.legendre(m, 40, z)
            got = oracle.spin_lambda(0, m, 40, z)[m:]
            np.testing.assert_allclose(got, want, rtol=0, atol=1e-14 * max(1.0, np.abs(want).max()))


def test_spin_two_closed_forms():
    """l = 2 spin-2 harmonics, obtained by applying the spin-raising operator
    twice to Y_2m (Newman-Penrose convention):
    2Y_22 = sqrt(5/pi)/8 (1 - cos)^2, 2Y_21 = -sqrt(5/pi)/4 sin (1 - cos),
    2Y_20 = sqrt(15/(2 pi))/4 sin^2, 2Y_2,-2 = sqrt(5/pi)/8 (1 + cos)^2."""
    for th in (0.2, 0.7, 1.9, 2.8):
        z, s = math.cos(th), math.sin(th)
        want = {2: math.sqrt(5 / math.pi) / 8 * (1 - z) ** 2,
                1: -math.sqrt(5 / math.pi) / 4 * s * (1 - z),
                0: math.sqrt(15 / (2 * math.pi)) / 4 * s * s,
                -2: math.sqrt(5 / math.pi) / 8 * (1 + z) ** 2}
        for m, w in want.items():
            assert oracle.spin_lambda(2, m, 2, z)[2] == pytest.approx(w, rel=1e-14, abs=1e-16)


def _eth(f, s, m, th, h=1e-5):
    """Spin raising (Newman-Penrose): -(sin)^s [d/dth - m/sin] (sin^-s f)."""
    g = lambda t: f(t) / math.sin(t) ** s  # noqa: E731
    dg = (g(th + h) - g(th - h)) / (2 * h)
    return -(math.sin(th) ** s) * (dg - m / math.sin(th) * g(th))


def _eth_bar(f, s, m, th, h=1e-5):
    """Spin lowering: -(sin)^-s [d/dth + m/sin] (sin^s f)."""
    g = lambda t: f(t) * math.sin(t) ** s  # noqa: E731
    dg = (g(th + h) - g(th - h)) / (2 * h)
    return -(math.sin(th) ** (-s)) * (dg + m / math.sin(th) * g(th))


def test_spin_raising_and_lowering_relations():
    """(s+1)Y_lm = eth sY_lm / sqrt((l-s)(l+s+1)) and (s-1)Y_lm =
    -eth_bar sY_lm / sqrt((l+s)(l-s+1)), by central differences in theta:
    this fixes the sign convention of every spin relative to s = 0."""
    def lam(s, l, m):
        return lambda t: oracle.spin_lambda(s, m, l, math.cos(t), math.sin(t))[l]
    for th in (0.4, 1.3, 2.5):
        for l, m in ((3, 0), (4, 1), (5, 2), (6, -3), (7, 5), (9, -8)):
            for s in (0, 1):
                up = _eth(lam(s, l, m), s, m, th) / math.sqrt((l - s) * (l + s + 1))
                assert up == pytest.approx(lam(s + 1, l, m)(th), abs=1e-8)
            for s in (0, -1):
                dn = -_eth_bar(lam(s, l, m), s, m, th) / math.sqrt((l + s) * (l - s + 1))
                assert dn == pytest.approx(lam(s - 1, l, m)(th), abs=1e-8)


@pytest.mark.parametrize("s", [-2, -1, 1, 2])
def test_spin_addition_theorem(s):
    """sum_m |sY_lm|^2 = (2l+1)/(4 pi) for every spin weight."""
    lmax = 40
    for z in (0.999, 0.6, -0.2, -0.9):
        tot = np.zeros(lmax + 1)
        for m in range(-lmax, lmax + 1):
            tot += oracle.spin_lambda(s, m, lmax, z) ** 2
        ls = np.arange(abs(s), lmax + 1)
        np.testing.assert_allclose(tot[abs(s):], (2 * ls + 1) / (4 * math.pi), rtol=1e-13)


def test_spin_parity_and_negative_m():
    """s_lambda_lm(-z) = (-1)^(l+m) (-s)_lambda_lm(z) and
    s_lambda_l,-m = (-1)^(s+m) (-s)_lambda_lm."""
    lmax = 30
    for z in (0.8, 0.15):
        for m in (0, 1, 2, 5, 17):
            for s in (2, -2):
                a = oracle.spin_lambda(s, m, lmax, -z)
                b = oracle.spin_lambda(-s, m, lmax, z)
                sign = np.array([(-1) ** (l + m) for l in range(lmax + 1)])
                np.testing.assert_allclose(a, sign * b, atol=1e-15)
                c = oracle.spin_lambda(s, -m, lmax, z)
                np.testing.assert_allclose(c, (-1) ** (s + m) * b, atol=1e-15)


def test_spin_gauss_legendre_orthonormality():
    """2 pi sum_k w_k 2lambda_lm(z_k) 2lambda_l'm(z_k) = delta_ll' for
    2 <= l, l' <= L on L+1 Gauss-Legendre nodes (the products are
    polynomials of degree <= 2L in z)."""
    lmax = 16
    rings, w = oracle.gauss_legendre_rings(lmax + 1, 2 * lmax + 1)
    for m in range(0, lmax + 1):
        P = np.array([oracle.spin_lambda(2, m, lmax, z, s) for z, s in zip(rings.z, rings.sinth)])
        l0 = max(m, 2)
        G = 2 * math.pi * (P[:, l0:].T * w) @ P[:, l0:]
        np.testing.assert_allclose(G, np.eye(lmax + 1 - l0), atol=2e-14)


def test_polarised_single_modes_brute_force():
    """One coefficient at a time, pixel by pixel: a_E,lm = 1 gives
    Q = -2 F+ cos(m phi), U = -2 F- sin(m phi); a_B,lm = 1 gives
    Q = 2 F- sin(m phi), U = -2 F+ cos(m phi) (m >= 1; F+- = (2_lambda +-
    (-2)_lambda)/2); at m = 0, a_E,l0 = 1 gives Q = -F+, U = 0."""
    nside, lmax = 4, 8
    rings = oracle.healpix_rings(nside)
    z, phi = _expand(rings)
    for l, m in ((2, 0), (3, 1), (5, 2), (8, 7)):
        for which in ("E", "B"):
            aE = np.zeros(oracle.nalm(lmax), dtype=np.complex128)
            aB = np.zeros_like(aE)
            (aE if which == "E" else aB)[_alm_index(lmax, l, m)] = 1.0
            Q, U = oracle.spin_synthesize(rings, lmax, aE, aB)
            Fp = np.array([0.5 * (oracle.spin_lambda(2, m, lmax, zz)[l] + oracle.spin_lambda(-2, m, lmax, zz)[l])
                           for zz in z])
            Fm = np.array([0.5 * (oracle.spin_lambda(2, m, lmax, zz)[l] - oracle.spin_lambda(-2, m, lmax, zz)[l])
                           for zz in z])
            c = 1.0 if m == 0 else 2.0
            if which == "E":
                wantQ, wantU = -c * Fp * np.cos(m * phi), -c * Fm * np.sin(m * phi)
            else:
                wantQ, wantU = c * Fm * np.sin(m * phi), -c * Fp * np.cos(m * phi)
            np.testing.assert_allclose(Q[0], wantQ, atol=1e-14)
            np.testing.assert_allclose(U[0], wantU, atol=1e-14)


def test_polarised_rotation_of_e_into_b():
    """(a_E, a_B) -> (-a_B, a_E) multiplies Q + iU by i: (Q, U) -> (-U, Q)."""
    nside, lmax = 8, 16
    rings = oracle.healpix_rings(nside)
    aE = _random_alm(lmax, 2, 51)
    aB = _random_alm(lmax, 2, 52)
    Q, U = oracle.spin_synthesize(rings, lmax, aE, aB)
    Q2, U2 = oracle.spin_synthesize(rings, lmax, -aB, aE)
    np.testing.assert_allclose(Q2, -U, atol=1e-13)
    np.testing.assert_allclose(U2, Q, atol=1e-13)


def test_polarised_adjoint_dot_product_identity():
    """<Y_pol (a_E, a_B), (Q, U)> = <a_E, g_E> + <a_B, g_B> with real inner
    products over (Re, Im); Im of the m = 0 outputs is 0."""
    nside, lmax = 8, 16
    rings = oracle.healpix_rings(nside)
    aE = _random_alm(lmax, 2, 61)
    aB = _random_alm(lmax, 2, 62)
    rng = np.random.default_rng(63)
    Q = rng.standard_normal((2, rings.npix))
    U = rng.standard_normal((2, rings.npix))
    Qa, Ua = oracle.spin_synthesize(rings, lmax, aE, aB)
    gE, gB = oracle.spin_adjoint(rings, lmax, Q, U)
    lhs = np.sum(Qa * Q + Ua * U)
    rhs = np.sum(aE.real * gE.real + aE.imag * gE.imag + aB.real * gB.real + aB.imag * gB.imag)
    assert lhs == pytest.approx(rhs, rel=1e-13)
    m0 = [_alm_index(lmax, l, 0) for l in range(lmax + 1)]
    assert np.all(gE[:, m0].imag == 0) and np.all(gB[:, m0].imag == 0)


def test_polarised_adjoint_is_explicit_transpose():
    """Dense polarised operator from synthesising every real unit
    coefficient (Re and Im of a_E and a_B; Im a_l0 has no effect), compared
    with the adjoint applied to every unit pixel of Q and U."""
    nside, lmax = 2, 4
    rings = oracle.healpix_rings(nside)
    n = oracle.nalm(lmax)
    cols = []
    for field in range(2):
        for part in (1.0, 1j):
            for i in range(n):
                a = [np.zeros(n, dtype=np.complex128), np.zeros(n, dtype=np.complex128)]
                a[field][i] = part
                Q, U = oracle.spin_synthesize(rings, lmax, a[0], a[1])
                cols.append(np.concatenate([Q[0], U[0]]))
    Y = np.array(cols).T                      # [2 npix, 4 nalm]
    npix = rings.npix
    eye = np.eye(2 * npix)
    gE, gB = oracle.spin_adjoint(rings, lmax, eye[:, :npix], eye[:, npix:])
    YT = np.concatenate([gE.real, gE.imag, gB.real, gB.imag], axis=1)   # [2 npix, 4 nalm]
    m0 = np.array([m == 0 for m in range(lmax + 1) for _ in range(m, lmax + 1)])
    keep = np.concatenate([np.ones(n, bool), ~m0, np.ones(n, bool), ~m0])
    np.testing.assert_allclose(YT[:, keep], Y[:, keep], atol=1e-13)


def test_polarised_analysis_exact_on_gauss_legendre_grid():
    """On a Gauss-Legendre grid (L+1 rings, J = 2L+1) the quadrature is exact
    for the spin-2 harmonics too: spin_analyze recovers band-limited a_E, a_B
    (l >= 2; the l < 2 coefficients do not enter the maps and come back 0)."""
    lmax = 12
    rings, w = oracle.gauss_legendre_rings(lmax + 1, 2 * lmax + 1)
    aE = _random_alm(lmax, 2, 71)
    aB = _random_alm(lmax, 2, 72)
    lcol = np.array([l for m in range(lmax + 1) for l in range(m, lmax + 1)])
    aE[:, lcol < 2] = 0
    aB[:, lcol < 2] = 0
    Q, U = oracle.spin_synthesize(rings, lmax, aE, aB)
    gE, gB = oracle.spin_analyze(rings, lmax, Q, U, 2 * math.pi * w / rings.J)
    np.testing.assert_allclose(gE, aE, atol=5e-14)
    np.testing.assert_allclose(gB, aB, atol=5e-14)


def test_polarised_analysis_refinement_converges_on_healpix():
    nside, lmax = 8, 16
    rings = oracle.healpix_rings(nside)
    w = np.full(rings.nrings, 4 * math.pi / rings.npix)
    aE = _random_alm(lmax, 1, 73)
    aB = _random_alm(lmax, 1, 74)
    lcol = np.array([l for m in range(lmax + 1) for l in range(m, lmax + 1)])
    aE[:, lcol < 2] = 0
    aB[:, lcol < 2] = 0
    Q, U = oracle.spin_synthesize(rings, lmax, aE, aB)
    err = []
    for k in (0, 2, 4, 8, 16):
        gE, gB = oracle.spin_analyze(rings, lmax, Q, U, w, niter=k)
        err.append(max(np.abs(gE - aE).max(), np.abs(gB - aB).max()))
    assert err[0] > 1e-3
    assert all(e1 < 0.2 * e0 for e0, e1 in zip(err[:-1], err[1:]) if e0 > 1e-13)
    assert err[-1] < 1e-12
