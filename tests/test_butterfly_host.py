"""Host-side (no GPU) checks of the butterfly compression: the interpolative
decomposition against the guarantees of Sec. 3.1 (Eq. ID, Eq. ID-approximation),
and the compressed operator of Sec. 3.2 applied on the CPU against the dense
Legendre matrix built independently from the oracle."""
import math

import numpy as np
import pytest

import oracle
import paper_1110_4874_gb300 as sh


def test_id_exact_for_low_rank():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((60, 7)) @ rng.standard_normal((7, 25))
    k, skel, T = sh.shtb_test_host_id(A, 1e-13)
    assert k == 7
    np.testing.assert_array_equal(T[:, skel], np.eye(k))          # identity on the skeleton
    assert np.abs(A - A[:, skel] @ T).max() < 1e-12 * np.abs(A).max()


@pytest.mark.parametrize("eps", [1e-6, 1e-10, 1e-13])
def test_id_error_bound_on_legendre_blocks(eps):
    """||A - A[:, skel] T|| <= sqrt(4k(n-k)+1) sigma_{k+1} (Eq. ID-approximation)
    up to the truncation level, on blocks of the Legendre matrix."""
    nside, lmax = 256, 512
    rings = oracle.healpix_rings(nside)
    for m, rows, cols in [(0, (100, 356), (30, 94)), (200, (0, 120), (300, 364)),
                          (10, (256, 512), (0, 64))]:
        ls = np.arange(m, lmax + 1)[rows[0]:rows[1]]
        A = np.array([oracle.legendre(m, lmax, rings.z[c], rings.sinth[c], rings.zlo[c],
                                      rings.sinlo[c])[ls - m] for c in range(*cols)]).T
        k, skel, T = sh.shtb_test_host_id(A, eps)
        n = A.shape[1]
        s = np.linalg.svd(A, compute_uv=False)
        err = np.linalg.norm(A - A[:, skel] @ T, 2)
        bound = math.sqrt(4 * k * (n - k) + 1) * (s[k] if k < len(s) else 0.0)
        assert err <= max(bound, 0.0) + 4 * eps * s[0] * math.sqrt(n)
        assert err <= 4 * eps * s[0] * math.sqrt(n)
        # the truncated QR keeps the interpolation coefficients modest
        assert np.abs(T).max() < 50
        assert k <= min(A.shape)


def test_id_zero_and_empty_blocks():
    k, skel, T = sh.shtb_test_host_id(np.zeros((10, 5)), 1e-10)
    assert k == 0
    A = np.zeros((8, 4))
    A[:, 2] = np.arange(8)
    k, skel, T = sh.shtb_test_host_id(A, 1e-10)
    assert k == 1 and skel[0] == 2
    np.testing.assert_array_equal(T, [[0, 0, 1, 0]])


@pytest.mark.parametrize("nside,lmax,eps", [(128, 256, 1e-10), (256, 512, 1e-12),
                                            (512, 1024, 1e-8), (64, 200, 1e-10)])
def test_compressed_operator_matches_dense(nside, lmax, eps):
    rng = np.random.default_rng(nside)
    for m in [0, 1, lmax // 3, lmax // 2, lmax - 5, lmax]:
        for t in (0, 1):
            n = (lmax - m - t) // 2 + 1 if m + t <= lmax else 0
            if n == 0:
                continue
            a = rng.standard_normal(n) / (m + 2 * np.arange(n) + 1 + t)
            q, qe, info = sh.shtb_test_host_butterfly(nside, lmax, eps, m, t, a)
            # the dense product from the oracle's (independent) Legendre values
            rings = oracle.healpix_rings(nside)
            lam = np.array([oracle.legendre(m, lmax, rings.z[r], rings.sinth[r], rings.zlo[r],
                                            rings.sinlo[r])[t::2][:n] for r in range(2 * nside)])
            want = lam @ a
            scale = np.linalg.norm(want)
            assert np.linalg.norm(qe - want) <= 1e-12 * scale + 1e-300
            assert np.linalg.norm(q - want) <= 100 * eps * scale + 1e-300
            if info["depth"] > 0:
                assert info["n_dense"] + info["n_r"] < n * 2 * nside


def test_compression_shrinks_with_resolution():
    """The rank property (Sec. 3.2): the stored fraction of the m = 0 matrix
    falls as L grows at fixed eps."""
    fracs = []
    for nside, lmax in [(128, 256), (512, 1024), (1024, 2048)]:
        n = lmax // 2 + 1
        q, qe, info = sh.shtb_test_host_butterfly(nside, lmax, 1e-10, 0, 0, np.ones(n))
        fracs.append((info["n_dense"] + info["n_r"] + info["n_ident"]) / (n * 2 * nside))
    assert fracs[0] > fracs[1] > fracs[2]
    assert fracs[2] < 0.35


@pytest.mark.parametrize("nside,lmax", [(16, 40), (64, 128), (512, 1024)])
def test_spin_columns_match_the_oracle(nside, lmax):
    """The spin-plan builder's s_lambda_lm (s = +-2; Wigner recurrence in l)
    against the oracle's Wigner-d closed form.  Near the poles both
    characteristic roots of the recurrence meet, so its FP64 rounding grows
    with l there, as it does for the scalar columns (about 2e-11 at l = 1024
    on the first polar ring); away from the poles it stays near 1e-13."""
    rings = oracle.healpix_rings(nside)
    for r in sorted({0, 1, 2, nside // 2, nside - 1, nside, 2 * nside - 2, 2 * nside - 1}):
        for m in sorted({0, 1, 2, 3, 5, lmax // 3, lmax - 1, lmax}):
            for s in (2, -2):
                got = sh.shtb_test_host_spin_column(nside, lmax, m, s, r)
                want = oracle.spin_lambda(s, m, lmax, rings.z[r], rings.sinth[r])[m:]
                tol = 5e-11 if r < nside // 2 else 2e-12
                # the builder drops values below 1e-30 (Appendix crop)
                assert np.abs(got - want).max() <= tol * np.abs(want).max() + 1e-30, (r, m, s)


def test_id_invariants_on_legendre_blocks():
    """The ID guarantees of Sec. 3.1 on blocks of the Legendre matrix: the
    interpolation matrix [I | T] has every entry of modulus <= 2 (guaranteed
    for a strong rank-revealing QR; the column-pivoted QR used here meets it
    on these blocks with room to spare), smallest singular value >= 1, and
    spectral norm <= sqrt(4 k (n - k) + 1)."""
    nside, lmax = 256, 512
    rings = oracle.healpix_rings(nside)
    for m, (r0, r1), (c0, c1) in [(0, (100, 356), (30, 94)), (200, (0, 120), (300, 364)),
                                  (10, (256, 503), (0, 64)), (50, (0, 230), (200, 328))]:
        P = np.array([oracle.legendre(m, lmax, rings.z[c], rings.sinth[c]) for c in range(c0, c1)]).T
        A = np.ascontiguousarray(P[r0:min(r1, P.shape[0])])
        n = A.shape[1]
        for eps in (1e-6, 1e-10, 1e-13):
            k, skel, T = sh.shtb_test_host_id(A, eps)
            assert np.abs(T).max() <= 2.0
            s = np.linalg.svd(T, compute_uv=False)
            assert s[-1] >= 1.0 - 1e-12
            assert s[0] <= math.sqrt(4 * k * (n - k) + 1)


@pytest.mark.parametrize("nside,lmax", [(4, 8), (8, 12), (16, 20)])
def test_depth_zero_chains_are_the_dense_operator(nside, lmax):
    """Where compression does not pay, the chain keeps depth 0: its stored
    residual blocks are the dense Legendre matrix, and applying them equals
    the dense product up to the order of the sums."""
    seen = 0
    for m in range(lmax + 1):
        for t in (0, 1):
            n = (lmax - m - t) // 2 + 1
            if n <= 0:
                continue
            a = np.random.default_rng(100 * m + t).standard_normal(n)
            q, qe, info = sh.shtb_test_host_butterfly(nside, lmax, 1e-10, m, t, a)
            if info["depth"] == 0:
                seen += 1
                assert info["n_dense"] == 0 and info["n_ident"] == 0
                np.testing.assert_allclose(q, qe, rtol=0, atol=1e-15 * max(np.abs(qe).max(), 1e-300))
    assert seen > 0


# ---------------------------------------------- interpolation variant (Sec. 3.4)
@pytest.mark.parametrize("m,t", [(0, 0), (32, 1), (64, 0), (96, 1)])
def test_interpolation_from_the_roots_reproduces_the_rings(m, t):
    """Eq. interpolation: q at the roots of P_{m+t+2n}^m determines q at every
    half-ring (the chain spans polynomials of degree < n in y^2)."""
    nside, lmax = 64, 128
    n = (lmax - m - t) // 2 + 1
    a = np.random.default_rng(m + t).normal(size=n) / (m + t + 2 * np.arange(n) + 1)
    q, qe, info = sh.shtb_test_host_interp(nside, lmax, 1e-10, m, t, a)
    assert info["n"] == n
    assert info["rings_dense"] == n * 2 * nside
    assert info["two_step_dense"] == n * n + n * 2 * nside
    assert np.linalg.norm(q - qe) <= 1e-11 * np.linalg.norm(qe)


def test_interpolation_variant_stores_more_than_the_butterfly():
    """The measured reason the interpolation variant is not built: Lambda at
    the roots plus the interpolation matrix, each compressed as well as the
    plan's builder (or a hierarchical FMM-style compression) can, hold more
    elements -- so cost more FP64 FMAs per map -- than the butterfly of Lambda
    at the HEALPix half-rings (Nside=256, L=512, eps=1e-10)."""
    nside, lmax = 256, 512
    for m in (0, 128, 256, 384):
        for t in (0, 1):
            n = (lmax - m - t) // 2 + 1
            a = np.random.default_rng(m).normal(size=n)
            _, _, info = sh.shtb_test_host_interp(nside, lmax, 1e-10, m, t, a)
            two_step = info["roots_butterfly"] + min(info["interp_butterfly"], info["interp_hierarchical"])
            assert two_step > info["rings_butterfly"], (m, t, info)


@pytest.mark.parametrize("nside,lmax,eps,m,t,bound", [
    (64, 128, 1e-10, 0, 0, 1e-13), (256, 512, 1e-12, 200, 1, 1e-13),
    (512, 1024, 1e-10, 0, 1, 2e-12), (512, 1024, 1e-10, 900, 1, 1e-13),
    (2048, 4096, 1e-10, 0, 0, 2e-11), (2048, 4096, 1e-10, 1000, 1, 2e-12)])
def test_regenerated_residual_blocks_match_the_stored_ones(nside, lmax, eps, m, t, bound):
    """Residual blocks rebuilt from the two recurrence start values per
    (block, column) that residual_recurrence plans keep (Eq. three-term,
    stepped as the kernel steps it) reproduce the stored blocks: same 1e-30
    crop, and the FP64 recurrence's rounding only (it grows with the chain
    length, to ~6e-12 of a column's largest value for m = 0 at L = 4096)."""
    err, info = sh.shtb_test_host_rec_blocks(nside, lmax, eps, m, t)
    assert info["blocks"] > 0 and info["elements"] > 0
    assert info["crop_mismatch"] == 0
    assert err <= bound
