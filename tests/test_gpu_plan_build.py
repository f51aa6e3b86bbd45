"""The GPU plan builder (gpu_build=True): its batched interpolative
decomposition against the host routine and the guarantees of Sec. 3.1, and
plans built with it against the oracle (Sec. 3.2 tolerance rules)."""
import numpy as np
import pytest

import oracle
from paper_1110_4874_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1110_4874_gb300 as sh  # noqa: E402


def rel_rms(x, y):
    x = np.asarray(x)
    y = np.asarray(y)
    return float(np.sqrt(np.sum(np.abs(x - y) ** 2) / np.sum(np.abs(x) ** 2)))


@pytest.mark.parametrize("rows,n,rank", [(60, 25, 7), (300, 64, 40), (1025, 32, 32), (5, 40, 5), (0, 8, 0)])
def test_gpu_id_matches_host_id(rows, n, rank):
    """Random matrices with well separated pivots: the same rank and skeleton
    as the host routine, and the same interpolation matrix to rounding."""
    rng = np.random.default_rng(rows + n)
    A = (rng.standard_normal((rows, rank)) * np.logspace(0, -6, rank)) @ rng.standard_normal((rank, n))
    A[:, 3] = 0.0                                      # a zero column
    kh, sh_, Th = sh.shtb_test_host_id(A, 1e-12)
    kg, sg, Tg = sh.shtb_test_gpu_id(A, 1e-12)
    assert kg == kh
    np.testing.assert_array_equal(sg, sh_)
    if kh:
        np.testing.assert_allclose(Tg, Th, rtol=0, atol=1e-9 * max(1.0, np.abs(Th).max()))
        assert np.abs(A - A[:, sg] @ Tg).max() <= 1e-10 * np.abs(A).max()


def test_gpu_id_on_legendre_blocks():
    """Blocks of the Legendre matrix: the GPU ID meets the ID error bound
    (Eq. ID-approximation) at the requested tolerance."""
    nside, lmax = 256, 512
    rings = oracle.healpix_rings(nside)
    for m, (r0, r1), (c0, c1) in [(0, (100, 356), (30, 94)), (200, (0, 120), (300, 364)), (10, (256, 512), (0, 64))]:
        P = np.array([oracle.legendre(m, lmax, rings.z[c], rings.sinth[c]) for c in range(c0, c1)]).T
        A = np.ascontiguousarray(P[r0:min(r1, P.shape[0])])
        for eps in (1e-6, 1e-10):
            k, skel, T = sh.shtb_test_gpu_id(A, eps)
            s = np.linalg.svd(A, compute_uv=False)
            err = np.linalg.norm(A - A[:, skel] @ T, 2)
            assert err <= np.sqrt(4 * k * (A.shape[1] - k) + 1) * max(s[k] if k < len(s) else 0.0,
                                                                      eps * s[0]) * 10


@pytest.mark.parametrize("nside,lmax,eps", [(64, 128, 1e-10), (32, 64, 1e-12), (13, 30, 1e-8)])
def test_gpu_built_plan_matches_oracle(nside, lmax, eps):
    gp = sh.Plan(nside, lmax, eps, gpu_build=True)
    hp = sh.Plan(nside, lmax, eps)
    rings = oracle.healpix_rings(nside)
    a = synthetic.gaussian_alm(lmax, 2, seed=910 + nside)
    want = oracle.synthesize(rings, lmax, a)
    got = gp.synthesize(torch.from_numpy(a).cuda()).cpu().numpy()
    tol = 1e-10 if eps <= 1e-12 else 100 * eps
    for b in range(2):
        assert rel_rms(want[b], got[b]) <= tol
    sg, sh_ = gp.stats(), hp.stats()
    for key in ("n_dense", "n_rstored", "n_ident"):
        assert abs(sg[key] - sh_[key]) <= 0.01 * max(sh_[key], 1), key
    f = torch.from_numpy(synthetic.gaussian_map(gp.npix, 2, seed=911)).cuda()
    at = gp.adjoint(f)
    x = torch.from_numpy(a).cuda()
    lhs = torch.sum(gp.synthesize(x) * f).item()
    rhs = torch.sum(x.real * at.real + x.imag * at.imag).item()
    assert lhs == pytest.approx(rhs, rel=1e-12)
    gp.close()
    hp.close()


def test_gpu_built_polarised_plan():
    nside, lmax, eps = 24, 48, 1e-10
    gp = sh.Plan(nside, lmax, eps, spin=2, gpu_build=True)
    rings = oracle.healpix_rings(nside)
    e = synthetic.gaussian_alm(lmax, 1, seed=920)
    b = synthetic.gaussian_alm(lmax, 1, seed=921)
    Q, U = oracle.spin_synthesize(rings, lmax, e, b)
    got = gp.synthesize_spin(torch.from_numpy(np.stack([e, b], axis=1)).cuda()).cpu().numpy()
    assert rel_rms(Q[0], got[0, 0]) <= 100 * eps and rel_rms(U[0], got[0, 1]) <= 100 * eps
    gp.close()
