"""Degenerate sizes through the C ABI against the oracle: the smallest grid
(Nside=1, 12 pixels), band limits 0 and 1, band limits far above the ring
lengths (heavy wrapping in Eq. tau), odd resolutions, compressed plans too
small to compress, and polarised plans whose band limit has no l >= 2
term."""
import numpy as np
import pytest

import oracle
from paper_1110_4874_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1110_4874_gb300 as sh  # noqa: E402


def rel_rms(x, y):
    x = np.asarray(x).view(np.float64) if np.iscomplexobj(x) else np.asarray(x)
    y = np.asarray(y).view(np.float64) if np.iscomplexobj(y) else np.asarray(y)
    den = np.sum(x ** 2)
    return float(np.sqrt(np.sum((x - y) ** 2) / den)) if den > 0 else float(np.abs(y).max())


EDGE = [(1, 0, 0.0), (1, 1, 0.0), (1, 4, 0.0), (2, 0, 0.0), (4, 40, 0.0), (3, 17, 0.0),
        (1, 4, 1e-10), (2, 8, 1e-12), (4, 40, 1e-10), (5, 2, 1e-10)]


@pytest.mark.parametrize("nside,lmax,eps", EDGE)
def test_degenerate_synthesis_and_adjoint(nside, lmax, eps):
    plan = sh.Plan(nside, lmax, eps)
    rings = oracle.healpix_rings(nside)
    a = synthetic.gaussian_alm(lmax, 2, seed=40 + nside + lmax)
    tol = 1e-12 if eps <= 0 else (1e-10 if eps <= 1e-12 else 100 * eps)
    got = plan.synthesize(torch.from_numpy(a).cuda()).cpu().numpy()
    want = oracle.synthesize(rings, lmax, a)
    for b in range(2):
        assert rel_rms(want[b], got[b]) <= tol
    f = synthetic.gaussian_map(rings.npix, 2, seed=41)
    gA = plan.adjoint(torch.from_numpy(f).cuda()).cpu().numpy()
    wA = oracle.adjoint(rings, lmax, f)
    for b in range(2):
        assert rel_rms(wA[b], gA[b]) <= tol
    plan.close()


@pytest.mark.parametrize("nside,lmax,eps", [(1, 4, 0.0), (2, 8, 1e-10), (3, 1, 0.0), (2, 1, 1e-10)])
def test_degenerate_polarised(nside, lmax, eps):
    """lmax = 1 has no l >= 2 term: the Q and U maps are exactly zero."""
    plan = sh.Plan(nside, lmax, eps, spin=2)
    rings = oracle.healpix_rings(nside)
    e = synthetic.gaussian_alm(lmax, 1, seed=50)
    b = synthetic.gaussian_alm(lmax, 1, seed=51)
    got = plan.synthesize_spin(torch.from_numpy(np.stack([e, b], axis=1)).cuda()).cpu().numpy()
    Q, U = oracle.spin_synthesize(rings, lmax, e, b)
    if lmax < 2:
        assert np.all(got == 0.0)
    else:
        tol = 1e-12 if eps <= 0 else 100 * eps
        assert rel_rms(Q[0], got[0, 0]) <= tol and rel_rms(U[0], got[0, 1]) <= tol
    plan.close()


@pytest.mark.parametrize("nside,lmax", [(1, 2), (2, 4)])
def test_degenerate_analysis(nside, lmax):
    plan = sh.Plan(nside, lmax, 0.0)
    rings = oracle.healpix_rings(nside)
    f = synthetic.gaussian_map(rings.npix, 1, seed=60)
    w = np.full(rings.nrings, 4 * np.pi / rings.npix)
    want = oracle.analyze(rings, lmax, f, w, niter=2)
    got = plan.analyze(torch.from_numpy(f).cuda(), niter=2).cpu().numpy()
    assert rel_rms(want[0], got[0]) <= 1e-12
    plan.close()
