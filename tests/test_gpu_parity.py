"""GPU parity of the CUDA path against the CPU oracle, stage by stage and end
to end, through the C ABI (the Python binding only marshals arguments).

Tolerances (relative RMS over all pixels / coefficients, Eq. relative-error):
uncompressed synthesis and adjoint <= 1e-12 (the FP64 recurrence and FFT
error is ~1e-15 * sqrt(L) away from the poles and the equator); single stages
of pure FFT arithmetic <= 1e-13 of the largest value.
"""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def plans():
    cache = {}

    def get(nside, lmax):
        if (nside, lmax) not in cache:
            cache[(nside, lmax)] = sh.Plan(nside, lmax, 0.0)
        return cache[(nside, lmax)]

    yield get
    for p in cache.values():
        p.close()


# (nside, lmax): powers of two (radix-2 rings) and odd sizes (Bluestein rings,
# ragged last warp of half-rings), L above and below 2*nside
CASES = [(32, 64), (16, 48), (6, 20), (13, 30), (64, 100), (8, 3)]


def test_fp64_peak_runs():
    dfma, dmma = sh.shtb_measure_fp64_peak(0)
    print(f"DFMA {dfma:.1f} GFLOP/s, DMMA {dmma:.1f} GFLOP/s")
    assert dfma > 0 and dmma > 0


@pytest.mark.parametrize("nside,lmax", CASES)
def test_phi_stage(plans, nside, lmax):
    p = plans(nside, lmax)
    rings = oracle.healpix_rings(nside)
    rng = np.random.default_rng(nside * 100 + lmax)
    q = rng.standard_normal((2, rings.nrings, lmax + 1)) + 1j * rng.standard_normal(
        (2, rings.nrings, lmax + 1))
    q[:, :, 0] = q[:, :, 0].real
    want = oracle.phi_synth(rings, lmax, q)
    out = torch.empty((2, rings.npix), dtype=torch.float64, device="cuda")
    sh.shtb_test_phi(p.handle, dev(q), out, 2)
    got = out.cpu().numpy()
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("nside,lmax", CASES)
def test_phi_adjoint_stage(plans, nside, lmax):
    p = plans(nside, lmax)
    rings = oracle.healpix_rings(nside)
    f = synthetic.gaussian_map(rings.npix, 2, seed=nside + lmax)
    want = oracle.phi_adjoint(rings, lmax, f)
    out = torch.empty((2, rings.nrings, lmax + 1), dtype=torch.complex128, device="cuda")
    sh.shtb_test_phi_adjoint(p.handle, dev(f), out, 2)
    got = out.cpu().numpy()
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("nside,lmax", CASES)
def test_legendre_stage(plans, nside, lmax):
    p = plans(nside, lmax)
    rings = oracle.healpix_rings(nside)
    a = synthetic.gaussian_alm(lmax, 3, seed=7)
    want = oracle.legendre_q(rings, lmax, a)
    out = torch.empty((3, rings.nrings, lmax + 1), dtype=torch.complex128, device="cuda")
    sh.shtb_test_legendre(p.handle, dev(a), out, 3)
    got = out.cpu().numpy()
    assert rel_rms(want, got) <= 1e-13


@pytest.mark.parametrize("nside,lmax", CASES)
def test_legendre_adjoint_stage(plans, nside, lmax):
    p = plans(nside, lmax)
    rings = oracle.healpix_rings(nside)
    rng = np.random.default_rng(3)
    F = rng.standard_normal((2, rings.nrings, lmax + 1)) + 1j * rng.standard_normal(
        (2, rings.nrings, lmax + 1))
    want = oracle.legendre_adjoint(rings, lmax, F)
    out = torch.empty((2, oracle.nalm(lmax)), dtype=torch.complex128, device="cuda")
    sh.shtb_test_legendre_adjoint(p.handle, dev(F), out, 2)
    got = out.cpu().numpy()
    assert rel_rms(want, got) <= 1e-13


@pytest.mark.parametrize("nside,lmax", CASES + [(128, 256)])
def test_synthesis_end_to_end(plans, nside, lmax):
    p = plans(nside, lmax)
    rings = oracle.healpix_rings(nside)
    a = synthetic.gaussian_alm(lmax, 2, seed=1000 * nside + lmax)
    want = oracle.synthesize(rings, lmax, a)
    got = p.synthesize(dev(a)).cpu().numpy()
    for b in range(2):
        assert rel_rms(want[b], got[b]) <= 1e-12


@pytest.mark.parametrize("nside,lmax", CASES + [(128, 256)])
def test_adjoint_end_to_end(plans, nside, lmax):
    p = plans(nside, lmax)
    rings = oracle.healpix_rings(nside)
    f = synthetic.gaussian_map(rings.npix, 2, seed=nside)
    want = oracle.adjoint(rings, lmax, f)
    got = p.adjoint(dev(f)).cpu().numpy()
    for b in range(2):
        assert rel_rms(want[b], got[b]) <= 1e-12


@pytest.mark.parametrize("nmaps", [1, 2, 3, 5, 8, 11, 16])
def test_map_batches_match_single_maps(plans, nmaps):
    """Every map of a batch (all map-group widths 8/4/2/1) equals the same map
    transformed alone, bit for bit (same per-map arithmetic order)."""
    p = plans(32, 64)
    a = dev(synthetic.gaussian_alm(64, nmaps, seed=nmaps))
    batch = p.synthesize(a)
    for b in range(nmaps):
        single = p.synthesize(a[b:b + 1])
        assert torch.equal(batch[b], single[0])
    f = dev(synthetic.gaussian_map(p.npix, nmaps, seed=nmaps))
    batch = p.adjoint(f)
    for b in range(nmaps):
        assert torch.equal(batch[b], p.adjoint(f[b:b + 1])[0])


def test_dot_product_identity(plans):
    """<Y a, f> = <a, Y^T f> with both sides computed by the CUDA path."""
    p = plans(64, 128)
    a = dev(synthetic.gaussian_alm(128, 3, seed=11))
    f = dev(synthetic.gaussian_map(p.npix, 3, seed=12))
    lhs = torch.sum(p.synthesize(a) * f).item()
    at = p.adjoint(f)
    rhs = torch.sum(a.real * at.real + a.imag * at.imag).item()
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_host_buffer_variants(plans):
    p = plans(32, 64)
    a = synthetic.gaussian_alm(64, 2, seed=5)
    ah = torch.from_numpy(a).pin_memory()
    mh = torch.empty((2, p.npix), dtype=torch.float64).pin_memory()
    sh.shtb_synthesize_host(p.handle, ah, mh, 2)
    torch.cuda.synchronize()
    dev_out = p.synthesize(dev(a)).cpu()
    assert torch.equal(mh, dev_out)
    back = torch.empty((2, p.nalm), dtype=torch.complex128).pin_memory()
    sh.shtb_adjoint_host(p.handle, mh, back, 2)
    assert torch.equal(back, p.adjoint(mh.cuda()).cpu())


def test_error_paths(plans):
    p = plans(8, 16)
    a = torch.zeros((1, p.nalm), dtype=torch.complex128, device="cuda")
    m = torch.zeros((1, p.npix), dtype=torch.float64, device="cuda")
    with pytest.raises(sh.ShtbError) as e:
        sh.shtb_synthesize(p.handle, a, m, 0)
    assert e.value.code == sh.SHTB_EINVAL
    with pytest.raises(sh.ShtbError) as e:
        sh.shtb_plan_create(0, 16)
    assert e.value.code == sh.SHTB_EINVAL
    with pytest.raises(sh.ShtbError) as e:
        sh.shtb_plan_create(8, -1)
    assert e.value.code == sh.SHTB_EINVAL
    with pytest.raises(sh.ShtbError) as e:
        sh.shtb_plan_create(8, 16, float("nan"))
    assert e.value.code == sh.SHTB_EINVAL
