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


@pytest.mark.parametrize("nmaps,pinned", [(11, True), (3, False)])
def test_host_buffer_synthesis_compressed(nmaps, pinned):
    """Compressed plans copy the maps back ring chunk by ring chunk while the
    ring stage runs: the host result equals the device-buffer call bit for
    bit, for map groups of 8 + 2 + 1 and for pageable host memory."""
    p = sh.Plan(64, 128, 1e-10)
    a = synthetic.gaussian_alm(128, nmaps, seed=15)
    ah = torch.from_numpy(a)
    mh = torch.full((nmaps, p.npix), float("nan"), dtype=torch.float64)
    if pinned:
        ah, mh = ah.pin_memory(), mh.pin_memory()
    sh.shtb_synthesize_host(p.handle, ah, mh, nmaps)
    torch.cuda.synchronize()
    assert torch.equal(mh, p.synthesize(dev(a)).cpu())
    p.close()


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


# ------------------------------------------------------------ compressed plans
COMPRESSED = [(32, 64, 1e-12), (128, 256, 1e-10), (64, 100, 1e-10), (13, 30, 1e-8),
              (256, 512, 1e-12), (16, 48, 1e-6)]


@pytest.mark.parametrize("nside,lmax,eps", COMPRESSED)
def test_compressed_synthesis_vs_oracle(nside, lmax, eps):
    """Butterfly-compressed synthesis (Sec. 3.2) within the tolerance rule:
    <= 1e-10 relative RMS at eps = 1e-12, <= 100 eps otherwise."""
    plan = sh.Plan(nside, lmax, eps)
    st = plan.stats()
    assert st["compressed"] == 1
    rings = oracle.healpix_rings(nside)
    a = synthetic.gaussian_alm(lmax, 3, seed=77)
    want = oracle.synthesize(rings, lmax, a)
    got = plan.synthesize(dev(a)).cpu().numpy()
    tol = 1e-10 if eps <= 1e-12 else 100 * eps
    for b in range(3):
        assert rel_rms(want[b], got[b]) <= tol
    plan.close()


@pytest.mark.parametrize("nside,lmax,eps", [(32, 64, 1e-12), (64, 100, 1e-10), (13, 30, 1e-8)])
def test_compressed_legendre_stage_parity_halves(nside, lmax, eps):
    """shtb_test_butterfly: residual blocks and butterfly levels alone give
    the parity halves q^0, q^1 on the half-rings (Eq. q-even-odd2); against
    the oracle's q_m(z) on a ring and its mirror, (q(z) + q(-z))/2 and
    (q(z) - q(-z))/2, within the compression tolerance."""
    plan = sh.Plan(nside, lmax, eps)
    Z = 2 * nside
    rings = oracle.healpix_rings(nside)
    a = synthetic.gaussian_alm(lmax, 2, seed=91)
    q = oracle.legendre_q(rings, lmax, a)                     # [b, nrings, L+1]
    nr = 4 * nside - 1
    north = q[:, :Z, :]
    south = q[:, [nr - 1 - r if r < Z - 1 else r for r in range(Z)], :]   # mirror (equator itself)
    want = np.stack([(north + south) / 2, (north - south) / 2], axis=1)    # [b, 2, Z, L+1]
    want[:, 1, Z - 1, :] = 0.0                                # odd parity vanishes on the equator
    qt = torch.empty((2, 2, Z, lmax + 1), dtype=torch.complex128, device="cuda")
    sh.shtb_test_butterfly(plan.handle, dev(a), qt, 2)
    got = qt.cpu().numpy()
    tol = 1e-10 if eps <= 1e-12 else 100 * eps
    scale = np.sqrt(np.mean(np.abs(want) ** 2))
    assert np.sqrt(np.mean(np.abs(got - want) ** 2)) <= tol * scale
    assert np.all(got[:, 1, :, lmax] == 0)                     # chain (m = L, t = 1) is empty
    plan.close()


def test_butterfly_stage_needs_compressed_plan():
    plan = sh.Plan(8, 16, 0.0)
    a = torch.zeros((1, plan.nalm), dtype=torch.complex128, device="cuda")
    qt = torch.empty((1, 2, 16, 17), dtype=torch.complex128, device="cuda")
    with pytest.raises(sh.ShtbError) as e:
        sh.shtb_test_butterfly(plan.handle, a, qt, 1)
    assert e.value.code == sh.SHTB_ENOTSUP
    plan.close()


def test_compressed_batches_match_single_maps():
    plan = sh.Plan(64, 128, 1e-10)
    a = dev(synthetic.gaussian_alm(128, 11, seed=3))
    batch = plan.synthesize(a)
    for b in range(11):
        assert torch.equal(batch[b], plan.synthesize(a[b:b + 1])[0])
    plan.close()


def test_compressed_stats_count_less_work_than_dense():
    plan = sh.Plan(256, 512, 1e-10)
    st = plan.stats()
    dense = sh.Plan(256, 512, 0.0).stats()
    assert st["n_dense"] + st["n_rstored"] > 0
    assert st["legendre_flops_per_map"] < dense["legendre_flops_per_map"]
    assert sum(st["depth_hist"]) == 2 * 513
    plan.close()


# ------------------------------------------------------------ differentiation
def test_autograd_matches_central_differences():
    """loss = 0.5 ||Y a - d||^2 (the data model of Eq. datamodel): the gradient
    from torch.autograd, whose backward is the adjoint kernel, equals central
    finite differences; the loss is quadratic, so central differences are exact
    up to rounding."""
    nside, lmax = 16, 32
    plan = sh.Plan(nside, lmax, 0.0)
    a_true = dev(synthetic.gaussian_alm(lmax, 1, seed=4100))[0]
    a0 = dev(synthetic.gaussian_alm(lmax, 1, seed=4000))[0]
    d = plan.synthesize(a_true) + 0.1 * dev(synthetic.gaussian_map(plan.npix, 1, seed=4200))[0]
    a = a0.clone().requires_grad_(True)
    loss = 0.5 * torch.sum((sh.synthesize(a, plan) - d) ** 2)
    loss.backward()
    g = a.grad.detach()
    m0 = torch.tensor(synthetic.m_of_index(lmax) == 0, device="cuda")
    assert torch.all(g.imag[m0] == 0)

    def L(x):
        return 0.5 * torch.sum((plan.synthesize(x) - d) ** 2).item()

    rng = np.random.default_rng(5)
    h = 1e-4 * torch.linalg.norm(a0).item()
    for _ in range(4):
        v = dev(rng.standard_normal(plan.nalm) + 1j * rng.standard_normal(plan.nalm))
        v = torch.where(m0, v.real.to(v.dtype), v)
        fd = (L(a0 + h * v) - L(a0 - h * v)) / (2 * h)
        an = torch.sum(g.real * v.real + g.imag * v.imag).item()
        assert an == pytest.approx(fd, rel=1e-9)
    plan.close()


@pytest.mark.parametrize("nside,lmax,eps", COMPRESSED)
def test_compressed_adjoint_vs_oracle(nside, lmax, eps):
    """Transposed butterfly: Y^T f within the same tolerance rule."""
    plan = sh.Plan(nside, lmax, eps)
    rings = oracle.healpix_rings(nside)
    f = synthetic.gaussian_map(rings.npix, 2, seed=78)
    want = oracle.adjoint(rings, lmax, f)
    got = plan.adjoint(dev(f)).cpu().numpy()
    tol = 1e-10 if eps <= 1e-12 else 100 * eps
    for b in range(2):
        assert rel_rms(want[b], got[b]) <= tol
    plan.close()


@pytest.mark.parametrize("nside,lmax,eps", [(64, 128, 1e-10), (13, 30, 1e-6), (128, 256, 1e-12)])
def test_compressed_adjoint_is_exact_transpose(nside, lmax, eps):
    """The compressed adjoint is the transpose of the compressed synthesis:
    <Y a, f> = <a, Y^T f> to rounding, whatever eps."""
    plan = sh.Plan(nside, lmax, eps)
    a = dev(synthetic.gaussian_alm(lmax, 3, seed=21))
    f = dev(synthetic.gaussian_map(plan.npix, 3, seed=22))
    lhs = torch.sum(plan.synthesize(a) * f).item()
    at = plan.adjoint(f)
    rhs = torch.sum(a.real * at.real + a.imag * at.imag).item()
    assert lhs == pytest.approx(rhs, rel=1e-12)
    # batches equal single maps
    for b in range(3):
        assert torch.equal(at[b], plan.adjoint(f[b:b + 1])[0])
    plan.close()
