"""Parity at the configured full sizes, in the launch configuration bench.py
times (one synthesize call over all maps of a plan), on outputs the oracle can
compute one by one: whole rings sampled at both poles, the equator, the
polar-cap / belt boundaries and at random in between.  Rule of the other
parity tests (Eq. relative-error over the sampled pixels): <= 1e-10 at
eps = 1e-12, <= 100 eps otherwise.  The adjoint is checked at full size by the
dot-product identity <Y a, f> = <a, Y^T f>, which holds at any size."""
import numpy as np
import pytest

import oracle
from paper_1110_4874_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1110_4874_gb300 as sh  # noqa: E402


def rel_rms(x, y):
    return float(np.sqrt(np.sum((x - y) ** 2) / np.sum(x ** 2)))


def ring_sample(nside, n):
    nr = 4 * nside - 1
    fixed = [0, 1, 2, nside - 2, nside - 1, nside, 2 * nside - 2, 2 * nside - 1, 2 * nside,
             3 * nside - 1, 3 * nside, nr - 3, nr - 2, nr - 1]
    rest = np.setdiff1d(np.arange(nr), fixed)
    extra = np.random.default_rng(nside).choice(rest, n - len(fixed), replace=False)
    return np.unique(np.concatenate([fixed, extra]))


def check_rings(nside, lmax, eps, a, maps, which, nrings):
    rings = oracle.healpix_rings(nside)
    idx = ring_sample(nside, nrings)
    want = oracle.synthesize(rings.subset(idx), lmax, a[which])
    maps = maps.cpu().numpy()
    got = np.concatenate([maps[:, rings.start[k]:rings.start[k] + rings.J[k]] for k in idx], axis=1)
    tol = 1e-10 if eps <= 1e-12 else 100 * eps
    for i, b in enumerate(which):
        assert rel_rms(want[i], got[b]) <= tol, (b, rel_rms(want[i], got[b]))


@pytest.mark.parametrize("eps", [1e-10, 1e-12])
def test_nside512_one_and_sixteen_maps(eps):
    """Nside=512, L=1024, 1 map and 16 maps sharing one plan."""
    nside, lmax = 512, 1024
    plan = sh.Plan(nside, lmax, eps)
    for nmaps in (1, 16):
        a = synthetic.gaussian_alm(lmax, nmaps, seed=1000 + nmaps)
        maps = plan.synthesize(torch.from_numpy(a).cuda())
        check_rings(nside, lmax, eps, a, maps, sorted({0, nmaps - 1}), 40)
    plan.close()


@pytest.fixture(scope="module")
def planck_plan():
    # built by the GPU plan builder, as bench.py builds it
    plan = sh.Plan(2048, 4096, 1e-10, gpu_build=True)
    yield plan
    plan.close()


def test_nside2048_batch_of_eight(planck_plan):
    """Nside=2048, L=4096, eps=1e-10, 8 maps in one call (the benchmark's
    workload), maps 0 and 7 on a 24-ring sample."""
    a = synthetic.gaussian_alm(4096, 8, seed=2048)
    maps = planck_plan.synthesize(torch.from_numpy(a).cuda())
    check_rings(2048, 4096, 1e-10, a, maps, [0, 7], 24)


def test_nside2048_dot_product_identity(planck_plan):
    a = torch.from_numpy(synthetic.gaussian_alm(4096, 2, seed=2049)).cuda()
    f = torch.from_numpy(synthetic.gaussian_map(planck_plan.npix, 2, seed=2050)).cuda()
    ya = planck_plan.synthesize(a)
    ytf = planck_plan.adjoint(f)
    lhs = float((ya * f).sum())
    rhs = float((a.conj() * ytf).real.sum())
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)
