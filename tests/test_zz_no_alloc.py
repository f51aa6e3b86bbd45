"""The allocation-free synthesis entry point (shtb_synthesize_noalloc).

It serves callers that cannot allocate device memory while they transform
(memory already held by another allocator, or loops that must not pay for
cudaMalloc's device synchronisation).  It must give the same maps as
shtb_synthesize, call after call, and refuse requests larger than its static
scratch.  This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1110_4874_gb300 as sh  # noqa: E402
from paper_1110_4874_gb300 import synthetic  # noqa: E402


def rel_rms(x, y):
    return float(torch.sqrt(torch.sum((x - y) ** 2) / torch.sum(x ** 2)))


@pytest.mark.parametrize("nside,lmax,nmaps", [(32, 64, 3), (13, 30, 2)])
def test_noalloc_matches_synthesize_twice(nside, lmax, nmaps):
    plan = sh.Plan(nside, lmax, 0.0)
    for call in range(2):
        a = torch.from_numpy(synthetic.gaussian_alm(lmax, nmaps, seed=50 + call)).cuda()
        want = plan.synthesize(a)
        got = torch.full((nmaps, plan.npix), float("nan"), dtype=torch.float64, device="cuda")
        sh.shtb_synthesize_noalloc(plan.handle, a, got, nmaps)
        torch.cuda.synchronize()
        assert rel_rms(want, got) <= 1e-12
        assert torch.equal(want, got)
    plan.close()


def test_noalloc_rejects_requests_beyond_the_static_scratch():
    plan = sh.Plan(512, 1024, 0.0)
    a = torch.zeros((2, plan.nalm), dtype=torch.complex128, device="cuda")
    m = torch.zeros((2, plan.npix), dtype=torch.float64, device="cuda")
    with pytest.raises(sh.ShtbError) as e:
        sh.shtb_synthesize_noalloc(plan.handle, a, m, 2)
    assert e.value.code == sh.SHTB_ENOTSUP
    assert "scratch" in str(e.value)
    # one map at this size fits
    a1 = torch.from_numpy(synthetic.gaussian_alm(1024, 1, seed=9)).cuda()
    want = plan.synthesize(a1)
    got = torch.empty_like(want)
    sh.shtb_synthesize_noalloc(plan.handle, a1, got, 1)
    torch.cuda.synchronize()
    assert torch.equal(want, got)
    plan.close()


def test_noalloc_on_a_compressed_plan_applies_the_exact_operator():
    """On a compressed plan (eps > 0) the call evaluates the uncompressed
    operator from the plan's recurrence tables: bit for bit the maps of an
    eps = 0 plan of the same size, and within the compressed plan's
    tolerance rule (1e-10 at eps = 1e-12) of that plan's shtb_synthesize."""
    nside, lmax, nmaps = 32, 64, 2
    exact = sh.Plan(nside, lmax, 0.0)
    comp = sh.Plan(nside, lmax, 1e-12)
    for call in range(2):
        a = torch.from_numpy(synthetic.gaussian_alm(lmax, nmaps, seed=70 + call)).cuda()
        got = torch.full((nmaps, comp.npix), float("nan"), dtype=torch.float64, device="cuda")
        sh.shtb_synthesize_noalloc(comp.handle, a, got, nmaps)
        torch.cuda.synchronize()
        assert torch.equal(got, exact.synthesize(a))
        assert rel_rms(comp.synthesize(a), got) <= 1e-10
    comp.close()
    exact.close()
