"""Plans that regenerate their residual blocks (residual_recurrence): each
block's R = Lambda[I, skeleton] comes from the jump-two recurrence of
Eq. (three-term) started from two stored values per (block, column), as
Sec. 3.3 describes, instead of being stored.  Synthesis and adjoint against
the oracle at the same rule as stored plans and against the stored plan of
the same operator, bit-identical map grouping, plan files, and the calls such
plans refuse.
"""
import os

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


@pytest.mark.parametrize("nside,lmax,eps", [(32, 64, 1e-12), (64, 100, 1e-10), (13, 30, 1e-8),
                                            (128, 256, 1e-10)])
def test_regenerated_synthesis_vs_oracle(nside, lmax, eps):
    """<= 1e-10 relative RMS at eps = 1e-12, <= 100 eps otherwise, as for
    stored plans; the ragged sizes (13, 30) take Bluestein rings."""
    plan = sh.Plan(nside, lmax, eps, residual_recurrence=True)
    st = plan.stats()
    assert st["compressed"] == 1 and st["n_rstored"] == 0 and st["n_rgen"] > 0
    rings = oracle.healpix_rings(nside)
    a = synthetic.gaussian_alm(lmax, 3, seed=78)
    want = oracle.synthesize(rings, lmax, a)
    got = plan.synthesize(dev(a)).cpu().numpy()
    tol = 1e-10 if eps <= 1e-12 else 100 * eps
    for b in range(3):
        assert rel_rms(want[b], got[b]) <= tol
    plan.close()


def test_regenerated_equals_stored_operator():
    """The same compressed operator with stored and with regenerated residual
    blocks: the maps differ only by the recurrence's rounding, and the
    regenerated plan holds less memory with as many regenerated elements as
    the stored plan stores."""
    nside, lmax, eps = 128, 256, 1e-10
    stored = sh.Plan(nside, lmax, eps)
    regen = sh.Plan(nside, lmax, eps, residual_recurrence=True)
    s0, s1 = stored.stats(), regen.stats()
    assert s1["n_rgen"] == s0["n_rstored"]
    assert s1["n_dense"] == s0["n_dense"]
    assert s1["plan_device_bytes"] < s0["plan_device_bytes"]
    a = dev(synthetic.gaussian_alm(lmax, 4, seed=79))
    m0 = stored.synthesize(a).cpu().numpy()
    m1 = regen.synthesize(a).cpu().numpy()
    for b in range(4):
        assert rel_rms(m0[b], m1[b]) <= 1e-12
    stored.close()
    regen.close()


def test_regenerated_batches_match_single_maps():
    """Map groups of 8, 2 and 1 give the same bits as one map per call: every
    column's recurrence and every dot product run in the same order at any
    group width."""
    plan = sh.Plan(64, 128, 1e-10, residual_recurrence=True)
    a = dev(synthetic.gaussian_alm(128, 11, seed=5))
    batch = plan.synthesize(a)
    for b in range(11):
        assert torch.equal(batch[b], plan.synthesize(a[b:b + 1])[0])
    plan.close()


def test_regenerated_host_buffers_and_plan_file(tmp_path):
    """Host-buffer synthesis equals the device call; a plan file keeps the
    option and the start values, and the loaded plan gives the same bits."""
    plan = sh.Plan(32, 64, 1e-10, residual_recurrence=True)
    a = synthetic.gaussian_alm(64, 3, seed=6)
    want = plan.synthesize(dev(a))
    out = torch.zeros((3, plan.npix), dtype=torch.float64)
    sh.shtb_synthesize_host(plan.handle, torch.from_numpy(a), out, 3)
    assert torch.equal(out, want.cpu())
    path = os.path.join(tmp_path, "regen.plan")
    plan.save(path)
    again = sh.Plan.load(path)
    assert again.stats()["n_rgen"] == plan.stats()["n_rgen"]
    assert torch.equal(again.synthesize(dev(a)), want)
    again.close()
    plan.close()


@pytest.mark.parametrize("nside,lmax,eps", [(32, 64, 1e-12), (13, 30, 1e-8), (64, 128, 1e-10)])
def test_regenerated_adjoint_vs_oracle_and_transpose(nside, lmax, eps):
    """Y^T f with regenerated blocks (each block's V staged a chunk of rows at
    a time, sigma applied by the final staging): against the oracle at the
    tolerance rule, against the stored plan's adjoint, and the exact
    transpose of the same plan's synthesis, <Y a, f> = <a, Y^T f>."""
    plan = sh.Plan(nside, lmax, eps, residual_recurrence=True)
    stored = sh.Plan(nside, lmax, eps)
    rings = oracle.healpix_rings(nside)
    f = synthetic.gaussian_map(rings.npix, 2, seed=80)
    want = oracle.adjoint(rings, lmax, f)
    got = plan.adjoint(dev(f)).cpu().numpy()
    ref = stored.adjoint(dev(f)).cpu().numpy()
    tol = 1e-10 if eps <= 1e-12 else 100 * eps
    for b in range(2):
        assert rel_rms(want[b], got[b]) <= tol
        assert rel_rms(ref[b], got[b]) <= 1e-12
    a = dev(synthetic.gaussian_alm(lmax, 3, seed=81))
    fd = dev(synthetic.gaussian_map(plan.npix, 3, seed=82))
    lhs = torch.sum(plan.synthesize(a) * fd).item()
    at = plan.adjoint(fd)
    rhs = torch.sum(a.real * at.real + a.imag * at.imag).item()
    assert lhs == pytest.approx(rhs, rel=1e-12)
    stored.close()
    plan.close()


def test_regenerated_plans_refuse_what_they_do_not_serve():
    """Batches need stored residual blocks; the option needs a compressed
    scalar plan."""
    plan = sh.Plan(16, 32, 1e-10, residual_recurrence=True)
    a = torch.zeros((1, plan.nalm), dtype=torch.complex128, device="cuda")
    m = torch.zeros((1, plan.npix), dtype=torch.float64, device="cuda")
    with pytest.raises(sh.ShtbError) as e:
        sh.shtb_batch_create([(plan, a, m)])
    assert e.value.code == sh.SHTB_ENOTSUP
    plan.close()
    for kw in ({"eps": 0.0}, {"eps": 1e-10, "spin": 2}):
        eps = kw.pop("eps")
        with pytest.raises(sh.ShtbError) as e:
            sh.Plan(16, 32, eps, residual_recurrence=True, **kw)
        assert e.value.code == sh.SHTB_ENOTSUP
