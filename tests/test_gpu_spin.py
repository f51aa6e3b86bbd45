"""Polarised (spin-2) synthesis on the GPU against the oracle's Wigner-d
route: compressed and uncompressed polarised plans, batches of (E, B)
pairs, the E-to-B rotation, sampled rings at the 3-million-pixel map, and
the calls a polarised plan refuses.

Tolerances (relative RMS over each map): uncompressed 1e-12, compressed
1e-10 at eps <= 1e-12, else 100 eps (the scalar rules)."""
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
    return float(np.sqrt(np.sum((x - y) ** 2) / np.sum(x ** 2)))


def tol_of(eps):
    return 1e-12 if eps <= 0 else (1e-10 if eps <= 1e-12 else 100 * eps)


def pairs(lmax, npairs, seed):
    e = synthetic.gaussian_alm(lmax, npairs, seed=seed)
    b = synthetic.gaussian_alm(lmax, npairs, seed=seed + 1000)
    return e, b, np.ascontiguousarray(np.stack([e, b], axis=1))


@pytest.mark.parametrize("nside,lmax,eps", [
    (16, 32, 0.0), (16, 32, 1e-12), (13, 40, 1e-10), (32, 64, 1e-10), (64, 128, 1e-12)])
def test_polarised_synthesis_vs_oracle(nside, lmax, eps):
    plan = sh.Plan(nside, lmax, eps, spin=2)
    st = plan.stats()
    assert st["spin"] == 2 and st["compressed"] == (1 if eps > 0 else 0)
    rings = oracle.healpix_rings(nside)
    e, b, eb = pairs(lmax, 3, seed=700 + nside)
    Q, U = oracle.spin_synthesize(rings, lmax, e, b)
    got = plan.synthesize_spin(torch.from_numpy(eb).cuda()).cpu().numpy()
    for p in range(3):
        assert rel_rms(Q[p], got[p, 0]) <= tol_of(eps)
        assert rel_rms(U[p], got[p, 1]) <= tol_of(eps)
    plan.close()


def test_pairs_in_a_batch_match_single_pairs():
    """Every pair of a batch of 5 (10 inputs: map groups 8 + 2) equals the
    same pair transformed alone, to rounding."""
    plan = sh.Plan(32, 64, 1e-10, spin=2)
    _, _, eb = pairs(64, 5, seed=900)
    a = torch.from_numpy(eb).cuda()
    both = plan.synthesize_spin(a)
    for p in range(5):
        one = plan.synthesize_spin(a[p])
        scale = float(one.abs().max())
        assert float((both[p] - one).abs().max()) <= 1e-14 * scale
    plan.close()


def test_rotation_of_e_into_b():
    """(E, B) -> (-B, E) multiplies Q + iU by i: (Q, U) -> (-U, Q)."""
    plan = sh.Plan(24, 48, 1e-10, spin=2)
    _, _, eb = pairs(48, 2, seed=950)
    a = torch.from_numpy(eb).cuda()
    r = torch.stack([-a[:, 1], a[:, 0]], dim=1).contiguous()
    m0 = plan.synthesize_spin(a)
    m1 = plan.synthesize_spin(r)
    scale = float(m0.abs().max())
    assert float((m1[:, 0] + m0[:, 1]).abs().max()) <= 1e-14 * scale
    assert float((m1[:, 1] - m0[:, 0]).abs().max()) <= 1e-14 * scale
    plan.close()


def test_polarised_nside512_sampled_rings():
    """Nside=512, L=1024, eps=1e-10, 2 pairs: every pixel of 12 rings (poles,
    equator, polar caps, belt) against the oracle on those rings."""
    nside, lmax, eps = 512, 1024, 1e-10
    plan = sh.Plan(nside, lmax, eps, spin=2)
    e, b, eb = pairs(lmax, 2, seed=5120)
    got = plan.synthesize_spin(torch.from_numpy(eb).cuda()).cpu().numpy()
    rings = oracle.healpix_rings(nside)
    idx = np.array([0, 1, 7, 100, 400, 511, 800, 1023, 1500, 2000, 2045, 2046])
    sub = rings.subset(idx)
    qQ, qU = oracle.spin_q(sub, lmax, e, b)
    Q, U = oracle.phi_synth(sub, lmax, qQ), oracle.phi_synth(sub, lmax, qU)
    cols = np.concatenate([np.arange(rings.start[k], rings.start[k + 1]) for k in idx])
    for p in range(2):
        assert rel_rms(Q[p], got[p, 0][cols]) <= tol_of(eps)
        assert rel_rms(U[p], got[p, 1][cols]) <= tol_of(eps)
    plan.close()


def test_polarised_plan_refuses_scalar_calls(tmp_path):
    plan = sh.Plan(8, 16, 1e-10, spin=2)
    a = torch.zeros((1, plan.nalm), dtype=torch.complex128, device="cuda")
    f = torch.zeros((1, plan.npix), dtype=torch.float64, device="cuda")
    for call in (lambda: plan.synthesize(a), lambda: plan.adjoint(f), lambda: plan.analyze(f),
                 lambda: sh.shtb_batch_create([(plan, a, f)])):
        with pytest.raises(sh.ShtbError) as e:
            call()
        assert e.value.code == sh.SHTB_ENOTSUP
    scalar = sh.Plan(8, 16, 1e-10)
    with pytest.raises(sh.ShtbError) as e:
        sh.shtb_synthesize_spin(scalar.handle, torch.zeros((1, 2, scalar.nalm), dtype=torch.complex128,
                                                           device="cuda"),
                                torch.zeros((1, 2, scalar.npix), dtype=torch.float64, device="cuda"), 1)
    assert e.value.code == sh.SHTB_ENOTSUP
    with pytest.raises(sh.ShtbError) as e:
        sh.Plan(8, 16, 1e-10, spin=1)
    assert e.value.code == sh.SHTB_EINVAL
    plan.close()
    scalar.close()


@pytest.mark.parametrize("nside,lmax,eps", [(16, 32, 0.0), (16, 32, 1e-12), (13, 40, 1e-10)])
def test_polarised_adjoint_vs_oracle(nside, lmax, eps):
    plan = sh.Plan(nside, lmax, eps, spin=2)
    rings = oracle.healpix_rings(nside)
    rng = np.random.default_rng(800 + nside)
    Q = rng.standard_normal((2, rings.npix))
    U = rng.standard_normal((2, rings.npix))
    gE, gB = oracle.spin_adjoint(rings, lmax, Q, U)
    f = torch.from_numpy(np.ascontiguousarray(np.stack([Q, U], axis=1))).cuda()
    got = plan.adjoint_spin(f).cpu().numpy()
    for p in range(2):
        assert rel_rms(gE[p].view(np.float64), got[p, 0].view(np.float64)) <= tol_of(eps)
        assert rel_rms(gB[p].view(np.float64), got[p, 1].view(np.float64)) <= tol_of(eps)
    plan.close()


@pytest.mark.parametrize("nside,lmax,eps", [(64, 128, 1e-10), (33, 64, 1e-6), (16, 32, 0.0)])
def test_polarised_adjoint_is_exact_transpose(nside, lmax, eps):
    """<Y a, f> = <a, Y^T f> to rounding for the plan's own (compressed)
    operator, whatever eps."""
    plan = sh.Plan(nside, lmax, eps, spin=2)
    _, _, eb = pairs(lmax, 3, seed=850)
    a = torch.from_numpy(eb).cuda()
    f = torch.from_numpy(np.random.default_rng(851).standard_normal((3, 2, plan.npix))).cuda()
    lhs = torch.sum(plan.synthesize_spin(a) * f).item()
    g = plan.adjoint_spin(f)
    rhs = torch.sum(a.real * g.real + a.imag * g.imag).item()
    assert lhs == pytest.approx(rhs, rel=1e-12)
    plan.close()


def test_polarised_autograd_directional_derivative():
    """loss = 1/2 ||Y_pol a - d||^2 through sh.synthesize_spin: the gradient
    from the adjoint kernels matches a central difference (exact for a
    quadratic loss up to rounding)."""
    plan = sh.Plan(32, 64, 1e-10, spin=2)
    _, _, eb = pairs(64, 2, seed=870)
    _, _, eb2 = pairs(64, 2, seed=880)
    d = plan.synthesize_spin(torch.from_numpy(eb2).cuda())
    a0 = torch.from_numpy(eb).cuda()
    a = a0.clone().requires_grad_(True)
    loss = 0.5 * ((sh.synthesize_spin(a, plan) - d) ** 2).sum()
    loss.backward()
    _, _, vv = pairs(64, 2, seed=890)
    v = torch.from_numpy(vv).cuda()
    h = 1e-3
    with torch.no_grad():
        lp = 0.5 * ((plan.synthesize_spin(a0 + h * v) - d) ** 2).sum()
        lm = 0.5 * ((plan.synthesize_spin(a0 - h * v) - d) ** 2).sum()
    fd = float((lp - lm) / (2 * h))
    dd = float((a.grad.conj() * v).real.sum())
    assert fd == pytest.approx(dd, rel=1e-9)
    plan.close()


@pytest.mark.parametrize("nside,lmax,eps,niter", [(16, 32, 0.0, 0), (16, 32, 0.0, 2), (24, 48, 1e-10, 1)])
def test_polarised_analysis_vs_oracle(nside, lmax, eps, niter):
    plan = sh.Plan(nside, lmax, eps, spin=2)
    rings = oracle.healpix_rings(nside)
    rng = np.random.default_rng(820 + nside)
    Q = rng.standard_normal((2, rings.npix))
    U = rng.standard_normal((2, rings.npix))
    w = np.full(rings.nrings, 4 * np.pi / rings.npix)
    wE, wB = oracle.spin_analyze(rings, lmax, Q, U, w, niter=niter)
    f = torch.from_numpy(np.ascontiguousarray(np.stack([Q, U], axis=1))).cuda()
    got = plan.analyze_spin(f, niter=niter).cpu().numpy()
    tol = tol_of(eps) * (1 + niter)
    for p in range(2):
        assert rel_rms(wE[p].view(np.float64), got[p, 0].view(np.float64)) <= tol
        assert rel_rms(wB[p].view(np.float64), got[p, 1].view(np.float64)) <= tol
    plan.close()


def test_polarised_refinement_recovers_band_limited_alm():
    """(Q, U) from the plan's own operator: Jacobi steps converge to (E, B)
    for l >= 2 (the l < 2 coefficients do not enter the maps)."""
    nside, lmax = 128, 256
    plan = sh.Plan(nside, lmax, 1e-10, spin=2)
    _, _, eb = pairs(lmax, 2, seed=830)
    lcol = np.array([l for m in range(lmax + 1) for l in range(m, lmax + 1)])
    eb[:, :, lcol < 2] = 0
    a = torch.from_numpy(eb).cuda()
    f = plan.synthesize_spin(a)
    errs = [float((plan.analyze_spin(f, niter=k) - a).abs().max() / a.abs().max()) for k in (0, 2, 4, 8)]
    for e0, e1 in zip(errs[:-1], errs[1:]):
        assert e1 < 0.3 * e0 or e1 < 1e-12
    assert errs[-1] < 1e-6 * errs[0]
    plan.close()
