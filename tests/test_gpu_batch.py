"""Batched serving: many uneven synthesis requests in one persistent launch
(captured in a CUDA graph), checked request by request against the
one-request-per-launch path on the same plans."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1110_4874_gb300 as sh  # noqa: E402
from paper_1110_4874_gb300 import synthetic  # noqa: E402

# Both schedules (the persistent kernel and the stage-kernel graph) run the
# single-request path's item bodies, and every dot product sums in one order
# whatever the map-group width, so a batched map equals the same request
# transformed alone, bit for bit.


def same_map(got, want):
    return torch.equal(got, want)


@pytest.fixture(scope="module")
def setup():
    rng = np.random.default_rng(3000)
    plans = {n: sh.Plan(n, 2 * n, 1e-10) for n in (16, 32, 64)}
    reqs = []
    for i in range(12):
        n = int(rng.choice([16, 32, 64]))
        b = int(rng.integers(1, 9))
        p = plans[n]
        alm = torch.from_numpy(synthetic.gaussian_alm(2 * n, b, seed=3000 + 10 * i)).cuda()
        maps = torch.full((b, p.npix), float("nan"), dtype=torch.float64, device="cuda")
        reqs.append((p, alm, maps))
    yield plans, reqs
    for p in plans.values():
        p.close()


def test_batch_equals_plain_requests(setup):
    plans, reqs = setup
    batch = sh.shtb_batch_create(reqs, autotune=True)
    info = sh.shtb_batch_info(batch)
    assert info["schedule"] in (0, 1) and info["tuned_ms"] > 0
    if info["schedule"] == 0:
        assert info["warps_per_block"] in (4, 8) and info["grid"] > 0 and info["npacks"] > 0
    else:
        assert info["streams"] in (1, 2, 4, 8)
    torch.cuda.synchronize()
    first = None
    for it in range(2):          # first run captures the graph, second replays it
        for _, _, maps in reqs:
            maps.fill_(float("nan"))
        sh.shtb_batch_run(batch)
        sh.shtb_batch_status(batch)
        for p, alm, maps in reqs:
            want = p.synthesize(alm)
            assert same_map(maps, want), f"run {it}"
        if first is None:
            first = [maps.clone() for _, _, maps in reqs]
        else:            # the replay repeats the captured run bit for bit
            assert all(torch.equal(a, m) for a, (_, _, m) in zip(first, reqs))
    sh.shtb_batch_destroy(batch)


def test_batch_on_a_user_stream(setup):
    plans, reqs = setup
    batch = sh.shtb_batch_create(reqs[:4], autotune=False, warps_per_block=8)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        sh.shtb_batch_run(batch, s)
    sh.shtb_batch_status(batch, s)
    for p, alm, maps in reqs[:4]:
        assert same_map(maps, p.synthesize(alm))
    sh.shtb_batch_destroy(batch)


@pytest.mark.parametrize("streams", [1, 3])
def test_stage_kernel_schedule(setup, streams):
    """The stage-kernel graph schedule (stand-alone kernels over merged map
    groups, spread over streams): same maps as the single-request path to
    rounding, and a graph replay repeats the captured run bit for bit."""
    plans, reqs = setup
    batch = sh.shtb_batch_create(reqs, autotune=False, schedule=1, streams=streams)
    assert sh.shtb_batch_schedule(batch) == {"schedule": 1, "streams": streams}
    first = None
    for _ in range(2):
        for _, _, maps in reqs:
            maps.fill_(float("nan"))
        sh.shtb_batch_run(batch)
        sh.shtb_batch_status(batch)
        if first is None:
            first = [m.clone() for _, _, m in reqs]
    for (p, alm, maps), f in zip(reqs, first):
        assert torch.equal(maps, f)
        assert same_map(maps, p.synthesize(alm))
    with pytest.raises(sh.ShtbError) as e:
        sh.shtb_test_batch_stall(batch, True)
    assert e.value.code == sh.SHTB_ENOTSUP
    sh.shtb_batch_destroy(batch)


def test_batch_wait_timeout_reports_status(setup):
    """A stage wait that never completes (the first stage claims one item
    more than it has) runs out of its bounded spin: the run ends, the status
    reports SHTB_ETIMEOUT, and the context stays usable."""
    plans, reqs = setup
    batch = sh.shtb_batch_create(reqs[:3], autotune=False, spin_limit=20000)
    sh.shtb_test_batch_stall(batch, True)
    sh.shtb_batch_run(batch)
    with pytest.raises(sh.ShtbError) as e:
        sh.shtb_batch_status(batch)
    assert e.value.code == sh.SHTB_ETIMEOUT
    sh.shtb_test_batch_stall(batch, False)
    sh.shtb_batch_run(batch)
    sh.shtb_batch_status(batch)
    for p, alm, maps in reqs[:3]:
        assert same_map(maps, p.synthesize(alm))
    sh.shtb_batch_destroy(batch)


def test_batch_rejects_bad_requests(setup):
    plans, reqs = setup
    dense = sh.Plan(16, 32, 0.0)
    alm = torch.zeros((1, dense.nalm), dtype=torch.complex128, device="cuda")
    maps = torch.zeros((1, dense.npix), dtype=torch.float64, device="cuda")
    with pytest.raises(sh.ShtbError) as e:
        sh.shtb_batch_create([(dense, alm, maps)])
    assert e.value.code == sh.SHTB_ENOTSUP
    with pytest.raises(sh.ShtbError) as e:
        sh.shtb_batch_create([])
    assert e.value.code == sh.SHTB_EINVAL
    dense.close()


@pytest.mark.parametrize("warps,lpt", [(4, 1), (8, 0)])
def test_persistent_schedule(setup, warps, lpt):
    """The persistent kernel over every request (three plans, map groups of
    1-8 maps): each map equals its single-request result bit for bit, and a
    graph replay repeats the captured run."""
    plans, reqs = setup
    batch = sh.shtb_batch_create(reqs, autotune=False, warps_per_block=warps, lpt=bool(lpt), schedule=0)
    info = sh.shtb_batch_info(batch)
    assert info["schedule"] == 0 and info["warps_per_block"] == warps and info["npacks"] > 0
    first = None
    for _ in range(2):
        for _, _, maps in reqs:
            maps.fill_(float("nan"))
        sh.shtb_batch_run(batch)
        sh.shtb_batch_status(batch)
        if first is None:
            first = [m.clone() for _, _, m in reqs]
    for (p, alm, maps), f in zip(reqs, first):
        assert torch.equal(maps, f)
        assert same_map(maps, p.synthesize(alm))
    sh.shtb_batch_destroy(batch)
