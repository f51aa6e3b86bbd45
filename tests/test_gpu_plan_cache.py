"""Plan files: a saved plan loads back and synthesizes the same maps bit for
bit; a cache directory serves the second plan creation from the file; and
damaged files -- flipped byte, truncation, wrong magic, another plan's file
under this plan's name -- are rejected with SHTB_ECORRUPT (a missing file
with SHTB_EIO) and, through the cache directory, rebuilt.  The faults are
made on the host, in the files."""
import os

import numpy as np
import pytest

from paper_1110_4874_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1110_4874_gb300 as sh  # noqa: E402


def maps_of(plan, seed=7):
    a = torch.from_numpy(synthetic.gaussian_alm(plan.lmax, 3, seed=seed)).cuda()
    return plan.synthesize(a)


@pytest.mark.parametrize("eps", [1e-10, 0.0])
def test_save_load_round_trip(tmp_path, eps):
    plan = sh.Plan(32, 64, eps)
    path = str(tmp_path / "p.bin")
    plan.save(path)
    back = sh.Plan.load(path)
    st0, st1 = plan.stats(), back.stats()
    assert (back.nside, back.lmax, back.eps) == (32, 64, eps)
    assert st1["from_cache"] == 1 and st0["from_cache"] == 0
    for k in ("compressed", "n_dense", "n_rstored", "n_ident", "n_recurrence", "plan_device_bytes"):
        assert st0[k] == st1[k], k
    assert torch.equal(maps_of(plan), maps_of(back))
    assert torch.equal(plan.adjoint(maps_of(plan)), back.adjoint(maps_of(plan)))
    plan.close()
    back.close()


def test_cache_dir_serves_the_second_creation(tmp_path):
    d = str(tmp_path)
    first = sh.Plan(24, 50, 1e-8, cache_dir=d)
    files = os.listdir(d)
    assert len(files) == 1 and first.stats()["from_cache"] == 0
    second = sh.Plan(24, 50, 1e-8, cache_dir=d)
    assert second.stats()["from_cache"] == 1
    assert torch.equal(maps_of(first), maps_of(second))
    other = sh.Plan(24, 50, 1e-6, cache_dir=d)          # another key: its own file
    assert other.stats()["from_cache"] == 0 and len(os.listdir(d)) == 2
    for p in (first, second, other):
        p.close()


def damage(path, how):
    data = bytearray(open(path, "rb").read())
    if how == "flip":
        data[len(data) // 2] ^= 0x40
    elif how == "truncate":
        data = data[: len(data) - 1000]
    elif how == "magic":
        data[0:8] = b"NOTAPLAN"
    open(path, "wb").write(bytes(data))


@pytest.mark.parametrize("how", ["flip", "truncate", "magic"])
def test_damaged_file_is_rejected_and_rebuilt(tmp_path, how):
    d = str(tmp_path)
    plan = sh.Plan(16, 40, 1e-10, cache_dir=d)
    want = maps_of(plan)
    path = os.path.join(d, os.listdir(d)[0])
    damage(path, how)
    with pytest.raises(sh.ShtbError) as e:
        sh.Plan.load(path)
    assert e.value.code == sh.SHTB_ECORRUPT
    again = sh.Plan(16, 40, 1e-10, cache_dir=d)           # rebuilt, file rewritten
    assert again.stats()["from_cache"] == 0
    assert torch.equal(maps_of(again), want)
    third = sh.Plan(16, 40, 1e-10, cache_dir=d)
    assert third.stats()["from_cache"] == 1
    for p in (plan, again, third):
        p.close()


def test_foreign_file_under_this_name_and_missing_file(tmp_path):
    d = str(tmp_path)
    a = sh.Plan(16, 40, 1e-10, cache_dir=d)
    name_a = os.listdir(d)[0]
    b = sh.Plan(20, 40, 1e-10, cache_dir=d)
    name_b = [f for f in os.listdir(d) if f != name_a][0]
    os.replace(os.path.join(d, name_a), os.path.join(d, name_b))   # a's plan under b's name
    c = sh.Plan(20, 40, 1e-10, cache_dir=d)                      # key check rejects it: rebuilt
    assert c.stats()["from_cache"] == 0 and c.nside == 20
    assert torch.equal(maps_of(c), maps_of(b))
    with pytest.raises(sh.ShtbError) as e:
        sh.Plan.load(os.path.join(d, "no_such_plan.bin"))
    assert e.value.code == sh.SHTB_EIO
    for p in (a, b, c):
        p.close()


def test_polarised_plan_files(tmp_path):
    """A polarised plan's file holds both operators: the loaded plan
    synthesizes bit-identical Q/U maps; the cache directory keys on spin."""
    d = str(tmp_path)
    plan = sh.Plan(16, 32, 1e-10, spin=2, cache_dir=d)
    assert plan.stats()["from_cache"] == 0 and plan.stats()["spin"] == 2
    eb = np.stack([synthetic.gaussian_alm(32, 2, seed=5), synthetic.gaussian_alm(32, 2, seed=6)], axis=1)
    a = torch.from_numpy(np.ascontiguousarray(eb)).cuda()
    want = plan.synthesize_spin(a)
    again = sh.Plan(16, 32, 1e-10, spin=2, cache_dir=d)
    st0, st1 = plan.stats(), again.stats()
    assert st1["from_cache"] == 1 and st1["spin"] == 2
    for k in ("n_dense", "n_rstored", "n_ident", "plan_device_bytes"):
        assert st0[k] == st1[k], k
    assert torch.equal(again.synthesize_spin(a), want)
    f = torch.from_numpy(np.random.default_rng(7).standard_normal((2, 2, plan.npix))).cuda()
    assert torch.equal(again.adjoint_spin(f), plan.adjoint_spin(f))
    scalar = sh.Plan(16, 32, 1e-10, cache_dir=d)          # same key but spin: its own file
    assert scalar.stats()["from_cache"] == 0 and len(os.listdir(d)) == 2
    path = str(tmp_path / "pol.bin")
    plan.save(path)
    back = sh.Plan.load(path)
    assert back.stats()["spin"] == 2
    assert torch.equal(back.synthesize_spin(a), want)
    for p in (plan, again, scalar, back):
        p.close()
