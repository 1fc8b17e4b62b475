"""Step groups (many microstructures in one set of launches per step)
against the same microstructures stepped alone, through the C ABI: the state
(every box and every value of phi), the grain volumes and the owner map bit
for bit, with members of different domains, grain counts and box tiers, FP32
and BF16 state storage, per-member step limits, group steps mixed with
single steps, and a member whose arena runs out of room mid-group."""
import numpy as np
import pytest

from paper_1701_06658_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1701_06658_gb300 import lsgg
    lsgg.lib()
    return lsgg


# (nx, ny, nz, grains, seed, storage): cubic and non-cubic domains; boxes of
# every tier (the 80^3 / 6-grain member has boxes wider than 64 cells and
# full periodic axes)
MEMBERS = [(48, 48, 48, 40, 11, "fp32"), (64, 64, 64, 50, 12, "fp32"), (40, 56, 64, 30, 13, "fp32"),
           (96, 96, 96, 260, 14, "fp32"), (80, 80, 80, 6, 15, "fp32"), (64, 64, 64, 50, 16, "bf16")]


def _make(L, m):
    nx, ny, nz, g, seed, st = m
    storage = L.STORAGE_BF16 if st == "bf16" else L.STORAGE_FP32
    return L.Microstructure(nx, ny, nz, g, seeds=I.voronoi_seeds(seed, g, (nx, ny, nz)), storage=storage)


def _snapshot(L, ms):
    ms.sync()
    return {"phi": L.get_phi(ms.ctx), "boxes": ms.boxes(), "vol": ms.grain_volumes(),
            "own": ms.voxel_owner(), "steps": ms.stats().steps_done}


def _assert_same(a, b):
    assert a["steps"] == b["steps"]
    assert np.array_equal(a["boxes"], b["boxes"])
    assert a["phi"].dtype == b["phi"].dtype and np.array_equal(a["phi"], b["phi"])
    assert np.array_equal(a["vol"], b["vol"])
    assert np.array_equal(a["own"], b["own"])


def test_group_equals_members_alone(L):
    n_steps = 7
    want = []
    for m in MEMBERS:
        with _make(L, m) as ms:
            ms.step(n_steps, 1.0)
            want.append(_snapshot(L, ms))
    mss = [_make(L, m) for m in MEMBERS]
    try:
        with L.Group(mss) as g:
            g.step(3, 1.0)
            g.step(4, 1.0)
        for ms, w in zip(mss, want):
            _assert_same(_snapshot(L, ms), w)
        # the tiers beyond 48 and the general tier did run
        assert mss[4].stats().pass_cells[4] > 0 or mss[4].stats().pass_cells[3] > 0
    finally:
        for ms in mss:
            ms.close()


def test_step_limits_and_single_steps_mixed(L):
    """Member k stops at its own step count inside a shared chunk; single
    steps of a member before and after group steps keep its result that of
    stepping it alone."""
    mem = MEMBERS[:4]
    limits = [2, 5, 9, 0]
    extra = [1, 0, 2, 3]                      # single steps after the group steps
    want = []
    for m, lim, ex in zip(mem, limits, extra):
        with _make(L, m) as ms:
            ms.step(1 + lim + ex, 1.0)
            want.append(_snapshot(L, ms))
    mss = [_make(L, m) for m in mem]
    try:
        for ms in mss:
            ms.step(1, 1.0)                   # one step alone first
        with L.Group(mss) as g:
            g.step(6, 1.0, [1 + lim for lim in limits])
            g.step(6, 1.0, [1 + lim for lim in limits])
        for ms, ex in zip(mss, extra):
            ms.step(ex, 1.0)
        for ms, w in zip(mss, want):
            _assert_same(_snapshot(L, ms), w)
    finally:
        for ms in mss:
            ms.close()


def test_member_arena_overflow_is_recovered(L):
    """A member whose arena is cut to its initial need halts inside the group
    (the others carry on); lsgg_sync on it grows the arena and finishes its
    steps alone, with the result of an untouched run."""
    from tests.test_gpu_failures import _need
    mem = MEMBERS[:3]
    want = []
    for m in mem:
        with _make(L, m) as ms:
            ms.step(8, 1.0)
            want.append(_snapshot(L, ms))
    mss = [_make(L, m) for m in mem]
    try:
        L.debug_set_capacity(mss[1].ctx, _need(mss[1].boxes()))
        with L.Group(mss) as g:
            g.step(8, 1.0)
        for ms, w in zip(mss, want):
            _assert_same(_snapshot(L, ms), w)
    finally:
        for ms in mss:
            ms.close()


def test_many_small_members(L):
    """Forty 32^3 members of 10 grains each (the serving mix's smallest
    requests) in one group equal their runs alone."""
    mem = [(32, 32, 32, 10, 100 + k, "fp32") for k in range(40)]
    want = []
    for m in mem:
        with _make(L, m) as ms:
            ms.step(5, 1.0)
            want.append(_snapshot(L, ms))
    mss = [_make(L, m) for m in mem]
    try:
        with L.Group(mss) as g:
            g.step(5, 1.0)
        for ms, w in zip(mss, want):
            _assert_same(_snapshot(L, ms), w)
    finally:
        for ms in mss:
            ms.close()


def test_group_refuses_other_configurations(L):
    a = _make(L, MEMBERS[0])
    rs = L.Microstructure(32, 32, 32, 8, seeds=I.voronoi_seeds(3, 8, (32, 32, 32)), physics=L.PHYSICS_READ_SHOCKLEY)
    try:
        with pytest.raises(L.LsggError) as e:
            L.group_create([a.ctx, rs.ctx])
        assert e.value.code == L.ERR_UNSUPPORTED
        with pytest.raises(L.LsggError) as e:
            L.group_create([a.ctx, a.ctx])
        assert e.value.code == L.ERR_INVALID_ARG
        with pytest.raises(L.LsggError) as e:
            L.group_create([a.ctx] * (L.MAX_GROUP + 1))
        assert e.value.code == L.ERR_INVALID_ARG
    finally:
        a.close()
        rs.close()


def test_membership_changes_between_steps(L):
    """One group whose members are replaced between steps (members leaving,
    joining and coming back) gives every microstructure the result of its
    steps alone."""
    mem = [MEMBERS[0], MEMBERS[1], MEMBERS[2], MEMBERS[5]]
    plan = [[0, 1], [0, 1, 2], [2, 3], [1, 3, 0]]      # members of each group step of 2 steps
    counts = [0] * len(mem)
    for grp in plan:
        for k in grp:
            counts[k] += 2
    want = []
    for m, c in zip(mem, counts):
        with _make(L, m) as ms:
            ms.step(c, 1.0)
            want.append(_snapshot(L, ms))
    mss = [_make(L, m) for m in mem]
    try:
        with L.Group([mss[k] for k in plan[0]]) as g:
            for i, grp in enumerate(plan):
                if i:
                    g.set_members([mss[k] for k in grp])
                g.step(2, 1.0)
        for ms, w in zip(mss, want):
            _assert_same(_snapshot(L, ms), w)
    finally:
        for ms in mss:
            ms.close()
