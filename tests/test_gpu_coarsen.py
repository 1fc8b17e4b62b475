"""GPU parity of the grid coarsening (Sec. 4.1, reading R12 of the oracle).

lsgg_coarsen projects every grain's function trilinearly onto a coarser grid
of the same periodic domain, scales distances by N'/N, re-initialises and
updates the boxes.  The oracle does the same in FP64 from the GPU's own FP32
state.  Boxes must match exactly and phi to the step tolerance, except within
the re-initialisation's reach of a cell whose projected value is so close to
0 that FP32 and FP64 may give it different signs.
"""
import numpy as np
import pytest

from oracle import lsgg_oracle as O
from paper_1701_06658_gb300 import inputs as I
from tests.parity import oracle_from_gpu

pytestmark = pytest.mark.gpu

TOL_PHI = 1e-4
NEAR_ZERO = 1e-5      # |projected value| below which FP32 and FP64 signs may differ
REACH = 7             # cells a sign decision can move in the re-initialisation


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1701_06658_gb300 import lsgg
    lsgg.lib()
    return lsgg


def _near_zero_mask(ref_ms, gid, shape2):
    """Coarse-domain cells within REACH face steps (periodic) of a cell where
    the oracle's projection of grain gid is within NEAR_ZERO of 0."""
    p = O.coarse_project(ref_ms.grains[gid], ref_ms.shape, shape2, ref_ms.eps)
    dom = np.zeros(shape2, dtype=bool)
    idx = np.ix_(*[(p.origin[a] + np.arange(p.phi.shape[a])) % shape2[a] for a in range(3)])
    dom[idx] = np.abs(p.phi) < NEAR_ZERO
    for _ in range(REACH if dom.any() else 0):
        grown = dom.copy()
        for ax in range(3):
            grown |= np.roll(dom, 1, axis=ax) | np.roll(dom, -1, axis=ax)
        dom = grown
    return dom


def _compare(L, ms_shape2, boxes2, phi2, ref_ms, ref):
    """GPU coarsened state vs the oracle's: boxes exact and phi within
    TOL_PHI outside the near-zero masks; returns (worst, excluded cells)."""
    worst, excluded = 0.0, 0
    for g, gr in enumerate(ref.grains):
        assert bool(boxes2[g, 0]) == gr.alive, g
        if not gr.alive:
            continue
        mask = _near_zero_mask(ref_ms, g, ms_shape2)
        if not mask.any():
            assert (boxes2[g, 3], boxes2[g, 2], boxes2[g, 1]) == gr.origin, g
            assert (boxes2[g, 6], boxes2[g, 5], boxes2[g, 4]) == gr.dims, g
        gv = O.Grain(g, (int(boxes2[g, 3]), int(boxes2[g, 2]), int(boxes2[g, 1])), phi2[g].astype(np.float64))
        pos = O.box_positions(gv, ms_shape2)
        want, _ = O.sample(gr, pos, ms_shape2, -7.0)
        skip = mask[np.ix_(*pos)]
        d = np.abs(gv.phi - want)
        d[skip] = 0.0
        excluded += int(skip.sum())
        worst = max(worst, float(d.max()))
    return worst, excluded


@pytest.mark.parametrize("shape,shape2,G,seed,steps", [
    ((64, 64, 64), (48, 48, 48), 50, 1, 3),
    ((64, 64, 64), (32, 32, 32), 40, 2, 2),
    ((40, 60, 80), (30, 45, 60), 30, 3, 2),
    ((48, 48, 48), (48, 48, 48), 30, 10, 2),       # ratio 1: the projection is the identity
])
def test_coarsen_matches_oracle(L, shape, shape2, G, seed, steps):
    nz, ny, nx = shape
    seeds = I.voronoi_seeds(seed, G, shape)
    with L.Microstructure(nx, ny, nz, G, seeds=seeds) as ms:
        ms.step(steps, 1.0)
        ms.sync()
        ref_ms = oracle_from_gpu(shape, ms.boxes(), ms.phi())
        done = L.get_stats(ms.ctx).steps_done
        ms.coarsen(shape2[2], shape2[1], shape2[0])
        assert ms.shape == shape2
        assert L.get_stats(ms.ctx).steps_done == done      # no step counted
        boxes2, phi2 = ms.boxes(), ms.phi()
    ref = O.coarsen(ref_ms, shape2)
    worst, excluded = _compare(L, shape2, boxes2, phi2, ref_ms, ref)
    print(f"coarsen {shape} -> {shape2}: max |phi - oracle| {worst:.2e}, {excluded} cells near sign ties")
    assert worst <= TOL_PHI


def test_coarsen_godunov_matches_oracle(L):
    """The re-initialisation after the projection follows the configured
    metric (LSGG_REDIST_GODUNOV: the oracle's Euclidean update, R11)."""
    N, G = 64, 40
    seeds = I.voronoi_seeds(4, G, (N, N, N))
    with L.Microstructure(N, N, N, G, seeds=seeds, redist=L.REDIST_GODUNOV) as ms:
        ms.step(2, 1.0)
        ms.sync()
        ref_ms = oracle_from_gpu((N, N, N), ms.boxes(), ms.phi())
        ref_ms.redist = "godunov"
        ms.coarsen(48, 48, 48)
        boxes2, phi2 = ms.boxes(), ms.phi()
    ref = O.coarsen(ref_ms, (48, 48, 48))
    worst, _ = _compare(L, (48, 48, 48), boxes2, phi2, ref_ms, ref)
    assert worst <= TOL_PHI


def test_steps_after_coarsening_match_oracle(L):
    """The coarsened state is an ordinary state of the coarse grid: the next
    steps equal the oracle's steps from it (boxes exact, phi within TOL_PHI
    outside near-tie sign flips)."""
    from tests.test_gpu_parity import _check_step
    N, G = 64, 50
    seeds = I.voronoi_seeds(5, G, (N, N, N))
    with L.Microstructure(N, N, N, G, seeds=seeds) as ms:
        ms.step(2, 1.0)
        ms.coarsen(40, 40, 40)
        _check_step(L, ms)
        ms.step(2, 1.0)
        _check_step(L, ms)


def test_coarsening_scales_grain_volumes(L):
    """Halving the cells per axis divides every grain's volume by 8 up to the
    interpolation's displacement of the interface: per-grain within 5 % for
    grains above 4000 fine cells, the total within 0.5 % (the grains tile the
    domain before and after)."""
    N, G = 96, 40
    seeds = I.voronoi_seeds(6, G, (N, N, N))
    with L.Microstructure(N, N, N, G, seeds=seeds) as ms:
        ms.step(4, 1.0)
        v1 = ms.grain_volumes()
        ms.coarsen(48, 48, 48)
        v2 = ms.grain_volumes()
        ms.step(2, 1.0)
        v3 = ms.grain_volumes()
    big = v1 > 4000
    rel = np.abs(8.0 * v2[big] - v1[big]) / v1[big]
    print(f"coarsened volumes x 8 vs fine: max rel {rel.max():.3e}, mean {rel.mean():.3e}; "
          f"total {v2.sum():.1f} of {48 ** 3}")
    assert rel.max() < 0.05
    assert abs(v2.sum() - 48 ** 3) / 48 ** 3 < 5e-3
    assert abs(v3.sum() - 48 ** 3) / 48 ** 3 < 5e-3


def test_coarsen_rejects_unequal_ratios_and_finer_grids(L):
    N, G = 32, 8
    seeds = I.voronoi_seeds(7, G, (N, N, N))
    with L.Microstructure(N, N, N, G, seeds=seeds) as ms:
        for dims in ((16, 16, 24), (40, 40, 40), (0, 0, 0)):
            with pytest.raises(L.LsggError) as e:
                ms.coarsen(*dims)
            assert e.value.code == L.ERR_INVALID_ARG
        assert ms.shape == (N, N, N)
        ms.step(1, 1.0)          # the context is unchanged and usable
        ms.sync()
    # a 2D domain (no 3D pass path) is refused
    seeds2 = I.voronoi_seeds(7, 6, (1, 32, 32))
    with L.Microstructure(32, 32, 1, 6, seeds=seeds2) as m2:
        with pytest.raises(L.LsggError) as e:
            m2.coarsen(16, 16, 1)
        assert e.value.code == L.ERR_UNSUPPORTED


def test_coarsen_with_read_shockley_rebuilds_the_id_field(L):
    """Read-Shockley physics: the coarsening matches the oracle's, and the next
    step -- whose predictor blends with the pair weights the ID-field selects
    -- matches the oracle's step from the oracle's coarsened state (its
    rebuilt ID-field), so the GPU's ID-field is the oracle's."""
    from tests.test_gpu_physics import _compare_step
    N, N2, G = 48, 36, 24
    seeds = I.voronoi_seeds(8, G, (N, N, N))
    quats = I.random_quaternions(8, G)
    phys = O.read_shockley_physics(quats)
    with L.Microstructure(N, N, N, G, seeds=seeds, quats=quats, physics=L.PHYSICS_READ_SHOCKLEY) as ms:
        ms.step(2, 1.0)
        ms.sync()
        ref_ms = oracle_from_gpu((N, N, N), ms.boxes(), ms.phi(), physics=phys)
        ms.coarsen(N2, N2, N2)
        boxes2, phi2 = ms.boxes(), ms.phi()
        ref = O.coarsen(ref_ms, (N2, N2, N2))
        worst, excluded = _compare(L, (N2, N2, N2), boxes2, phi2, ref_ms, ref)
        assert worst <= TOL_PHI
        assert excluded == 0
        idf = {g: ref.grains[g].idf for g in range(G) if ref.grains[g].alive}
        nxt = oracle_from_gpu((N2, N2, N2), boxes2, phi2, idf_by_grain=idf, physics=phys)
        _compare_step(L, ms, nxt)


def test_coarsen_with_bf16_storage(L):
    """BF16 state storage: the projection reads the FP32 view of the state and
    the re-initialisation stores BF16 again.  From the same FP32-exact start
    the coarsened BF16 state equals the FP32 run's coarsened state up to the
    storage rounding (2^-8 relative) and a few sign-tie cells, with the same
    grains alive."""
    N, G = 64, 40
    seeds = I.voronoi_seeds(9, G, (N, N, N))
    out = {}
    for st in (L.STORAGE_FP32, L.STORAGE_BF16):
        with L.Microstructure(N, N, N, G, seeds=seeds, storage=st) as ms:
            ms.coarsen(48, 48, 48)
            out[st] = (ms.boxes(), ms.phi(), ms.grain_volumes())
    b32, p32, v32 = out[L.STORAGE_FP32]
    b16, p16, v16 = out[L.STORAGE_BF16]
    assert np.array_equal(b32[:, 0], b16[:, 0])
    same = 0
    for g in range(G):
        if not b32[g, 0] or not np.array_equal(b32[g], b16[g]):
            continue
        same += 1
        d = np.abs(p16[g] - p32[g]) - 2.0 ** -7 * np.abs(p32[g]) - 2e-2
        assert np.mean(d > 0) < 0.01, g
    assert same >= G - 2
    alive = v32 > 50
    assert np.max(np.abs(v16[alive] - v32[alive]) / v32[alive]) < 5e-3
