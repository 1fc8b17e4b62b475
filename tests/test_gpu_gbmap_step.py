"""The anisotropy map inside the step (Sec. 2.1.4, reading R15): with
gb_map_tube set, Eq. (10)'s pair (i, j) of every cell within the tube of
grain i's zero level comes from the closest point of grain i's triangulated
boundary instead of the cell's ID-field entry.

The map is checked like the stateless op (tests/test_gpu_gbmap.py): exact
where one grain's triangles are the closest by more than 1e-4, one of the
tied grains elsewhere.  The step is then checked with the map it used: the
oracle's step whose predictor takes the same pairs equals the device's step
stage by stage at the parity tolerances."""
import numpy as np
import pytest

from oracle import lsgg_oracle as O
from paper_1701_06658_gb300 import inputs as I
from tests.parity import box_full, oracle_from_gpu, sign_flip_exclusion
from tests.test_gpu_gbmap import check_box

pytestmark = pytest.mark.gpu

TUBE = 3.0


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1701_06658_gb300 import lsgg
    lsgg.lib()
    return lsgg


def _rs(L, N, G, seed):
    seeds = I.voronoi_seeds(seed, G, (N, N, N))
    quats = I.random_quaternions(seed, G)
    return seeds, quats, L.Microstructure(N, N, N, G, seeds=seeds, quats=quats, physics=L.PHYSICS_READ_SHOCKLEY,
                                          gb_map_tube=TUBE)


def _sampled_map_check(phi, idf, mp, rng, per_box=60):
    """The device map against R15 on up to per_box band cells per grain (exact
    where unique, a tied grain otherwise) and on every other cell exactly."""
    unique = picked = 0
    for g in phi:
        cells = np.argwhere(np.abs(phi[g]) < TUBE)
        if len(cells) > per_box:
            cells = cells[rng.choice(len(cells), size=per_box, replace=False)]
        u, k = check_box(phi[g], idf[g], mp[g], TUBE, cells)
        unique, picked = unique + u, picked + k
    return unique, picked


def test_step_map_and_step_match_the_oracle(L):
    """40^3, 20 Read-Shockley grains, tube 3, after two steps: the map the next
    step uses is R15's on the state and ID-field on the current boxes, and
    the step with it equals the oracle's step whose predictor takes the same
    pairs, stage by stage."""
    N, G = 40, 20
    seeds, quats, ms = _rs(L, N, G, 31)
    rng = np.random.default_rng(31)
    with ms:
        ms.step(2, 1.0)
        boxes = ms.boxes()
        phi = ms.phi()
        idf, mp = L.debug_pair_ids(ms.ctx, boxes)
        unique, picked = _sampled_map_check(phi, idf, mp, rng)
        assert picked > 600 and unique > 0.6 * picked, (unique, picked)
        changed = sum(int(np.sum(mp[g] != idf[g])) for g in phi)
        assert changed > 0                                   # the map differs from the ID-field somewhere
        ref_ms = oracle_from_gpu(ms.shape, boxes, phi, idf_by_grain=mp, physics=O.read_shockley_physics(quats))
        ref = O.step_parts(ref_ms, 1.0)
        b2, (phip, m, idm, phic, phin) = ms.debug_step(1.0)
    assert np.array_equal(b2, boxes)
    for g in phin:
        assert np.max(np.abs(phip[g] - ref.phip[g])) <= 3e-5, g
        assert np.max(np.abs(phic[g] - ref.phic[g])) <= 3e-5, g
        excl = sign_flip_exclusion(ref.phic[g], phic[g], box_full(boxes[g], (N, N, N)))
        d = np.abs(phin[g] - ref.phi[g])
        d[excl] = 0
        assert d.max() <= 1e-4, g


def test_step_map_evolution_over_6_steps(L):
    """Six steps with the map: before every step the device's map is checked
    against R15 on sampled band cells and handed to the oracle, which takes
    its own step with those pairs (so near-tied cells, where R15 admits either
    grain, take the device's choice); per-grain volumes after six steps
    within 0.1 % for grains above 50 cells, boxes equal, every cell owned."""
    N, G, steps = 40, 20, 6
    seeds, quats, ms = _rs(L, N, G, 33)
    rng = np.random.default_rng(33)
    ref = O.tessellate((N, N, N), seeds, physics=O.read_shockley_physics(quats))
    with ms:
        for _ in range(steps):
            boxes = ms.boxes()
            idf, mp = L.debug_pair_ids(ms.ctx, boxes)
            unique, picked = _sampled_map_check(ms.phi(), idf, mp, rng, per_box=20)
            assert unique > 0.6 * picked, (unique, picked)
            for g, gr in enumerate(ref.grains):
                if gr.alive:
                    assert (boxes[g, 3], boxes[g, 2], boxes[g, 1]) == gr.origin
                    assert (boxes[g, 6], boxes[g, 5], boxes[g, 4]) == gr.dims
                    gr.idf = mp[g].astype(np.int64)
            ref = O.step(ref, 1.0)
            ms.step(1, 1.0)
        vg = ms.grain_volumes()
        own = ms.voxel_owner()
    vo = O.volumes(ref)
    big = vo > 50
    assert np.max(np.abs(vg - vo)[big] / vo[big]) <= 1e-3
    assert (own >= 0).all()
