"""The label-field initialisation (reading R17) on the GPU against the FP64
oracle: from the same label field both sides build the same boxes (bit for
bit), the same starting functions (the re-initialisation of +-1/2 by
membership, to the FP32 tolerance of a step's re-initialisation), the same
ID-field with physics (checked through one step whose velocity reads it) and
the same grain volumes after several steps.  The label fields are Voronoi
tessellations of seeded points, edited to add a grain that spans two full
periodic axes, a grain split across the periodic boundary, and labels that
hold no cell (extinct from the start)."""
import numpy as np
import pytest

from oracle import lsgg_oracle as O
from paper_1701_06658_gb300 import inputs as I
from tests.parity import box_full, sign_flip_exclusion

pytestmark = pytest.mark.gpu

TOL_PHI = 1e-4


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1701_06658_gb300 import lsgg
    lsgg.lib()
    return lsgg


def _labels(shape, G, seed):
    """A Voronoi label field of G - 3 seeds plus three edited labels: G - 3 a
    slab spanning the x and y axes, G - 2 a block split by the periodic
    boundary of every axis, G - 1 no cell at all."""
    nz, ny, nx = shape
    lab = O.labels_of_tessellation(shape, I.voronoi_seeds(seed, G - 3, (nx, ny, nz))).astype(np.int32)
    lab[nz // 2:nz // 2 + 3, :, :] = G - 3
    idx = np.r_[-3:3]
    lab[np.ix_(idx % nz, idx % ny, idx % nx)] = G - 2
    return lab


def _assert_same_start(ms, ref, tol=TOL_PHI):
    boxes = ms.boxes()
    phi = ms.phi()
    for g, gr in enumerate(ref.grains):
        assert bool(boxes[g, 0]) == gr.alive, g
        if not gr.alive:
            continue
        assert (boxes[g, 3], boxes[g, 2], boxes[g, 1]) == gr.origin, g
        assert (boxes[g, 6], boxes[g, 5], boxes[g, 4]) == gr.dims, g
        assert np.max(np.abs(phi[g] - gr.phi)) <= tol, g
        assert np.array_equal(phi[g] > 0, gr.phi > 0), g
    return boxes, phi


@pytest.mark.parametrize("shape,G,seed", [((48, 48, 48), 30, 61), ((29, 41, 37), 16, 62)])
def test_label_start_matches_oracle(L, shape, G, seed):
    nz, ny, nx = shape
    lab = _labels(shape, G, seed)
    ref = O.tessellate_labels(lab, G)
    with L.Microstructure(nx, ny, nz, G, labels=lab) as ms:
        boxes, _ = _assert_same_start(ms, ref)
        assert not boxes[G - 1, 0]                                 # the label without a cell
        assert boxes[G - 3, 4] == nx and boxes[G - 3, 5] == ny     # the slab spans x and y
        # every cell is owned by its label
        own = ms.voxel_owner().reshape(shape)
        assert np.array_equal(own, lab)


def test_label_start_godunov_matches_oracle(L):
    """The Godunov re-initialisation (reading R11) builds the starting
    functions when the microstructure uses it."""
    shape, G = (40, 40, 40), 20
    lab = _labels(shape, G, 63)
    ref = O.tessellate_labels(lab, G, redist="godunov")
    with L.Microstructure(40, 40, 40, G, labels=lab, redist=L.REDIST_GODUNOV) as ms:
        _assert_same_start(ms, ref)


def test_label_start_read_shockley_step(L):
    """With Read-Shockley physics the ID-field of the start is the largest
    other function (lowest id on ties); one step whose per-pair velocity reads
    it matches the oracle's step from its own label start."""
    shape, G = (40, 40, 40), 20
    lab = _labels(shape, G, 64)
    quats = I.random_quaternions(64, G)
    ref_ms = O.tessellate_labels(lab, G, physics=O.read_shockley_physics(quats))
    with L.Microstructure(40, 40, 40, G, labels=lab, quats=quats, physics=L.PHYSICS_READ_SHOCKLEY) as ms:
        _assert_same_start(ms, ref_ms)
        ref = O.step_parts(ref_ms, 1.0)
        b, (phip, m, idm, phic, phin) = ms.debug_step(1.0)
    for g in phin:
        assert np.max(np.abs(phip[g] - ref.phip[g])) <= 3e-5, g
        assert np.max(np.abs(phic[g] - ref.phic[g])) <= 3e-5, g
        excl = sign_flip_exclusion(ref.phic[g], phic[g], box_full(b[g], shape))
        d = np.abs(phin[g] - ref.phi[g])
        d[excl] = 0
        assert d.max() <= TOL_PHI, g


def test_label_start_volumes_after_steps(L):
    """Eight ideal steps from a label start: per-grain volumes within 0.1 % of
    the oracle's eight steps from the same labels."""
    shape, G, steps = (48, 48, 48), 30, 8
    lab = _labels(shape, G, 65)
    ref = O.run(O.tessellate_labels(lab, G), steps, 1.0)
    with L.Microstructure(48, 48, 48, G, labels=lab) as ms:
        ms.step(steps, 1.0)
        vol = ms.grain_volumes()
    want = O.volumes(ref)
    big = want > 50
    assert np.max(np.abs(vol - want)[big] / want[big]) <= 1e-3
    assert np.all(np.abs(vol - want)[~big] <= 0.05)


def test_label_start_of_a_voronoi_field_has_its_cells(L):
    """The label start of the Voronoi labels of a set of seeds: every grain
    positive exactly on its label cells, the boxes of the seed start of the
    same seeds, and the seed start's signs wherever the seed start's own
    bisector function (reading R7, which looks only at face neighbours) agrees
    with the labels."""
    N, G = 64, 50
    seeds = I.voronoi_seeds(1, G, (N, N, N))
    lab = O.labels_of_tessellation((N, N, N), seeds).astype(np.int32)
    seed_ref = O.tessellate((N, N, N), seeds)
    with L.Microstructure(N, N, N, G, labels=lab) as a, L.Microstructure(N, N, N, G, seeds=seeds) as b:
        assert np.array_equal(a.boxes(), b.boxes())
        pa, pb = a.phi(), b.phi()
    n_r7 = 0
    for g in pa:
        gr = seed_ref.grains[g]
        mine = lab[np.ix_(*O.box_positions(gr, (N, N, N)))] == g
        assert np.array_equal(pa[g] > 0, mine), g
        agree = (gr.phi > 0) == mine
        n_r7 += int((~agree).sum())
        assert np.array_equal((pb[g] > 0)[agree], mine[agree]), g
    assert n_r7 < 10
