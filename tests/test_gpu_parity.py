"""GPU parity of the batched CUDA path against the FP64 oracle.

Every test calls the library through its C ABI (ctypes binding) on cuda:0 and
compares element by element with the oracle on the same seeded inputs.
Tolerances: max |phi_gpu - phi_oracle| <= 1e-4 except within 7 cells of a
cell whose sign the two disagree on at |phi_c| < 1e-4; boxes exact; voxel
ownership exact except where the two largest functions differ by < 1e-4;
per-grain volumes within 0.1 % after 20 steps.
"""
import numpy as np
import pytest

from oracle import lsgg_oracle as O
from paper_1701_06658_gb300 import inputs as I
from tests.parity import box_full, oracle_from_gpu, sign_flip_exclusion

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


def _check_step(L, ms, dt=1.0, tol_p=2e-5):
    """One debug step on the GPU vs the oracle's step on the same FP32 state."""
    shape = ms.shape
    boxes = ms.boxes()
    phi = ms.phi()
    ref_ms = oracle_from_gpu(shape, boxes, phi)
    ref = O.step_parts(ref_ms, dt)
    b2, (phip, m, idm, phic, phin) = ms.debug_step(dt)
    assert np.array_equal(b2, boxes)
    worst = {"phip": 0.0, "m": 0.0, "phic": 0.0, "phin": 0.0}
    flips = 0
    for g in phin:
        worst["phip"] = max(worst["phip"], float(np.max(np.abs(phip[g] - ref.phip[g]))))
        worst["m"] = max(worst["m"], float(np.max(np.abs(m[g] - ref.m[g]))))
        worst["phic"] = max(worst["phic"], float(np.max(np.abs(phic[g] - ref.phic[g]))))
        excl = sign_flip_exclusion(ref.phic[g], phic[g], box_full(boxes[g], shape))
        flips += int(excl.sum())
        d = np.abs(phin[g] - ref.phi[g])
        d[excl] = 0
        worst["phin"] = max(worst["phin"], float(d.max()))
    assert worst["phip"] <= tol_p, worst
    assert worst["m"] <= tol_p, worst
    assert worst["phic"] <= tol_p, worst
    assert worst["phin"] <= TOL_PHI, worst
    # ID-field: equal except near-ties of the neighbour max
    for g in phin:
        bad = idm[g] != ref.idm[g]
        if bad.any():
            pos = O.box_positions(ref_ms.grains[g], shape)
            for (z, y, x) in zip(*np.nonzero(bad)):
                j = int(idm[g][z, y, x])
                if j < 0:     # GPU max rounded to -eps: a near-tie with "no neighbour"
                    assert ref.m[g][z, y, x] < -7.0 + 1e-4
                    continue
                view = O.Grain(j, ref_ms.grains[j].origin, ref.phip[j])
                v, _ = O.sample(view, (pos[0][[z]], pos[1][[y]], pos[2][[x]]), shape, -7.0)
                assert abs(float(v.ravel()[0]) - ref.m[g][z, y, x]) < 1e-4, (g, j, worst)
    return ref_ms, ref, worst, flips


def test_init_matches_oracle(L):
    """64^3, 50 Voronoi grains (seed 1): boxes bit-exact, phi = oracle cast to FP32."""
    N, G = 64, 50
    seeds = I.voronoi_seeds(1, G, (N, N, N))
    ref = O.tessellate((N, N, N), seeds)
    with L.Microstructure(N, N, N, G, seeds=seeds) as ms:
        boxes = ms.boxes()
        phi = ms.phi()
    for g, gr in enumerate(ref.grains):
        assert bool(boxes[g, 0]) == gr.alive
        if not gr.alive:
            continue
        assert (boxes[g, 3], boxes[g, 2], boxes[g, 1]) == gr.origin
        assert (boxes[g, 6], boxes[g, 5], boxes[g, 4]) == gr.dims
        assert np.max(np.abs(phi[g] - gr.phi.astype(np.float32))) <= 1e-6


def test_single_step_parity_64(L):
    N, G = 64, 50
    seeds = I.voronoi_seeds(1, G, (N, N, N))
    with L.Microstructure(N, N, N, G, seeds=seeds) as ms:
        ms.step(3, 1.0)
        ref_ms, ref, worst, _ = _check_step(L, ms)
        # the box update of the oracle on its own result
        boxes_after = ms.boxes()
        for g, gr in enumerate(ref_ms.grains):
            if not gr.alive:
                continue
            upd = O.box_update(O.Grain(g, gr.origin, ref.phi[g]), ref_ms.shape, 5, 7.0)
            assert bool(boxes_after[g, 0]) == upd.alive
            if upd.alive:
                assert (boxes_after[g, 3], boxes_after[g, 2], boxes_after[g, 1]) == upd.origin
                assert (boxes_after[g, 6], boxes_after[g, 5], boxes_after[g, 4]) == upd.dims


@pytest.mark.parametrize("shape,G,seed", [((1, 96, 96), 12, 4), ((24, 24, 24), 3, 5), ((29, 41, 37), 20, 6),
                                          ((1, 50, 300), 9, 8)])
def test_single_step_parity_edge_domains(L, shape, G, seed):
    """2D, tiny 3D with full periodic boxes, ragged sizes, a long 2D strip."""
    nz, ny, nx = shape
    seeds = I.voronoi_seeds(seed, G, (nx, ny, nz))
    with L.Microstructure(nx, ny, nz, G, seeds=seeds) as ms:
        ms.step(2, 1.0)
        _check_step(L, ms)


def test_multistep_volumes_and_owner_64(L):
    """20 steps of the 64^3 / 50-grain workload: per-grain volumes within 0.1 %
    of the oracle's 20 steps from the same seeds; ownership exact except at
    near-ties."""
    N, G, steps = 64, 50, 20
    seeds = I.voronoi_seeds(1, G, (N, N, N))
    with L.Microstructure(N, N, N, G, seeds=seeds) as ms:
        ms.step(steps, 1.0)
        ms.sync()
        vg = ms.grain_volumes()
        own = ms.voxel_owner()
    ref = O.run(O.tessellate((N, N, N), seeds), steps, 1.0)
    vo = O.volumes(ref)
    big = vo > 50
    rel = np.abs(vg - vo)[big] / vo[big]
    assert rel.max() <= 1e-3, rel.max()
    assert np.all(np.abs(vg - vo)[~big] <= 0.05)
    ro = O.owner_map(ref)
    diff = own != ro
    if diff.any():
        # a mismatch must be a near-tie of the top two functions in the oracle
        allpos = tuple(np.arange(s) for s in ref.shape)
        vals = np.stack([O.sample(g, allpos, ref.shape, -np.inf)[0] for g in ref.grains if g.alive])
        top = np.sort(vals, axis=0)
        gap = top[-1] - top[-2]
        assert np.all(gap[diff] < 1e-4), int(diff.sum())
    assert (own >= 0).all()
    assert np.bincount(own.ravel(), minlength=G).sum() == N ** 3


def test_deterministic(L):
    N, G = 48, 20
    seeds = I.voronoi_seeds(11, G, (N, N, N))
    out = []
    for _ in range(2):
        with L.Microstructure(N, N, N, G, seeds=seeds) as ms:
            ms.step(5, 1.0)
            out.append((ms.boxes(), L.get_phi(ms.ctx), ms.grain_volumes()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][2], out[1][2])


def test_extinction_matches_oracle(L):
    """A small sphere in a matrix shrinks away: the GPU and the oracle agree on
    the step at which it becomes extinct (and the matrix then fills the domain)."""
    N = 32
    c = N / 2.0
    ref = O.single_grain_state((N, N, N), lambda z, y, x: 4.5 - np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2))
    boxes = np.zeros((2, 7), np.int32)
    phi = {}
    for g in ref.grains:
        oz, oy, ox = g.origin
        nz, ny, nx = g.dims
        boxes[g.gid] = (1, ox, oy, oz, nx, ny, nz)
        phi[g.gid] = g.phi.astype(np.float32)
    seeds = np.array([[c, c, c], [1.0, 1.0, 1.0]])
    with L.Microstructure(N, N, N, 2, seeds=seeds) as ms:
        ms.set_state(boxes, phi)
        for k in range(12):
            ms.step(1, 1.0)
            ref = O.step(ref, 1.0)
            assert bool(ms.boxes()[0, 0]) == ref.grains[0].alive, k
        assert not ref.grains[0].alive
        assert (ms.voxel_owner() == 1).all()


def test_large_domain_properties_and_sampled_parity(L):
    """The 256^3 / 5000-grain workload: every cell owned after 2 steps, volumes
    sum to N^3, and one step of 6 sampled grains equals the oracle's step of
    those grains computed from the same state (the oracle evaluates only the
    sampled grains and the grains whose boxes meet theirs)."""
    N, G = 256, 5000
    seeds = I.voronoi_seeds(2, G, (N, N, N))
    with L.Microstructure(N, N, N, G, seeds=seeds) as ms:
        ms.step(2, 1.0)
        boxes = ms.boxes()
        phi = ms.phi()
        ref_ms = oracle_from_gpu((N, N, N), boxes, phi)
        b2, (phip, m, idm, phic, phin) = ms.debug_step(1.0)
        own = ms.voxel_owner()
        vol = ms.grain_volumes()
    assert (own >= 0).all()
    assert abs(vol.sum() - N ** 3) / N ** 3 < 2e-3
    rng = np.random.default_rng(0)
    alive = [g for g in range(G) if boxes[g, 0]]
    sample = rng.choice(alive, 6, replace=False)
    taps = O.heat_kernel_taps(1.0, 5)
    for g in sample:
        gi = ref_ms.grains[g]
        cand = [j for j in alive if j != g and O.boxes_intersect(gi, ref_ms.grains[j], (N, N, N))]
        pp = {j: O.predict(ref_ms.grains[j], (N, N, N), taps, 7.0) for j in cand + [int(g)]}
        mm, _ = O.neighbour_max(int(g), ref_ms.grains, pp, (N, N, N), 7.0, cand)
        pc = O.compare(pp[int(g)], mm)
        full = box_full(boxes[g], (N, N, N))
        pn = np.clip(O.redistance(pc, full, 7.0, (0, 1, 2)), -7, 7)
        assert np.max(np.abs(phip[g] - pp[int(g)])) <= 2e-5
        assert np.max(np.abs(m[g] - mm)) <= 2e-5
        excl = sign_flip_exclusion(pc, phic[g], full)
        d = np.abs(phin[g] - pn)
        d[excl] = 0
        assert d.max() <= TOL_PHI


def test_plain_path_matches_batched_and_oracle(L):
    """The per-grain comparator path (separate launches per grain and
    sub-step) gives the batched path's result: same boxes, phi within 1e-5."""
    N, G = 48, 24
    seeds = I.voronoi_seeds(21, G, (N, N, N))
    out = {}
    for mode in (L.EXEC_BATCHED, L.EXEC_PLAIN):
        with L.Microstructure(N, N, N, G, seeds=seeds, exec_mode=mode) as ms:
            ms.step(3, 1.0)
            ms.sync()
            out[mode] = (ms.boxes(), L.get_phi(ms.ctx), ms.grain_volumes())
    assert np.array_equal(out[0][0], out[1][0])
    assert np.max(np.abs(out[0][1] - out[1][1])) <= 1e-5
    assert np.max(np.abs(out[0][2] - out[1][2])) <= 1e-3


def test_graph_replay_equals_eager_launches(L):
    """Steps replayed from the captured CUDA graph equal eager launches bit for bit."""
    N, G = 40, 16
    seeds = I.voronoi_seeds(22, G, (N, N, N))
    res = []
    for prof in (False, True):
        with L.Microstructure(N, N, N, G, seeds=seeds) as ms:
            L.profile(ms.ctx, prof)       # profiling forces eager launches
            ms.step(4, 1.0)
            ms.sync()
            res.append(L.get_phi(ms.ctx))
    assert np.array_equal(res[0], res[1])


def test_grain_neighbours_are_the_id_field(L):
    """Contact neighbours after a step = the distinct grains of the step's
    ID-field (Sec. 3.1), and the relation is symmetric between touching grains."""
    N, G = 48, 24
    seeds = I.voronoi_seeds(23, G, (N, N, N))
    with L.Microstructure(N, N, N, G, seeds=seeds) as ms:
        ms.step(2, 1.0)
        with pytest.raises(L.LsggError) as e:      # the pass path keeps the field only on request
            L.grain_neighbours(ms.ctx, G)
        assert e.value.code == L.ERR_NOT_READY
        L.keep_field(ms.ctx, True)
        _, (phip, m, idm, phic, phin) = ms.debug_step(1.0)
        nb = L.grain_neighbours(ms.ctx, G)
    for g in phin:
        assert nb[g] == sorted(set(np.unique(idm[g][idm[g] >= 0]).tolist()))
    touching = {(a, b) for a in phin for b in nb[a]}
    assert len(touching) > 0
    # a grain that sees b at its interface is seen by b (both are the top two there)
    asym = [(a, b) for (a, b) in touching if (b, a) not in touching]
    assert len(asym) <= 0.05 * len(touching)


def test_autotune_keeps_results_bitwise(L):
    """The tile variants the autotuner tries give bit-identical steps: a tuned
    run (3 x 2 tuning steps) equals an untuned run of as many steps."""
    N, G = 64, 50
    seeds = I.voronoi_seeds(24, G, (N, N, N))
    with L.Microstructure(N, N, N, G, seeds=seeds, exec_mode=L.EXEC_STREAMED) as a:
        a.step(6, 1.0)
        pa = L.get_phi(a.ctx)
        ba = a.boxes()
    with L.Microstructure(N, N, N, G, seeds=seeds, exec_mode=L.EXEC_STREAMED) as b:
        chosen = L.autotune(b.ctx, 2, 1.0)
        assert b.stats().steps_done == 6
        pb = L.get_phi(b.ctx)
        bb = b.boxes()
    assert any(v >= 0 for v in chosen["k_predict"])
    assert np.array_equal(ba, bb)
    assert np.array_equal(pa, pb)


@pytest.mark.parametrize("shape,G,seed", [((64, 64, 64), 50, 31), ((40, 72, 56), 30, 32), ((24, 24, 24), 5, 33),
                                          ((96, 96, 96), 12, 34)])
def test_pass_path_matches_box_streaming(L, shape, G, seed):
    """The pass path (five passes over plane / column work items) and the
    box-streaming kernels compute the same step: same boxes, phi within 1e-5
    over 6 steps, on cubic, non-cubic, full-axis (few grains in a small
    domain) and large-box (x, y sides above 64) cases."""
    nx, ny, nz = shape
    seeds = I.voronoi_seeds(seed, G, (nx, ny, nz))
    out = {}
    for mode in (L.EXEC_BATCHED, L.EXEC_STREAMED):
        with L.Microstructure(nx, ny, nz, G, seeds=seeds, exec_mode=mode) as ms:
            ms.step(6, 1.0)
            ms.sync()
            out[mode] = (ms.boxes(), L.get_phi(ms.ctx), ms.grain_volumes())
    a, b = out[L.EXEC_BATCHED], out[L.EXEC_STREAMED]
    assert np.array_equal(a[0], b[0])
    assert np.max(np.abs(a[1] - b[1])) <= 1e-5
    assert np.max(np.abs(a[2] - b[2])) <= 1e-3


def test_pass_times_cover_every_pass(L):
    """Profiled steps on the pass path report each pass of each tier once per step."""
    N, G = 64, 50
    seeds = I.voronoi_seeds(35, G, (N, N, N))
    with L.Microstructure(N, N, N, G, seeds=seeds) as ms:
        L.profile(ms.ctx, True)
        ms.step(3, 1.0)
        L.kernel_times(ms.ctx)
        pt = L.pass_times(ms.ctx)
        L.profile(ms.ctx, False)
    assert len(pt) == 4 * L.PASS_TIERS + 2
    for name, (ms_, n) in pt.items():
        assert n == 3, (name, n)
        assert ms_ >= 0.0


def test_field_pass_with_overflowing_tile_lists(L):
    """Dense small grains put more boxes on a domain tile than its list holds
    (over 128): the field pass then tests every box for those tiles, and the
    step still equals the box-streaming kernels' step."""
    N, G = 64, 2000
    seeds = I.voronoi_seeds(36, G, (N, N, N))
    out = {}
    for mode in (L.EXEC_BATCHED, L.EXEC_STREAMED):
        with L.Microstructure(N, N, N, G, seeds=seeds, exec_mode=mode) as ms:
            s = ms.stats()
            assert s.superimposition > 20          # about 260 boxes per 32 x 8 x 16 tile
            ms.step(2, 1.0)
            ms.sync()
            out[mode] = (ms.boxes(), L.get_phi(ms.ctx))
    a, b = out[L.EXEC_BATCHED], out[L.EXEC_STREAMED]
    assert np.array_equal(a[0], b[0])
    assert np.max(np.abs(a[1] - b[1])) <= 1e-5


def test_godunov_single_step_matches_oracle(L):
    """LSGG_REDIST_GODUNOV: one step from the GPU's state equals the oracle's
    step with the Godunov re-initialisation (reading R11) to the FP32
    tolerance; the predictor and comparison parts are the taxicab run's."""
    N, G = 64, 50
    seeds = I.voronoi_seeds(1, G, (N, N, N))
    with L.Microstructure(N, N, N, G, seeds=seeds, redist=L.REDIST_GODUNOV) as ms:
        ms.step(3, 1.0)
        boxes = ms.boxes()
        phi = ms.phi()
        ref_ms = oracle_from_gpu((N, N, N), boxes, phi)
        ref_ms.redist = "godunov"
        ref = O.step_parts(ref_ms, 1.0)
        b2, (phip, m, idm, phic, phin) = ms.debug_step(1.0)
    assert np.array_equal(b2, boxes)
    worst = 0.0
    for g in phin:
        assert np.max(np.abs(phic[g] - ref.phic[g])) <= 2e-5
        excl = sign_flip_exclusion(ref.phic[g], phic[g], box_full(boxes[g], (N, N, N)))
        d = np.abs(phin[g] - ref.phi[g])
        d[excl] = 0
        worst = max(worst, float(d.max()))
    assert worst <= TOL_PHI, worst


def test_godunov_multistep_volumes(L):
    """Six Godunov steps of a 48^3 / 24-grain microstructure: per-grain volumes
    within 0.1 % of the oracle's, every cell owned."""
    N, G = 48, 24
    seeds = I.voronoi_seeds(41, G, (N, N, N))
    ref = O.tessellate((N, N, N), seeds)
    ref.redist = "godunov"
    ref = O.run(ref, 6, 1.0)
    with L.Microstructure(N, N, N, G, seeds=seeds, redist=L.REDIST_GODUNOV) as ms:
        ms.step(6, 1.0)
        vol = ms.grain_volumes()
        own = ms.voxel_owner()
    want = O.volumes(ref)
    alive = want > 1.0
    assert np.max(np.abs(vol[alive] - want[alive]) / want[alive]) < 1e-3
    assert (own >= 0).all()


def test_grain_statistics_on_device(L):
    """The device statistics equal the oracle's definition evaluated on the
    device's own volumes (to rounding), and on the oracle's volumes after the
    20-step run (to the 0.1 % volume tolerance)."""
    N, G = 64, 50
    seeds = I.voronoi_seeds(1, G, (N, N, N))
    with L.Microstructure(N, N, N, G, seeds=seeds) as ms:
        ms.step(20, 1.0)
        st = ms.grain_statistics(16, 2.5)
        vol = ms.grain_volumes()
    want = O.grain_statistics(vol, 3, 16, 2.5)
    assert st["alive"] == want["alive"]
    for k in ("mean_volume", "mean_radius", "rms_radius", "max_radius", "overflow", "rho", "var_z"):
        assert abs(st[k] - want[k]) <= 1e-12 * max(1.0, abs(want[k])), k
    assert np.array_equal(st["hist"], want["hist"])
    ref = O.run(O.tessellate((N, N, N), seeds), 20, 1.0)
    ow = O.grain_statistics(O.volumes(ref), 3, 16, 2.5)
    assert st["alive"] == ow["alive"]
    assert abs(st["mean_radius"] - ow["mean_radius"]) / ow["mean_radius"] < 1e-3



def test_texture_shares_on_device(L):
    """Volume fractions of grain classes (Sec. 5.3's texture components): the
    device's compensated sums equal the oracle's shares of the device's own
    volumes to rounding, and the shares of a partition sum to 1."""
    N, G = 64, 50
    seeds = I.voronoi_seeds(2, G, (N, N, N))
    cls = (np.arange(G) * 7) % 3
    cls[5] = -1                       # a grain in no class
    with L.Microstructure(N, N, N, G, seeds=seeds) as ms:
        ms.step(5, 1.0)
        sh = ms.texture_shares(cls, 3)
        vol = ms.grain_volumes()
        full = ms.texture_shares(np.zeros(G, np.int32), 1)
    want = O.texture_shares(vol, cls, 3)
    assert np.max(np.abs(sh - want)) <= 1e-14
    assert abs(full[0] - 1.0) <= 1e-15
    assert sh.sum() < 1.0


def test_single_grain_fills_the_domain(L):
    """Degenerate case: one grain.  No bisector exists, so its function is eps
    everywhere, its box is the whole periodic domain, the comparison step sees
    no other grain (m = -eps), and the state is a fixed point: after steps the
    grain still covers all N^3 cells and matches the oracle."""
    N = 32
    seeds = I.voronoi_seeds(12, 1, (N, N, N))
    ref = O.run(O.tessellate((N, N, N), seeds), 3, 1.0)
    with L.Microstructure(N, N, N, 1, seeds=seeds) as ms:
        ms.step(3, 1.0)
        boxes, phi, vol = ms.boxes(), ms.phi(), ms.grain_volumes()
    assert boxes[0, 0] == 1 and tuple(boxes[0, 4:7]) == (N, N, N)
    assert np.max(np.abs(phi[0] - ref.grains[0].phi)) <= 1e-6
    assert np.all(phi[0] == 7.0)
    assert vol[0] == N ** 3


def test_hartmann_single_step_matches_oracle(L):
    """LSGG_REDIST_HARTMANN: one step from the GPU's state equals the oracle's
    step with the constrained reinitialization (reading R16: 20 pseudo-time
    steps in FP32 against FP64) to the FP32 tolerance; the predictor and
    comparison parts are the taxicab run's."""
    N, G = 64, 50
    seeds = I.voronoi_seeds(1, G, (N, N, N))
    with L.Microstructure(N, N, N, G, seeds=seeds, redist=L.REDIST_HARTMANN) as ms:
        ms.step(3, 1.0)
        boxes = ms.boxes()
        phi = ms.phi()
        ref_ms = oracle_from_gpu((N, N, N), boxes, phi)
        ref_ms.redist = "hartmann"
        ref = O.step_parts(ref_ms, 1.0)
        b2, (phip, m, idm, phic, phin) = ms.debug_step(1.0)
        after = ms.boxes()
    assert np.array_equal(b2, boxes)
    worst = 0.0
    for g in phin:
        assert np.max(np.abs(phic[g] - ref.phic[g])) <= 2e-5
        excl = sign_flip_exclusion(ref.phic[g], phic[g], box_full(boxes[g], (N, N, N)))
        d = np.abs(phin[g] - ref.phi[g])
        d[excl] = 0
        worst = max(worst, float(d.max()))
    assert worst <= TOL_PHI, worst
    for g, gr in enumerate(ref_ms.grains):
        if gr.alive:
            upd = O.box_update(O.Grain(g, gr.origin, ref.phi[g]), ref_ms.shape, 5, 7.0)
            assert bool(after[g, 0]) == upd.alive
            if upd.alive:
                assert (after[g, 3], after[g, 2], after[g, 1]) == upd.origin
                assert (after[g, 6], after[g, 5], after[g, 4]) == upd.dims


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_hartmann_multistep_volumes(L, storage):
    """Six Hartmann steps of a 48^3 / 24-grain microstructure: per-grain volumes
    within 0.1 % of the oracle's (FP32 state; with BF16 storage within the
    BF16 variant's 0.5 %), every cell owned."""
    N, G = 48, 24
    seeds = I.voronoi_seeds(41, G, (N, N, N))
    ref = O.tessellate((N, N, N), seeds)
    ref.redist = "hartmann"
    ref = O.run(ref, 6, 1.0)
    st = L.STORAGE_FP32 if storage == "fp32" else L.STORAGE_BF16
    with L.Microstructure(N, N, N, G, seeds=seeds, redist=L.REDIST_HARTMANN, storage=st) as ms:
        ms.step(6, 1.0)
        vol = ms.grain_volumes()
        own = ms.voxel_owner()
    want = O.volumes(ref)
    alive = want > 1.0
    tol = 1e-3 if storage == "fp32" else 5e-3
    assert np.max(np.abs(vol[alive] - want[alive]) / want[alive]) < tol
    assert (own >= 0).all()


def test_pass_path_autotune_keeps_results_bitwise(L):
    """The pass path's autotuner (grid sizes per tier and pass, slab depth)
    runs 4 x 2 real steps under different settings; the result equals an
    untuned run of 8 steps bit for bit, and the chosen settings are within
    their ranges."""
    N, G = 64, 50
    seeds = I.voronoi_seeds(24, G, (N, N, N))
    with L.Microstructure(N, N, N, G, seeds=seeds) as a:
        a.step(8, 1.0)
        a.sync()
        pa, ba = L.get_phi(a.ctx), a.boxes()
    with L.Microstructure(N, N, N, G, seeds=seeds) as b:
        chosen = L.autotune(b.ctx, 2, 1.0)
        assert b.stats().steps_done == 8
        assert all(v == -1 for v in chosen["k_predict"])
        tune = L.pass_tuning(b.ctx)
        pb, bb = L.get_phi(b.ctx), b.boxes()
        b.step(2, 1.0)                        # the tuned settings step on
        b.sync()
    assert np.array_equal(ba, bb)
    assert np.array_equal(pa, pb)
    assert tune["slab"] in (4, 8, 16)
    assert all(1 <= v <= 32 for k, v in tune.items() if k != "slab")
