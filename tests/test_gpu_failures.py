"""Failure handling without faulting a GPU: a box arena that runs out of room
mid-run (grown on the host, steps resumed, same result), a bounded device
wait that nothing completes (gives up and reports it), a host wait that
times out while work is still running."""
import numpy as np
import pytest

from oracle import lsgg_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1701_06658_gb300 import lsgg
    lsgg.lib()
    return lsgg


def _growing_sphere(L, N=40, r0=8.0, de=0.5):
    """A low-energy sphere in a matrix grain: it grows (Eq. (19) bulk term),
    so its box and the arena's need grow with it."""
    c = N / 2.0
    ref = O.single_grain_state((N, N, N), lambda z, y, x: r0 - np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2))
    boxes = np.zeros((2, 7), np.int32)
    phi, idf = {}, {}
    for g in ref.grains:
        oz, oy, ox = g.origin
        nz, ny, nx = g.dims
        boxes[g.gid] = (1, ox, oy, oz, nx, ny, nz)
        phi[g.gid] = g.phi.astype(np.float32)
        idf[g.gid] = np.full(g.dims, 1 - g.gid, np.int32)
    seeds = np.array([[c, c, c], [1.0, 1.0, 1.0]])
    ms = L.Microstructure(N, N, N, 2, seeds=seeds, physics=L.PHYSICS_MAGNETIC, energy=np.array([0.0, de]))
    ms.set_state(boxes, phi, idf)
    return ms


def _need(boxes):
    n = 0
    for b in boxes:
        if b[0]:
            ps = (int(b[4]) * int(b[5]) + 7) & ~7
            n += (ps * int(b[6]) + 31) & ~31
    return n


def test_arena_overflow_is_recovered_bit_for_bit(L):
    with _growing_sphere(L) as a:
        a.step(12, 1.0)
        a.sync()
        want_phi, want_boxes = L.get_phi(a.ctx), a.boxes()
    with _growing_sphere(L) as b:
        cap = _need(b.boxes())
        L.debug_set_capacity(b.ctx, cap)
        assert b.stats().arena_capacity == (cap + 31) & ~31
        b.step(12, 1.0)
        b.sync()                                   # detects the overflow, grows, resumes
        st = b.stats()
        assert st.steps_done == 12
        assert st.arena_capacity > cap
        assert np.array_equal(b.boxes(), want_boxes)
        assert np.array_equal(L.get_phi(b.ctx), want_phi)
    assert want_boxes[0, 4] > 2 * 8 + 10          # the sphere did grow


def test_bounded_device_wait_gives_up(L):
    assert L.debug_wait_timeout(0, 2000) is True


def test_host_wait_times_out_while_work_runs(L):
    from paper_1701_06658_gb300 import inputs as I
    N, G = 64, 50
    with L.Microstructure(N, N, N, G, seeds=I.voronoi_seeds(1, G, (N, N, N))) as ms:
        ms.step(300, 1.0)
        code = L.lib().lsgg_sync(ms.ctx, 0)
        assert code in (L.OK, L.ERR_TIMEOUT)
        ms.sync()
        assert ms.stats().steps_done == 300


def test_step_waits_give_up_and_the_context_recovers(L):
    """The pass kernels' own bounded waits: with the poll limit lowered to zero
    every plane pass gives up at its first wait on a bulk copy, records
    LSGG_ERR_TIMEOUT, halts the step and drains its copies; lsgg_sync reports
    the timeout once.  Nothing was written to the state, so with the default
    limit restored the steps run as in a context that never timed out."""
    from paper_1701_06658_gb300 import inputs as I
    N, G = 64, 50
    seeds = I.voronoi_seeds(1, G, (N, N, N))
    with L.Microstructure(N, N, N, G, seeds=seeds) as a:
        a.step(3, 1.0)
        a.sync()
        want_phi, want_boxes = L.get_phi(a.ctx), a.boxes()
    with L.Microstructure(N, N, N, G, seeds=seeds) as b:
        L.debug_set_wait_limit(b.ctx, 0)
        b.step(2, 1.0)
        assert L.lib().lsgg_sync(b.ctx, -1) == L.ERR_TIMEOUT
        assert L.lib().lsgg_sync(b.ctx, -1) == L.OK          # reported once
        assert b.stats().steps_done == 0
        L.debug_set_wait_limit(b.ctx, -1)
        b.step(3, 1.0)
        b.sync()
        assert b.stats().steps_done == 3
        assert np.array_equal(b.boxes(), want_boxes)
        assert np.array_equal(L.get_phi(b.ctx), want_phi)
