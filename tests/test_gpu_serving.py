"""GPU tests of the serving loop: continuous batching under an HBM budget.

Each request's result must be the same alone and in a mix with others that
overlap it on the device (bit for bit: the requests share no state and run
the same kernels); requests larger than the budget are refused; a small
budget serialises admissions without changing results.
"""
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


MIX = [(48, 30, 7, 12), (32, 20, 8, 30), (64, 60, 9, 9), (40, 25, 10, 17), (56, 40, 11, 5), (32, 20, 12, 21)]


def _direct(L, n, g, seed, steps):
    with L.Microstructure(n, n, n, g, seeds=I.voronoi_seeds(seed, g, (n, n, n))) as ms:
        ms.step(steps, 1.0)
        return ms.grain_volumes()


@pytest.mark.parametrize("mode", ["shared", "per_context"])
def test_result_alone_equals_result_in_the_mix(L, mode):
    """Shared launches (one step group over the running requests, rebuilt as
    they join and finish) and per-context streams give every request the
    result of running it alone."""
    n, g, seed, steps = MIX[0]
    seeds = I.voronoi_seeds(seed, g, (n, n, n))
    m = L.SERVE_SHARED if mode == "shared" else L.SERVE_PER_CONTEXT
    with L.Server(budget_bytes=8 << 30, max_active=8, steps_per_round=3, mode=m) as srv:
        t = srv.submit(n, n, n, g, steps, seeds=seeds)
        srv.wait(t)
        alone = srv.volumes(t)
        tickets = []
        for (nn, gg, sd, st) in MIX:
            tickets.append(srv.submit(nn, nn, nn, gg, st, seeds=I.voronoi_seeds(sd, gg, (nn, nn, nn))))
        infos = [srv.wait(tk) for tk in tickets]
        mixed = srv.volumes(tickets[0])
        # the requests did overlap: some were admitted before others finished
        assert min(i.t_done for i in infos) > max(i.t_admit for i in infos[:3])
        assert np.array_equal(alone, mixed)
        assert np.array_equal(alone, _direct(L, n, g, seed, steps))
        for (nn, gg, sd, st), tk in zip(MIX[1:], tickets[1:]):
            assert np.array_equal(srv.volumes(tk), _direct(L, nn, gg, sd, st))
        s = srv.stats()
        assert s.completed == len(MIX) + 1 and s.active == 0 and s.queued == 0


def test_budget_serialises_and_refuses(L):
    n, g, seed, steps = MIX[1]
    seeds = I.voronoi_seeds(seed, g, (n, n, n))
    # room for about one 32^3 request at a time
    with L.Server(budget_bytes=(64 << 20) + 3 * 4 * 18 * 32 ** 3 + 21 * 32 ** 3 + 4096, max_active=8,
                  steps_per_round=5) as srv:
        a = srv.submit(n, n, n, g, steps, seeds=seeds)
        b = srv.submit(n, n, n, g, steps, seeds=seeds)
        big = srv.submit(128, 128, 128, 200, 2)
        ia, ib = srv.wait(a), srv.wait(b)
        assert ib.t_admit >= ia.t_done          # the second waited for the first's memory
        assert np.array_equal(srv.volumes(a), srv.volumes(b))
        with pytest.raises(L.LsggError) as e:
            srv.wait(big)
        assert e.value.code == L.ERR_OVER_BUDGET


def test_shared_launches_with_requests_outside_the_group(L):
    """A server with shared launches runs requests the step group does not
    take (Read-Shockley physics; another dt; a domain above 128^3 cells) on
    their own streams beside the group; every result equals the request run
    alone."""
    reqs = [(40, 25, 21, 9, 1.0, {}), (48, 30, 22, 7, 1.0, {"physics": L.PHYSICS_READ_SHOCKLEY}),
            (32, 20, 23, 11, 0.5, {}), (36, 24, 24, 8, 1.0, {}), (132, 690, 25, 3, 1.0, {})]
    with L.Server(budget_bytes=8 << 30, max_active=8, steps_per_round=4, mode=L.SERVE_SHARED) as srv:
        tks = [srv.submit(n, n, n, g, st, dt=dt, seeds=I.voronoi_seeds(sd, g, (n, n, n)), **kw)
               for (n, g, sd, st, dt, kw) in reqs]
        for tk in tks:
            srv.wait(tk)
        for (n, g, sd, st, dt, kw), tk in zip(reqs, tks):
            with L.Microstructure(n, n, n, g, seeds=I.voronoi_seeds(sd, g, (n, n, n)), **kw) as ms:
                ms.step(st, dt)
                assert np.array_equal(srv.volumes(tk), ms.grain_volumes())


def test_label_request_is_copied_at_submit(L):
    """A request starting from a label field holds its own copy of the
    labels from submission on (the caller's array is overwritten right after
    submit), and ends with the volumes of the same start stepped alone."""
    from oracle import lsgg_oracle as O
    n, g, steps = 40, 20, 6
    lab = O.labels_of_tessellation((n, n, n), I.voronoi_seeds(81, g, (n, n, n))).astype(np.int32)
    with L.Microstructure(n, n, n, g, labels=lab) as ms:
        ms.step(steps, 1.0)
        want = ms.grain_volumes()
    with L.Server(budget_bytes=8 << 30, max_active=8, steps_per_round=3) as srv:
        buf = lab.copy()
        t = srv.submit(n, n, n, g, steps, labels=buf)
        buf[:] = -5
        srv.wait(t)
        assert np.array_equal(srv.volumes(t), want)
