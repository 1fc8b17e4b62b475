"""lsgg_neighbour_max_noalloc against lsgg_neighbour_max.

The no-allocation entry point is for callers that cannot allocate device
memory (hosts that give all of it to their own pool, or keep cudaMalloc and
cudaFree out of latency-critical loops).  It must return exactly what the
allocating entry point returns on the same inputs, call after call, although
its scratch field is one static device array shared by every call.  This file
is collected last so a failure here comes after every other test has run.
"""
import numpy as np
import pytest

from tests.test_gpu_ops import neighbour_max_case, run_neighbour_max

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1701_06658_gb300 import lsgg
    lsgg.lib()
    return torch, lsgg


def test_no_alloc_matches_allocating_entry_point_twice(env):
    torch, L = env
    # two calls in a row on different inputs: the second must not see the first's field
    for seed, shape, n in ((11, (16, 20, 24), 12), (12, (1, 64, 48), 20)):
        boxes, phip = neighbour_max_case(seed, shape, n)
        want_m, want_id = run_neighbour_max(torch, L, boxes, phip, shape)
        got_m, got_id = run_neighbour_max(torch, L, boxes, phip, shape, fn=L.neighbour_max_noalloc)
        assert np.array_equal(got_m, want_m)        # the op is exact: tolerance 0
        assert np.array_equal(got_id, want_id)


def test_no_alloc_rejects_domains_above_its_limit(env):
    torch, L = env
    boxes, phip = neighbour_max_case(13, (4, 4, 4), 2)
    with pytest.raises(L.LsggError) as e:
        run_neighbour_max(torch, L, boxes, phip, (128, 128, 65), fn=L.neighbour_max_noalloc)
    assert e.value.code == L.ERR_CAPACITY
