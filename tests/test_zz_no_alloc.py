"""lsgg_neighbour_max_noalloc against lsgg_neighbour_max.

The no-allocation entry point is for callers that cannot allocate device
memory (hosts that give all of it to their own pool, or keep cudaMalloc and
cudaFree out of latency-critical loops).  It must return exactly what the
allocating entry point returns on the same inputs, call after call, although
its scratch field is one static device array shared by every call, and it
must leave the device's free memory unchanged.  This file is collected last
so a failure here comes after every other test has run.
"""
import numpy as np
import pytest

from tests.test_gpu_ops import neighbour_max_case, run_neighbour_max

pytestmark = pytest.mark.gpu

# domains of different sizes, in an order that puts a larger domain after a
# smaller one and a smaller one after a larger one: a clear of the shared field
# that covered only part of it would leave stale keys that a later call reads
CASES = ((11, (16, 20, 24), 12), (12, (1, 64, 48), 20), (14, (40, 48, 44), 30), (15, (6, 9, 7), 5))


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1701_06658_gb300 import lsgg
    lsgg.lib()
    return torch, lsgg


def _device_case(torch, boxes, phip):
    dev = torch.device("cuda:0")
    tb = torch.from_numpy(boxes.view(np.uint8).copy()).to(dev)
    tp = torch.from_numpy(phip).to(dev)
    tm = torch.full((phip.size,), 123.0, dtype=torch.float32, device=dev)
    ti = torch.full((phip.size,), -99, dtype=torch.int32, device=dev)
    return tb, tp, tm, ti


def test_no_alloc_matches_allocating_entry_point_call_after_call(env):
    torch, L = env
    cases = []
    for seed, shape, n in CASES:
        boxes, phip = neighbour_max_case(seed, shape, n)
        want = run_neighbour_max(torch, L, boxes, phip, shape)
        cases.append((boxes, phip, shape, want, _device_case(torch, boxes, phip)))
    stream = torch.cuda.current_stream().cuda_stream

    def call(k):
        boxes, phip, shape, _, (tb, tp, tm, ti) = cases[k]
        nz, ny, nx = shape
        L.neighbour_max_noalloc(tb.data_ptr(), len(boxes), tp.data_ptr(), phip.size, nx, ny, nz, 7.0,
                                tm.data_ptr(), ti.data_ptr(), stream)

    call(0)                              # the first call on the device loads the module
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    order = [0, 1, 2, 3, 2, 0, 3, 1]     # two calls in a row on different inputs, both size orders
    for k in order:
        call(k)
        torch.cuda.synchronize()
        want_m, want_id = cases[k][3]
        tm, ti = cases[k][4][2], cases[k][4][3]
        assert np.array_equal(tm.cpu().numpy(), want_m), k     # the op is exact: tolerance 0
        assert np.array_equal(ti.cpu().numpy(), want_id), k
    assert torch.cuda.mem_get_info()[0] == free_before


def test_no_alloc_rejects_domains_above_its_limit(env):
    torch, L = env
    boxes, phip = neighbour_max_case(13, (4, 4, 4), 2)
    with pytest.raises(L.LsggError) as e:
        run_neighbour_max(torch, L, boxes, phip, (128, 128, 65), fn=L.neighbour_max_noalloc)
    assert e.value.code == L.ERR_CAPACITY
