"""GPU tests of the stateless device ops of the C ABI (device pointers from
torch tensors; torch is only the allocator here)."""
import numpy as np
import pytest

from oracle import lsgg_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1701_06658_gb300 import lsgg
    lsgg.lib()
    return torch, lsgg


def neighbour_max_case(seed, shape_zyx, n_boxes):
    """Random boxes (some spanning a whole axis) with values in [-7, 7], a share
    of exact -7 values and exact ties between boxes."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape_zyx
    rows, vals, off = [], [], 0
    for i in range(n_boxes):
        dims = []
        for n in (nx, ny, nz):
            dims.append(n if rng.uniform() < 0.15 else int(rng.integers(1, n + 1)))
        org = [int(rng.integers(0, n)) for n in (nx, ny, nz)]
        cnt = dims[0] * dims[1] * dims[2]
        v = rng.uniform(-7, 7, cnt).astype(np.float32)
        v[rng.uniform(size=cnt) < 0.2] = -7.0
        v[rng.uniform(size=cnt) < 0.1] = 1.25            # ties across boxes
        rows.append((org[0], org[1], org[2], dims[0], dims[1], dims[2], off))
        vals.append(v)
        off += cnt
    boxes = np.array(rows, dtype=[("ox", "<i4"), ("oy", "<i4"), ("oz", "<i4"), ("nx", "<i4"), ("ny", "<i4"),
                                   ("nz", "<i4"), ("offset", "<i8")])
    return boxes, np.concatenate(vals)


def oracle_neighbour_max(boxes, phip, shape_zyx, eps=7.0):
    grains, pp = [], {}
    for i, b in enumerate(boxes):
        arr = phip[b["offset"]:b["offset"] + b["nx"] * b["ny"] * b["nz"]].reshape(b["nz"], b["ny"], b["nx"])
        grains.append(O.Grain(i, (int(b["oz"]), int(b["oy"]), int(b["ox"])), arr.astype(np.float64)))
        pp[i] = grains[-1].phi
    m_all, id_all = [], []
    for i in range(len(boxes)):
        m, idm = O.neighbour_max(i, grains, pp, shape_zyx, eps)
        m_all.append(m.ravel())
        id_all.append(idm.ravel())
    return np.concatenate(m_all), np.concatenate(id_all)


def run_neighbour_max(torch, L, boxes, phip, shape_zyx, fn="alloc"):
    nz, ny, nx = shape_zyx
    dev = torch.device("cuda:0")
    tb = torch.from_numpy(boxes.view(np.uint8).copy()).to(dev)
    tp = torch.from_numpy(phip).to(dev)
    tm = torch.full((phip.size,), 123.0, dtype=torch.float32, device=dev)
    ti = torch.full((phip.size,), -99, dtype=torch.int32, device=dev)
    if fn == "alloc":
        scratch = torch.empty(2 * nx * ny * nz, dtype=torch.int64, device=dev)
        L.neighbour_max(tb.data_ptr(), len(boxes), tp.data_ptr(), phip.size, nx, ny, nz, 7.0,
                        scratch.data_ptr(), tm.data_ptr(), ti.data_ptr(), torch.cuda.current_stream().cuda_stream)
    else:
        fn(tb.data_ptr(), len(boxes), tp.data_ptr(), phip.size, nx, ny, nz, 7.0, tm.data_ptr(), ti.data_ptr(),
           torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return tm.cpu().numpy(), ti.cpu().numpy()


@pytest.mark.parametrize("seed,shape,n", [(1, (12, 15, 17), 9), (2, (1, 40, 33), 14), (3, (20, 20, 20), 25)])
def test_neighbour_max_matches_oracle(env, seed, shape, n):
    torch, L = env
    boxes, phip = neighbour_max_case(seed, shape, n)
    m, idm = run_neighbour_max(torch, L, boxes, phip, shape)
    m_ref, id_ref = oracle_neighbour_max(boxes, phip, shape)
    assert np.array_equal(m, m_ref.astype(np.float32))
    assert np.array_equal(idm, id_ref)


def test_neighbour_max_skips_invalid_boxes(env):
    torch, L = env
    shape = (10, 10, 10)
    boxes, phip = neighbour_max_case(4, shape, 5)
    spans = [(int(b["offset"]), int(b["nx"] * b["ny"] * b["nz"])) for b in boxes]
    boxes[2]["offset"] = phip.size        # reaches past n_elems
    boxes[3]["nx"] = 11                   # wider than the domain
    m, idm = run_neighbour_max(torch, L, boxes, phip, shape)
    for k in (2, 3):                      # skipped: their original cells keep the fill value
        o, n = spans[k]
        assert np.all(m[o:o + n] == 123.0) and np.all(idm[o:o + n] == -99)
    for k in (0, 1, 4):
        o, n = spans[k]
        assert np.all(m[o:o + n] != 123.0)
