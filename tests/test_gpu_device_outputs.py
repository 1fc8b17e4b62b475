"""The device-pointer output variants (lsgg_grain_volumes_device,
lsgg_voxel_owner_device) against the host variants, through the C ABI with
torch-allocated outputs: bit for bit, on the context's stream and on a
caller's stream, with FP32 and BF16 state storage, and the step status they
report when a step stopped on a full box arena."""
import numpy as np
import pytest

from paper_1701_06658_gb300 import inputs as I
from tests.test_gpu_failures import _growing_sphere, _need

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1701_06658_gb300 import lsgg
    lsgg.lib()
    return torch, lsgg


def _device_outputs(torch, L, ms, stream):
    G = ms.n_grains
    nz, ny, nx = ms.shape
    vol = torch.full((G,), -1.0, dtype=torch.float64, device="cuda:0")
    own = torch.full((nz * ny * nx,), -7, dtype=torch.int32, device="cuda:0")
    st = torch.full((2,), 99, dtype=torch.int32, device="cuda:0")
    sp = 0 if stream is None else stream.cuda_stream
    L.grain_volumes_device(ms.ctx, vol.data_ptr(), G, st.data_ptr(), sp)
    L.voxel_owner_device(ms.ctx, own.data_ptr(), own.numel(), st.data_ptr() + 4, sp)
    (stream or torch.cuda.ExternalStream(ms.stream)).synchronize()
    return vol.cpu().numpy(), own.cpu().numpy().reshape(ms.shape), st.cpu().numpy()


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_device_outputs_equal_host_outputs(env, storage):
    torch, L = env
    N, G = 64, 50
    st_kind = L.STORAGE_FP32 if storage == "fp32" else L.STORAGE_BF16
    with L.Microstructure(N, N, N, G, seeds=I.voronoi_seeds(1, G, (N, N, N)), storage=st_kind) as ms:
        ms.step(3, 1.0)
        for stream in (None, torch.cuda.Stream()):
            ms.step(1, 1.0)                      # enqueued, not waited for: the outputs order after it
            vol_d, own_d, status = _device_outputs(torch, L, ms, stream)
            vol_h = ms.grain_volumes()
            own_h = ms.voxel_owner()
            assert np.array_equal(vol_d, vol_h)
            assert np.array_equal(own_d, own_h)
            assert list(status) == [0, 0]
        assert ms.stats().steps_done == 5


def test_device_outputs_report_a_stopped_step(env):
    """A step that stops on a full box arena is reported through the status
    word; after lsgg_sync grows the arena and finishes the steps, the device
    outputs equal the host outputs again."""
    torch, L = env
    with _growing_sphere(L) as ms:
        L.debug_set_capacity(ms.ctx, _need(ms.boxes()))
        ms.step(12, 1.0)
        _, _, status = _device_outputs(torch, L, ms, None)
        assert list(status) == [L.ERR_CAPACITY] * 2
        ms.sync()
        assert ms.stats().steps_done == 12
        vol_d, own_d, status = _device_outputs(torch, L, ms, None)
        assert list(status) == [0, 0]
        assert np.array_equal(vol_d, ms.grain_volumes())
        assert np.array_equal(own_d, ms.voxel_owner())


def test_device_outputs_check_their_arguments(env):
    torch, L = env
    N, G = 24, 4
    with L.Microstructure(N, N, N, G, seeds=I.voronoi_seeds(2, G, (N, N, N))) as ms:
        out = torch.zeros(G, dtype=torch.float64, device="cuda:0")
        with pytest.raises(L.LsggError) as e:
            L.grain_volumes_device(ms.ctx, out.data_ptr(), G - 1)
        assert e.value.code == L.ERR_CAPACITY
        with pytest.raises(L.LsggError) as e:
            L.voxel_owner_device(ms.ctx, 0, N ** 3)
        assert e.value.code == L.ERR_INVALID_ARG
