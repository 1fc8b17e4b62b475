"""The C-ABI library without a GPU: it loads, exports every function that
include/lsgg.h declares, agrees with the binding's struct layout, implements
the seed generator bit for bit like the inputs module, and refuses to compute
without a CUDA device (no CPU fallback)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1701_06658_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    L = pytest.importorskip("paper_1701_06658_gb300.lsgg")
    try:
        L.lib()
    except ImportError as e:
        pytest.fail(f"liblsgg.so not built: {e}")
    return L


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lsgg_\w+)\s*\(", src))
    return sorted(names)


def test_exports_every_declared_symbol():
    L = _lib()
    h = ctypes.CDLL(L.LIB_PATH)
    names = declared_functions()
    assert "lsgg_create_microstructure" in names and "lsgg_step" in names
    missing = [n for n in names if not hasattr(h, n)]
    assert not missing, missing


def test_config_layout_and_defaults():
    L = _lib()
    assert L.lib().lsgg_abi_config_size() == ctypes.sizeof(L.Config)
    cfg = L.config_default()
    assert (cfg.nx, cfg.ny, cfg.nz, cfg.n_grains, cfg.halo, cfg.radius) == (64, 64, 64, 50, 5, 5)
    assert cfg.eps == 7.0 and cfg.arena_slack == 1.5 and cfg.gb_map_tube == 0.0


@pytest.mark.parametrize("seed,n,shape", [(1, 50, (64, 64, 64)), (2, 5000, (256, 256, 256)),
                                          (7, 33, (40, 30, 1)), (2 ** 63 + 5, 10, (17, 19, 23))])
def test_seed_generator_matches_inputs_module(seed, n, shape):
    L = _lib()
    got = L.generate_seeds(seed, n, *shape)
    want = I.voronoi_seeds(seed, n, shape)
    assert np.array_equal(got, want)


def test_status_strings():
    L = _lib()
    assert L.status_string(0) == "ok"
    assert L.status_string(L.ERR_CUDA) == "CUDA error"
    assert L.status_string(-99) == "unknown status"


def test_invalid_arguments_rejected_before_any_device_work():
    L = _lib()
    cfg = L.config_default()
    cfg.n_grains = 0
    with pytest.raises(L.LsggError) as e:
        L.create_microstructure(cfg)
    assert e.value.code == L.ERR_INVALID_ARG
    with pytest.raises(L.LsggError):
        L.generate_seeds(1, 0, 4, 4, 4)
    with pytest.raises(L.LsggError) as e:
        L.coarsen(None, 16, 16, 16)          # no context
    assert e.value.code == L.ERR_INVALID_ARG
    for args in ((0, 1, 8, 8, 10, 3.0, 8), (8, 1, 8, 8, 10, 0.0, 8), (8, 1, 8, 8, 10, 17.0, 8),
                 (8, -1, 8, 8, 10, 3.0, 8), (8, 1, 8, 8, 10, float("nan"), 8)):
        with pytest.raises(L.LsggError) as e:    # checked before any launch: the pointers are never read
            L.closest_gb_map(*args)
        assert e.value.code == L.ERR_INVALID_ARG


def test_no_cpu_fallback_without_a_device():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = _lib()
    with pytest.raises(L.LsggError) as e:
        L.Microstructure(16, 16, 16, 4)
    assert e.value.code == L.ERR_CUDA


@pytest.mark.parametrize("exec_mode", ["EXEC_PLAIN", "EXEC_STREAMED"])
def test_bf16_storage_only_on_the_batched_path(exec_mode):
    """BF16 state storage is refused before any device work on the execution
    modes whose kernels keep FP32 only."""
    L = _lib()
    cfg = L.config_default()
    cfg.storage = L.STORAGE_BF16
    cfg.exec = getattr(L, exec_mode)
    ctx = ctypes.c_void_p()
    assert L.lib().lsgg_create_microstructure(ctypes.byref(cfg), None, ctypes.byref(ctx)) == L.ERR_UNSUPPORTED


def test_smoke_exclusion_equals_the_parity_helpers():
    """smoke() carries its own copy of the parity tests' sign-flip exclusion
    (it imports nothing from tests/): both give the same cells on random
    boxes, with and without full periodic axes."""
    import numpy as np

    import __graft_entry__ as ge
    from tests.parity import box_full, sign_flip_exclusion
    rng = np.random.default_rng(5)
    # (box array shape z, y, x; domain z, y, x): full on every axis, on x and z only, 2D full on y only
    for shape, dom in (((9, 11, 13), (9, 11, 13)), ((9, 11, 13), (9, 40, 13)), ((1, 12, 10), (1, 12, 30))):
        box = (1, 0, 0, 0, shape[2], shape[1], shape[0])
        ref = rng.uniform(-2e-4, 2e-4, shape)
        gpu = ref + rng.uniform(-1e-4, 1e-4, shape)
        a = ge._sign_flip_exclusion(ref, gpu, box, dom)
        b = sign_flip_exclusion(ref, gpu, box_full(box, dom))
        assert np.array_equal(a, b)


@pytest.mark.parametrize("case", ["plain", "streamed", "2d", "unknown"])
def test_sweep_reinitialisations_only_on_the_batched_3d_path(case):
    """The Godunov and Hartmann re-initialisations run as column sweeps of the
    batched 3D path; other execution modes, 2D domains and unknown schemes
    are refused before any device work."""
    L = _lib()
    cfg = L.config_default()
    cfg.redist = L.REDIST_HARTMANN
    if case == "plain":
        cfg.exec = L.EXEC_PLAIN
    elif case == "streamed":
        cfg.exec = L.EXEC_STREAMED
    elif case == "2d":
        cfg.nz = 1
    else:
        cfg.redist = 3
    ctx = ctypes.c_void_p()
    code = L.lib().lsgg_create_microstructure(ctypes.byref(cfg), None, ctypes.byref(ctx))
    assert code in (L.ERR_INVALID_ARG, L.ERR_UNSUPPORTED)


@pytest.mark.parametrize("case", ["ideal", "wide", "negative", "streamed"])
def test_anisotropy_map_configuration_is_checked(case):
    """The in-step anisotropy map needs physics that reads pairs, a tube
    inside the band and the batched path; anything else is refused before any
    device work."""
    L = _lib()
    cfg = L.config_default()
    cfg.physics = L.PHYSICS_READ_SHOCKLEY
    cfg.gb_map_tube = 3.0
    if case == "ideal":
        cfg.physics = L.PHYSICS_IDEAL
    elif case == "wide":
        cfg.gb_map_tube = 7.0
    elif case == "negative":
        cfg.gb_map_tube = -1.0
    else:
        cfg.exec = L.EXEC_STREAMED
    ctx = ctypes.c_void_p()
    code = L.lib().lsgg_create_microstructure(ctypes.byref(cfg), None, ctypes.byref(ctx))
    assert code in (L.ERR_INVALID_ARG, L.ERR_UNSUPPORTED)


def test_group_arguments_checked_before_any_device_work():
    """Step groups: no members, too many members or a NULL member are refused
    without touching a device; a NULL group is refused by the step and the
    destroy calls."""
    L = _lib()
    h = ctypes.c_void_p()
    assert L.lib().lsgg_group_create(None, 0, ctypes.byref(h)) == L.ERR_INVALID_ARG
    arr = (ctypes.c_void_p * 2)(None, None)
    assert L.lib().lsgg_group_create(arr, 2, ctypes.byref(h)) == L.ERR_INVALID_ARG
    assert L.lib().lsgg_group_create(arr, L.MAX_GROUP + 1, ctypes.byref(h)) == L.ERR_INVALID_ARG
    assert L.lib().lsgg_group_step(None, 1, 1.0, None) == L.ERR_INVALID_ARG
    assert L.lib().lsgg_group_destroy(None) == L.ERR_INVALID_ARG


@pytest.mark.parametrize("case", ["null", "low", "high", "streamed", "2d"])
def test_label_field_configuration_is_checked(case):
    """A label-field start needs the labels, every label in [0, n_grains) and
    the batched 3D path; anything else is refused before any device work."""
    L = _lib()
    cfg = L.config_default()
    cfg.nx, cfg.ny, cfg.nz, cfg.n_grains = 8, 8, 8, 4
    cfg.init_kind = L.INIT_LABELS
    lab = np.zeros(8 * 8 * 8, dtype=np.int32)
    lab[::3] = 3
    want = L.ERR_INVALID_ARG
    if case == "low":
        lab[17] = -1
    elif case == "high":
        lab[-1] = 4
    elif case == "streamed":
        cfg.exec = L.EXEC_STREAMED
        want = L.ERR_UNSUPPORTED
    elif case == "2d":
        cfg.nz = 1
        want = L.ERR_UNSUPPORTED
    if case != "null":
        cfg.labels = lab.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    ctx = ctypes.c_void_p()
    assert L.lib().lsgg_create_microstructure(ctypes.byref(cfg), None, ctypes.byref(ctx)) == want


@pytest.mark.parametrize("kw", [{"labels": np.zeros(100, dtype=np.int32)}, {"seeds": np.zeros((3, 3))},
                                {"weights": np.zeros(5)}, {"quats": np.zeros((4, 3))}, {"energy": np.zeros(2)}])
def test_input_array_sizes_are_checked_by_the_binding(kw):
    """The C ABI reads the config's arrays through plain pointers (3 n_grains
    seeds, n_grains weights and energies, 4 n_grains quaternions, nx ny nz
    labels); the binding refuses an array of another size before calling it."""
    L = _lib()
    with pytest.raises(ValueError):
        L.Microstructure(8, 8, 8, 4, **kw)
