"""Python binding of the ``liblsgg`` C ABI (include/lsgg.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  The functions keep the C names without the ``lsgg_`` prefix
(``create_microstructure``, ``step``, ``grain_volumes``, ``voxel_owner``, ...);
``Microstructure`` wraps a context.  The library must have been built in-tree
(``paper_1701_06658_gb300.build.build()``); importing this module without it
raises ``ImportError`` -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblsgg.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_OUT_OF_MEMORY = -2
ERR_OVER_BUDGET = -3
ERR_CUDA = -4
ERR_TIMEOUT = -5
ERR_NOT_READY = -6
ERR_CAPACITY = -7
ERR_UNSUPPORTED = -8

INIT_VORONOI, INIT_LAGUERRE, INIT_LABELS = 0, 1, 2
PHYSICS_IDEAL, PHYSICS_READ_SHOCKLEY, PHYSICS_MAGNETIC = 0, 1, 2
STORAGE_FP32, STORAGE_BF16 = 0, 1
EXEC_BATCHED, EXEC_PLAIN, EXEC_STREAMED = 0, 1, 2
MOBILITY_STEP, MOBILITY_EQ20 = 0, 1
REDIST_TAXICAB, REDIST_GODUNOV, REDIST_HARTMANN = 0, 1, 2

_dp = C.POINTER(C.c_double)


class Config(C.Structure):
    """Mirror of ``lsgg_config`` (field order and types as in lsgg.h)."""
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("n_grains", C.c_int32),
        ("seed", C.c_uint64),
        ("halo", C.c_int32), ("radius", C.c_int32),
        ("eps", C.c_float),
        ("init_kind", C.c_int32), ("physics", C.c_int32), ("storage", C.c_int32),
        ("exec", C.c_int32), ("mobility_law", C.c_int32), ("device", C.c_int32),
        ("redist", C.c_int32), ("reserved", C.c_int32),
        ("theta_max_deg", C.c_double), ("mob_low", C.c_double),
        ("lognormal_sigma", C.c_double), ("big_fraction", C.c_double), ("big_volume", C.c_double),
        ("field_dir", C.c_double * 3),
        ("energy_scale", C.c_double),
        ("arena_slack", C.c_double),
        ("gb_map_tube", C.c_double),
        ("seeds", _dp), ("weights", _dp), ("quats", _dp), ("energy", _dp),
        ("labels", C.POINTER(C.c_int32)),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("steps_done", C.c_int64), ("cell_updates", C.c_int64), ("alive", C.c_int64), ("box_cells", C.c_int64),
        ("arena_capacity", C.c_int64), ("superimposition", C.c_double),
        ("device_bytes", C.c_int64), ("n_classes", C.c_int32), ("class_count", C.c_int32 * 8),
        ("pass_cells", C.c_int64 * 5),
    ]


class GrainStats(C.Structure):
    """Mirror of ``lsgg_grain_stats``."""
    _fields_ = [("alive", C.c_int64), ("mean_volume", C.c_double), ("mean_radius", C.c_double),
                ("rms_radius", C.c_double), ("max_radius", C.c_double), ("overflow", C.c_double),
                ("rho", C.c_double), ("var_z", C.c_double)]


class LsggError(RuntimeError):
    def __init__(self, fn: str, code: int):
        self.code = code
        super().__init__(f"{fn}: {status_string(code)} ({code})")


_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "lsgg_config_default": (None, [C.POINTER(Config)]),
    "lsgg_create_microstructure": (C.c_int, [C.POINTER(Config), C.c_void_p, C.POINTER(C.c_void_p)]),
    "lsgg_step": (C.c_int, [C.c_void_p, C.c_int32, C.c_double]),
    "lsgg_sync": (C.c_int, [C.c_void_p, C.c_int64]),
    "lsgg_grain_volumes": (C.c_int, [C.c_void_p, _dp, C.c_int64, C.POINTER(C.c_int64)]),
    "lsgg_voxel_owner": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int64]),
    "lsgg_grain_volumes_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "lsgg_voxel_owner_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "lsgg_grain_statistics": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.POINTER(GrainStats), _dp]),
    "lsgg_coarsen": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32]),
    "lsgg_texture_shares": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32, _dp]),
    "lsgg_rios_pdf": (C.c_double, [C.c_double, C.c_double, C.c_double]),
    "lsgg_hillert_pdf": (C.c_double, [C.c_double]),
    "lsgg_fit_rios_nu": (C.c_int, [_dp, C.c_int32, C.c_double, C.c_double, _dp]),
    "lsgg_fit_growth_exponent": (C.c_int, [_dp, _dp, C.c_int32, _dp, _dp]),
    "lsgg_destroy": (C.c_int, [C.c_void_p]),
    "lsgg_status_string": (C.c_char_p, [C.c_int]),
    "lsgg_get_stream": (C.c_void_p, [C.c_void_p]),
    "lsgg_abi_config_size": (C.c_size_t, []),
    "lsgg_get_stats": (C.c_int, [C.c_void_p, C.POINTER(Stats)]),
    "lsgg_get_boxes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int64]),
    "lsgg_get_phi": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.c_int64, C.POINTER(C.c_int64)]),
    "lsgg_set_state": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_float), C.POINTER(C.c_int32)]),
    "lsgg_debug_step": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                  C.POINTER(C.c_int32), C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    "lsgg_generate_seeds": (C.c_int, [C.c_uint64, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _dp]),
    "lsgg_neighbour_max": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.c_int32, C.c_int32,
                                     C.c_int32, C.c_float, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "lsgg_neighbour_max_noalloc": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.c_int32, C.c_int32,
                                             C.c_int32, C.c_float, C.c_void_p, C.c_void_p, C.c_void_p]),
    "lsgg_closest_gb_map": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int64, C.c_float,
                                      C.c_void_p, C.c_void_p]),
    "lsgg_server_create": (C.c_int, [C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_void_p)]),
    "lsgg_server_create_mode": (C.c_int, [C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                          C.POINTER(C.c_void_p)]),
    "lsgg_server_submit": (C.c_int, [C.c_void_p, C.POINTER(Config), C.c_int32, C.c_double, C.POINTER(C.c_int64)]),
    "lsgg_server_poll": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p]),
    "lsgg_server_wait": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p]),
    "lsgg_server_volumes": (C.c_int, [C.c_void_p, C.c_int64, _dp, C.c_int64, C.POINTER(C.c_int64)]),
    "lsgg_server_release": (C.c_int, [C.c_void_p, C.c_int64]),
    "lsgg_server_get_stats": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lsgg_server_destroy": (C.c_int, [C.c_void_p]),
    "lsgg_grain_neighbours": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.c_int32]),
    "lsgg_keep_field": (C.c_int, [C.c_void_p, C.c_int32]),
    "lsgg_autotune": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.POINTER(C.c_int32)]),
    "lsgg_pass_tuning": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "lsgg_debug_set_capacity": (C.c_int, [C.c_void_p, C.c_int64]),
    "lsgg_debug_wait_timeout": (C.c_int, [C.c_int32, C.c_int32, C.POINTER(C.c_int32)]),
    "lsgg_debug_set_wait_limit": (C.c_int, [C.c_void_p, C.c_int32]),
    "lsgg_debug_pair_ids": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.c_int64]),
    "lsgg_group_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_void_p)]),
    "lsgg_group_step": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.POINTER(C.c_int64)]),
    "lsgg_group_set_members": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.c_int32]),
    "lsgg_group_destroy": (C.c_int, [C.c_void_p]),
    "lsgg_profile": (C.c_int, [C.c_void_p, C.c_int32]),
    "lsgg_kernel_times": (C.c_int, [C.c_void_p, _dp, C.POINTER(C.c_int64)]),
    "lsgg_pass_times": (C.c_int, [C.c_void_p, _dp, C.POINTER(C.c_int64)]),
}


def lib():
    """The loaded library (ImportError if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_1701_06658_gb300.build.build() "
                              "(needs nvcc); there is no non-CUDA implementation")
        h = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(h, name)
            f.restype = res
            f.argtypes = args
        if h.lsgg_abi_config_size() != C.sizeof(Config):
            raise ImportError("lsgg_config layout mismatch between liblsgg.so and the binding")
        _lib = h
    return _lib


def status_string(code: int) -> str:
    return lib().lsgg_status_string(code).decode()


def _check(fn: str, code: int):
    if code != OK:
        raise LsggError(fn, code)


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


def config_default() -> Config:
    cfg = Config()
    lib().lsgg_config_default(C.byref(cfg))
    return cfg


def generate_seeds(seed: int, n: int, nx: int, ny: int, nz: int) -> np.ndarray:
    out = np.zeros((n, 3), dtype=np.float64)
    _check("generate_seeds", lib().lsgg_generate_seeds(seed, n, nx, ny, nz, _ptr(out, C.c_double)))
    return out


def create_microstructure(cfg: Config, stream=None):
    ctx = C.c_void_p()
    _check("create_microstructure", lib().lsgg_create_microstructure(C.byref(cfg), stream, C.byref(ctx)))
    return ctx


def step(ctx, n: int, dt: float):
    _check("step", lib().lsgg_step(ctx, int(n), float(dt)))


def sync(ctx, timeout_ms: int = -1):
    _check("sync", lib().lsgg_sync(ctx, int(timeout_ms)))


def destroy(ctx):
    _check("destroy", lib().lsgg_destroy(ctx))


def get_stream(ctx) -> int:
    return lib().lsgg_get_stream(ctx) or 0


def grain_volumes(ctx, n_grains: int, out=None) -> np.ndarray:
    out = np.zeros(n_grains, dtype=np.float64) if out is None else out
    n = C.c_int64()
    _check("grain_volumes", lib().lsgg_grain_volumes(ctx, _ptr(out, C.c_double), out.size, C.byref(n)))
    return out


def grain_statistics(ctx, n_bins: int = 20, r_max: float = 3.0) -> dict:
    """Device-computed grain statistics (see lsgg.h): a dict of the struct's
    fields plus the R / <R> histogram."""
    st = GrainStats()
    hist = np.zeros(n_bins, np.float64)
    _check("grain_statistics", lib().lsgg_grain_statistics(ctx, n_bins, r_max, C.byref(st), _ptr(hist, C.c_double)))
    out = {f: getattr(st, f) for f, _ in GrainStats._fields_}
    out["hist"] = hist
    return out


def texture_shares(ctx, grain_class, n_classes: int) -> np.ndarray:
    """Volume fraction of each grain class (see lsgg.h)."""
    cls = np.ascontiguousarray(grain_class, dtype=np.int32)
    out = np.zeros(n_classes, np.float64)
    _check("texture_shares", lib().lsgg_texture_shares(ctx, _ptr(cls, C.c_int32), n_classes, _ptr(out, C.c_double)))
    return out


def rios_pdf(z: float, nu: float, rho: float) -> float:
    return lib().lsgg_rios_pdf(z, nu, rho)


def hillert_pdf(z: float) -> float:
    return lib().lsgg_hillert_pdf(z)


def fit_rios_nu(hist, r_max_rel: float, rho: float) -> float:
    h = np.ascontiguousarray(hist, dtype=np.float64)
    nu = C.c_double()
    _check("fit_rios_nu", lib().lsgg_fit_rios_nu(_ptr(h, C.c_double), h.size, r_max_rel, rho, C.byref(nu)))
    return nu.value


def fit_growth_exponent(t, mean_r):
    """(n, k) of <R> ~ t^n fitted as <R>^(1/n) - <R_0>^(1/n) = k t (see lsgg.h)."""
    tt = np.ascontiguousarray(t, dtype=np.float64)
    rr = np.ascontiguousarray(mean_r, dtype=np.float64)
    n, k = C.c_double(), C.c_double()
    _check("fit_growth_exponent", lib().lsgg_fit_growth_exponent(_ptr(tt, C.c_double), _ptr(rr, C.c_double),
                                                                 tt.size, C.byref(n), C.byref(k)))
    return n.value, k.value


def coarsen(ctx, nx: int, ny: int, nz: int):
    """Grid coarsening onto nx x ny x nz cells of the same domain (see lsgg.h)."""
    _check("coarsen", lib().lsgg_coarsen(ctx, nx, ny, nz))


def voxel_owner(ctx, shape_zyx, out=None) -> np.ndarray:
    out = np.zeros(shape_zyx, dtype=np.int32) if out is None else out
    _check("voxel_owner", lib().lsgg_voxel_owner(ctx, _ptr(out, C.c_int32), out.size))
    return out


def grain_volumes_device(ctx, out_dev: int, cap: int, status_dev: int = 0, stream: int = 0):
    """lsgg_grain_volumes_device: device pointers in, enqueued, no synchronisation."""
    _check("grain_volumes_device", lib().lsgg_grain_volumes_device(ctx, out_dev, cap, status_dev or None,
                                                                   stream or None))


def voxel_owner_device(ctx, out_dev: int, n_cells: int, status_dev: int = 0, stream: int = 0):
    """lsgg_voxel_owner_device: device pointers in, enqueued, no synchronisation."""
    _check("voxel_owner_device", lib().lsgg_voxel_owner_device(ctx, out_dev, n_cells, status_dev or None,
                                                               stream or None))


def get_stats(ctx) -> Stats:
    s = Stats()
    _check("get_stats", lib().lsgg_get_stats(ctx, C.byref(s)))
    return s


def autotune(ctx, steps_per_trial: int = 2, dt: float = 1.0) -> dict:
    """Run the tile autotuner; returns {"k_predict": [...], "k_correct": [...]} variant per class."""
    chosen = np.full(16, -1, np.int32)
    _check("autotune", lib().lsgg_autotune(ctx, steps_per_trial, float(dt), _ptr(chosen, C.c_int32)))
    return {"k_predict": chosen[0:5].tolist(), "k_correct": chosen[5:10].tolist()}


def pass_tuning(ctx) -> dict:
    """The pass path's tuning: CTAs per SM per tier and pass, and the slab depth."""
    ctas = np.zeros(4 * PASS_TIERS, np.int32)
    slab = C.c_int32()
    _check("pass_tuning", lib().lsgg_pass_tuning(ctx, _ptr(ctas, C.c_int32), C.byref(slab)))
    return {f"{PASS_NAMES[k]}[tier{t}]": int(ctas[t * 4 + k]) for t in range(PASS_TIERS) for k in range(4)} | {
        "slab": int(slab.value)}


def debug_set_capacity(ctx, capacity: int):
    _check("debug_set_capacity", lib().lsgg_debug_set_capacity(ctx, int(capacity)))


def debug_wait_timeout(device: int, iterations: int) -> bool:
    out = C.c_int32(-1)
    _check("debug_wait_timeout", lib().lsgg_debug_wait_timeout(device, iterations, C.byref(out)))
    return out.value == 1


def debug_pair_ids(ctx, boxes: np.ndarray):
    """Test hook: (ID-field, anisotropy map) per grain on the current boxes, as
    dicts of box-shaped int32 arrays (see lsgg.h)."""
    n = packed_size(boxes)
    idf = np.zeros(max(n, 1), np.int32)
    mp = np.zeros(max(n, 1), np.int32)
    _check("debug_pair_ids", lib().lsgg_debug_pair_ids(ctx, _ptr(idf, C.c_int32), _ptr(mp, C.c_int32), n))
    return unpack(boxes, idf), unpack(boxes, mp)


def debug_set_wait_limit(ctx, polls: int):
    """Test hook: polls of the pass kernels' bounded waits (< 0: the default)."""
    _check("debug_set_wait_limit", lib().lsgg_debug_set_wait_limit(ctx, polls))


def profile(ctx, enable: bool):
    _check("profile", lib().lsgg_profile(ctx, 1 if enable else 0))


KERNEL_GROUPS = ("field_clear", "k_predict", "k_correct", "k_box_update")


def kernel_times(ctx):
    """(ms, launches) per kernel group since the previous call (see lsgg.h)."""
    ms = np.zeros(4, np.float64)
    cnt = np.zeros(4, np.int64)
    _check("kernel_times", lib().lsgg_kernel_times(ctx, _ptr(ms, C.c_double), _ptr(cnt, C.c_int64)))
    return dict(zip(KERNEL_GROUPS, ms.tolist())), dict(zip(KERNEL_GROUPS, cnt.tolist()))


PASS_NAMES = ("p_conv_xy", "p_conv_z", "p_redist_xy", "p_redist_z")
PASS_TIERS = 5          # LSGG_PASS_TIERS: boxes of x, y side <= 32, <= 40, <= 48, <= 64, larger


def pass_times(ctx):
    """{name: (ms, launches)} of the pass path since the previous call: the
    per-tier passes as "name[tierT]", plus "k_bin" and "p_field"."""
    ms = np.zeros(4 * PASS_TIERS + 2, np.float64)
    cnt = np.zeros(4 * PASS_TIERS + 2, np.int64)
    _check("pass_times", lib().lsgg_pass_times(ctx, _ptr(ms, C.c_double), _ptr(cnt, C.c_int64)))
    out = {f"{PASS_NAMES[k]}[tier{t}]": (float(ms[t * 4 + k]), int(cnt[t * 4 + k]))
           for t in range(PASS_TIERS) for k in range(4)}
    out["k_bin"] = (float(ms[4 * PASS_TIERS]), int(cnt[4 * PASS_TIERS]))
    out["p_field"] = (float(ms[4 * PASS_TIERS + 1]), int(cnt[4 * PASS_TIERS + 1]))
    return out


class Box(C.Structure):
    """Mirror of ``lsgg_box`` (stateless ops)."""
    _fields_ = [("ox", C.c_int32), ("oy", C.c_int32), ("oz", C.c_int32),
                ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("offset", C.c_int64)]


BOX_DTYPE = np.dtype([("ox", "<i4"), ("oy", "<i4"), ("oz", "<i4"), ("nx", "<i4"), ("ny", "<i4"),
                      ("nz", "<i4"), ("offset", "<i8")])


def neighbour_max(boxes_dev: int, n_boxes: int, phip_dev: int, n_elems: int, nx: int, ny: int, nz: int,
                  eps: float, scratch_dev: int, m_dev: int, id_dev: int, stream: int = 0):
    """lsgg_neighbour_max on device pointers (ints, e.g. torch ``data_ptr()``)."""
    _check("neighbour_max", lib().lsgg_neighbour_max(boxes_dev, n_boxes, phip_dev, n_elems, nx, ny, nz, eps,
                                                      scratch_dev, m_dev, id_dev, stream or None))


NOALLOC_MAX_CELLS = 1 << 20


def neighbour_max_noalloc(boxes_dev: int, n_boxes: int, phip_dev: int, n_elems: int, nx: int, ny: int, nz: int,
                          eps: float, m_dev: int, id_dev: int, stream: int = 0):
    """lsgg_neighbour_max_noalloc: the same op without caller scratch and without
    any device allocation (its field is a static array of NOALLOC_MAX_CELLS cells)."""
    _check("neighbour_max_noalloc", lib().lsgg_neighbour_max_noalloc(boxes_dev, n_boxes, phip_dev, n_elems, nx, ny,
                                                                      nz, eps, m_dev, id_dev, stream or None))


def closest_gb_map(boxes_dev: int, n_boxes: int, phi_dev: int, idf_dev: int, n_elems: int, tube: float,
                   out_dev: int, stream: int = 0):
    """lsgg_closest_gb_map on device pointers: the grain across the closest
    triangulated boundary point for every cell with |phi| < tube."""
    _check("closest_gb_map", lib().lsgg_closest_gb_map(boxes_dev, n_boxes, phi_dev, idf_dev, n_elems, tube, out_dev,
                                                        stream or None))


def keep_field(ctx, on: bool = True):
    _check("keep_field", lib().lsgg_keep_field(ctx, 1 if on else 0))


def grain_neighbours(ctx, n_grains: int, cap: int = 96) -> list:
    """Contact neighbours (ascending ids) of every grain after the last step."""
    counts = np.zeros(n_grains, np.int32)
    ids = np.zeros((n_grains, cap), np.int32)
    _check("grain_neighbours", lib().lsgg_grain_neighbours(ctx, _ptr(counts, C.c_int32), _ptr(ids, C.c_int32), cap))
    return [ids[g, :min(int(counts[g]), cap)].tolist() for g in range(n_grains)]


def get_boxes(ctx, n_grains: int) -> np.ndarray:
    out = np.zeros((n_grains, 7), dtype=np.int32)
    _check("get_boxes", lib().lsgg_get_boxes(ctx, _ptr(out, C.c_int32), out.size))
    return out


def get_phi(ctx) -> np.ndarray:
    n = C.c_int64()
    code = lib().lsgg_get_phi(ctx, None, 0, C.byref(n))
    if code not in (OK, ERR_CAPACITY):
        _check("get_phi", code)
    out = np.zeros(n.value, dtype=np.float32)
    _check("get_phi", lib().lsgg_get_phi(ctx, _ptr(out, C.c_float), out.size, C.byref(n)))
    return out


def set_state(ctx, boxes: np.ndarray, phi: np.ndarray, idf: np.ndarray | None = None):
    b = np.ascontiguousarray(boxes, dtype=np.int32)
    p = np.ascontiguousarray(phi, dtype=np.float32)
    i = None if idf is None else np.ascontiguousarray(idf, dtype=np.int32)
    _check("set_state", lib().lsgg_set_state(ctx, _ptr(b, C.c_int32), _ptr(p, C.c_float), _ptr(i, C.c_int32)))


def packed_size(boxes: np.ndarray) -> int:
    alive = boxes[:, 0] != 0
    return int((boxes[alive, 4].astype(np.int64) * boxes[alive, 5] * boxes[alive, 6]).sum())


def debug_step(ctx, dt: float, boxes: np.ndarray):
    """One step returning the packed intermediates (phip, m, idm, phic, phin)
    on ``boxes`` (the boxes returned by get_boxes before the call)."""
    n = packed_size(boxes)
    phip = np.zeros(n, np.float32)
    m = np.zeros(n, np.float32)
    idm = np.zeros(n, np.int32)
    phic = np.zeros(n, np.float32)
    phin = np.zeros(n, np.float32)
    _check("debug_step", lib().lsgg_debug_step(ctx, float(dt), _ptr(phip, C.c_float), _ptr(m, C.c_float),
                                                _ptr(idm, C.c_int32), _ptr(phic, C.c_float), _ptr(phin, C.c_float)))
    return phip, m, idm, phic, phin


def unpack(boxes: np.ndarray, packed: np.ndarray) -> dict:
    """Split a packed array into per-grain (nz, ny, nx) arrays keyed by grain id."""
    out = {}
    o = 0
    for g, b in enumerate(boxes):
        if not b[0]:
            continue
        n = int(b[4]) * int(b[5]) * int(b[6])
        out[g] = packed[o:o + n].reshape(int(b[6]), int(b[5]), int(b[4]))
        o += n
    return out


def pack(boxes: np.ndarray, arrays: dict, dtype=np.float32) -> np.ndarray:
    parts = [np.asarray(arrays[g], dtype=dtype).ravel() for g, b in enumerate(boxes) if b[0]]
    return np.concatenate(parts) if parts else np.zeros(0, dtype)


MAX_GROUP = 64
SERVE_PER_CONTEXT, SERVE_SHARED = 0, 1


def group_create(ctxs) -> int:
    """A step group over contexts (handles); returns the group handle."""
    arr = (C.c_void_p * len(ctxs))(*ctxs)
    g = C.c_void_p()
    _check("group_create", lib().lsgg_group_create(arr, len(ctxs), C.byref(g)))
    return g.value


def group_step(group, n: int, dt: float, step_limits=None):
    lim = None
    if step_limits is not None:
        keep = np.ascontiguousarray(step_limits, dtype=np.int64)
        lim = _ptr(keep, C.c_int64)
    _check("group_step", lib().lsgg_group_step(group, n, dt, lim))


def group_set_members(group, ctxs):
    arr = (C.c_void_p * len(ctxs))(*ctxs)
    _check("group_set_members", lib().lsgg_group_set_members(group, arr, len(ctxs)))


def group_destroy(group):
    _check("group_destroy", lib().lsgg_group_destroy(group))


class Group:
    """Several microstructures stepped by one set of launches per step."""

    def __init__(self, members):
        self.members = list(members)
        self.handle = group_create([m.ctx for m in self.members])

    def step(self, n: int, dt: float, step_limits=None):
        group_step(self.handle, n, dt, step_limits)

    def set_members(self, members):
        group_set_members(self.handle, [m.ctx for m in members])
        self.members = list(members)

    def close(self):
        if self.handle:
            group_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Microstructure:
    """A context: create -> step / sync -> outputs -> close."""

    def __init__(self, nx: int, ny: int, nz: int, n_grains: int, seed: int = 1, seeds=None, weights=None,
                 quats=None, energy=None, physics: int = PHYSICS_IDEAL, exec_mode: int = EXEC_BATCHED,
                 storage: int = STORAGE_FP32, halo: int = 5, radius: int = 5, eps: float = 7.0,
                 init_kind: int | None = None, stream=None, device: int = 0, arena_slack: float = 1.5,
                 labels=None, **extra):
        cfg = config_default()
        cfg.nx, cfg.ny, cfg.nz, cfg.n_grains, cfg.seed = nx, ny, nz, n_grains, seed
        cfg.halo, cfg.radius, cfg.eps = halo, radius, eps
        cfg.physics, cfg.exec, cfg.storage, cfg.device = physics, exec_mode, storage, device
        cfg.arena_slack = arena_slack
        for k, v in extra.items():
            if k == "field_dir":
                for a in range(3):
                    cfg.field_dir[a] = float(v[a])
            else:
                setattr(cfg, k, v)
        self._keep = []

        def _sized(a, n, what):
            # the C ABI reads the arrays through plain pointers: their sizes are checked here
            if a.size != n:
                raise ValueError(f"{what}: {a.size} values where {n} are read")
            self._keep.append(a)
            return a

        if seeds is not None:
            s = _sized(np.ascontiguousarray(seeds, dtype=np.float64), 3 * n_grains, "seeds")
            cfg.seeds = _ptr(s, C.c_double)
        if weights is not None:
            w = _sized(np.ascontiguousarray(weights, dtype=np.float64), n_grains, "weights")
            cfg.weights = _ptr(w, C.c_double)
        cfg.init_kind = (INIT_LAGUERRE if weights is not None else INIT_VORONOI) if init_kind is None else init_kind
        if labels is not None:                       # (z, y, x) grain ids: the label-field initialisation
            lab = _sized(np.ascontiguousarray(labels, dtype=np.int32), nx * ny * nz, "labels")
            cfg.labels = _ptr(lab, C.c_int32)
            cfg.init_kind = INIT_LABELS
        if quats is not None:
            q = _sized(np.ascontiguousarray(quats, dtype=np.float64), 4 * n_grains, "quats")
            cfg.quats = _ptr(q, C.c_double)
        if energy is not None:
            e = _sized(np.ascontiguousarray(energy, dtype=np.float64), n_grains, "energy")
            cfg.energy = _ptr(e, C.c_double)
        self.shape = (nz, ny, nx)
        self.n_grains = n_grains
        self.ctx = create_microstructure(cfg, stream)
        self._keep.clear()

    def step(self, n: int, dt: float = 1.0):
        step(self.ctx, n, dt)

    def sync(self, timeout_ms: int = -1):
        sync(self.ctx, timeout_ms)

    def grain_volumes(self, out=None) -> np.ndarray:
        """Volumes into `out` (n_grains float64, e.g. a view of pinned memory) or a new array."""
        return grain_volumes(self.ctx, self.n_grains, out)

    def voxel_owner(self, out=None) -> np.ndarray:
        """Owner map into `out` ((nz, ny, nx) int32, e.g. a view of pinned memory) or a new array."""
        return voxel_owner(self.ctx, self.shape, out)

    def grain_statistics(self, n_bins: int = 20, r_max: float = 3.0) -> dict:
        return grain_statistics(self.ctx, n_bins, r_max)

    def texture_shares(self, grain_class, n_classes: int) -> np.ndarray:
        return texture_shares(self.ctx, grain_class, n_classes)

    def coarsen(self, nx: int, ny: int, nz: int):
        coarsen(self.ctx, nx, ny, nz)
        self.shape = (nz, ny, nx)

    def boxes(self) -> np.ndarray:
        return get_boxes(self.ctx, self.n_grains)

    def phi(self) -> dict:
        b = self.boxes()
        return unpack(b, get_phi(self.ctx))

    def set_state(self, boxes, phi_by_grain: dict, idf_by_grain: dict | None = None):
        p = pack(boxes, phi_by_grain)
        i = None if idf_by_grain is None else pack(boxes, idf_by_grain, np.int32)
        set_state(self.ctx, boxes, p, i)

    def debug_step(self, dt: float = 1.0):
        b = self.boxes()
        parts = debug_step(self.ctx, dt, b)
        return b, [unpack(b, p) for p in parts]

    def stats(self) -> Stats:
        return get_stats(self.ctx)

    @property
    def stream(self) -> int:
        return get_stream(self.ctx)

    def close(self):
        if self.ctx is not None:
            destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- serving

class RequestInfo(C.Structure):
    _fields_ = [("state", C.c_int32), ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("cell_updates", C.c_int64), ("device_bytes", C.c_int64), ("estimate_bytes", C.c_int64)]


class ServerStats(C.Structure):
    _fields_ = [("queued", C.c_int64), ("active", C.c_int64), ("completed", C.c_int64),
                ("used_bytes", C.c_int64), ("peak_bytes", C.c_int64), ("cell_updates", C.c_int64)]


class Server:
    """lsgg_server_*: continuous batching of independent simulations under an HBM budget."""

    def __init__(self, budget_bytes: int, max_active: int = 64, steps_per_round: int = 4, device: int = 0,
                 mode: int = SERVE_SHARED):
        h = C.c_void_p()
        _check("server_create", lib().lsgg_server_create_mode(int(budget_bytes), max_active, steps_per_round, device,
                                                               mode, C.byref(h)))
        self.h = h
        self._n_grains = {}

    def submit(self, nx: int, ny: int, nz: int, n_grains: int, n_steps: int, dt: float = 1.0, seed: int = 1,
               seeds=None, labels=None, **fields) -> int:
        """Queue a request (the library copies the config and its arrays)."""
        cfg = config_default()
        cfg.nx, cfg.ny, cfg.nz, cfg.n_grains, cfg.seed = nx, ny, nz, n_grains, seed
        for k, v in fields.items():
            setattr(cfg, k, v)
        keep = []
        if seeds is not None:
            s = np.ascontiguousarray(seeds, dtype=np.float64)
            if s.size != 3 * n_grains:
                raise ValueError(f"seeds: {s.size} values where {3 * n_grains} are read")
            keep.append(s)
            cfg.seeds = _ptr(s, C.c_double)
        if labels is not None:
            lab = np.ascontiguousarray(labels, dtype=np.int32)
            if lab.size != nx * ny * nz:
                raise ValueError(f"labels: {lab.size} values where {nx * ny * nz} are read")
            keep.append(lab)
            cfg.labels = _ptr(lab, C.c_int32)
            cfg.init_kind = INIT_LABELS
        t = C.c_int64()
        _check("server_submit", lib().lsgg_server_submit(self.h, C.byref(cfg), int(n_steps), float(dt), C.byref(t)))
        self._n_grains[t.value] = n_grains
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1) -> RequestInfo:
        info = RequestInfo()
        _check("server_wait", lib().lsgg_server_wait(self.h, ticket, timeout_ms, C.byref(info)))
        return info

    def poll(self, ticket: int):
        info = RequestInfo()
        code = lib().lsgg_server_poll(self.h, ticket, C.byref(info))
        return code, info

    def volumes(self, ticket: int) -> np.ndarray:
        out = np.zeros(self._n_grains[ticket], np.float64)
        n = C.c_int64()
        _check("server_volumes", lib().lsgg_server_volumes(self.h, ticket, _ptr(out, C.c_double), out.size,
                                                            C.byref(n)))
        return out

    def release(self, ticket: int):
        _check("server_release", lib().lsgg_server_release(self.h, ticket))
        self._n_grains.pop(ticket, None)

    def stats(self) -> ServerStats:
        s = ServerStats()
        _check("server_get_stats", lib().lsgg_server_get_stats(self.h, C.byref(s)))
        return s

    def close(self):
        if self.h is not None:
            lib().lsgg_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
