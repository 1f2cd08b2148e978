"""Thin Python binding of libsupa.so (the C ABI of include/supa.h).

Every function here has the name of the C entry point it calls and does
argument marshalling only: torch tensors provide device memory and streams,
and every step of the computation runs in the library's CUDA kernels.  There
is no CPU fallback: if the library cannot be loaded, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build
from . import inputs as _inputs

SUPA_OK = 0
SUPA_ERR_INVALID_ARG = -1
SUPA_ERR_OOM = -2
SUPA_ERR_OVERFLOW = -3
SUPA_ERR_TIMEOUT = -4
SUPA_ERR_CUDA = -5
SUPA_ERR_NOT_READY = -6

EXPORTED = (
    "supa_last_error", "supa_init_geometry", "supa_destroy_geometry", "supa_batch_create", "supa_destroy_batch",
    "supa_simulate", "supa_simulate_batch", "supa_batch_get_info", "supa_fetch_hits", "supa_fetch_hit_tags",
    "supa_voxelize", "supa_voxelize_hits", "supa_autotune", "supa_surrogate_param_count", "supa_surrogate_create",
    "supa_surrogate_destroy", "supa_surrogate_get_params", "supa_surrogate_gradients", "supa_surrogate_train_step",
    "supa_surrogate_forward", "supa_surrogate_check", "supa_surrogate_train_epoch", "supa_batch_set_surrogate",
    "supa_build_training_set", "supa_profiles", "supa_shower_offsets_noalloc", "supa_export_diverted",
    "supa_shower_shapes", "supa_layer_images_cells", "supa_voxelize_layers", "supa_voxelize_fetch",
    "supa_check_wait_expiry", "supa_export_surrogate", "supa_batch_warp_times", "supa_surrogate_average",
)


class SupaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class supa_geometry_desc(ctypes.Structure):
    _fields_ = [
        ("n_slices", ctypes.c_int32), ("dz", ctypes.c_float),
        ("slice_to_layer", ctypes.POINTER(ctypes.c_int32)), ("n_layers", ctypes.c_int32),
        ("p_stop", ctypes.POINTER(ctypes.c_double)), ("p_split", ctypes.POINTER(ctypes.c_double)),
        ("theta_mode", ctypes.c_int32), ("theta_lo", ctypes.c_double), ("theta_hi", ctypes.c_double),
        ("eps_mode", ctypes.c_int32), ("eps_frac", ctypes.c_double), ("split_mode", ctypes.c_int32),
        ("e_min", ctypes.c_double), ("uz_min", ctypes.c_double),
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("wx", ctypes.c_float), ("wy", ctypes.c_float),
        ("roi_mode", ctypes.c_int32),
        ("n_regions", ctypes.c_int32), ("region_radius", ctypes.POINTER(ctypes.c_double)),
        ("region_p_stop", ctypes.POINTER(ctypes.c_double)), ("region_p_split", ctypes.POINTER(ctypes.c_double)),
        ("region_theta_lo", ctypes.POINTER(ctypes.c_double)), ("region_theta_hi", ctypes.POINTER(ctypes.c_double)),
        ("region_eps_frac", ctypes.POINTER(ctypes.c_double)),
    ]


class supa_launch_config(ctypes.Structure):
    _fields_ = [
        ("warps_per_block", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("stack_depth", ctypes.c_int32),
        ("flush_threshold", ctypes.c_int32), ("record_tags", ctypes.c_int32), ("lpt_order", ctypes.c_int32),
        ("voxel_ctas_per_sm", ctypes.c_int32), ("max_hits", ctypes.c_int64), ("record_warp_times", ctypes.c_int32),
    ]


class supa_batch_info(ctypes.Structure):
    _fields_ = [
        ("n_showers", ctypes.c_int64), ("n_hits", ctypes.c_int64), ("n_steps", ctypes.c_int64),
        ("max_layers", ctypes.c_int32), ("status", ctypes.c_int32),
        ("offsets_dev", ctypes.c_void_p), ("counts_dev", ctypes.c_void_p), ("steps_dev", ctypes.c_void_p),
        ("layer_sums_dev", ctypes.c_void_p), ("dead_dev", ctypes.c_void_p), ("leak_dev", ctypes.c_void_p),
        ("escape_dev", ctypes.c_void_p), ("n_diverted", ctypes.c_int64), ("sur_leak_dev", ctypes.c_void_p),
    ]


_lib = None
_VP = ctypes.c_void_p
_I64 = ctypes.c_int64


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libsupa.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libsupa.so not found at {_build.LIB}; run the build first")
        L = ctypes.CDLL(_build.LIB)
        L.supa_last_error.restype = ctypes.c_char_p
        L.supa_init_geometry.argtypes = [ctypes.POINTER(supa_geometry_desc), ctypes.POINTER(_VP)]
        L.supa_destroy_geometry.argtypes = [_VP]
        L.supa_batch_create.argtypes = [ctypes.POINTER(_VP), ctypes.c_int32, _I64,
                                         ctypes.POINTER(supa_launch_config), ctypes.POINTER(_VP)]
        L.supa_destroy_batch.argtypes = [_VP]
        L.supa_simulate.argtypes = [_VP, _VP, _I64, ctypes.c_uint64, ctypes.c_uint64, _VP]
        L.supa_simulate_batch.argtypes = [ctypes.POINTER(_VP), ctypes.c_int32, _VP, _I64, ctypes.c_uint64,
                                          ctypes.c_uint64, ctypes.POINTER(supa_launch_config), ctypes.POINTER(_VP),
                                          _VP]
        L.supa_batch_get_info.argtypes = [_VP, ctypes.POINTER(supa_batch_info), _VP]
        L.supa_fetch_hits.argtypes = [_VP, _I64, _I64, _VP, ctypes.c_int32, ctypes.POINTER(_I64), _VP]
        L.supa_fetch_hit_tags.argtypes = [_VP, _I64, _I64, _VP, ctypes.POINTER(_I64), _VP]
        L.supa_voxelize.argtypes = [_VP, _I64, _I64, _VP, _VP, _VP]
        L.supa_voxelize_fetch.argtypes = [_VP, _I64, _I64, _VP, _VP, _VP, _I64, _VP]
        L.supa_check_wait_expiry.argtypes = [_I64, _VP]
        L.supa_voxelize_hits.argtypes = [_VP, _VP, _VP, _I64, _VP, _VP, _VP, _VP, _VP]
        L.supa_autotune.argtypes = [ctypes.POINTER(_VP), ctypes.c_int32, _VP, _I64, ctypes.c_uint64,
                                    ctypes.POINTER(supa_launch_config), ctypes.POINTER(ctypes.c_double), _VP]
        L.supa_surrogate_param_count.argtypes = []
        L.supa_surrogate_create.argtypes = [ctypes.c_int32, _VP, ctypes.POINTER(_VP)]
        L.supa_surrogate_destroy.argtypes = [_VP]
        L.supa_surrogate_get_params.argtypes = [_VP, _VP]
        L.supa_surrogate_gradients.argtypes = [_VP, _VP, _VP, _VP, ctypes.POINTER(ctypes.c_double), _VP]
        L.supa_surrogate_train_step.argtypes = [_VP, _VP, _VP, ctypes.c_float, _VP, _VP]
        L.supa_surrogate_forward.argtypes = [_VP, _VP, _I64, _VP, _I64, _VP]
        L.supa_surrogate_check.argtypes = [_VP]
        L.supa_surrogate_train_epoch.argtypes = [_VP, _VP, _VP, _I64, ctypes.c_uint64, ctypes.c_float, _VP, _VP]
        L.supa_surrogate_average.argtypes = [_VP, ctypes.c_int32, _VP]
        L.supa_batch_set_surrogate.argtypes = [_VP, _VP, ctypes.c_float, _I64, ctypes.c_int32]
        L.supa_build_training_set.argtypes = [_VP, ctypes.c_float, _VP, _VP, _VP]
        L.supa_profiles.argtypes = [_VP, _I64, _I64, ctypes.c_int32, ctypes.c_float, _VP, _VP, _VP]
        L.supa_shower_offsets_noalloc.argtypes = [_VP, _I64, _VP, _VP]
        L.supa_export_diverted.argtypes = [_VP, _VP, _I64, ctypes.POINTER(_I64), _VP]
        L.supa_export_surrogate.argtypes = [_VP, _VP, _I64, ctypes.POINTER(_I64), _VP]
        L.supa_batch_warp_times.argtypes = [_VP, _VP, _I64, ctypes.POINTER(_I64)]
        L.supa_shower_shapes.argtypes = [_VP, _I64, _I64, _VP, _VP, _VP]
        L.supa_layer_images_cells.argtypes = [_VP, ctypes.c_int32, _VP, ctypes.c_int32]
        L.supa_voxelize_layers.argtypes = [_VP, _I64, _I64, _VP, ctypes.c_int32, _VP, ctypes.c_int32, _VP, _VP,
                                           _VP]
        for name in EXPORTED[1:]:
            getattr(L, name).restype = ctypes.c_int
        L.supa_layer_images_cells.restype = ctypes.c_int64
        _lib = L
    return _lib


def _check(rc: int, name: str):
    if rc != SUPA_OK:
        msg = lib().supa_last_error().decode()
        raise SupaError(rc, f"{name}: {msg}")


def _ptr(x) -> int | None:
    """Device or host address of a torch tensor / numpy array / int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def supa_last_error() -> str:
    return lib().supa_last_error().decode()


def supa_init_geometry(geom) -> int:
    """Upload a geometry (an inputs.Geometry or any object with its fields)."""
    s2l = np.ascontiguousarray(geom.slice_to_layer, dtype=np.int32)
    ps = np.ascontiguousarray(geom.p_stop, dtype=np.float64)
    pp = np.ascontiguousarray(geom.p_split, dtype=np.float64)
    d = supa_geometry_desc(
        int(geom.n_slices), float(geom.dz), s2l.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(geom.n_layers),
        ps.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), pp.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        int(geom.theta_mode), float(geom.theta_lo), float(geom.theta_hi), int(geom.eps_mode), float(geom.eps_frac),
        int(geom.split_mode), float(geom.e_min), float(geom.uz_min), int(geom.nx), int(geom.ny), float(geom.wx),
        float(geom.wy), int(geom.roi_mode))
    keep = []
    reg = getattr(geom, "regions", None)
    if reg is not None and reg.n > 1:
        keep = [np.ascontiguousarray(a, dtype=np.float64) for a in
                (reg.radius, reg.p_stop, reg.p_split, reg.theta_lo, reg.theta_hi, reg.eps_frac)]
        d.n_regions = reg.n
        for name, a in zip(("region_radius", "region_p_stop", "region_p_split", "region_theta_lo",
                            "region_theta_hi", "region_eps_frac"), keep):
            setattr(d, name, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    out = _VP()
    _check(lib().supa_init_geometry(ctypes.byref(d), ctypes.byref(out)), "supa_init_geometry")
    del keep
    return out.value


def supa_destroy_geometry(g: int):
    _check(lib().supa_destroy_geometry(g), "supa_destroy_geometry")


def _cfg(cfg: dict | None):
    if cfg is None:
        return None
    c = supa_launch_config()
    for k, v in cfg.items():
        setattr(c, k, int(v))
    return ctypes.byref(c)


def supa_batch_create(geoms: list[int], max_showers: int, cfg: dict | None = None) -> int:
    arr = (_VP * len(geoms))(*geoms)
    out = _VP()
    _check(lib().supa_batch_create(arr, len(geoms), int(max_showers), _cfg(cfg), ctypes.byref(out)),
           "supa_batch_create")
    return out.value


def supa_batch_warp_times(b: int) -> np.ndarray:
    """[n_warps, 2] uint64 start / end times (ns, the GPU's global timer) of
    every step-kernel warp in the last simulation (record_warp_times)."""
    n = _I64(0)
    _check(lib().supa_batch_warp_times(b, None, 0, ctypes.byref(n)), "supa_batch_warp_times")
    out = np.zeros((n.value, 2), dtype=np.uint64)
    _check(lib().supa_batch_warp_times(b, out.ctypes.data, n.value, ctypes.byref(n)), "supa_batch_warp_times")
    return out


def supa_destroy_batch(b: int):
    _check(lib().supa_destroy_batch(b), "supa_destroy_batch")


def supa_simulate(b: int, prim_dev, n: int, seed: int, shower_id_base: int = 0, stream=None):
    _check(lib().supa_simulate(b, _ptr(prim_dev), int(n), int(seed) & (2**64 - 1), int(shower_id_base),
                               _stream(stream)), "supa_simulate")


def supa_simulate_batch(geoms: list[int], prim_dev, n: int, seed: int, shower_id_base: int = 0,
                        cfg: dict | None = None, stream=None) -> int:
    arr = (_VP * len(geoms))(*geoms)
    out = _VP()
    _check(lib().supa_simulate_batch(arr, len(geoms), _ptr(prim_dev), int(n), int(seed) & (2**64 - 1),
                                     int(shower_id_base), _cfg(cfg), ctypes.byref(out), _stream(stream)),
           "supa_simulate_batch")
    return out.value


def supa_batch_get_info(b: int, stream=None) -> supa_batch_info:
    info = supa_batch_info()
    _check(lib().supa_batch_get_info(b, ctypes.byref(info), _stream(stream)), "supa_batch_get_info")
    return info


def supa_fetch_hits(b: int, first_hit: int, max_hits: int, dst, dst_is_device: bool | None = None,
                    stream=None) -> int:
    if dst_is_device is None:
        dst_is_device = bool(getattr(dst, "is_cuda", False))
    n = _I64()
    _check(lib().supa_fetch_hits(b, int(first_hit), int(max_hits), _ptr(dst), int(dst_is_device), ctypes.byref(n),
                                 _stream(stream)), "supa_fetch_hits")
    return n.value


def supa_fetch_hit_tags(b: int, first_hit: int, max_hits: int, dst_dev, stream=None) -> int:
    n = _I64()
    _check(lib().supa_fetch_hit_tags(b, int(first_hit), int(max_hits), _ptr(dst_dev), ctypes.byref(n),
                                     _stream(stream)), "supa_fetch_hit_tags")
    return n.value


def supa_voxelize(b: int, shower_begin: int, shower_end: int, grid_dev, out_of_roi_dev=None, stream=None):
    _check(lib().supa_voxelize(b, int(shower_begin), int(shower_end), _ptr(grid_dev), _ptr(out_of_roi_dev),
                               _stream(stream)), "supa_voxelize")


def supa_voxelize_fetch(b: int, shower_begin: int, shower_end: int, grid_dev, out_of_roi_dev, hits_dev,
                        hits_base: int = 0, stream=None):
    """Images and point cloud of showers [shower_begin, shower_end) in one pass;
    hit i of shower s lands in row offsets[s] + i - hits_base of hits_dev."""
    _check(lib().supa_voxelize_fetch(b, int(shower_begin), int(shower_end), _ptr(grid_dev), _ptr(out_of_roi_dev),
                                     _ptr(hits_dev), int(hits_base), _stream(stream)), "supa_voxelize_fetch")


def supa_voxelize_hits(g: int, hits_dev, offsets_dev, n_showers: int, roi_x0_dev, roi_y0_dev, grid_dev,
                       out_of_roi_dev=None, stream=None):
    _check(lib().supa_voxelize_hits(g, _ptr(hits_dev), _ptr(offsets_dev), int(n_showers), _ptr(roi_x0_dev),
                                    _ptr(roi_y0_dev), _ptr(grid_dev), _ptr(out_of_roi_dev), _stream(stream)),
           "supa_voxelize_hits")


def supa_autotune(geoms: list[int], prim_dev, n: int, seed: int, cfg: dict | None = None,
                  stream=None) -> tuple[dict, float]:
    """Returns (tuned launch config as a dict, sample time in ms)."""
    arr = (_VP * len(geoms))(*geoms)
    c = supa_launch_config()
    for k, v in (cfg or {}).items():
        setattr(c, k, int(v))
    ms = ctypes.c_double()
    _check(lib().supa_autotune(arr, len(geoms), _ptr(prim_dev), int(n), int(seed) & (2**64 - 1), ctypes.byref(c),
                               ctypes.byref(ms), _stream(stream)), "supa_autotune")
    return {name: getattr(c, name) for name, _ in supa_launch_config._fields_}, ms.value


def supa_surrogate_param_count() -> int:
    return lib().supa_surrogate_param_count()


def supa_surrogate_create(batch: int, params: np.ndarray) -> int:
    p = np.ascontiguousarray(params, dtype=np.float32)
    assert p.size == supa_surrogate_param_count()
    out = _VP()
    _check(lib().supa_surrogate_create(int(batch), p.ctypes.data, ctypes.byref(out)), "supa_surrogate_create")
    return out.value


def supa_surrogate_destroy(s: int):
    _check(lib().supa_surrogate_destroy(s), "supa_surrogate_destroy")


def supa_surrogate_get_params(s: int) -> np.ndarray:
    p = np.zeros(supa_surrogate_param_count(), dtype=np.float32)
    _check(lib().supa_surrogate_get_params(s, p.ctypes.data), "supa_surrogate_get_params")
    return p


def supa_surrogate_gradients(s: int, x_dev, y_dev, stream=None) -> tuple[np.ndarray, float]:
    g = np.zeros(supa_surrogate_param_count(), dtype=np.float32)
    loss = ctypes.c_double()
    _check(lib().supa_surrogate_gradients(s, _ptr(x_dev), _ptr(y_dev), g.ctypes.data, ctypes.byref(loss),
                                          _stream(stream)), "supa_surrogate_gradients")
    return g, loss.value


def supa_surrogate_train_step(s: int, x_dev, y_dev, lr: float, loss_acc_dev=None, stream=None):
    _check(lib().supa_surrogate_train_step(s, _ptr(x_dev), _ptr(y_dev), float(lr), _ptr(loss_acc_dev),
                                           _stream(stream)), "supa_surrogate_train_step")


def supa_surrogate_forward(s: int, x_dev, n: int, out_dev, ld_out=None, stream=None):
    """ld_out: the row pitch of out_dev in floats (default: the tensor's row stride, else 90)."""
    if ld_out is None:
        ld_out = out_dev.stride(0) if hasattr(out_dev, "stride") and out_dev.dim() == 2 else 90
    _check(lib().supa_surrogate_forward(s, _ptr(x_dev), int(n), _ptr(out_dev), int(ld_out), _stream(stream)),
           "supa_surrogate_forward")


def supa_surrogate_check(s: int):
    _check(lib().supa_surrogate_check(s), "supa_surrogate_check")


SUPA_AVERAGE_STOP, SUPA_AVERAGE_START, SUPA_AVERAGE_APPLY = 0, 1, 2


def supa_surrogate_average(s: int, mode: int, stream=None):
    """Iterate averaging of the training (SUPA_AVERAGE_*): start adding the
    Adam steps that follow to a uniform average, stop, or replace the
    parameters by the average."""
    _check(lib().supa_surrogate_average(s, int(mode), _stream(stream)), "supa_surrogate_average")


def supa_surrogate_train_epoch(s: int, x_dev, y_dev, n: int, seed: int, lr: float, loss_acc_dev=None, stream=None):
    _check(lib().supa_surrogate_train_epoch(s, _ptr(x_dev), _ptr(y_dev), int(n), int(seed) & (2**64 - 1), float(lr),
                                            _ptr(loss_acc_dev), _stream(stream)), "supa_surrogate_train_epoch")


SUPA_SURROGATE_SAMPLE = 0
SUPA_SURROGATE_MEAN = 1


def supa_batch_set_surrogate(b: int, s: int | None, e_s: float, queue_capacity: int, mode: int = SUPA_SURROGATE_SAMPLE):
    _check(lib().supa_batch_set_surrogate(b, s, float(e_s), int(queue_capacity), int(mode)),
           "supa_batch_set_surrogate")


def supa_profiles(b: int, shower_begin: int, shower_end: int, nbins: int, r_max: float, longi_dev, lat_dev,
                  stream=None):
    _check(lib().supa_profiles(b, int(shower_begin), int(shower_end), int(nbins), float(r_max), _ptr(longi_dev),
                               _ptr(lat_dev), _stream(stream)), "supa_profiles")


def supa_shower_offsets_noalloc(counts_dev, n: int, offsets_dev, stream=None):
    """First-hit offsets from per-shower counts; allocates nothing (see include/supa.h)."""
    _check(lib().supa_shower_offsets_noalloc(_ptr(counts_dev), int(n), _ptr(offsets_dev), _stream(stream)),
           "supa_shower_offsets_noalloc")


def supa_build_training_set(b: int, e_s: float, x_dev, y_dev, stream=None):
    _check(lib().supa_build_training_set(b, float(e_s), _ptr(x_dev), _ptr(y_dev), _stream(stream)),
           "supa_build_training_set")


def supa_shower_shapes(b: int, shower_begin: int, shower_end: int, layer_feats_dev, shower_feats_dev, stream=None):
    """Shower shape variables: layer_feats_dev float32 [n][max_layers][18],
    shower_feats_dev float32 [n][5] (see include/supa.h)."""
    _check(lib().supa_shower_shapes(b, int(shower_begin), int(shower_end), _ptr(layer_feats_dev),
                                    _ptr(shower_feats_dev), _stream(stream)), "supa_shower_shapes")


class supa_layer_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("wx", ctypes.c_float), ("wy", ctypes.c_float)]


def _grid_args(grids, factors):
    g = (supa_layer_grid * len(grids))(*[supa_layer_grid(int(nx), int(ny), float(wx), float(wy))
                                         for (nx, ny, wx, wy) in grids])
    f = (ctypes.c_int32 * len(factors))(*[int(x) for x in factors])
    return g, f


def supa_layer_images_cells(grids, factors) -> int:
    """Cells per shower of supa_voxelize_layers for grids [(nx, ny, wx, wy)] per layer and factors."""
    g, f = _grid_args(grids, factors)
    c = lib().supa_layer_images_cells(g, len(grids), f, len(factors))
    if c < 0:
        _check(int(c), "supa_layer_images_cells")
    return int(c)


def supa_voxelize_layers(b: int, shower_begin: int, shower_end: int, grids, factors, images_dev,
                         out_of_roi_dev=None, stream=None):
    """Per-layer grids at every factor from one pass over the hits: images_dev
    float32 [n][cells], out_of_roi_dev float64 [n][len(factors)] or None."""
    g, f = _grid_args(grids, factors)
    _check(lib().supa_voxelize_layers(b, int(shower_begin), int(shower_end), g, len(grids), f, len(factors),
                                      _ptr(images_dev), _ptr(out_of_roi_dev), _stream(stream)),
           "supa_voxelize_layers")


def supa_export_diverted(b: int, out_dev=None, stream=None) -> int:
    """Diverted particles of the last hybrid run as sub-shower primaries into
    out_dev (a uint8 tensor of 24-byte records, or None to only count);
    returns how many the queue held."""
    n = _I64(0)
    cap = 0 if out_dev is None else out_dev.numel() * out_dev.element_size() // 24
    _check(lib().supa_export_diverted(b, _ptr(out_dev) if cap else None, cap, ctypes.byref(n), _stream(stream)),
           "supa_export_diverted")
    return int(n.value)


# supa_diverted_record of include/supa.h (528 bytes)
DIVERTED_RECORD_DTYPE = np.dtype([
    ("shower", "<u4"), ("slice", "<i4"), ("layer", "<i4"), ("x", "<f4"), ("y", "<f4"), ("tx", "<f4"),
    ("ty", "<f4"), ("E", "<f4"), ("lineage", "<u8"), ("lmu", "<f4", 30), ("s", "<f4", 30), ("rho", "<f4", 30),
    ("dep", "<f4", 30), ("n_hits", "<u4"), ("reserved", "<u4")])
assert DIVERTED_RECORD_DTYPE.itemsize == 528


def supa_export_surrogate(b: int, out_dev=None, stream=None) -> int:
    """Per diverted particle of the last hybrid run: key, state, network
    outputs and deposits (supa_diverted_record) into out_dev (a uint8 tensor
    of 528-byte records, or None to only count); returns how many the queue
    held."""
    n = _I64(0)
    size = DIVERTED_RECORD_DTYPE.itemsize
    cap = 0 if out_dev is None else out_dev.numel() * out_dev.element_size() // size
    _check(lib().supa_export_surrogate(b, _ptr(out_dev) if cap else None, cap, ctypes.byref(n), _stream(stream)),
           "supa_export_surrogate")
    return int(n.value)


def pack_mlp_params(params) -> np.ndarray:
    """[(W, b)] -> the packed float32 vector of the C ABI (W row-major, then b)."""
    return np.concatenate([np.concatenate([np.asarray(W).ravel(), np.asarray(b).ravel()]) for W, b in params]
                          ).astype(np.float32)


def unpack_mlp_params(vec: np.ndarray, shapes=((256, 6), (256, 256), (256, 256), (90, 256))):
    out, o = [], 0
    for r, c in shapes:
        W = vec[o:o + r * c].reshape(r, c)
        o += r * c
        b = vec[o:o + r]
        o += r
        out.append((W, b))
    return out


# ---- marshalling helpers ----------------------------------------------------

def primaries_to_device(prims: np.ndarray, device="cuda"):
    """Copy a PRIMARY_DTYPE array into a device byte tensor (24 bytes each)."""
    import torch
    assert prims.dtype == _inputs.PRIMARY_DTYPE
    t = torch.from_numpy(np.ascontiguousarray(prims).view(np.uint8))
    return t.to(device)


class _DeviceArray:
    """Exposes a library-owned device buffer through __cuda_array_interface__."""

    def __init__(self, ptr: int, shape: tuple, typestr: str):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def device_view(ptr: int, shape: tuple, dtype):
    """Zero-copy torch view of a library-owned device buffer."""
    import torch
    typestr = {torch.int64: "<i8", torch.int32: "<i4", torch.float64: "<f8", torch.float32: "<f4"}[dtype]
    if int(np.prod(shape)) == 0:
        return torch.zeros(shape, dtype=dtype, device="cuda")
    return torch.as_tensor(_DeviceArray(ptr, tuple(shape), typestr), device="cuda")


def info_arrays(info: supa_batch_info):
    """Per-shower result buffers of a batch as torch views (valid until the
    batch's next simulation).  counts and steps are uint32 read as int32."""
    import torch
    n, L = info.n_showers, info.max_layers
    return dict(
        offsets=device_view(info.offsets_dev, (n + 1,), torch.int64),
        counts=device_view(info.counts_dev, (n,), torch.int32),
        steps=device_view(info.steps_dev, (n,), torch.int32),
        layer_sum=device_view(info.layer_sums_dev, (n, L), torch.float64),
        dead=device_view(info.dead_dev, (n,), torch.float64),
        leak=device_view(info.leak_dev, (n,), torch.float64),
        escape=device_view(info.escape_dev, (n,), torch.float64),
    )
