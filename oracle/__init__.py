"""Plain FP64 CPU oracle for SUPA (arxiv 2202.05012) -- TEST INFRASTRUCTURE.

Only tests/, ``__graft_entry__.smoke()`` and the cpu_baseline / reference legs
of ``bench.py`` may import this package.  The product package never imports
it, and it imports nothing from the product: geometries and primaries arrive
as plain objects and numpy arrays (duck-typed), drawn by the seeded input
module.

Contents
  * supa_oracle.c  -- Philox4x32-10, Algorithm 1 per shower (Sec. 3), the
                      downsampling of App. A.5; FP64 except the float32
                      decisions named in its header.
  * roi_origins()  -- the region-of-interest corners of the downsampling grid
                      (App. A.5, "a rectangular region for each layer").
  * mlp.py         -- FP64 surrogate network forward/backward, loss and Adam.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile supa_oracle.c into liboracle.so with gcc (OpenMP, no FMA contraction)."""
    src = os.path.join(_HERE, "supa_oracle.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "supa_oracle.h"))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Geom(ctypes.Structure):
    _fields_ = [
        ("n_slices", ctypes.c_int), ("dz", ctypes.c_double),
        ("slice_to_layer", ctypes.POINTER(ctypes.c_int)), ("n_layers", ctypes.c_int),
        ("p_stop", ctypes.POINTER(ctypes.c_double)), ("p_split", ctypes.POINTER(ctypes.c_double)),
        ("theta_mode", ctypes.c_int), ("theta_lo", ctypes.c_double), ("theta_hi", ctypes.c_double),
        ("eps_mode", ctypes.c_int), ("eps_frac", ctypes.c_double),
        ("split_mode", ctypes.c_int), ("e_min", ctypes.c_double), ("uz_min", ctypes.c_double),
        ("e_s", ctypes.c_double),
        ("n_regions", ctypes.c_int), ("region_radius", ctypes.POINTER(ctypes.c_double)),
        ("region_p_stop", ctypes.POINTER(ctypes.c_double)), ("region_p_split", ctypes.POINTER(ctypes.c_double)),
        ("region_theta_lo", ctypes.POINTER(ctypes.c_double)), ("region_theta_hi", ctypes.POINTER(ctypes.c_double)),
        ("region_eps_frac", ctypes.POINTER(ctypes.c_double)),
    ]


class _Primary(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("x0", ctypes.c_double), ("y0", ctypes.c_double),
                ("theta", ctypes.c_double), ("phi", ctypes.c_double), ("start_slice", ctypes.c_int)]


_PRIMARY_NP = np.dtype([("E", "<f8"), ("x0", "<f8"), ("y0", "<f8"), ("theta", "<f8"), ("phi", "<f8"),
                        ("start_slice", "<i4"), ("pad", "<i4")])

_P = ctypes.POINTER


class _Result(ctypes.Structure):
    _fields_ = [
        ("n_hits", ctypes.c_int64),
        ("hx", _P(ctypes.c_double)), ("hy", _P(ctypes.c_double)), ("hz", _P(ctypes.c_double)),
        ("hE", _P(ctypes.c_double)), ("hslice", _P(ctypes.c_int32)), ("hlineage", _P(ctypes.c_uint64)),
        ("n_showers", ctypes.c_int64), ("hit_offset", _P(ctypes.c_int64)), ("steps", _P(ctypes.c_int64)),
        ("layer_sum", _P(ctypes.c_double)), ("dead", _P(ctypes.c_double)), ("leak", _P(ctypes.c_double)),
        ("escape", _P(ctypes.c_double)), ("n_splits", _P(ctypes.c_int64)), ("max_depth", _P(ctypes.c_int32)),
        ("status", ctypes.c_int),
        ("n_div", ctypes.c_int64), ("div_shower", _P(ctypes.c_int64)), ("div_k", _P(ctypes.c_int32)),
        ("div_layer", _P(ctypes.c_int32)), ("div_x", _P(ctypes.c_double)), ("div_y", _P(ctypes.c_double)),
        ("div_ux", _P(ctypes.c_double)), ("div_uy", _P(ctypes.c_double)), ("div_uz", _P(ctypes.c_double)),
        ("div_E", _P(ctypes.c_double)), ("div_lin", _P(ctypes.c_uint64)),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            L.ora_philox4x32_10.argtypes = [_P(ctypes.c_uint32), _P(ctypes.c_uint32), _P(ctypes.c_uint32)]
            L.ora_simulate.argtypes = [_P(_Geom), ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64,
                                       ctypes.c_uint64, ctypes.c_int, _P(_Result)]
            L.ora_simulate.restype = ctypes.c_int
            L.ora_free_result.argtypes = [_P(_Result)]
            L.ora_voxelize.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_void_p, ctypes.c_int64, ctypes.c_float,
                                                               ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                                               ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                                               ctypes.c_void_p, ctypes.c_void_p]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one counter block: ctr (4 x u32), key (2 x u32) -> 4 x u32."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().ora_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def simulate(geom, prims: np.ndarray, seed: int, shower_id_base: int = 0, n_threads: int = 1,
             e_s: float = 0.0) -> dict:
    """Run Algorithm 1 on every shower; returns numpy arrays (hits sorted per
    shower by slice then lineage) and per-shower FP64 bookkeeping.  With
    e_s > 0, particles below e_s on a readout slice are returned as the
    'div' records (hybrid path) instead of being stepped."""
    s2l = np.ascontiguousarray(geom.slice_to_layer, dtype=np.int32)
    ps = np.ascontiguousarray(geom.p_stop, dtype=np.float64)
    pp = np.ascontiguousarray(geom.p_split, dtype=np.float64)
    g = _Geom(int(geom.n_slices), float(geom.dz), s2l.ctypes.data_as(_P(ctypes.c_int)), int(geom.n_layers),
              ps.ctypes.data_as(_P(ctypes.c_double)), pp.ctypes.data_as(_P(ctypes.c_double)),
              int(geom.theta_mode), float(geom.theta_lo), float(geom.theta_hi), int(geom.eps_mode),
              float(geom.eps_frac), int(geom.split_mode), float(geom.e_min), float(geom.uz_min), float(e_s))
    keep = []
    reg = getattr(geom, "regions", None)
    if reg is not None and reg.n > 1:
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in
                (reg.radius, reg.p_stop, reg.p_split, reg.theta_lo, reg.theta_hi, reg.eps_frac)]
        keep.extend(arrs)
        g.n_regions = reg.n
        for name, a in zip(("region_radius", "region_p_stop", "region_p_split", "region_theta_lo",
                            "region_theta_hi", "region_eps_frac"), arrs):
            setattr(g, name, a.ctypes.data_as(_P(ctypes.c_double)))
    n = len(prims)
    assert ctypes.sizeof(_Primary) == _PRIMARY_NP.itemsize
    pr = np.zeros(max(n, 1), dtype=_PRIMARY_NP)
    for f in ("E", "x0", "y0", "theta", "phi"):
        pr[f][:n] = prims[f].astype(np.float64)
    pr["start_slice"][:n] = (prims["geom"].astype(np.uint32) >> np.uint32(16)).astype(np.int32)
    res = _Result()
    rc = lib().ora_simulate(ctypes.byref(g), _ptr(pr), n, int(seed) & (2**64 - 1), int(shower_id_base),
                            int(n_threads), ctypes.byref(res))
    if rc != 0:
        raise MemoryError("oracle simulation failed")
    try:
        nh = res.n_hits
        L = int(geom.n_layers)

        def arr(p, count, dt):
            if count == 0:
                return np.zeros(0, dtype=dt)
            return np.ctypeslib.as_array(p, shape=(count,)).astype(dt, copy=True)

        out = dict(
            x=arr(res.hx, nh, np.float64), y=arr(res.hy, nh, np.float64), z=arr(res.hz, nh, np.float64),
            E=arr(res.hE, nh, np.float64), slice=arr(res.hslice, nh, np.int32),
            lineage=arr(res.hlineage, nh, np.uint64), offsets=arr(res.hit_offset, n + 1, np.int64),
            steps=arr(res.steps, n, np.int64), layer_sum=arr(res.layer_sum, n * L, np.float64).reshape(n, L),
            dead=arr(res.dead, n, np.float64), leak=arr(res.leak, n, np.float64),
            escape=arr(res.escape, n, np.float64), n_splits=arr(res.n_splits, n, np.int64),
            max_depth=arr(res.max_depth, n, np.int32),
        )
        nd = res.n_div
        out["div"] = dict(
            shower=arr(res.div_shower, nd, np.int64), k=arr(res.div_k, nd, np.int32),
            layer=arr(res.div_layer, nd, np.int32), x=arr(res.div_x, nd, np.float64),
            y=arr(res.div_y, nd, np.float64), ux=arr(res.div_ux, nd, np.float64), uy=arr(res.div_uy, nd, np.float64),
            uz=arr(res.div_uz, nd, np.float64), E=arr(res.div_E, nd, np.float64),
            lineage=arr(res.div_lin, nd, np.uint64))
    finally:
        lib().ora_free_result(ctypes.byref(res))
    return out


def roi_origins(geom, prims: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Low corners [n, L] (float32) of each layer's region of interest.

    FIXED: centred on the z axis.  AXIS: centred on the nominal shower axis
    (the incidence direction through the origin) at the layer's mid depth,
    so an offset impact point shows up as a displacement in the image.
    """
    n, L = len(prims), int(geom.n_layers)
    f32 = np.float32
    half_x = f32(geom.nx) * f32(geom.wx) * f32(0.5)
    half_y = f32(geom.ny) * f32(geom.wy) * f32(0.5)
    x0 = np.full((n, L), -half_x, dtype=f32)
    y0 = np.full((n, L), -half_y, dtype=f32)
    if int(geom.roi_mode) == 1:
        th = prims["theta"].astype(f32)
        ph = prims["phi"].astype(f32)
        t = np.tan(th).astype(f32)
        tx = (t * np.cos(ph).astype(f32)).astype(f32)
        ty = (t * np.sin(ph).astype(f32)).astype(f32)
        for l in range(L):
            ks = np.nonzero(np.asarray(geom.slice_to_layer) == l)[0]
            zmid = f32(f32(geom.dz) * f32(int(ks.min()) + int(ks.max())) * f32(0.5))
            x0[:, l] = (zmid * tx).astype(f32) - half_x
            y0[:, l] = (zmid * ty).astype(f32) - half_y
    return x0, y0


def voxelize(hx, hy, hz, hE, offsets, geom, roi_x0, roi_y0) -> tuple[np.ndarray, np.ndarray]:
    """Downsample float32 hits into [n, L, ny, nx] FP64 cell sums plus the
    per-shower energy that falls outside every region of interest."""
    hx, hy, hz, hE = (np.ascontiguousarray(a, dtype=np.float32) for a in (hx, hy, hz, hE))
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    n = len(offsets) - 1
    L = int(geom.n_layers)
    s2l = np.ascontiguousarray(geom.slice_to_layer, dtype=np.int32)
    rx = np.ascontiguousarray(roi_x0, dtype=np.float32)
    ry = np.ascontiguousarray(roi_y0, dtype=np.float32)
    grid = np.zeros((n, L, int(geom.ny), int(geom.nx)), dtype=np.float64)
    oor = np.zeros(n, dtype=np.float64)
    lib().ora_voxelize(_ptr(hx), _ptr(hy), _ptr(hz), _ptr(hE), _ptr(offsets), n, float(geom.dz), _ptr(s2l),
                       int(geom.n_slices), L, _ptr(rx), _ptr(ry), int(geom.nx), int(geom.ny),
                       float(geom.wx), float(geom.wy), _ptr(grid), _ptr(oor))
    return grid, oor
