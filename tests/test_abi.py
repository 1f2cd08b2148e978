"""The C ABI library builds, loads, and exports every entry point of
include/supa.h; host-side argument checks answer before any CUDA call."""
import ctypes
import math
import re
import os

import numpy as np
import pytest

from paper_2202_05012_gb300 import inputs
from paper_2202_05012_gb300 import supa as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "supa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(supa_[a-z_0-9]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert declared_entry_points() == sorted(S.EXPORTED)


def declared_parameter_counts():
    src = open(os.path.join(ROOT, "include", "supa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for name, params in re.findall(r"\b(supa_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", src):
        params = " ".join(params.split())
        out[name] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_argument_counts_match_the_header():
    """Every prototype's parameter count equals the argtypes the binding sets."""
    L = S.lib()
    counts = declared_parameter_counts()
    assert set(counts) == set(declared_entry_points())
    for name, n in counts.items():
        argtypes = getattr(L, name).argtypes
        assert (len(argtypes) if argtypes is not None else 0) == n, (name, n, argtypes)
        assert argtypes is not None or n == 0, name


def test_library_exports_every_declared_symbol():
    L = S.lib()
    for name in declared_entry_points():
        assert hasattr(L, name), name
    assert S.supa_last_error() == ""


def _desc(**over):
    g = inputs.supa_d(3)
    for k, v in over.items():
        setattr(g, k, v)
    return g


@pytest.mark.parametrize("field,value,needle", [
    ("n_slices", 0, "n_slices"),
    ("n_slices", 256, "n_slices"),
    ("n_layers", 65, "n_layers"),
    ("dz", 0.0, "dz"),
    ("theta_lo", 0.0, "theta"),
    ("theta_hi", 2.0, "theta"),
    ("eps_frac", 0.5, "eps_frac"),
    ("uz_min", 0.0, "uz_min"),
    ("nx", 0, "nx*ny"),
    ("ny", -4, "nx*ny"),
    ("theta_mode", 7, "theta_mode"),
])
def test_geometry_validation_rejects(field, value, needle):
    g = _desc(**{field: value})
    with pytest.raises(S.SupaError) as ei:
        S.supa_init_geometry(g)
    assert ei.value.code == S.SUPA_ERR_INVALID_ARG
    assert needle in str(ei.value)


def test_probabilities_validated():
    g = _desc()
    g.p_stop = g.p_stop.copy()
    g.p_stop[4] = 0.6  # 0.6 + 0.5 > 1
    with pytest.raises(S.SupaError, match="slice 4"):
        S.supa_init_geometry(g)
    g = _desc()
    g.slice_to_layer = g.slice_to_layer.copy()
    g.slice_to_layer[2] = 3
    with pytest.raises(S.SupaError, match="layer 3 out of range"):
        S.supa_init_geometry(g)


def test_lineage_bound_needs_energy_cut():
    g = inputs.supa_d(25, e_min=0.0)  # 75 slices, no cut: lineage ids could overflow
    with pytest.raises(S.SupaError, match="62 slices"):
        S.supa_init_geometry(g)


def _three_regions(**over):
    g = inputs.supa_d(3)
    kw = dict(radius=[1.0, 2.0], p_stop=[0.02, 0.1, 0.3], p_split=[0.5, 0.4, 0.2], theta_lo=[0.1, 0.2, 0.3],
              theta_hi=[0.3, 0.4, 0.5], eps_frac=[0.25, 0.1, 0.0])
    kw.update(over)
    return inputs.with_regions(g, **kw)


@pytest.mark.parametrize("over,needle", [
    (dict(radius=[2.0, 1.0]), "radii"),
    (dict(radius=[0.0, 1.0]), "radii"),
    (dict(radius=[1.0, math.inf]), "radii"),
    (dict(eps_frac=[0.25, 0.5, 0.0]), "region 1: eps_frac"),
    (dict(theta_lo=[0.1, 0.2, 1.6], theta_hi=[0.3, 0.4, 1.7]), "region 2: need 0 < theta_lo"),
    (dict(p_stop=[0.02, 0.7, 0.3]), "region 1, slice 0"),
])
def test_region_validation_rejects(over, needle):
    with pytest.raises(S.SupaError, match=needle) as ei:
        S.supa_init_geometry(_three_regions(**over))
    assert ei.value.code == S.SUPA_ERR_INVALID_ARG


def test_too_many_regions_rejected():
    R = 9
    g = inputs.with_regions(inputs.supa_d(3), list(np.arange(1.0, R)), [0.02] * R, [0.5] * R, [0.1] * R,
                            [0.3] * R, [0.25] * R)
    with pytest.raises(S.SupaError, match="n_regions"):
        S.supa_init_geometry(g)


def test_null_arguments_rejected_without_gpu():
    L = S.lib()
    out = ctypes.c_void_p()
    assert L.supa_init_geometry(None, ctypes.byref(out)) == S.SUPA_ERR_INVALID_ARG
    assert L.supa_batch_create(None, 1, 10, None, ctypes.byref(out)) == S.SUPA_ERR_INVALID_ARG
    info = S.supa_batch_info()
    assert L.supa_batch_get_info(None, ctypes.byref(info), None) == S.SUPA_ERR_INVALID_ARG
    n = ctypes.c_int64()
    assert L.supa_fetch_hits(None, 0, 1, None, 1, ctypes.byref(n), None) == S.SUPA_ERR_INVALID_ARG
    assert L.supa_voxelize(None, 0, 1, None, None, None) == S.SUPA_ERR_INVALID_ARG
    assert L.supa_voxelize_fetch(None, 0, 1, None, None, None, 0, None) == S.SUPA_ERR_INVALID_ARG
    assert L.supa_check_wait_expiry(0, None) == S.SUPA_ERR_INVALID_ARG
    assert L.supa_surrogate_forward(None, None, 1, None, 96, None) == S.SUPA_ERR_INVALID_ARG
    assert L.supa_simulate(None, None, 1, 0, 0, None) == S.SUPA_ERR_INVALID_ARG
    assert "null" in S.supa_last_error()


def test_layer_image_sizes_and_their_validation():
    grids = inputs.calogan_grids()
    # 3x96 + 12x12 + 12x6 = 504 cells at 1x; x4 at 2x, x9 at 3x
    assert S.supa_layer_images_cells(grids, [1]) == 504
    assert S.supa_layer_images_cells(grids, [1, 2, 3]) == 504 * (1 + 4 + 9)
    for bad_grids, bad_factors in (([(0, 12, 1.0, 1.0)], [1]), ([(12, 12, -1.0, 1.0)], [1]),
                                   ([(12, 12, 1.0, float("nan"))], [1]), (grids, [0]), (grids, [17]),
                                   (grids, [1] * 9)):
        with pytest.raises(S.SupaError) as ei:
            S.supa_layer_images_cells(bad_grids, bad_factors)
        assert ei.value.code == S.SUPA_ERR_INVALID_ARG
