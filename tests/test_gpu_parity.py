"""GPU parity: the CUDA path of Algorithm 1 against the FP64 oracle, hit by
hit, on the same seeded primaries (keys: shower, slice, lineage id)."""
import math

import numpy as np
import pytest

import oracle
from paper_2202_05012_gb300 import inputs
from paper_2202_05012_gb300 import supa as S

from gpu_helpers import compare, oracle_multi, run_gpu

pytestmark = pytest.mark.gpu


def _check(geoms, prims, seed, cfg=None, base=0, pos_rtol=1e-5):
    gpu = run_gpu(geoms, prims, seed, cfg=cfg, shower_id_base=base)
    if len(geoms) == 1:
        ora = oracle.simulate(geoms[0], prims, seed, shower_id_base=base, n_threads=8)
    else:
        ora = oracle_multi(geoms, prims, seed, base)
    return compare(gpu, ora, geoms, prims, pos_rtol=pos_rtol), gpu, ora


def test_supav1_exact_on_gpu():
    g = inputs.supa_v1()
    p = inputs.primaries(64, 3, e_lo=65.0, e_hi=65.0)
    gpu = run_gpu([g], p, seed=11)
    assert np.array_equal(np.diff(gpu["offsets"]), [128] * 64)
    assert np.all(gpu["E"] == np.float32(65.0 / 128))
    assert np.all(gpu["z"] == 7.0)
    for s in range(64):
        lin = np.sort(gpu["lineage"][128 * s:128 * (s + 1)])
        assert np.array_equal(lin, np.arange(128, 256, dtype=np.uint64))
    assert np.all(gpu["layer_sum"][:, 0] == 65.0)
    assert np.all(gpu["steps"] == 255)


def test_c1_workload_parity():
    g, p = inputs.workload_plain10(1000)
    st, gpu, ora = _check([g], p, seed=0)
    assert gpu["n_hits"] == ora["offsets"][-1] or st["n_flip_showers"] > 0
    assert st["n_flip_showers"] <= 2


def test_error_report_30_layer_showers():
    """The error of each output against the FP64 oracle on showers shaped
    like the 30-layer workload (E U[1,100] GeV, 0-30 deg; printed as one JSON line; the asserts are the stated tolerances)."""
    import json

    import torch
    g = inputs.supa_d(30, grid=64, roi_mode=inputs.ROI_AXIS)
    p = inputs.primaries(400, 41, e_lo=1.0, e_hi=100.0, theta_max_deg=30.0, entry_halfwidth=0.25)
    st, gpu, ora = _check([g], p, seed=23)
    rx, ry = oracle.roi_origins(g, p)
    grid_o, oor_o = oracle.voxelize(ora["x"], ora["y"], ora["z"], ora["E"], ora["offsets"], g, rx, ry)
    gh = S.supa_init_geometry(g)
    b = S.supa_batch_create([gh], len(p), {})
    try:
        S.supa_simulate(b, S.primaries_to_device(p), len(p), 23)
        S.supa_batch_get_info(b)
        grid = torch.zeros((len(p), 30, 64, 64), dtype=torch.float32, device="cuda")
        oor = torch.zeros(len(p), dtype=torch.float64, device="cuda")
        S.supa_voxelize(b, 0, len(p), grid, oor)
        grid_g = grid.cpu().numpy().astype(np.float64)
        oor_g = oor.cpu().numpy()
    finally:
        S.supa_destroy_batch(b)
        S.supa_destroy_geometry(gh)
    on = (grid_o != 0) | (grid_g != 0)
    cell_err = np.abs(grid_g - grid_o)[on] / np.maximum(np.abs(grid_o[on]), 1e-30)
    st.update(cells_nonzero=int(on.sum()), cells_off_by_more_than_1e5=float(np.mean(cell_err > 1e-5)),
              max_err_out_of_roi=float((np.abs(oor_g - oor_o) / np.maximum(oor_o, 1e-9)).max()))
    print("ERROR_REPORT " + json.dumps(st))
    assert st["cells_off_by_more_than_1e5"] < 1e-4
    assert st["hit_counts_equal"] > 0.99 and st["steps_equal"] > 0.99


def test_inclined_showers_axis_roi_parity():
    g = inputs.supa_d(30, grid=64, roi_mode=inputs.ROI_AXIS)
    p = inputs.primaries(300, 21, e_lo=1.0, e_hi=100.0, theta_max_deg=45.0, entry_halfwidth=0.25)
    _check([g], p, seed=1, base=5000)


def test_dead_material_literal_split_fixed_angles():
    g = inputs.supa_d(8, n_dead_front=4, p_stop=0.05, p_split=0.4)
    g.theta_mode, g.theta_lo, g.theta_hi = inputs.THETA_FIXED, math.pi / 24, math.pi / 24
    g.eps_mode, g.eps_frac = inputs.EPS_ZERO, 0.0
    g.split_mode = inputs.SPLIT_LITERAL
    p = inputs.primaries(300, 22, e_lo=1.0, e_hi=40.0, theta_max_deg=20.0)
    st, gpu, ora = _check([g], p, seed=7)
    assert ora["dead"].sum() > 0


def test_escape_and_leak_paths():
    g = inputs.supa_d(10, p_stop=0.005, p_split=0.3, e_min=0.0)
    p = inputs.primaries(300, 23, e_lo=1.0, e_hi=5.0, theta_max_deg=88.0)
    # near the escape cut the slope u_x/u_z amplifies FP32 direction error by
    # up to 1/uz_min = 1000: positions are held to 1e-5 * 100 here
    st, gpu, ora = _check([g], p, seed=9, pos_rtol=1e-3)
    assert ora["escape"].sum() > 0 and ora["leak"].sum() > 0


@pytest.mark.parametrize("cfg", [
    {"stack_depth": 64, "flush_threshold": 32, "warps_per_block": 4},
    {"stack_depth": 256, "flush_threshold": 256, "warps_per_block": 8, "blocks_per_sm": 1},
    {"lpt_order": 1},
    {"flush_threshold": -1},
])
def test_launch_shapes_do_not_change_results(cfg):
    """Spills to global scratch (tiny stacks), small and large flush thresholds of
    the hit staging, one block per SM, LPT ordering, hits written without
    staging."""
    g = inputs.supa_d(50)
    p = inputs.primaries(60, 24, e_lo=100.0, e_hi=1000.0, log_uniform=True)
    _check([g], p, seed=3, cfg=cfg)


def test_mixed_geometries_in_one_launch():
    geoms, p = inputs.workload_mixed4(240)
    p["E"] = np.minimum(p["E"], 200.0)
    _check(geoms, p, seed=2)


def test_empty_and_single():
    g = inputs.supa_d(5)
    gpu = run_gpu([g], inputs.primaries(0, 1, e_lo=1, e_hi=1), seed=1)
    assert gpu["n_hits"] == 0 and len(gpu["offsets"]) == 1
    _check([g], inputs.primaries(1, 2, e_lo=30, e_hi=30), seed=1)


def test_max_slices_and_layers():
    g = inputs.supa_d(64, slices_per_layer=3, e_min=0.2)  # 192 slices, 64 layers
    p = inputs.primaries(40, 25, e_lo=10, e_hi=300, theta_max_deg=10)
    _check([g], p, seed=4)


def test_determinism_and_replay():
    g, p = inputs.workload_plain10(200)
    a = run_gpu([g], p, seed=5)
    b = run_gpu([g], p, seed=5, cfg={"warps_per_block": 2})
    for key in ("counts", "steps"):
        assert np.array_equal(a[key], b[key])
    np.testing.assert_allclose(a["layer_sum"], b["layer_sum"], rtol=1e-12)  # FP64 sums, order may differ
    # a single shower replayed alone with its global id gives the same hits
    one = run_gpu([g], p[17:18], seed=5, shower_id_base=17)
    sl = slice(a["offsets"][17], a["offsets"][18])
    ka = sorted(zip(a["lineage"][sl].tolist(), a["E"][sl].tolist(), a["x"][sl].tolist()))
    kb = sorted(zip(one["lineage"].tolist(), one["E"].tolist(), one["x"].tolist()))
    assert ka == kb


def test_invalid_primary_reported():
    g = inputs.supa_d(5)
    p = inputs.primaries(10, 1, e_lo=1, e_hi=2)
    p["E"][3] = -1.0
    with pytest.raises(S.SupaError) as ei:
        run_gpu([g], p, seed=1)
    assert ei.value.code == S.SUPA_ERR_INVALID_ARG


def test_hit_pool_overflow_is_an_error_not_a_fault():
    g = inputs.supa_d(50)
    p = inputs.primaries(3000, 26, e_lo=1000, e_hi=1000)
    with pytest.raises(S.SupaError) as ei:
        run_gpu([g], p, seed=1, cfg={"max_hits": 1}, tags=False)
    assert ei.value.code == S.SUPA_ERR_OVERFLOW


def test_fetch_chunks_and_host_destination():
    import torch
    g, p = inputs.workload_plain10(300)
    gh = S.supa_init_geometry(g)
    b = S.supa_batch_create([gh], 300, {"record_tags": 1})
    try:
        S.supa_simulate(b, S.primaries_to_device(p), 300, 0)
        nh = S.supa_batch_get_info(b).n_hits
        full = torch.zeros((nh, 4), dtype=torch.float32, device="cuda")
        assert S.supa_fetch_hits(b, 0, nh, full) == nh
        parts = []
        first = 0
        while first < nh:
            c = torch.zeros((777, 4), dtype=torch.float32, device="cuda")
            m = S.supa_fetch_hits(b, first, 777, c)
            parts.append(c[:m])
            first += m
        assert torch.equal(torch.cat(parts), full)
        host = np.zeros((nh, 4), dtype=np.float32)
        assert S.supa_fetch_hits(b, 0, nh + 10, host, dst_is_device=False) == nh
        assert np.array_equal(host, full.cpu().numpy())
        assert S.supa_fetch_hits(b, nh, 5, full) == 0
    finally:
        S.supa_destroy_batch(b)
        S.supa_destroy_geometry(gh)


def test_observable_distributions_ks():
    """Two-sample KS (p > 0.01) on shower observables: hit multiplicity, total
    deposit, longitudinal centroid and lateral width (Sec. 5.1)."""
    from scipy import stats
    g = inputs.supa_d(30, grid=64, roi_mode=inputs.ROI_AXIS)
    p = inputs.primaries(1000, 27, e_lo=1.0, e_hi=100.0, theta_max_deg=30.0)
    gpu = run_gpu([g], p, seed=13)
    ora = oracle.simulate(g, p, 13, n_threads=8)

    def obs(r):
        cnt = np.diff(r["offsets"])
        sh = np.repeat(np.arange(len(p)), cnt)
        E = np.asarray(r["E"], dtype=np.float64)
        tot = np.bincount(sh, weights=E, minlength=len(p))
        zc = np.bincount(sh, weights=E * np.asarray(r["z"], np.float64), minlength=len(p)) / tot
        rr = np.hypot(np.asarray(r["x"], np.float64), np.asarray(r["y"], np.float64))
        wr = np.bincount(sh, weights=E * rr, minlength=len(p)) / tot
        return dict(mult=cnt, tot=tot, zc=zc, wr=wr)

    a, b = obs(gpu), obs(ora)
    for k in a:
        assert stats.ks_2samp(a[k], b[k]).pvalue > 0.01, k
