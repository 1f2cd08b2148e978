"""GPU parity of the downsampling kernel (App. A.5) against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2202_05012_gb300 import inputs
from paper_2202_05012_gb300 import supa as S

from gpu_helpers import run_gpu

pytestmark = pytest.mark.gpu


def _synthetic_hits(geom, n, seed, per=200, spread=6.0):
    """Seeded float32 hits: normal lateral spread, uniform slices, some on
    exact cell edges and outside the region."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cnt = rng.integers(0, per, n)
    cnt[0] = 0
    off = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
    nh = int(off[-1])
    x = rng.normal(0, spread, nh).astype(np.float32)
    y = rng.normal(0, spread, nh).astype(np.float32)
    edge = rng.random(nh) < 0.1
    x[edge] = (np.round(x[edge] / geom.wx) * geom.wx).astype(np.float32)
    z = (rng.integers(0, geom.n_slices, nh) * geom.dz).astype(np.float32)
    E = rng.exponential(1.0, nh).astype(np.float32)
    return np.stack([x, y, z, E], 1), off


@pytest.mark.parametrize("layers,grid,roi", [(10, 32, inputs.ROI_FIXED), (30, 64, inputs.ROI_AXIS),
                                             (5, 128, inputs.ROI_AXIS), (3, 12, inputs.ROI_FIXED)])
def test_voxelize_hits_bin_exact(layers, grid, roi):
    import torch
    g = inputs.supa_d(layers, n_dead_front=2, grid=grid, roi_mode=roi)
    n = 97
    prims = inputs.primaries(n, 5, e_lo=1, e_hi=1, theta_max_deg=30)
    hits, off = _synthetic_hits(g, n, 11)
    rx, ry = oracle.roi_origins(g, prims)
    grid_o, oor_o = oracle.voxelize(hits[:, 0], hits[:, 1], hits[:, 2], hits[:, 3], off, g, rx, ry)
    gh = S.supa_init_geometry(g)
    try:
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        out = torch.full((n, layers, g.ny, g.nx), -1.0, dtype=torch.float32, device="cuda")
        oor = torch.zeros(n, dtype=torch.float64, device="cuda")
        S.supa_voxelize_hits(gh, dev(hits), dev(off), n, dev(rx), dev(ry), out, oor)
        grid_g = out.cpu().numpy().astype(np.float64)
        # the same cells receive energy (bin indices decided in float32 on both sides)
        assert np.array_equal(grid_g != 0, grid_o != 0)
        np.testing.assert_allclose(grid_g, grid_o, rtol=2e-6, atol=0)
        np.testing.assert_allclose(oor.cpu().numpy(), oor_o, rtol=1e-12, atol=1e-12)
    finally:
        S.supa_destroy_geometry(gh)


def test_batch_voxelize_matches_oracle_and_conserves():
    import torch
    g = inputs.supa_d(30, grid=64, roi_mode=inputs.ROI_AXIS)
    p = inputs.primaries(200, 31, e_lo=1.0, e_hi=100.0, theta_max_deg=30.0, entry_halfwidth=0.25)
    ora = oracle.simulate(g, p, 17, n_threads=8)
    rx, ry = oracle.roi_origins(g, p)
    grid_o, oor_o = oracle.voxelize(ora["x"], ora["y"], ora["z"], ora["E"], ora["offsets"], g, rx, ry)
    gh = S.supa_init_geometry(g)
    b = S.supa_batch_create([gh], 200, {})
    try:
        S.supa_simulate(b, S.primaries_to_device(p), 200, 17)
        info = S.supa_batch_get_info(b)
        grid = torch.full((200, 30, 64, 64), -1.0, dtype=torch.float32, device="cuda")
        oor = torch.zeros(200, dtype=torch.float64, device="cuda")
        S.supa_voxelize(b, 0, 200, grid, oor)
        # chunked voxelisation gives the same images (float32 cell sums from
        # shared-memory atomics: equal up to the order of additions)
        g2 = torch.full((120, 30, 64, 64), -1.0, dtype=torch.float32, device="cuda")
        S.supa_voxelize(b, 80, 200, g2, None)
        assert torch.equal(g2 != 0, grid[80:] != 0)
        assert torch.allclose(g2, grid[80:], rtol=1e-6, atol=0)
        grid_g = grid.cpu().numpy().astype(np.float64)
        arr = S.info_arrays(info)
        ls = arr["layer_sum"].cpu().numpy()
        # conservation: image + out-of-region = all deposits (per shower)
        np.testing.assert_allclose(grid_g.sum((1, 2, 3)) + oor.cpu().numpy(), ls.sum(1), rtol=1e-5)
        # against the oracle: cells can move only where a rounding difference
        # crosses a cell edge
        diff = np.abs(grid_g - grid_o)
        tol = 1e-5 * np.maximum(np.abs(grid_o), 1e-3)
        frac_bad = np.mean(diff > tol)
        assert frac_bad < 1e-5, frac_bad
        np.testing.assert_allclose(grid_g.sum((1, 2, 3)), grid_o.sum((1, 2, 3)), rtol=1e-4)
    finally:
        S.supa_destroy_batch(b)
        S.supa_destroy_geometry(gh)


def test_profiles_match_oracle():
    """Longitudinal (layer energy / E0) and lateral (energy / E0 in rings
    around the incidence axis) profiles against the same sums over the
    oracle's showers."""
    import torch
    g = inputs.supa_d(30, grid=64, roi_mode=inputs.ROI_AXIS)
    n = 500
    p = inputs.primaries(n, 41, e_lo=1.0, e_hi=50.0, theta_max_deg=30.0, entry_halfwidth=0.25)
    gh = S.supa_init_geometry(g)
    b = S.supa_batch_create([gh], n, {})
    try:
        S.supa_simulate(b, S.primaries_to_device(p), n, 21)
        S.supa_batch_get_info(b)
        lo = torch.zeros(30, dtype=torch.float64, device="cuda")
        la = torch.zeros(64, dtype=torch.float64, device="cuda")
        S.supa_profiles(b, 0, n, 64, 8.0, lo, la)
        lo, la = lo.cpu().numpy(), la.cpu().numpy()
    finally:
        S.supa_destroy_batch(b)
        S.supa_destroy_geometry(gh)
    ora = oracle.simulate(g, p, 21, n_threads=8)
    E0 = p["E"].astype(np.float64)
    np.testing.assert_allclose(lo, (ora["layer_sum"] / E0[:, None]).sum(0), rtol=1e-4, atol=1e-6)
    sh = np.repeat(np.arange(n), np.diff(ora["offsets"]))
    th, ph = p["theta"].astype(np.float64)[sh], p["phi"].astype(np.float64)[sh]
    ax = p["x0"].astype(np.float64)[sh] + ora["z"] * np.tan(th) * np.cos(ph)
    ay = p["y0"].astype(np.float64)[sh] + ora["z"] * np.tan(th) * np.sin(ph)
    r = np.hypot(ora["x"] - ax, ora["y"] - ay)
    bins = np.minimum((r * 8.0).astype(int), 63)
    ref = np.bincount(bins, weights=ora["E"] / E0[sh], minlength=64)
    np.testing.assert_allclose(la, ref, rtol=2e-3, atol=1e-3)
    np.testing.assert_allclose(la.sum(), ref.sum(), rtol=1e-5)


def test_voxelize_rejects_bad_ranges():
    import torch
    g = inputs.supa_d(3)
    gh = S.supa_init_geometry(g)
    b = S.supa_batch_create([gh], 10, {})
    try:
        grid = torch.zeros((10, 3, 32, 32), dtype=torch.float32, device="cuda")
        with pytest.raises(S.SupaError):
            S.supa_voxelize(b, 0, 10, grid)  # before any simulation
        S.supa_simulate(b, S.primaries_to_device(inputs.primaries(10, 1, e_lo=1, e_hi=2)), 10, 1)
        S.supa_batch_get_info(b)
        with pytest.raises(S.SupaError):
            S.supa_voxelize(b, 5, 11, grid)
        S.supa_voxelize(b, 3, 3, grid)  # empty range is fine
    finally:
        S.supa_destroy_batch(b)
        S.supa_destroy_geometry(gh)


@pytest.mark.parametrize("hybrid", [False, True])
def test_voxelize_fetch_equals_voxelize_then_fetch(hybrid):
    """One pass for images and point cloud gives what supa_voxelize followed by
    supa_fetch_hits gives (the point cloud bit for bit), also in chunks with a
    hit offset and with the surrogate's hits after the stepped ones."""
    import torch
    g = inputs.supa_d(20, grid=32, roi_mode=inputs.ROI_AXIS)
    n = 3000
    p = inputs.primaries(n, 17, e_lo=1.0, e_hi=60.0, theta_max_deg=25.0, entry_halfwidth=0.5)
    gh = S.supa_init_geometry(g)
    sur = S.supa_surrogate_create(1024, S.pack_mlp_params(inputs.mlp_init(3))) if hybrid else None
    b = S.supa_batch_create([gh], n, {})
    try:
        if hybrid:
            S.supa_batch_set_surrogate(b, sur, 1.0, 2_000_000, S.SUPA_SURROGATE_MEAN)
        S.supa_simulate(b, S.primaries_to_device(p), n, 8)
        info = S.supa_batch_get_info(b)
        if hybrid:
            assert info.n_diverted > 0
        nh = info.n_hits
        off = S.info_arrays(info)["offsets"].cpu().numpy()
        L = info.max_layers
        ref_img = torch.empty((n, L, 32, 32), device="cuda")
        ref_oor = torch.empty(n, dtype=torch.float64, device="cuda")
        S.supa_voxelize(b, 0, n, ref_img, ref_oor)
        ref_hits = torch.empty((nh, 4), device="cuda")
        assert S.supa_fetch_hits(b, 0, nh, ref_hits) == nh
        img = torch.full((n, L, 32, 32), float("nan"), device="cuda")
        oor = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        hits = torch.full((nh, 4), float("nan"), device="cuda")
        S.supa_voxelize_fetch(b, 0, n, img, oor, hits)
        torch.cuda.synchronize()
        assert torch.equal(hits, ref_hits) and torch.equal(oor, ref_oor)
        # cells sum in shared-memory float atomics: the order of the additions,
        # and so the last bits, may differ from run to run
        torch.testing.assert_close(img, ref_img, rtol=1e-5, atol=1e-6)
        # two chunks into their own buffers, each indexed from its first hit
        c = 1234
        for s0, s1 in ((0, c), (c, n)):
            m = int(off[s1] - off[s0])
            part = torch.full((max(m, 1), 4), float("nan"), device="cuda")
            S.supa_voxelize_fetch(b, s0, s1, img[s0:s1], oor[s0:s1], part, int(off[s0]))
            torch.cuda.synchronize()
            assert torch.equal(part[:m], ref_hits[off[s0]:off[s1]])
        torch.testing.assert_close(img, ref_img, rtol=1e-5, atol=1e-6)
        with pytest.raises(S.SupaError):
            S.supa_voxelize_fetch(b, 0, n, img, oor, hits[:, 1:], 0)  # not 16-byte aligned
    finally:
        S.supa_destroy_batch(b)
        if sur is not None:
            S.supa_surrogate_destroy(sur)
        S.supa_destroy_geometry(gh)


def test_voxelize_windows_and_oversized_layer_groups():
    """Showers whose hits overflow the shared-memory list: layers taken in
    several windows, a layer group with more hits than the list holds binned
    straight from the hits, an empty shower -- all against the oracle."""
    import torch
    g = inputs.supa_d(6, grid=128, roi_mode=inputs.ROI_FIXED)  # 64 KB per layer: one layer per group
    rng = np.random.Generator(np.random.PCG64(21))

    def shower(n_hits, slices):
        x = rng.normal(0, 3.0, n_hits).astype(np.float32)
        y = rng.normal(0, 3.0, n_hits).astype(np.float32)
        z = (rng.choice(slices, n_hits) * g.dz).astype(np.float32)
        E = rng.exponential(1.0, n_hits).astype(np.float32)
        return np.stack([x, y, z, E], 1)

    parts = [shower(30000, np.arange(g.n_slices)),                 # ~5,000 per layer: one window per layer
             np.concatenate([shower(12000, [3, 4, 5]), shower(300, np.arange(g.n_slices))]),  # one layer > list
             np.zeros((0, 4), np.float32),
             shower(100, np.arange(g.n_slices))]
    hits = np.concatenate(parts)
    off = np.concatenate([[0], np.cumsum([len(q) for q in parts])]).astype(np.int64)
    n = len(parts)
    prims = inputs.primaries(n, 5, e_lo=1, e_hi=1)
    rx, ry = oracle.roi_origins(g, prims)
    grid_o, oor_o = oracle.voxelize(hits[:, 0], hits[:, 1], hits[:, 2], hits[:, 3], off, g, rx, ry)
    gh = S.supa_init_geometry(g)
    try:
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        out = torch.full((n, g.n_layers, g.ny, g.nx), -1.0, dtype=torch.float32, device="cuda")
        oor = torch.zeros(n, dtype=torch.float64, device="cuda")
        S.supa_voxelize_hits(gh, dev(hits), dev(off), n, dev(rx), dev(ry), out, oor)
        grid_g = out.cpu().numpy().astype(np.float64)
        assert np.array_equal(grid_g != 0, grid_o != 0)
        np.testing.assert_allclose(grid_g, grid_o, rtol=2e-6, atol=1e-6)
        np.testing.assert_allclose(oor.cpu().numpy(), oor_o, rtol=1e-12, atol=1e-12)
        assert np.all(grid_g[2] == 0)
    finally:
        S.supa_destroy_geometry(gh)
