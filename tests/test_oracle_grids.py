"""Pins of the per-layer-grid / multi-resolution downsampling oracle: at
factor 1 with the geometry's own grid it is the pinned uniform downsampler;
power-of-two cells nest exactly across factors; a CaloGAN-like layer grid
matches numpy.histogram2d (library routine) away from cell edges; energy is
conserved at every factor."""
import numpy as np

import oracle
from oracle import grids as G
from paper_2202_05012_gb300 import inputs


def _sim(g, n, seed, **kw):
    p = inputs.primaries(n, seed, **kw)
    return p, oracle.simulate(g, p, seed, n_threads=8)


def test_factor_one_is_the_uniform_downsampler():
    for roi in (inputs.ROI_FIXED, inputs.ROI_AXIS):
        g = inputs.supa_d(6, grid=32, roi_mode=roi)
        p, r = _sim(g, 60, 3, e_lo=1.0, e_hi=30.0, theta_max_deg=25.0, entry_halfwidth=0.5)
        rx, ry = oracle.roi_origins(g, p)
        ref, oor_ref = oracle.voxelize(r["x"], r["y"], r["z"], r["E"], r["offsets"], g, rx, ry)
        grids = [(g.nx, g.ny, g.wx, g.wy)] * g.n_layers
        img, oor = G.voxelize_layers(r["x"], r["y"], r["z"], r["E"], r["offsets"], g, p, grids, [1])
        np.testing.assert_array_equal(img, ref.reshape(len(p), -1))
        np.testing.assert_array_equal(oor[:, 0], oor_ref)


def test_power_of_two_cells_nest_exactly():
    g = inputs.supa_d(4, grid=16, roi_mode=inputs.ROI_FIXED)  # cells of 1.0
    p, r = _sim(g, 40, 5, e_lo=1.0, e_hi=20.0, theta_max_deg=20.0)
    grids = [(16, 16, 1.0, 1.0), (8, 8, 2.0, 2.0), (16, 8, 1.0, 2.0), (4, 16, 4.0, 1.0)]
    img, oor = G.voxelize_layers(r["x"], r["y"], r["z"], r["E"], r["offsets"], g, p, grids, [1, 2, 4])
    c1 = G.cells(grids, [1])
    c2 = G.cells(grids, [2])
    o = 0
    for l, (nx, ny, _, _) in enumerate(grids):
        a = img[:, o:o + nx * ny].reshape(-1, ny, nx)
        o2 = c1 + sum(2 * grids[m][1] * 2 * grids[m][0] for m in range(l))
        b = img[:, o2:o2 + 4 * nx * ny].reshape(-1, 2 * ny, 2 * nx)
        o4 = c1 + c2 + sum(4 * grids[m][1] * 4 * grids[m][0] for m in range(l))
        c = img[:, o4:o4 + 16 * nx * ny].reshape(-1, 4 * ny, 4 * nx)
        np.testing.assert_allclose(b.reshape(-1, ny, 2, nx, 2).sum((2, 4)), a, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(c.reshape(-1, ny, 4, nx, 4).sum((2, 4)), a, rtol=1e-12, atol=1e-12)
        o += nx * ny
    np.testing.assert_array_equal(oor[:, 0], oor[:, 1])
    np.testing.assert_array_equal(oor[:, 0], oor[:, 2])


def test_calogan_like_layer_matches_histogram2d_away_from_edges():
    g = inputs.supa_calogan()
    grids = inputs.calogan_grids()
    rng = np.random.default_rng(4)
    m = 20000
    x = rng.uniform(-9, 9, m).astype(np.float32)
    y = rng.uniform(-9, 9, m).astype(np.float32)
    E = rng.uniform(0.1, 1.0, m).astype(np.float32)
    z = np.full(m, 10.0, dtype=np.float32)  # slice 10: layer 1
    p = inputs.primaries(1, 0, e_lo=1.0, e_hi=1.0)  # normal incidence at the origin
    img, oor = G.voxelize_layers(x, y, z, E, np.array([0, m]), g, p, grids, [1, 3])
    for fi, f in enumerate((1, 3)):
        nx, ny, wx, wy = grids[1]
        ex = -nx * wx / 2 + np.arange(nx * f + 1) * (wx / f)
        ey = -ny * wy / 2 + np.arange(ny * f + 1) * (wy / f)
        h, _, _ = np.histogram2d(y.astype(np.float64), x.astype(np.float64), bins=[ey, ex], weights=E.astype(np.float64))
        near = (np.min(np.abs(x[:, None].astype(np.float64) - ex[None, :]), 1) < 1e-4) | \
               (np.min(np.abs(y[:, None].astype(np.float64) - ey[None, :]), 1) < 1e-4)
        assert near.mean() < 0.01
        hn, _, _ = np.histogram2d(y[near], x[near], bins=[ey, ex], weights=E[near].astype(np.float64))
        off = G.cells(grids, [1]) if f == 3 else 0
        off += sum(grids[l][1] * f * grids[l][0] * f for l in range(1))
        mine = img[0, off:off + nx * f * ny * f].reshape(ny * f, nx * f)
        # cells agree exactly once the points within rounding of an edge are set aside
        assert np.all(np.abs(mine - h) <= hn + 1e-9)
        inside = (np.abs(x) < nx * wx / 2) & (np.abs(y) < ny * wy / 2)
        np.testing.assert_allclose(mine.sum() + oor[0, fi], E.astype(np.float64).sum(), rtol=1e-12)
        assert abs(mine.sum() - E[inside].astype(np.float64).sum()) <= E[near].sum() + 1e-9


def test_energy_is_conserved_at_every_factor():
    g = inputs.supa_calogan()
    p, r = _sim(g, 50, 9, e_lo=1.0, e_hi=100.0)
    grids = inputs.calogan_grids()
    img, oor = G.voxelize_layers(r["x"], r["y"], r["z"], r["E"], r["offsets"], g, p, grids, [1, 2, 3])
    # the hits enter as float32 (the GPU's hit format)
    E32 = r["E"].astype(np.float32).astype(np.float64)
    tot = np.array([E32[a:b].sum() for a, b in zip(r["offsets"][:-1], r["offsets"][1:])])
    o = 0
    for fi, f in enumerate((1, 2, 3)):
        c = G.cells(grids, [f])
        np.testing.assert_allclose(img[:, o:o + c].sum(1) + oor[:, fi], tot, rtol=1e-12)
        o += c
