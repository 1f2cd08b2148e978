"""Pins of the lateral-region extension of the oracle (Sec. 4.2: slices
divided into regions with their own meta-parameters): identical regions
change nothing; a track stops at the slice where it first reaches a
stopping region (closed form); each region's stop law and split angle are
its own."""
import math

import numpy as np

import oracle
from paper_2202_05012_gb300 import inputs


def _geom(n_layers=10, **kw):
    g = inputs.supa_d(n_layers, e_min=0.0, **kw)
    return g


def test_identical_regions_change_nothing():
    g = inputs.supa_d(10)
    p = inputs.primaries(200, 3, e_lo=1.0, e_hi=30.0, theta_max_deg=20.0, entry_halfwidth=3.0)
    a = oracle.simulate(g, p, 5)
    inputs.with_regions(g, [1.0, 2.5], [g.p_stop] * 3, [g.p_split] * 3, [g.theta_lo] * 3, [g.theta_hi] * 3,
                        [g.eps_frac] * 3)
    b = oracle.simulate(g, p, 5)
    for k in ("x", "y", "E", "slice", "lineage", "steps", "layer_sum"):
        assert np.array_equal(a[k], b[k]), k


def test_track_stops_where_it_reaches_the_stopping_region():
    g = _geom(10)
    g.p_stop[:] = 0.0
    g.p_split[:] = 0.0
    # inner region (r < 2): pass; outer: stop
    inputs.with_regions(g, [2.0], [0.0, 1.0], [0.0, 0.0], [g.theta_lo] * 2, [g.theta_hi] * 2, [0.0, 0.0])
    th = np.array([0.05, 0.1, 0.2, 0.3, 0.45])
    p = inputs.primaries(len(th), 0, e_lo=5.0, e_hi=5.0)
    p["x0"], p["y0"], p["phi"] = 0.3, 0.0, 0.0
    p["theta"] = th
    r = oracle.simulate(g, p, 1)
    t = np.tan(p["theta"].astype(np.float64))
    x0 = float(p["x0"][0])
    # first slice k with x0 + k tan(theta) >= 2 (no ties for these angles)
    k_star = np.ceil((2.0 - x0) / t).astype(int)
    k_star = np.where(k_star < g.n_slices, k_star, -1)
    for s in range(len(th)):
        a, b = r["offsets"][s], r["offsets"][s + 1]
        if k_star[s] < 0:
            assert b == a and r["leak"][s] == 5.0
        else:
            assert b - a == 1 and r["slice"][a] == k_star[s] and r["lineage"][a] == 1 and r["E"][a] == 5.0


def test_each_region_has_its_own_stop_law():
    g = _geom(20)
    g.p_split[:] = 0.0
    # normal incidence: r stays at the entry radius
    inputs.with_regions(g, [1.0], [0.05, 0.25], [0.0, 0.0], [g.theta_lo] * 2, [g.theta_hi] * 2, [0.25, 0.25])
    n = 20000
    p = inputs.primaries(n, 7, e_lo=1.0, e_hi=1.0)
    p["x0"] = np.where(np.arange(n) % 2 == 0, 0.5, 1.5)
    p["y0"] = 0.0
    r = oracle.simulate(g, p, 11, n_threads=8)
    cnt = np.diff(r["offsets"])
    first = r["offsets"][:-1]
    for region, ps in ((0, 0.05), (1, 0.25)):
        sel = (np.arange(n) % 2 == region) & (cnt == 1)
        k = r["slice"][first[sel]]
        # P(stop at k) = ps (1 - ps)^k, k < n_slices: mean of the truncated geometric law
        N = g.n_slices
        ks = np.arange(N)
        pk = ps * (1 - ps) ** ks
        mean = (ks * pk).sum() / pk.sum()
        var = (ks ** 2 * pk).sum() / pk.sum() - mean ** 2
        assert abs(k.mean() - mean) < 4 * math.sqrt(var / len(k)), (region, k.mean(), mean)
        assert abs(sel.sum() / (n / 2) - pk.sum()) < 0.02


def test_each_region_splits_with_its_own_angle():
    g = _geom(3)
    g.p_stop[:] = 0.0
    g.p_split[:] = 0.0
    g.theta_mode = inputs.THETA_UNIFORM
    ps = np.zeros(g.n_slices)
    st = np.zeros(g.n_slices)
    ps[0] = 1.0   # split on slice 0
    st[6] = 1.0   # stop on slice 6
    th0, th1 = math.pi / 24, math.pi / 8
    inputs.with_regions(g, [1.0], [st, st], [ps, ps], [th0, th1], [th0, th1], [0.0, 0.0])
    p = inputs.primaries(40, 9, e_lo=2.0, e_hi=2.0)
    p["x0"] = np.where(np.arange(40) % 2 == 0, 0.2, 3.0)
    p["y0"] = 0.0
    r = oracle.simulate(g, p, 2)
    for s in range(40):
        a = r["offsets"][s]
        assert r["offsets"][s + 1] - a == 2
        d = math.hypot(r["x"][a] - r["x"][a + 1], r["y"][a] - r["y"][a + 1])
        th = th0 if s % 2 == 0 else th1
        # two daughters deflected by theta/2 in opposite azimuths, 6 slices on
        np.testing.assert_allclose(d, 12.0 * math.tan(th / 2), rtol=1e-9)
