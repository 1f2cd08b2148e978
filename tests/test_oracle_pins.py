"""Pins of the FP64 oracle to facts the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks it against a
library routine, a closed form of the splitting process, a brute-force
enumeration, the paper's worked example (SUPAv1, Table 2 / App. A.2.1), or a
geometric invariant of the split kinematics (Sec. 3, Algorithm 1).
"""
import ctypes
import ctypes.util
import math
import os
from collections import Counter

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2202_05012_gb300 import inputs


def _tiny_geom(n, p_stop, p_split, **kw):
    g = inputs.supa_d(1, slices_per_layer=n, p_stop=0.0, p_split=0.0, e_min=0.0)
    g.p_stop = np.asarray(p_stop, dtype=np.float64)
    g.p_split = np.asarray(p_split, dtype=np.float64)
    for k, v in kw.items():
        setattr(g, k, v)
    return g


# ---------------------------------------------------------------- Philox ---

def _curand():
    for cand in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if not cand:
            continue
        try:
            return ctypes.CDLL(cand)
        except OSError:
            continue
    return None


def _curand_host_blocks(seed, n_blocks, offset=0):
    cr = _curand()
    if cr is None:
        pytest.skip("cuRAND host library not available")
    gen = ctypes.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    assert cr.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert cr.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        buf = (ctypes.c_uint32 * (4 * n_blocks))()
        assert cr.curandGenerate(gen, buf, ctypes.c_size_t(4 * n_blocks)) == 0
        return np.frombuffer(buf, dtype=np.uint32).reshape(n_blocks, 4).copy()
    finally:
        cr.curandDestroyGenerator(gen)


@pytest.mark.parametrize("seed", [0, 0x123456789ABCDEF, 2**64 - 1])
def test_philox_matches_curand_host_generator(seed):
    """cuRAND's host Philox4x32-10 emits, for seed s, block j = Philox(ctr =
    (j div 65536, 0, j mod 65536, 0), key = (s_lo, s_hi)); offsets of 2^50
    outputs step counter word 1.  This pins counter words 0-2 and the key."""
    key = (seed & 0xFFFFFFFF, seed >> 32)
    blocks = _curand_host_blocks(seed, 70000)
    for j in list(range(0, 300)) + [65535, 65536, 65537, 69999]:
        ctr = (j // 65536, 0, j % 65536, 0)
        assert np.array_equal(oracle.philox(ctr, key), blocks[j]), j
    blocks = _curand_host_blocks(seed, 4, offset=(1 << 50) * 3)
    for j in range(4):
        assert np.array_equal(oracle.philox((0, 3, j, 0), key), blocks[j])


def test_philox_statistics_including_counter_word_3():
    """Uniformity (chi^2 over 256 bins) of every output word, also when only
    counter word 3 varies -- the one word the library pin cannot reach --
    and avalanche: flipping one counter bit flips about half the output bits."""
    key = (0x1234, 0xBEEF)
    outs = np.array([oracle.philox((7, 9, 11, i), key) for i in range(20000)], dtype=np.uint32)
    for w in range(4):
        h = np.bincount(outs[:, w] >> 24, minlength=256)
        assert stats.chisquare(h).pvalue > 1e-4
    base = oracle.philox((1, 2, 3, 4), key)
    flips = []
    for word in range(4):
        for bit in range(0, 32, 3):
            c = [1, 2, 3, 4]
            c[word] ^= 1 << bit
            d = oracle.philox(c, key) ^ base
            flips.append(sum(bin(int(v)).count("1") for v in d))
    assert 56 < np.mean(flips) < 72


# ------------------------------------------------- SUPAv1 worked example ---

def test_supav1_worked_example():
    """SUPAv1 (Table 2, App. A.2.1): splits on slices 0..6 and stops on slice 7
    give exactly 2^7 = 128 points, all of energy E0/128, all in layer L0."""
    g = inputs.supa_v1()
    p = inputs.primaries(5, 3, e_lo=65.0, e_hi=65.0)
    r = oracle.simulate(g, p, seed=11)
    assert np.array_equal(np.diff(r["offsets"]), [128] * 5)
    assert np.all(r["slice"] == 7)
    assert np.all(r["E"] == 65.0 / 128)
    assert np.all(r["z"] == 7.0)
    for s in range(5):
        lin = np.sort(r["lineage"][r["offsets"][s]:r["offsets"][s + 1]])
        assert np.array_equal(lin, np.arange(128, 256, dtype=np.uint64))
    assert np.all(r["layer_sum"][:, 0] == 65.0)
    assert np.all(r["dead"] == 0) and np.all(r["leak"] == 0) and np.all(r["escape"] == 0)
    assert np.all(r["steps"] == 255)  # 1 + 2 + ... + 128 visits


# ------------------------------------------------ closed forms, p_split=0 ---

def test_straight_line_propagation():
    """Without splits a particle keeps its velocity (Sec. 3): at slice k it
    sits at x0 + k dz tan(theta) cos(phi)."""
    g = _tiny_geom(40, np.full(40, 0.06), np.zeros(40))
    p = inputs.primaries(3000, 5, e_lo=1, e_hi=2, theta_max_deg=60.0, entry_halfwidth=3.0)
    r = oracle.simulate(g, p, seed=2)
    cnt = np.diff(r["offsets"])
    assert set(np.unique(cnt)) <= {0, 1}
    idx = np.nonzero(cnt)[0]
    th = p["theta"][idx].astype(np.float64)
    ph = p["phi"][idx].astype(np.float64)
    k = r["slice"].astype(np.float64)
    ex = p["x0"][idx].astype(np.float64) + k * np.tan(th) * np.cos(ph)
    ey = p["y0"][idx].astype(np.float64) + k * np.tan(th) * np.sin(ph)
    np.testing.assert_allclose(r["x"], ex, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(r["y"], ey, rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(r["E"], p["E"][idx].astype(np.float64))


def test_stop_depth_distribution_is_geometric():
    """With p_split = 0 the stop slice follows P(k) = p_stop[k] prod_{j<k}(1 - p_stop[j])
    and the leak probability is prod_k (1 - p_stop[k])."""
    n = 8
    ps = np.array([0.05, 0.1, 0.2, 0.0, 0.3, 0.15, 0.25, 0.1])
    g = _tiny_geom(n, ps, np.zeros(n))
    N = 100_000
    p = inputs.primaries(N, 6, e_lo=1, e_hi=1)
    r = oracle.simulate(g, p, seed=99, n_threads=4)
    surv = np.concatenate([[1.0], np.cumprod(1 - ps)])
    expect = np.append(ps * surv[:-1], surv[-1]) * N
    obs = np.append(np.bincount(r["slice"], minlength=n), np.count_nonzero(r["leak"] > 0))
    keep = expect > 0
    assert obs[~keep].sum() == 0
    assert stats.chisquare(obs[keep], expect[keep]).pvalue > 1e-3


# -------------------------------------------------- brute-force enumeration ---

def _exact_outcome_distribution(p_stop, p_split):
    """Distribution of (hits at each slice..., number leaked) for one primary,
    enumerated from the three rules of Algorithm 1 (stop / split / pass)."""
    n = len(p_stop)

    def conv(a, b):
        out = Counter()
        for ka, pa in a.items():
            for kb, pb in b.items():
                out[tuple(x + y for x, y in zip(ka, kb))] += pa * pb
        return out

    def dist(k):
        if k == n:
            return Counter({tuple([0] * n + [1]): 1.0})
        nxt = dist(k + 1)
        out = Counter()
        e = [0] * (n + 1)
        e[k] = 1
        out[tuple(e)] += p_stop[k]
        for key, pr in conv(nxt, nxt).items():
            out[key] += p_split[k] * pr
        for key, pr in nxt.items():
            out[key] += (1 - p_stop[k] - p_split[k]) * pr
        return out

    return dist(0)


def test_splitting_tree_matches_brute_force_enumeration():
    ps = np.array([0.1, 0.2, 0.3, 0.25])
    pp = np.array([0.6, 0.5, 0.4, 0.5])
    g = _tiny_geom(4, ps, pp, theta_lo=0.05, theta_hi=0.1)
    exact = _exact_outcome_distribution(ps, pp)
    assert abs(sum(exact.values()) - 1) < 1e-12
    N = 200_000
    r = oracle.simulate(g, inputs.primaries(N, 8, e_lo=1, e_hi=1), seed=2024, n_threads=4)
    hits = np.zeros((N, 4), dtype=np.int64)
    sh = np.repeat(np.arange(N), np.diff(r["offsets"]))
    np.add.at(hits, (sh, r["slice"]), 1)
    # compare the joint law of the hit counts per slice (the leak count is a
    # function of the whole history and is pinned by the expected values below)
    marg = Counter()
    for key, pr in exact.items():
        marg[key[:4]] += pr
    keys = Counter(map(tuple, hits))
    items = sorted(marg.items(), key=lambda kv: -kv[1])
    exp_, obs_ = [], []
    rest_e, rest_o = 0.0, 0
    for key, pr in items:
        if pr * N >= 20:
            exp_.append(pr * N)
            obs_.append(keys.get(key, 0))
        else:
            rest_e += pr * N
            rest_o += keys.get(key, 0)
    exp_.append(rest_e)
    obs_.append(N - sum(obs_))
    assert stats.chisquare(obs_, exp_).pvalue > 1e-3


def test_expected_hits_per_slice_closed_form():
    """E[hits at k] = p_stop[k] prod_{j<k} (1 - p_stop[j] + p_split[j]) (each
    particle yields 0, 1 or 2 successors with probabilities stop, pass, split)."""
    n = 10
    ps = np.linspace(0.05, 0.3, n)
    pp = np.linspace(0.5, 0.2, n)
    g = _tiny_geom(n, ps, pp, theta_lo=0.02, theta_hi=0.05)
    N = 40_000
    r = oracle.simulate(g, inputs.primaries(N, 9, e_lo=1, e_hi=1), seed=77, n_threads=4)
    sh = np.repeat(np.arange(N), np.diff(r["offsets"]))
    hits = np.zeros((N, n))
    np.add.at(hits, (sh, r["slice"]), 1)
    grow = np.concatenate([[1.0], np.cumprod(1 - ps + pp)])
    expect = ps * grow[:-1]
    mean = hits.mean(0)
    se = hits.std(0) / math.sqrt(N)
    assert np.all(np.abs(mean - expect) < 5 * se + 1e-12)


def test_longitudinal_energy_profile_independent_of_splits():
    """With e_min = 0, energy is conserved at every split and every particle
    stops with the same slice probability, so the mean deposit at slice k is
    E0 p_stop[k] prod_{j<k}(1 - p_stop[j]) whatever p_split, theta and eps."""
    n = 12
    ps = np.full(n, 0.12)
    pp = np.full(n, 0.45)
    g = _tiny_geom(n, ps, pp)
    N = 20_000
    p = inputs.primaries(N, 10, e_lo=2.0, e_hi=2.0)
    r = oracle.simulate(g, p, seed=5, n_threads=4)
    sh = np.repeat(np.arange(N), np.diff(r["offsets"]))
    dep = np.zeros((N, n))
    np.add.at(dep, (sh, r["slice"]), r["E"])
    surv = np.concatenate([[1.0], np.cumprod(1 - ps)])
    expect = 2.0 * ps * surv[:-1]
    se = dep.std(0) / math.sqrt(N)
    assert np.all(np.abs(dep.mean(0) - expect) < 5 * se)
    se_l = r["leak"].std() / math.sqrt(N)
    assert abs(r["leak"].mean() - 2.0 * surv[-1]) < 5 * se_l


# ------------------------------------------------------- split kinematics ---

def test_split_geometry_and_momentum_balance():
    """One split then a stop: reconstruct each daughter's direction from its
    hit.  The opening angle is theta, the daughters are coplanar with the
    parent on opposite sides, E_0 delta_0 = E_1 delta_1 (momentum balance,
    Sec. 3) and E_0 / E = (theta/2 + eps) / theta (Algorithm 1)."""
    g = _tiny_geom(2, [0.0, 1.0], [1.0, 0.0], theta_lo=math.pi / 32, theta_hi=math.pi / 16)
    N = 4000
    p = inputs.primaries(N, 12, e_lo=3, e_hi=3, theta_max_deg=40.0, entry_halfwidth=1.0)
    r = oracle.simulate(g, p, seed=31)
    assert np.array_equal(np.diff(r["offsets"]), [2] * N)
    th = p["theta"].astype(np.float64)
    ph = p["phi"].astype(np.float64)
    u = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    a = slice(0, None, 2)  # lineage 2 (daughter 0) sorts before 3
    b = slice(1, None, 2)
    assert np.all(r["lineage"][a] == 2) and np.all(r["lineage"][b] == 3)

    def direction(sel):
        d = np.stack([r["x"][sel] - p["x0"], r["y"][sel] - p["y0"], np.ones(N)], 1)
        return d / np.linalg.norm(d, axis=1, keepdims=True)

    da, db = direction(a), direction(b)
    ang = lambda v, w: np.arccos(np.clip(np.sum(v * w, 1), -1, 1))
    d0, d1 = ang(u, da), ang(u, db)
    theta = ang(da, db)
    np.testing.assert_allclose(d0 + d1, theta, rtol=1e-9, atol=1e-12)
    assert np.all(theta >= math.pi / 32 - 1e-9) and np.all(theta <= math.pi / 16 + 1e-9)
    eps = (d1 - d0) / 2
    assert np.all(np.abs(eps) <= theta / 4 + 1e-9)
    Ea, Eb = r["E"][a], r["E"][b]
    np.testing.assert_allclose(Ea + Eb, 3.0, rtol=1e-15)
    np.testing.assert_allclose(Ea * d0, Eb * d1, rtol=1e-9)
    np.testing.assert_allclose(Ea / 3.0, (theta / 2 + eps) / theta, rtol=1e-9)
    det = np.einsum("ij,ij->i", u, np.cross(da, db))
    assert np.max(np.abs(det)) < 1e-9
    # the distributions of theta, eps/theta and the azimuth are uniform
    assert stats.kstest((theta - math.pi / 32) / (math.pi / 32), "uniform").pvalue > 1e-3
    assert stats.kstest(eps / theta * 2 + 0.5, "uniform").pvalue > 1e-3
    # azimuth of daughter 0 about the parent, measured from a fixed
    # perpendicular reference: uniform on [0, 2 pi)
    ref = np.cross(u, np.array([0.0, 1.0, 0.0]))
    ref /= np.linalg.norm(ref, axis=1, keepdims=True)
    ref2 = np.cross(u, ref)
    perp = da - np.sum(da * u, 1, keepdims=True) * u
    az = np.mod(np.arctan2(np.sum(perp * ref2, 1), np.sum(perp * ref, 1)), 2 * math.pi)
    assert stats.kstest(az / (2 * math.pi), "uniform").pvalue > 1e-3


def test_literal_split_reading_deflects_both_by_half_theta_plus_eps():
    g = _tiny_geom(2, [0.0, 1.0], [1.0, 0.0], split_mode=inputs.SPLIT_LITERAL)
    N = 500
    p = inputs.primaries(N, 13, e_lo=1, e_hi=1)
    r = oracle.simulate(g, p, seed=3)
    da = np.stack([r["x"][0::2], r["y"][0::2], np.ones(N)], 1)
    db = np.stack([r["x"][1::2], r["y"][1::2], np.ones(N)], 1)
    d0 = np.arctan(np.linalg.norm(da[:, :2], axis=1))
    d1 = np.arctan(np.linalg.norm(db[:, :2], axis=1))
    np.testing.assert_allclose(d0, d1, rtol=1e-9)


def test_symmetric_split_halves_energy_exactly():
    """eps = 0: all splits symmetric, energy halved exactly (App. A.2.1)."""
    g = _tiny_geom(6, [0, 0, 0, 0, 0, 1.0], [1.0] * 5 + [0.0], eps_mode=inputs.EPS_ZERO,
                   theta_mode=inputs.THETA_FIXED, theta_lo=math.pi / 24, theta_hi=math.pi / 24)
    r = oracle.simulate(g, inputs.primaries(10, 1, e_lo=5, e_hi=5), seed=1)
    assert np.all(r["E"] == 5.0 / 32)


# ---------------------------------------------------- bookkeeping and cuts ---

@pytest.mark.parametrize("theta_max", [0.0, 45.0, 88.0])
def test_energy_bookkeeping(theta_max):
    """Hits + dead + leak + escape = E0 (energy conserved at every split)."""
    g = inputs.supa_d(10, n_dead_front=2)
    p = inputs.primaries(400, 14, e_lo=1, e_hi=30, theta_max_deg=theta_max)
    r = oracle.simulate(g, p, seed=4, n_threads=2)
    tot = r["layer_sum"].sum(1) + r["dead"] + r["leak"] + r["escape"]
    np.testing.assert_allclose(tot, p["E"].astype(np.float64), rtol=1e-12)
    sh = np.repeat(np.arange(len(p)), np.diff(r["offsets"]))
    per = np.bincount(sh, weights=r["E"], minlength=len(p))
    np.testing.assert_allclose(per, r["layer_sum"].sum(1), rtol=1e-12)
    assert np.all(np.isin(r["slice"], np.arange(2, g.n_slices)))
    if theta_max == 88.0:
        assert r["escape"].sum() > 0


def test_energy_cut_bounds_depth_and_stops_low_energy():
    g = inputs.supa_d(30, e_min=0.05)
    p = inputs.primaries(300, 15, e_lo=50, e_hi=100)
    r = oracle.simulate(g, p, seed=8, n_threads=2)
    # every split keeps at most 3/4 of the parent's energy (eps in [-theta/4, theta/4])
    bound = np.ceil(np.log(p["E"].astype(np.float64) / 0.05) / np.log(4 / 3)) + 1
    assert np.all(r["max_depth"] <= bound)
    assert np.all(r["E"][r["E"] < 0.05] > 0)


def test_escape_and_leak_rules():
    g = _tiny_geom(5, np.zeros(5), np.zeros(5))
    p = inputs.primaries(4, 1, e_lo=2, e_hi=2)
    r = oracle.simulate(g, p, seed=1)
    assert np.all(r["leak"] == 2.0) and np.all(r["steps"] == 5) and r["offsets"][-1] == 0
    p["theta"] = np.float32(math.acos(5e-4))
    r = oracle.simulate(g, p, seed=1)
    assert np.all(r["escape"] == 2.0) and np.all(r["steps"] == 1)


def test_results_independent_of_partition_and_threads():
    g, p = inputs.workload_plain10(200)
    a = oracle.simulate(g, p, seed=0, n_threads=1)
    b = oracle.simulate(g, p, seed=0, n_threads=4)
    lo = oracle.simulate(g, p[:77], seed=0, shower_id_base=0)
    hi = oracle.simulate(g, p[77:], seed=0, shower_id_base=77)
    for key in ("x", "y", "z", "E", "lineage"):
        assert np.array_equal(a[key], b[key])
        assert np.array_equal(a[key], np.concatenate([lo[key], hi[key]]))
    assert np.array_equal(a["layer_sum"], np.concatenate([lo["layer_sum"], hi["layer_sum"]]))


# ----------------------------------------------------------- downsampling ---

def _random_hits(n_showers, seed, geom, per=50):
    rng = np.random.Generator(np.random.PCG64(seed))
    counts = rng.integers(0, per, n_showers)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    nh = int(off[-1])
    hx = rng.normal(0, 3.0, nh).astype(np.float32)
    hy = rng.normal(0, 3.0, nh).astype(np.float32)
    hz = (rng.integers(0, geom.n_slices, nh) * geom.dz).astype(np.float32)
    hE = rng.exponential(1.0, nh).astype(np.float32)
    return hx, hy, hz, hE, off


def test_voxelize_matches_histogram2d_and_conserves():
    """Each cell holds the energy of the points inside it (App. A.5),
    checked against numpy's histogram2d; grid + out-of-ROI = all hits."""
    g = inputs.supa_d(4, grid=16)
    prims = inputs.primaries(30, 2, e_lo=1, e_hi=1)
    hx, hy, hz, hE, off = _random_hits(30, 1, g)
    rx, ry = oracle.roi_origins(g, prims)
    grid, oor = oracle.voxelize(hx, hy, hz, hE, off, g, rx, ry)
    for s in range(30):
        sl = slice(off[s], off[s + 1])
        layer = g.slice_to_layer[np.rint(hz[sl] / g.dz).astype(int)]
        for l in range(4):
            m = layer == l
            edges_x = rx[s, l] + g.wx * np.arange(g.nx + 1)
            edges_y = ry[s, l] + g.wy * np.arange(g.ny + 1)
            h, _, _ = np.histogram2d(hy[sl][m].astype(np.float64), hx[sl][m].astype(np.float64),
                                     bins=[edges_y, edges_x], weights=hE[sl][m].astype(np.float64))
            np.testing.assert_allclose(grid[s, l], h, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(grid[s].sum() + oor[s], hE[sl].astype(np.float64).sum(), rtol=1e-12)


def test_voxelize_single_hit_floor_cell():
    g = inputs.supa_d(2, grid=8)  # wx = 2, ROI [-8, 8)
    prims = inputs.primaries(1, 0, e_lo=1, e_hi=1)
    rx, ry = oracle.roi_origins(g, prims)
    assert rx[0, 0] == -8.0 and ry[0, 1] == -8.0
    cases = [(-8.0, -8.0, 0, 0), (-6.0, 7.9, 1, 7), (7.99, 0.0, 7, 4), (8.0, 0.0, None, None),
             (-8.001, 0.0, None, None), (0.0, -0.001, 4, 3)]
    for x, y, ix, iy in cases:
        grid, oor = oracle.voxelize([x], [y], [4.0], [1.5], [0, 1], g, rx, ry)
        if ix is None:
            assert oor[0] == 1.5 and grid.sum() == 0
        else:
            assert grid[0, 1, iy, ix] == 1.5 and oor[0] == 0


def test_roi_axis_centred_follows_incidence_direction():
    g = inputs.supa_d(3, grid=16, roi_mode=inputs.ROI_AXIS)
    p = inputs.primaries(5, 3, e_lo=1, e_hi=1, theta_max_deg=30)
    rx, ry = oracle.roi_origins(g, p)
    for l in range(3):
        zmid = (3 * l + 3 * l + 2) / 2
        cx = zmid * np.tan(p["theta"].astype(np.float64)) * np.cos(p["phi"].astype(np.float64))
        np.testing.assert_allclose(rx[:, l] + 8.0, cx, rtol=1e-5, atol=1e-5)
