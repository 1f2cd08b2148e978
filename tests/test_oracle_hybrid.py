"""Pins of the FP64 hybrid-path oracle (no counterpart in the paper; the
rules are the library's): the gamma variates follow the gamma law
(scipy.stats), a network with zero spread deposits exactly its means, SAMPLE
splits the MEAN total by a Dirichlet draw whose means are the MEAN shares
and whose spread matches the predicted variances, sums above E are
scaled to E, hits
lie on the particle's straight line when the predicted mean distance is zero
and at distances that follow the measured lateral law scaled to it
otherwise, the law is the plain sub-showers' (remeasured), the hybrid stepping reduces to the plain one when nothing is set
aside, energy is conserved, and the lateral training targets (mean
distances) of a single symmetric split are their closed form."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from oracle import hybrid, mlp
from paper_2202_05012_gb300 import inputs


@pytest.mark.parametrize("alpha", [0.05, 0.3, 1.0, 2.5, 40.0])
def test_gamma_variates_follow_the_gamma_law(alpha):
    """Marsaglia-Tsang with the alpha < 1 boost against scipy's gamma law,
    over independent counters (showers) and two layers' streams."""
    g = np.array([hybrid.gamma_variate(alpha, s, 5, 2 * s + 1, s % 2, 4242) for s in range(4000)])
    assert np.all(g >= 0)
    assert stats.kstest(g, "gamma", args=(alpha,)).pvalue > 1e-3
    assert abs(g.mean() - alpha) < 4 * math.sqrt(alpha / len(g))
    assert abs(g.var() / alpha - 1) < 0.25


def test_gamma_streams_differ_by_layer_and_attempt():
    a = [hybrid.gamma_variate(2.0, 7, 3, 9, j, 1) for j in range(30)]
    assert len(set(a)) == 30
    # a layer's draw depends on the shower, slice and lineage of its particle
    assert hybrid.gamma_variate(2.0, 8, 3, 9, 0, 1) != a[0]
    assert hybrid.gamma_variate(2.0, 7, 4, 9, 0, 1) != a[0]
    assert hybrid.gamma_variate(2.0, 7, 3, 10, 0, 1) != a[0]


def _law_cdf(q):
    """CDF of the lateral law (linear quantile function between the table
    points, equal u steps of 1 / 64)."""
    Q = hybrid.LATERAL_Q
    i = np.clip(np.searchsorted(Q, q, side="right") - 1, 0, 63)
    span = Q[i + 1] - Q[i]
    f = np.where(span > 0, (q - Q[i]) / np.where(span > 0, span, 1.0), 1.0)
    return np.clip((i + np.clip(f, 0.0, 1.0)) / 64.0, 0.0, 1.0)


def test_lateral_law_has_mean_one():
    Q = hybrid.LATERAL_Q
    assert len(Q) == 65 and Q[0] == 0.0 and np.all(np.diff(Q) >= 0)
    # mean of a quantile function linear on each of 64 equal steps
    assert abs(((Q[:-1] + Q[1:]) / 2).mean() - 1.0) < 1e-5
    # spike at 0 (the first deposits on the axis), wider than a 2-D Gaussian
    m2 = ((Q[:-1] ** 2 + Q[:-1] * Q[1:] + Q[1:] ** 2) / 3).mean()
    assert 4 / math.pi + 0.05 < m2 < 1.5, m2
    assert hybrid.lateral_quantile(0.0) == 0.0 and hybrid.lateral_quantile(1.0 / 64) == 0.0
    assert abs(hybrid.lateral_quantile(0.5 + 1 / 128) - (Q[32] + Q[33]) / 2) < 1e-12


def test_lateral_offsets_follow_the_law():
    m = np.array([hybrid.lateral_offset(s, 2 + s % 5, 3 * s + 1, 777) for s in range(6000)])
    q = np.hypot(m[:, 0], m[:, 1])
    # u uniform on [0, 1): the law's quantiles, its atom at 0 and its mean
    assert abs(np.mean(q == 0.0) - 2 / 64) < 4 * math.sqrt(2 / 64 / len(q))
    pos = q[q > 0]
    assert stats.kstest((_law_cdf(pos) - 2 / 64) / (62 / 64), "uniform").pvalue > 1e-3
    assert abs(q.mean() - 1.0) < 4 * q.std() / math.sqrt(len(q))
    # isotropic direction, independent of the distance
    phi = np.arctan2(m[q > 0, 1], m[q > 0, 0])
    assert stats.kstest((phi + math.pi) / (2 * math.pi), "uniform").pvalue > 1e-3
    assert abs(np.corrcoef(phi, pos)[0, 1]) < 0.05
    # a different stream (tag 2) from the decision block (tag 0) of the same particle
    w0 = oracle.philox((0, 2, 1, 0), (777, 0))
    w2 = oracle.philox((0, 2 | (2 << 16), 1, 0), (777, 0))
    assert not np.array_equal(w0, w2)


def test_plain_path_when_nothing_is_set_aside():
    g = inputs.supa_d(10)
    p = inputs.primaries(200, 3, e_lo=1, e_hi=20)
    a = oracle.simulate(g, p, 5)
    b = oracle.simulate(g, p, 5, e_s=0.01)  # below the energy cut: never diverts
    assert len(b["div"]["E"]) == 0
    for k in ("x", "E", "lineage", "steps"):
        assert np.array_equal(a[k], b[k])


def test_energy_conservation_with_diversion():
    g = inputs.supa_d(30)
    p = inputs.primaries(100, 4, e_lo=5, e_hi=60, theta_max_deg=30)
    r = oracle.simulate(g, p, 6, e_s=1.0)
    div = r["div"]
    assert len(div["E"]) > 0 and np.all(div["E"] < 1.0)
    assert np.all(np.asarray(g.slice_to_layer)[div["k"]] == div["layer"])
    tot = r["layer_sum"].sum(1) + r["dead"] + r["leak"] + r["escape"]
    tot += np.bincount(div["shower"], weights=div["E"], minlength=len(p))
    np.testing.assert_allclose(tot, p["E"].astype(np.float64), rtol=1e-12)


def _raw_mu(mu):
    """Network outputs o_j that give the means mu_j = exp(o_j - 4) (a very
    negative output for mu <= 0: a mean far below every cut)."""
    mu = np.asarray(mu, dtype=float)
    return np.where(mu > 0, np.log(np.where(mu > 0, mu, 1.0)) + mlp.MU_SHIFT, -100.0)


def _const_net(mu, s, rho=0.0):
    params = inputs.mlp_init(2)
    W4 = np.zeros((90, 256))
    b4 = np.concatenate([np.full(30, _raw_mu(mu)), np.full(30, s), np.full(30, rho)])
    return params[:3] + [(W4, b4)]


def test_zero_spread_deposits_the_means_and_scales_to_E():
    g = inputs.supa_d(30)
    p = inputs.primaries(40, 5, e_lo=5, e_hi=20)
    r = oracle.simulate(g, p, 7, e_s=1.0)
    div = r["div"]
    dep = hybrid.deposits(div, _const_net(0.02, -80.0), g, 1.0, 7)
    L = g.n_layers
    for i in range(len(div["E"])):
        m = min(30, L - div["layer"][i])
        np.testing.assert_allclose(dep["d"][i, :m], 0.02 * div["E"][i], rtol=1e-12)
        assert np.all(dep["d"][i, m:] == 0)
    dep = hybrid.deposits(div, _const_net(0.5, -80.0), g, 1.0, 7)  # 30 x 0.5 > 1: scaled
    inside = np.minimum(30, L - div["layer"])
    full = inside * 0.5 > 1
    np.testing.assert_allclose(dep["d"][full].sum(1), div["E"][full], rtol=1e-12)
    # hits sit on the particle's straight line at the layers' mid depths
    h = dep["hits"]
    assert np.all(np.isin(h[:, 3], 1.0 + 3.0 * np.arange(L)))
    x, y = _straight_line(div, h, g)
    np.testing.assert_allclose(h[:, 1], x, atol=1e-12)
    np.testing.assert_allclose(h[:, 2], y, atol=1e-12)


def _straight_line(div, h, g):
    """Position of each hit's particle continued straight to the hit's depth."""
    idx = {}
    for i in range(len(div["E"])):
        idx.setdefault(int(div["shower"][i]), []).append(i)
    xs, ys = [], []
    pos = {}
    for row in h:
        s, lay = int(row[0]), int(row[5])
        # hits of one particle follow each other in layer order
        key = (s, pos.get(s, 0))
        i = idx[s][key[1]]
        dz = row[3] - div["k"][i] * g.dz
        xs.append(div["x"][i] + dz * div["ux"][i] / div["uz"][i])
        ys.append(div["y"][i] + dz * div["uy"][i] / div["uz"][i])
        last = lay == min(g.n_layers, div["layer"][i] + 30) - 1
        if last:
            pos[s] = key[1] + 1
    return np.array(xs), np.array(ys)


def test_hits_spread_by_the_lateral_law_about_the_mean_distance():
    g = inputs.supa_d(30)
    p = inputs.primaries(60, 9, e_lo=5, e_hi=20)
    r = oracle.simulate(g, p, 3, e_s=1.0)
    div = r["div"]
    R = 0.7
    dep = hybrid.deposits(div, _const_net(0.02, -80.0, R), g, 1.0, 3)
    h = dep["hits"]
    x, y = _straight_line(div, h, g)
    dist = np.hypot(h[:, 1] - x, h[:, 2] - y)
    # the distance over the predicted mean distance R follows the lateral law
    # (mean 1); one draw per particle, so test the first layer of each particle
    first = np.concatenate([[True], (h[1:, 0] != h[:-1, 0]) | (h[1:, 5] <= h[:-1, 5])])
    q = dist[first] / R
    assert len(q) > 300
    assert abs(q.mean() - 1.0) < 4 * q.std() / math.sqrt(len(q))
    pos = q[q > 1e-9]
    assert stats.kstest((_law_cdf(pos) - 2 / 64) / (62 / 64), "uniform").pvalue > 1e-3
    # all layers of a particle share the direction and size of the displacement
    d1 = dist[first]
    assert np.allclose(dist[~first], np.repeat(d1, np.diff(np.append(np.nonzero(first)[0], len(first))))[~first],
                       rtol=1e-9, atol=1e-12)


def test_training_targets_of_a_single_symmetric_split():
    # one split on slice 0 with fixed theta and eps = 0: two halves of E
    # deflected by theta/2 in opposite azimuths; every particle stops on
    # slice 7 (layer 2), at distance 7 dz tan(theta/2) from the axis
    g = inputs.supa_d(4, e_min=0.0)
    g.p_split[:] = 0.0
    g.p_stop[:] = 0.0
    g.p_split[0] = 1.0
    g.p_stop[7] = 1.0
    g.theta_mode, g.theta_lo, g.theta_hi = inputs.THETA_FIXED, math.pi / 24, math.pi / 24
    g.eps_mode = inputs.EPS_ZERO
    p = inputs.primaries(5, 2, e_lo=0.5, e_hi=0.9)
    p["theta"] = 0.0
    r = oracle.simulate(g, p, 1)
    Y = hybrid.training_targets(g, p, r)
    assert np.all(r["offsets"][1:] - r["offsets"][:-1] == 2)
    np.testing.assert_allclose(Y[:, 2], 1.0, rtol=1e-12)
    np.testing.assert_allclose(Y[:, [0, 1, 3]], 0.0, atol=0)
    np.testing.assert_allclose(Y[:, 32], 7.0 * math.tan(math.pi / 48), rtol=1e-9)
    np.testing.assert_allclose(Y[:, [30, 31, 33]], 0.0, atol=0)


def _layer_net(mu, s, rho=0.0):
    """A network whose outputs are the given per-layer mu_j, s_j (and rho)
    whatever its inputs."""
    params = inputs.mlp_init(2)
    W4 = np.zeros((90, 256))
    b4 = np.concatenate([_raw_mu(mu), np.asarray(s, float), np.full(30, rho)])
    return params[:3] + [(W4, b4)]


def _diverted_on_layer0(n, E=0.5):
    """n diverted particles at the front of a 30-layer detector (all 30
    predicted layers inside), distinct showers and lineages."""
    return dict(shower=np.arange(n), k=np.zeros(n, int), lineage=2 * np.arange(n) + 3, layer=np.zeros(n, int),
                E=np.full(n, E), x=np.zeros(n), y=np.zeros(n), ux=np.zeros(n), uy=np.zeros(n), uz=np.ones(n))


def test_sample_concentration_matches_the_predicted_variance():
    # equal layers: T = 30 mu, m = 1/30, V = 30 v with v = sd^2 + the
    # network's variance floor -> c + 1 = T^2 (1 - 1/30) / V
    mu, sd = 0.02, 0.01
    v = sd * sd + mlp.VAR_FLOOR
    f = np.full(30, mu)
    c = hybrid.sample_concentration(f, np.full(30, math.log(sd * sd)))
    T = 30 * mu
    assert c == pytest.approx(T * T * (1 - 1 / 30) / (30 * v) - 1, rel=1e-12)
    # a Dirichlet share then has variance T^2 m (1 - m) / (c + 1) = v
    assert T * T * (1 / 30) * (1 - 1 / 30) / (c + 1) == pytest.approx(v, rel=1e-12)
    # a negligible spread takes the means (no draw); a huge one the lowest c
    assert math.isinf(hybrid.sample_concentration(f, np.full(30, -200.0)))
    v_edge = T * T * (1 - 1 / 30) / (30 * (hybrid.SAMPLE_C_MAX + 1))  # c = C_MAX exactly
    s_just_below = math.log(1.01 * v_edge - mlp.VAR_FLOOR)  # c slightly below C_MAX
    assert hybrid.sample_concentration(f, np.full(30, s_just_below)) == pytest.approx(
        (hybrid.SAMPLE_C_MAX + 1) / 1.01 - 1, rel=1e-9)
    s_just_above = math.log(0.99 * v_edge - mlp.VAR_FLOOR)
    assert math.isinf(hybrid.sample_concentration(f, np.full(30, s_just_above)))
    assert hybrid.sample_concentration(f, np.full(30, 5.0)) == hybrid.SAMPLE_C_MIN
    assert math.isinf(hybrid.sample_concentration(np.zeros(30), np.zeros(30)))
    # layers without a mean deposit do not count towards V
    f2 = f.copy()
    f2[10:] = 0.0
    s2 = np.full(30, math.log(sd * sd))
    s2[10:] = 3.0
    T2 = 10 * mu
    assert hybrid.sample_concentration(f2, s2) == pytest.approx(T2 * T2 * 0.9 / (10 * v) - 1, rel=1e-12)


def test_sample_mode_is_an_unbiased_dirichlet_split():
    g = inputs.supa_d(30)
    n = 3000
    div = _diverted_on_layer0(n)
    # uneven means (a peak and a long tail, two layers empty) and spreads
    j = np.arange(30)
    mu = 0.08 * np.exp(-0.5 * ((j - 6) / 3.0) ** 2) + 0.002  # total 0.65: no scaling to E
    mu[[20, 25]] = -0.01
    sd = 0.4 * np.abs(mu)
    net = _layer_net(mu, np.log(sd * sd))
    dep = hybrid.deposits(div, net, g, 1.0, 4, mode=0)
    mean = hybrid.deposits(div, net, g, 1.0, 4, mode=1)
    E = div["E"][:, None]
    fr = dep["d"] / E
    # every particle keeps the MEAN total; layers without a mean get nothing
    np.testing.assert_allclose(dep["d"].sum(1), mean["d"].sum(1), rtol=1e-12)
    assert np.all(dep["d"][:, [20, 25]] == 0)
    f = np.maximum(0.0, mu)
    T = f.sum()
    m = f / T
    c = hybrid.sample_concentration(f, np.log(sd * sd))
    # each layer's mean fraction is its MEAN fraction (Dirichlet means), its
    # variance T^2 m (1 - m) / (c + 1)
    var = T * T * m * (1 - m) / (c + 1)
    se = np.sqrt(var / n)
    ok = f > 0
    assert np.all(np.abs(fr.mean(0)[ok] - f[ok]) < 4.5 * se[ok])
    np.testing.assert_allclose(fr.var(0)[ok], var[ok], rtol=0.2)
    # and the spread summed over the layers is the predicted one
    assert abs((fr.var(0)[ok]).sum() / (sd[ok] ** 2 + mlp.VAR_FLOOR).sum() - 1) < 0.1
    # replayable: the same counters give the same draws
    again = hybrid.deposits({k: v[:50] for k, v in div.items()}, net, g, 1.0, 4, mode=0)
    np.testing.assert_array_equal(again["d"], dep["d"][:50])


def test_sample_mode_is_truncated_at_the_back():
    g = inputs.supa_d(30)
    div = _diverted_on_layer0(200)
    div["layer"][:] = 25  # five layers inside
    div["k"][:] = 75
    net = _layer_net(np.full(30, 0.05), np.full(30, math.log(1e-4)))
    dep = hybrid.deposits(div, net, g, 1.0, 4, mode=0)
    assert np.all(dep["d"][:, 5:] == 0)
    np.testing.assert_allclose(dep["d"].sum(1), 0.25 * div["E"], rtol=1e-12)


def test_features_follow_their_definition():
    g = inputs.supa_d(30)
    div = dict(E=np.array([0.5, 0.05]), ux=np.array([0.1, 0.0]), uy=np.array([0.2, 0.0]),
               uz=np.array([math.sqrt(0.95), 1.0]), k=np.array([4, 89]), layer=np.array([1, 29]))
    f = hybrid.features(div, g, 1.0)
    np.testing.assert_allclose(f[0], [math.log(0.5), 0.1, 0.2, math.sqrt(0.95), 1 / 3, 29 / 30])
    np.testing.assert_allclose(f[1], [math.log(0.05), 0, 0, 1, 2 / 3, 1 / 30])


def test_log_link_means_and_the_millionth_cut():
    """mu_j = exp(o_j - 4); a layer whose mean fraction is below 10^-6 gets
    no deposit and no hit in either mode, one just above it does."""
    out = np.zeros((1, 90))
    out[0, :3] = [4.0, 4.0 + math.log(0.5), 0.0]
    np.testing.assert_allclose(mlp.deposit_means(out)[0, :3], [1.0, 0.5, math.exp(-4.0)], rtol=1e-15)
    g = inputs.supa_d(30)
    div = _diverted_on_layer0(40)
    mu = np.full(30, 0.02)
    mu[3], mu[4] = 0.99e-6, 1.01e-6
    for mode in (0, 1):
        dep = hybrid.deposits(div, _layer_net(mu, np.full(30, math.log(1e-10))), g, 1.0, 4, mode=mode)
        assert np.all(dep["d"][:, 3] == 0) and np.all(dep["d"][:, 4] > 0)
        assert not np.any(dep["hits"][:, 5] == 3)
        assert np.sum(dep["hits"][:, 5] == 4) == len(div["E"])


def test_lateral_law_is_the_plain_sub_showers():
    """LATERAL_Q restates a measurement (tests/golden/lateral_law.py, 80,000
    sub-showers, seed 5): remeasured on 40,000 other sub-showers, the
    quantiles agree to the measurement's statistical spread."""
    import sys
    import os
    sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
    import lateral_law
    Q = lateral_law.measure(40_000, seed=6, n_threads=8)
    d = np.abs(Q - hybrid.LATERAL_Q)
    assert d[:63].max() < 0.02, d[:63].max()
    assert d[63] < 0.02 and d[64] < 0.6, (d[63], d[64])
