"""Pins of the FP64 hybrid-path oracle (no counterpart in the paper; the
rules are the library's): the normals are standard normal, a network with
zero spread deposits exactly its means, SAMPLE draws are log-normal with the
predicted mean and variance, rescaled to the MEAN total, sums above E are
scaled to E, hits
lie on the particle's straight line when the predicted distance is zero and
at that mean distance otherwise, the hybrid stepping reduces to the plain
one when nothing is set aside, energy is conserved, and the lateral
training targets of a single symmetric split are its closed form."""
import math

import numpy as np
from scipy import stats

import oracle
from oracle import hybrid
from paper_2202_05012_gb300 import inputs


def test_box_muller_normals_are_standard():
    z = np.concatenate([hybrid.normals(s, 3 + s % 7, 2 * s + 1, 12345) for s in range(700)])
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(z.mean()) < 0.03 and abs(z.std() - 1) < 0.03


def test_offset_normals_are_standard_pairs():
    m = np.array([hybrid.offset_normals(s, 2 + s % 5, 3 * s + 1, 777) for s in range(6000)])
    assert stats.kstest(m.ravel(), "norm").pvalue > 1e-3
    assert abs(np.corrcoef(m[:, 0], m[:, 1])[0, 1]) < 0.05
    # a different stream from the deposit normals
    assert not np.isclose(m[0, 0], hybrid.normals(0, 2, 1, 777)[0])


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


def _const_net(mu, s, rho=0.0):
    params = inputs.mlp_init(2)
    W4 = np.zeros((90, 256))
    b4 = np.concatenate([np.full(30, mu), np.full(30, s), np.full(30, rho)])
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


def test_hits_spread_at_the_predicted_mean_distance():
    g = inputs.supa_d(30)
    p = inputs.primaries(60, 9, e_lo=5, e_hi=20)
    r = oracle.simulate(g, p, 3, e_s=1.0)
    div = r["div"]
    R = 0.7
    dep = hybrid.deposits(div, _const_net(0.02, -80.0, R), g, 1.0, 3)
    h = dep["hits"]
    x, y = _straight_line(div, h, g)
    dist = np.hypot(h[:, 1] - x, h[:, 2] - y)
    # per layer an isotropic 2-D Gaussian with sigma = R sqrt(2/pi): the
    # distances are Rayleigh with mean R; one pair per particle, so test the
    # first layer of each particle (independent draws)
    first = np.concatenate([[True], (h[1:, 0] != h[:-1, 0]) | (h[1:, 5] <= h[:-1, 5])])
    d1 = dist[first]
    assert len(d1) > 300
    sig = R * math.sqrt(2 / math.pi)
    assert abs(d1.mean() - R) < 4 * sig * math.sqrt(2 - math.pi / 2) / math.sqrt(len(d1))
    assert stats.kstest(d1, "rayleigh", args=(0, sig)).pvalue > 1e-3
    # all layers of a particle share the direction of the displacement
    assert np.allclose(dist[~first], R * math.sqrt(2 / math.pi) * np.repeat(
        d1 / sig, np.diff(np.append(np.nonzero(first)[0], len(first))))[~first], rtol=1e-9)


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


def test_sample_mode_is_the_moment_matched_log_normal():
    g = inputs.supa_d(30)
    p = inputs.primaries(150, 12, e_lo=5, e_hi=20)
    r = oracle.simulate(g, p, 4, e_s=1.0)
    div = r["div"]
    mu, sd = 0.02, 0.01
    net = _const_net(mu, math.log(sd * sd))
    dep = hybrid.deposits(div, net, g, 1.0, 4, mode=0)
    mean = hybrid.deposits(div, net, g, 1.0, 4, mode=1)
    # the total of every particle is the MEAN total; the shape fluctuates
    np.testing.assert_allclose(dep["d"].sum(1), mean["d"].sum(1), rtol=1e-12)
    assert np.std(dep["d"][:, 0] / div["E"]) > 0.5 * sd
    # before that rescaling the draws are log-normal with mean mu and
    # variance sd^2 (a^2 = ln 1.25, below the cap): undo it per particle
    inside = div["layer"][:, None] + np.arange(30) < g.n_layers  # [n, 30]
    n_in = inside.sum(1)
    raw = []
    for i in range(len(div["E"])):
        norm = hybrid.normals(int(div["shower"][i]), int(div["k"][i]), int(div["lineage"][i]), 4)[:n_in[i]]
        raw.append(norm)
    z = np.concatenate(raw)
    assert z.size > 20000
    a2 = math.log1p(sd * sd / (mu * mu))
    g_draw = mu * np.exp(math.sqrt(a2) * z - 0.5 * a2)
    assert abs(g_draw.mean() - mu) < 4 * sd / math.sqrt(g_draw.size)
    assert abs(g_draw.var() / sd ** 2 - 1) < 0.05
    ratio = np.concatenate([dep["d"][i, :n_in[i]] / div["E"][i] / (mu * np.exp(math.sqrt(a2) * raw[i] - 0.5 * a2))
                            for i in range(len(raw))])
    # one factor per particle: sum of means / sum of draws
    for i in range(0, len(raw), 37):
        r = dep["d"][i, :n_in[i]] / div["E"][i] / (mu * np.exp(math.sqrt(a2) * raw[i] - 0.5 * a2))
        np.testing.assert_allclose(r, r[0], rtol=1e-12)
    assert ratio.size == z.size


def test_features_follow_their_definition():
    g = inputs.supa_d(30)
    div = dict(E=np.array([0.5, 0.05]), ux=np.array([0.1, 0.0]), uy=np.array([0.2, 0.0]),
               uz=np.array([math.sqrt(0.95), 1.0]), k=np.array([4, 89]), layer=np.array([1, 29]))
    f = hybrid.features(div, g, 1.0)
    np.testing.assert_allclose(f[0], [math.log(0.5), 0.1, 0.2, math.sqrt(0.95), 1 / 3, 29 / 30])
    np.testing.assert_allclose(f[1], [math.log(0.05), 0, 0, 1, 2 / 3, 1 / 30])
