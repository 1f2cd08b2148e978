"""Pins of the FP64 hybrid-path oracle (no counterpart in the paper; the
rules are the library's): the normals are standard normal, a network with
zero spread deposits exactly its means, sums above E are scaled to E, the
hybrid stepping reduces to the plain one when nothing is set aside, and
energy is conserved."""
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


def _const_net(mu, s):
    params = inputs.mlp_init(2)
    W4 = np.zeros((60, 256))
    b4 = np.concatenate([np.full(30, mu), np.full(30, s)])
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


def test_features_follow_their_definition():
    g = inputs.supa_d(30)
    div = dict(E=np.array([0.5, 0.05]), ux=np.array([0.1, 0.0]), uy=np.array([0.2, 0.0]),
               uz=np.array([math.sqrt(0.95), 1.0]), k=np.array([4, 89]), layer=np.array([1, 29]))
    f = hybrid.features(div, g, 1.0)
    np.testing.assert_allclose(f[0], [math.log(0.5), 0.1, 0.2, math.sqrt(0.95), 1 / 3, 29 / 30])
    np.testing.assert_allclose(f[1], [math.log(0.05), 0, 0, 1, 2 / 3, 1 / 30])
