"""FP64 oracle of the surrogate side of the hybrid path -- TEST INFRASTRUCTURE.

The SUPA paper has no surrogate; this follows the library's stated rule for
it.  For every particle set aside below E_s (oracle.simulate(..., e_s=...)
returns them):
  1. features: log(E / E_s), direction cosines, position of the slice in its
     layer (k - first slice) / slices in the layer, layers left from the
     particle's layer to the back over 30 (capped at 1);
  2. the FP64 network (oracle.mlp) gives o_j, s_j and rho_j, j = 0..29;
     the mean deposit fraction of layer start + j is mu_j = exp(o_j - 4)
     (oracle.mlp.deposit_means);
  3. SAMPLE draws: gamma variates by Marsaglia and Tsang's method ("A
     simple method for generating gamma variables", ACM TOMS 26(3), 2000)
     for shape a = alpha (alpha >= 1) or a = alpha + 1 (alpha < 1, then
     multiplied by U^(1/alpha)): d = a - 1/3, c = 1 / sqrt(9 d); attempt t
     (t = 0..3) of layer j takes the Philox4x32-10 block with counter
     (shower id, slice | 3 << 16 | (4 j + t) << 20, lineage lo, lineage
     hi), key = seed, words (w0, w1, w2, w3): a standard normal
     x = sqrt(-2 ln u1) cos(2 pi u2) with u1 = ((w0 >> 8) + 1) 2^-24,
     u2 = (w1 >> 8) 2^-24; v = (1 + c x)^3; accepted when 1 + c x > 0 and
     ln u < x^2 / 2 + d (1 - v + ln v), u = ((w2 >> 8) + 1) 2^-24, giving
     d v (times u3^(1/alpha), u3 = ((w3 >> 8) + 1) 2^-24, when alpha < 1).
     Four rejections in a row (probability below 10^-5 for a >= 1) give the
     mean alpha.  The accept test is taken in float32 with the operations in
     the order written (the precision the library takes it in); the value is
     formed in FP64;
  4. d_j = E f_j for layers inside the detector.  MEAN: f_j = mu_j, and
     0 where mu_j < 10^-6 (a layer that would get less than a millionth of
     the particle's energy gets no hit).  SAMPLE: the total T = sum_j f_j of
     the MEAN fractions is kept and its split over their layers is drawn
     from a Dirichlet distribution whose means are the MEAN shares
     m_j = f_j / T, so every layer's expected deposit is its MEAN deposit:
     f_j = T G_j / sum_i G_i with independent G_j ~ Gamma(alpha_j = c m_j)
     (gamma_variate); a layer whose drawn share T G_j / sum_i G_i is below
     10^-6 gets nothing and the sum over the others normalises (the draws'
     only departure from the MEAN expectation, at most 3 10^-5 of E per
     particle moved between layers).  The concentration c is
     matched to the predicted spreads: a Dirichlet share has variance
     m_j (1 - m_j) / (c + 1), so T^2 (1 - sum m_j^2) / (c + 1) is set equal
     to V = sum (exp(s_j) + 10^-8) over the layers with f_j > 0 (the
     predicted variances of their deposit fractions, with the network's
     variance floor), c raised to 1 where it falls
     below; where c exceeds 10^4 (V = 0 included) the spread is negligible
     and the MEAN fractions are taken without a draw.  Both: scaled by
     E / sum d when the sum exceeds E;
  5. one hit per layer with d_j > 0 at the layer's mid depth, displaced
     from the particle's straight-line position by max(0, rho_j) q
     (cos phi, sin phi), one (q, phi) per particle (all its layers: the
     sub-shower drifts one way), from words (w0, w1) of the Philox block
     with counter (shower id, slice | 2 << 16, lineage lo, lineage hi):
     phi = 2 pi (w1 >> 8) 2^-24 and q = lateral_quantile(u), u = (w0 >> 8)
     2^-24, the quantile function of the lateral law LATERAL_Q.  The law is
     measured with this oracle (tests/golden/lateral_law.py): the
     energy-weighted distribution of plain sub-showers' hit distances from
     their axis divided by the mean distance of sub-showers alike in energy,
     start slice and layer offset -- the quantity rho_j estimates -- with
     mean 1, so each layer's mean displacement is rho_j.  It has a spike at
     0 (a sub-shower's first deposits lie on its axis), a core narrower and
     a tail longer than a 2-D Gaussian's (E q^2 = 1.38 against 4 / pi =
     1.27); a Gaussian of either moment left the shower's lateral profile
     2-3 % off in its rings.

training_targets() writes out the network's targets from a plain
simulation of sub-showers: deposit fractions y_j of layers start + j and
the energy-weighted mean distance R_j of those layers' hits from the
sub-shower's axis (the straight line of its start direction through its
entry point), 0 for an empty layer.
"""
from __future__ import annotations

import math

import numpy as np

from . import mlp, philox


def features(div: dict, geom, e_s: float) -> np.ndarray:
    s2l = np.asarray(geom.slice_to_layer)
    L = int(geom.n_layers)
    first = np.array([np.nonzero(s2l == l)[0].min() for l in range(L)])
    count = np.array([np.count_nonzero(s2l == l) for l in range(L)])
    lay = div["layer"]
    return np.stack([np.log(div["E"] / e_s), div["ux"], div["uy"], div["uz"],
                     (div["k"] - first[lay]) / count[lay], np.minimum(1.0, (L - lay) / 30.0)], 1)


# The lateral law: its quantile function at u = i / 64, i = 0..64 (the last
# value is the measured quantile at u = 0.998, which leaves the far 0.2 % of
# the tail short), linear in between, scaled to mean 1.  Written by
# tests/golden/lateral_law.py (80,000 sub-showers, seed 5).
LATERAL_Q = np.array([
    0.00000, 0.00000, 0.00000, 0.13168, 0.19840, 0.24732, 0.28922, 0.32671,
    0.36028, 0.39115, 0.42114, 0.44900, 0.47602, 0.50152, 0.52699, 0.55146,
    0.57525, 0.59910, 0.62231, 0.64475, 0.66703, 0.68907, 0.71090, 0.73253,
    0.75422, 0.77610, 0.79778, 0.81916, 0.84060, 0.86253, 0.88486, 0.90712,
    0.92884, 0.95082, 0.97305, 0.99593, 1.01889, 1.04247, 1.06618, 1.09030,
    1.11503, 1.14011, 1.16589, 1.19201, 1.21890, 1.24660, 1.27561, 1.30556,
    1.33609, 1.36810, 1.40167, 1.43705, 1.47402, 1.51349, 1.55558, 1.60084,
    1.65098, 1.70647, 1.77006, 1.84258, 1.92934, 2.03901, 2.19413, 2.48104,
    4.43834])


def lateral_quantile(u: float) -> float:
    """q(u), u in [0, 1), of the lateral law: linear between LATERAL_Q[i] at
    u = i / 64 and LATERAL_Q[i + 1]."""
    x = u * 64.0
    i = min(63, int(x))
    return float(LATERAL_Q[i] + (x - i) * (LATERAL_Q[i + 1] - LATERAL_Q[i]))


def lateral_offset(shower_id: int, k: int, lineage: int, seed: int) -> np.ndarray:
    """(q cos phi, q sin phi) of a particle's hit displacements (step 5)."""
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    w = philox(((shower_id) & 0xFFFFFFFF, k | (2 << 16), lineage & 0xFFFFFFFF, (lineage >> 32) & 0xFFFFFFFF), key)
    q = lateral_quantile((int(w[0]) >> 8) * 2.0 ** -24)
    phi = 2 * math.pi * (int(w[1]) >> 8) * 2.0 ** -24
    return np.array([q * math.cos(phi), q * math.sin(phi)])


def training_targets(geom, prims, res) -> np.ndarray:
    """Y [n, 60] of sub-showers `prims` (start slice in geom >> 16) from
    their plain simulation `res` (oracle.simulate)."""
    s2l = np.asarray(geom.slice_to_layer)
    L = int(geom.n_layers)
    n = len(prims)
    Y = np.zeros((n, 60))
    off = res["offsets"]
    for s in range(n):
        k0 = int(prims["geom"][s]) >> 16
        l0 = int(s2l[k0])
        E0 = float(prims["E"][s])
        m = min(30, L - l0)
        Y[s, :m] = res["layer_sum"][s, l0:l0 + m] / E0
        th, ph = float(prims["theta"][s]), float(prims["phi"][s])
        tx, ty = math.tan(th) * math.cos(ph), math.tan(th) * math.sin(ph)
        x0, y0, z0 = float(prims["x0"][s]), float(prims["y0"][s]), k0 * geom.dz
        er = np.zeros(30)
        e = np.zeros(30)
        for h in range(off[s], off[s + 1]):
            j = int(s2l[int(round(res["z"][h] / geom.dz))]) - l0
            if 0 <= j < 30:
                dz = res["z"][h] - z0
                r = math.hypot(res["x"][h] - x0 - dz * tx, res["y"][h] - y0 - dz * ty)
                er[j] += res["E"][h] * r
                e[j] += res["E"][h]
        Y[s, 30:] = np.where(e > 0, er / np.where(e > 0, e, 1.0), 0.0)
    return Y


def _u24p(w: int) -> float:
    """((w >> 8) + 1) 2^-24, a uniform on (0, 1]."""
    return ((int(w) >> 8) + 1) * 2.0 ** -24


def gamma_variate(alpha: float, shower_id: int, k: int, lineage: int, j: int, seed: int) -> float:
    """Gamma(alpha, 1) variate of layer j of a diverted particle (step 3 of
    the module's rule); alpha is taken at float32 precision."""
    f32 = np.float32
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    al = f32(alpha)
    boost = al < f32(1.0)
    a = f32(al + f32(1.0)) if boost else al
    d = f32(a - f32(1.0 / 3.0))
    c = f32(f32(1.0) / f32(np.sqrt(f32(f32(9.0) * d))))
    for t in range(4):
        w = philox((shower_id & 0xFFFFFFFF, k | (3 << 16) | ((4 * j + t) << 20), lineage & 0xFFFFFFFF,
                    (lineage >> 32) & 0xFFFFFFFF), key)
        u1, u2, u, u3 = _u24p(w[0]), (int(w[1]) >> 8) * 2.0 ** -24, _u24p(w[2]), _u24p(w[3])
        # the decision in float32, the operations in the order written
        rad = f32(np.sqrt(f32(f32(-2.0) * f32(math.log(u1)))))
        x = f32(rad * f32(math.cos(2.0 * math.pi * u2)))
        t1 = f32(f32(1.0) + f32(c * x))
        if not t1 > f32(0.0):
            continue
        v = f32(f32(t1 * t1) * t1)
        rhs = f32(f32(f32(0.5) * f32(x * x)) + f32(d * f32(f32(f32(1.0) - v) + f32(math.log(float(v))))))
        if not f32(math.log(u)) < rhs:
            continue
        # the value in FP64 from the same draws
        x64 = math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)
        d64 = float(a) - 1.0 / 3.0
        g = d64 * (1.0 + x64 / math.sqrt(9.0 * d64)) ** 3
        if boost:
            g *= u3 ** (1.0 / float(al))
        return g
    return float(al)


SAMPLE_C_MIN, SAMPLE_C_MAX = 1.0, 1.0e4
FRACTION_MIN = 1.0e-6


def sample_concentration(f: np.ndarray, s: np.ndarray) -> float:
    """Dirichlet concentration c of step 4 from the MEAN fractions f_j
    (>= 0) and the predicted log-variances s_j; math.inf where the MEAN
    fractions are taken without a draw (c above SAMPLE_C_MAX)."""
    T = float(f.sum())
    pos = f > 0
    V = float((np.exp(s[pos]) + mlp.VAR_FLOOR).sum())
    if T <= 0:
        return math.inf
    m = f / T
    num = T * T * (1.0 - float((m * m).sum()))
    if V <= 0 or num > (SAMPLE_C_MAX + 1.0) * V:
        return math.inf
    return max(SAMPLE_C_MIN, num / V - 1.0)


def sample_fractions(f: np.ndarray, s: np.ndarray, shower_id: int, k: int, lineage: int, seed: int) -> np.ndarray:
    """SAMPLE fractions: the MEAN total T = sum f split by a Dirichlet draw
    with means f / T (step 4)."""
    T = float(f.sum())
    if T <= 0:
        return np.zeros_like(f)
    c = sample_concentration(f, s)
    if math.isinf(c):
        return f.copy()
    G = np.zeros_like(f)
    for j in np.nonzero(f > 0)[0]:
        G[j] = gamma_variate(c * f[j] / T, shower_id, k, lineage, int(j), seed)
    tot = G.sum()
    if tot <= 0:
        return f.copy()
    G[T * G / tot < FRACTION_MIN] = 0.0
    kept = G.sum()
    if kept <= 0:
        return f.copy()
    return T * G / kept


def deposits(div: dict, params, geom, e_s: float, seed: int, shower_id_base: int = 0, mode: int = 0,
             out=None) -> dict:
    """Per diverted particle: the drawn deposits d [n_div, 30] and the hits
    [n_hits, 7] (shower, x, y, z, E, layer, index of the particle in div).
    mode 0 (SAMPLE): Dirichlet split of the MEAN total; mode 1 (MEAN): the
    means.  `out` [n_div, 90] replaces the FP64 network's outputs when given
    (to apply the rule to another implementation's network outputs)."""
    X = features(div, geom, e_s)
    if out is None:
        out, _ = mlp.forward(params, X) if len(X) else (np.zeros((0, 90)), None)
    L = int(geom.n_layers)
    s2l = np.asarray(geom.slice_to_layer)
    zmid = np.array([geom.dz * (np.nonzero(s2l == l)[0].min() + np.nonzero(s2l == l)[0].max()) * 0.5
                     for l in range(L)])
    nd = len(X)
    d = np.zeros((nd, 30))
    hits = []
    for i in range(nd):
        l0 = int(div["layer"][i])
        E = div["E"][i]
        inside = l0 + np.arange(30) < L
        mu = mlp.deposit_means(out[i:i + 1])[0]
        f = np.where(inside & (mu >= FRACTION_MIN), mu, 0.0)
        if mode != 1:
            f = sample_fractions(f, out[i, 30:60], shower_id_base + int(div["shower"][i]), int(div["k"][i]),
                                 int(div["lineage"][i]), seed)
        d[i] = E * f
        tot = d[i].sum()
        if tot > E:
            d[i] *= E / tot
        zk = div["k"][i] * geom.dz
        mo = lateral_offset(shower_id_base + int(div["shower"][i]), int(div["k"][i]), int(div["lineage"][i]), seed)
        for j in range(30):
            if d[i, j] > 0:
                zm = zmid[l0 + j]
                sig = max(0.0, out[i, 60 + j])
                hits.append((int(div["shower"][i]),
                             div["x"][i] + (zm - zk) * div["ux"][i] / div["uz"][i] + sig * mo[0],
                             div["y"][i] + (zm - zk) * div["uy"][i] / div["uz"][i] + sig * mo[1], zm, d[i, j],
                             l0 + j, i))
    return dict(d=d, out=out, hits=np.array(hits).reshape(-1, 7))
