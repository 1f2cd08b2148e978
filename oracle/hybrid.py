"""FP64 oracle of the surrogate side of the hybrid path -- TEST INFRASTRUCTURE.

The SUPA paper has no surrogate; this follows the library's stated rule for
it.  For every particle set aside below E_s (oracle.simulate(..., e_s=...)
returns them):
  1. features: log(E / E_s), direction cosines, position of the slice in its
     layer (k - first slice) / slices in the layer, layers left from the
     particle's layer to the back over 30 (capped at 1);
  2. the FP64 network (oracle.mlp) gives mu_j and s_j, j = 0..29;
  3. n_j: standard normals by Box-Muller from Philox4x32-10 blocks with
     counter (shower id, slice | 1 << 16 | block << 20, lineage lo, lineage
     hi), block = 0..7, key = seed; from each block's words (w0, w1, w2, w3)
     the pairs (w0, w1) and (w2, w3) give u1 = ((w >> 8) + 1) 2^-24 and
     u2 = (w >> 8) 2^-24, z = sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2);
  4. d_j = E f_j for layers inside the detector.  MEAN: f_j = max(0, mu_j).
     SAMPLE: g_j = mu_j exp(a_j n_j - a_j^2 / 2), the log-normal with mean
     mu_j and variance exp(s_j) (a_j^2 = ln(1 + exp(s_j) / mu_j^2), capped at
     4 -- the mean stays mu_j), 0 when mu_j <= 0, then rescaled to the MEAN
     total: f_j = g_j sum_i max(0, mu_i) / sum_i g_i (the shape fluctuates,
     the total does not).  Both: scaled by E / sum d when the sum exceeds E;
  5. one hit per layer with d_j > 0 at the layer's mid depth, displaced
     from the particle's straight-line position by sigma_j (m1, m2):
     sigma_j = max(0, rho_j) sqrt(2 / pi), so that each layer's displacement
     is an isotropic 2-D Gaussian whose mean distance is the predicted rho_j;
     (m1, m2) is one Box-Muller pair per particle (all its layers: the
     sub-shower drifts one way), from words (w0, w1) of the Philox block
     with counter (shower id, slice | 2 << 16, lineage lo, lineage hi).

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


def _box_muller(w0: int, w1: int):
    u1 = ((int(w0) >> 8) + 1) * 2.0 ** -24
    u2 = (int(w1) >> 8) * 2.0 ** -24
    rad = math.sqrt(-2.0 * math.log(u1))
    return rad * math.cos(2 * math.pi * u2), rad * math.sin(2 * math.pi * u2)


def offset_normals(shower_id: int, k: int, lineage: int, seed: int) -> np.ndarray:
    """The standard normal pair (m1, m2) of a particle's hit displacements."""
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    w = philox(((shower_id) & 0xFFFFFFFF, k | (2 << 16), lineage & 0xFFFFFFFF, (lineage >> 32) & 0xFFFFFFFF), key)
    return np.array(_box_muller(w[0], w[1]))


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


def normals(shower_id: int, k: int, lineage: int, seed: int) -> np.ndarray:
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    z = []
    for blk in range(8):
        w = philox(((shower_id) & 0xFFFFFFFF, k | (1 << 16) | (blk << 20), lineage & 0xFFFFFFFF,
                    (lineage >> 32) & 0xFFFFFFFF), key)
        for p in range(2):
            u1 = ((int(w[2 * p]) >> 8) + 1) * 2.0 ** -24
            u2 = (int(w[2 * p + 1]) >> 8) * 2.0 ** -24
            rad = math.sqrt(-2.0 * math.log(u1))
            z.append(rad * math.cos(2 * math.pi * u2))
            z.append(rad * math.sin(2 * math.pi * u2))
    return np.array(z)


def deposits(div: dict, params, geom, e_s: float, seed: int, shower_id_base: int = 0, mode: int = 0) -> dict:
    """Per diverted particle: the drawn deposits d [n_div, 30] and the hits.
    mode 0 (SAMPLE): moment-matched log-normal draws; mode 1 (MEAN): the means."""
    X = features(div, geom, e_s)
    out, _ = mlp.forward(params, X) if len(X) else (np.zeros((0, 90)), None)
    L = int(geom.n_layers)
    s2l = np.asarray(geom.slice_to_layer)
    zmid = np.array([geom.dz * (np.nonzero(s2l == l)[0].min() + np.nonzero(s2l == l)[0].max()) * 0.5
                     for l in range(L)])
    nd = len(X)
    d = np.zeros((nd, 30))
    hits = []
    for i in range(nd):
        n = normals(shower_id_base + int(div["shower"][i]), int(div["k"][i]), int(div["lineage"][i]), seed)
        l0 = int(div["layer"][i])
        E = div["E"][i]
        for j in range(30):
            if l0 + j < L:
                mu = out[i, j]
                if mode == 1 or mu <= 0.0:
                    f = max(0.0, mu)
                else:
                    a2 = min(4.0, math.log1p(math.exp(out[i, 30 + j]) / (mu * mu)))
                    f = mu * math.exp(math.sqrt(a2) * n[j] - 0.5 * a2)
                d[i, j] = E * f
        if mode != 1:
            inside = l0 + np.arange(30) < L
            mean_tot = E * np.maximum(0.0, out[i, :30][inside]).sum()
            if d[i].sum() > 0:
                d[i] *= mean_tot / d[i].sum()
        tot = d[i].sum()
        if tot > E:
            d[i] *= E / tot
        zk = div["k"][i] * geom.dz
        mo = offset_normals(shower_id_base + int(div["shower"][i]), int(div["k"][i]), int(div["lineage"][i]), seed)
        for j in range(30):
            if d[i, j] > 0:
                zm = zmid[l0 + j]
                sig = max(0.0, out[i, 60 + j]) * math.sqrt(2.0 / math.pi)
                hits.append((int(div["shower"][i]),
                             div["x"][i] + (zm - zk) * div["ux"][i] / div["uz"][i] + sig * mo[0],
                             div["y"][i] + (zm - zk) * div["uy"][i] / div["uz"][i] + sig * mo[1], zm, d[i, j],
                             l0 + j))
    return dict(d=d, out=out, hits=np.array(hits).reshape(-1, 6))
