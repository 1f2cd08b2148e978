"""Measures the radial law of the surrogate's hit displacements
(oracle.hybrid.LATERAL_Q) with the FP64 oracle and prints it.

Plain sub-showers started at the front of the 30-layer detector at normal
incidence, energies log-uniform from the energy cut to 2 GeV: every hit's
distance d from its sub-shower's axis is divided by the energy-weighted mean
distance of the hits of sub-showers alike in energy (16 log bins), start
slice within the layer and layer offset from the start -- the quantity the
network predicts per layer.  The law is the energy-weighted distribution of
q = d / mean: its quantile function sampled at u = i / 64 (i = 0..63) and
at u = 0.998 (the end of the last interval), then scaled so that the law
with linear interpolation between the samples has mean exactly 1.

    python tests/golden/lateral_law.py [n_subshowers]   (80,000 for the table)
"""
from __future__ import annotations

import os
import sys

import numpy as np

K = 64
U_END = 0.998


def measure(n: int, seed: int = 5, e_hi: float = 2.0, n_threads: int = 16) -> np.ndarray:
    import oracle
    from paper_2202_05012_gb300 import inputs
    g = inputs.supa_d(30)
    p, _ = inputs.subshower_primaries(n, seed, e_lo=g.e_min, e_hi=e_hi)
    p["theta"] = 0.0
    r = oracle.simulate(g, p, 3, n_threads=n_threads)
    s2l = np.asarray(g.slice_to_layer)
    sh = np.repeat(np.arange(len(p)), np.diff(r["offsets"]))
    k0 = (p["geom"].astype(np.int64) >> 16)[sh]
    first = np.array([np.nonzero(s2l == l)[0].min() for l in range(g.n_layers)])
    j = s2l[np.rint(r["z"] / g.dz).astype(int)] - s2l[k0]
    d = np.hypot(r["x"] - p["x0"][sh], r["y"] - p["y0"][sh])
    w = r["E"]
    ebin = np.clip((np.log(p["E"][sh] / g.e_min) / np.log(e_hi / g.e_min) * 16).astype(int), 0, 15)
    key = (ebin * 8 + (k0 - first[s2l[k0]])) * 64 + j
    mean_d = np.bincount(key, weights=w * d) / np.maximum(np.bincount(key, weights=w), 1e-300)
    ok = mean_d[key] > 0
    q, w = d[ok] / mean_d[key][ok], w[ok]
    o = np.argsort(q)
    q, w = q[o], w[o]
    cw = (np.cumsum(w) - 0.5 * w) / w.sum()
    Q = np.interp(np.append(np.arange(K) / K, U_END), cw, q)
    Q[0] = 0.0
    return Q / ((Q[:-1] + Q[1:]) / 2).mean()


if __name__ == "__main__":
    sys.path.insert(0, os.path.join(os.path.dirname(__file__), "..", ".."))
    Q = measure(int(sys.argv[1]) if len(sys.argv) > 1 else 80_000)
    print(",\n".join(", ".join(f"{v:.5f}" for v in Q[i:i + 8]) for i in range(0, len(Q), 8)))
