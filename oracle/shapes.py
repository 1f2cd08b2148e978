"""FP64 oracle of the shower shape variables -- TEST INFRASTRUCTURE.

Sec. 5.1 ("Shower Shape Variables") and App. A.1 ("More shower shape
variables") define them for point clouds.  For shower s and layer i, with
the points j of the layer (eta_j, phi_j) = the lateral position relative to
the shower's incidence axis at the point's depth, r_j = sqrt(eta_j^2 +
phi_j^2), and E_j the point's energy:

  per layer (18 values, in this order)
    n_i                          number of points
    Ebar_i = sum_j E_j           layer energy (the FP64 layer sum)
    f_i = Ebar_i / E_tot         layer energy fraction
    <eta>, <phi>, <r>, <E>       feature means (unweighted over the points)
    sigma of eta, phi, r, E      feature spreads sqrt(mean of squares - mean^2)
    <eta>_E, <phi>_E, <r>_E      layer centroids (energy weighted)
    sigma_E of eta, phi, r       layer lateral widths (energy weighted)
    E_ratio = (E[1] - E[2]) / (E[1] + E[2]), E[1] >= E[2] the two largest
              point energies of the layer (E[2] = 0 for a single point)
  per shower (5 values)
    E_tot = sum_i Ebar_i; depth d = deepest layer with energy (-1: none);
    l_d = sum_i i Ebar_i; s_d = l_d / E_tot;
    sigma_sd = sqrt(sum_i i^2 Ebar_i / E_tot - s_d^2)

Layers are numbered from 0; an empty layer's values are all 0 (E_tot = 0
makes f, s_d, sigma_sd 0).  Plain numpy float64, one formula per value.
"""
from __future__ import annotations

import math

import numpy as np

N_LAYER_FEATS = 18
N_SHOWER_FEATS = 5


def shower_shapes(geom, prims, res):
    """(layer_feats [n, L, 18], shower_feats [n, 5]) of the showers `prims`
    simulated in `res` (oracle.simulate output)."""
    s2l = np.asarray(geom.slice_to_layer)
    L = int(geom.n_layers)
    n = len(prims)
    lf = np.zeros((n, L, N_LAYER_FEATS))
    sf = np.zeros((n, N_SHOWER_FEATS))
    off = res["offsets"]
    for s in range(n):
        th, ph = float(prims["theta"][s]), float(prims["phi"][s])
        tx, ty = math.tan(th) * math.cos(ph), math.tan(th) * math.sin(ph)
        x0, y0 = float(prims["x0"][s]), float(prims["y0"][s])
        a, b = off[s], off[s + 1]
        z = res["z"][a:b]
        eta = res["x"][a:b] - (x0 + z * tx)
        phi = res["y"][a:b] - (y0 + z * ty)
        r = np.sqrt(eta ** 2 + phi ** 2)
        E = res["E"][a:b]
        lay = s2l[np.rint(z / geom.dz).astype(int)]
        Ebar = res["layer_sum"][s, :L]
        Etot = Ebar.sum()
        for i in range(L):
            m = lay == i
            k = int(m.sum())
            out = lf[s, i]
            out[1] = Ebar[i]
            out[2] = Ebar[i] / Etot if Etot > 0 else 0.0
            if k == 0:
                continue
            out[0] = k
            for c, v in enumerate((eta[m], phi[m], r[m], E[m])):
                mean = v.sum() / k
                out[3 + c] = mean
                out[7 + c] = math.sqrt(max(0.0, (v ** 2).sum() / k - mean ** 2))
            Ei = E[m].sum()
            for c, v in enumerate((eta[m], phi[m], r[m])):
                cen = (E[m] * v).sum() / Ei
                out[11 + c] = cen
                out[14 + c] = math.sqrt(max(0.0, (E[m] * v ** 2).sum() / Ei - cen ** 2))
            top = np.sort(E[m])[::-1]
            e1, e2 = top[0], (top[1] if k > 1 else 0.0)
            out[17] = (e1 - e2) / (e1 + e2)
        idx = np.arange(L)
        nz = np.nonzero(Ebar > 0)[0]
        sf[s, 0] = Etot
        sf[s, 1] = nz.max() if len(nz) else -1
        sf[s, 2] = (idx * Ebar).sum()
        if Etot > 0:
            sf[s, 3] = sf[s, 2] / Etot
            sf[s, 4] = math.sqrt(max(0.0, (idx ** 2 * Ebar).sum() / Etot - sf[s, 3] ** 2))
    return lf, sf
