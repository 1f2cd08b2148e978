"""Oracle of per-layer grids and multi-resolution images -- TEST INFRASTRUCTURE.

App. A.5 ("Downsampling") and the grid experiments: each layer l has its own
region of interest and cell grid (the CaloGAN-like detector: 3 x 96, 12 x 12
and 12 x 6 cells over one square region), and "2x", "3x" resolutions divide
every cell of a layer f times in both directions.  For layer l with nx_l x
ny_l cells of wx_l x wy_l and resolution factor f:
  region low corner (float32): FIXED -> (-nx_l wx_l / 2, -ny_l wy_l / 2);
    AXIS -> (zmid_l tan(theta) cos(phi) - nx_l wx_l / 2, ... sin ...), as
    for the uniform grid;
  cell widths w' = w / f (float32), cells nx_l f x ny_l f, half-open cells
    [lo + i w', lo + (i + 1) w'), i = floor((x - lo) / w') in float32;
  a point outside the region adds to that resolution's out-of-region sum.
Cell sums in FP64.  Image layout per shower: for each factor (in the given
order), for each layer, ny_l f rows of nx_l f cells (x fastest).
"""
from __future__ import annotations

import numpy as np


def cells(grids, factors) -> int:
    return int(sum(int(ny) * f * int(nx) * f for f in factors for (nx, ny, _, _) in grids))


def voxelize_layers(hx, hy, hz, hE, offsets, geom, prims, grids, factors):
    """grids: [(nx, ny, wx, wy)] per layer; factors: resolution factors.
    Returns (images [n, C] FP64, out_of_roi [n, len(factors)] FP64)."""
    f32 = np.float32
    hx, hy, hz, hE = (np.asarray(a, dtype=f32) for a in (hx, hy, hz, hE))
    n = len(offsets) - 1
    L = int(geom.n_layers)
    s2l = np.asarray(geom.slice_to_layer)
    C = cells(grids, factors)
    img = np.zeros((n, C))
    oor = np.zeros((n, len(factors)))
    half_x = [f32(nx) * f32(wx) * f32(0.5) for (nx, ny, wx, wy) in grids]
    half_y = [f32(ny) * f32(wy) * f32(0.5) for (nx, ny, wx, wy) in grids]
    zmid = [f32(f32(geom.dz) * f32(int(np.nonzero(s2l == l)[0].min()) + int(np.nonzero(s2l == l)[0].max()))
                * f32(0.5)) for l in range(L)]
    # image offsets of (factor index, layer)
    base = {}
    o = 0
    for fi, f in enumerate(factors):
        for l, (nx, ny, _, _) in enumerate(grids):
            base[fi, l] = o
            o += int(ny) * f * int(nx) * f
    for s in range(n):
        if int(geom.roi_mode) == 1:
            t = f32(np.tan(f32(prims["theta"][s])))
            tx = f32(t * f32(np.cos(f32(prims["phi"][s]))))
            ty = f32(t * f32(np.sin(f32(prims["phi"][s]))))
            lo_x = [f32(f32(zmid[l] * tx) - half_x[l]) for l in range(L)]
            lo_y = [f32(f32(zmid[l] * ty) - half_y[l]) for l in range(L)]
        else:
            lo_x = [-half_x[l] for l in range(L)]
            lo_y = [-half_y[l] for l in range(L)]
        for j in range(offsets[s], offsets[s + 1]):
            k = int(np.rint(hz[j] / f32(geom.dz)))
            l = int(s2l[k]) if 0 <= k < len(s2l) else -1
            for fi, f in enumerate(factors):
                if l < 0:
                    oor[s, fi] += float(hE[j])
                    continue
                nx, ny, wx, wy = grids[l]
                ix = np.floor(f32(hx[j] - lo_x[l]) / f32(f32(wx) / f32(f)))
                iy = np.floor(f32(hy[j] - lo_y[l]) / f32(f32(wy) / f32(f)))
                if 0 <= ix < int(nx) * f and 0 <= iy < int(ny) * f:
                    img[s, base[fi, l] + int(iy) * int(nx) * f + int(ix)] += float(hE[j])
                else:
                    oor[s, fi] += float(hE[j])
    return img, oor
