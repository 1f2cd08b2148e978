"""GPU parity of per-layer grids at several resolutions (App. A.5; the
CaloGAN-like 3 x 96 / 12 x 12 / 12 x 6 detector at 1x, 2x, 3x) against the
oracle, and energy conservation per factor."""
import numpy as np
import pytest

import oracle
from oracle import grids as G
from paper_2202_05012_gb300 import inputs
from paper_2202_05012_gb300 import supa as S

pytestmark = pytest.mark.gpu


def _run(g, p, seed, grids, factors):
    import torch
    n = len(p)
    gh = S.supa_init_geometry(g)
    b = S.supa_batch_create([gh], n, {})
    try:
        S.supa_simulate(b, S.primaries_to_device(p), n, seed)
        info = S.supa_batch_get_info(b)
        C = S.supa_layer_images_cells(grids, factors)
        img = torch.full((n, C), -1.0, dtype=torch.float32, device="cuda")
        oor = torch.zeros((n, len(factors)), dtype=torch.float64, device="cuda")
        S.supa_voxelize_layers(b, 0, n, grids, factors, img, oor)
        ls = S.info_arrays(info)["layer_sum"].cpu().numpy()
        torch.cuda.synchronize()
        return img.cpu().numpy().astype(np.float64), oor.cpu().numpy(), ls
    finally:
        S.supa_destroy_batch(b)
        S.supa_destroy_geometry(gh)


def _check(g, p, seed, grids, factors):
    img, oor, ls = _run(g, p, seed, grids, factors)
    r = oracle.simulate(g, p, seed, n_threads=8)
    ref, oor_ref = G.voxelize_layers(r["x"], r["y"], r["z"], r["E"], r["offsets"], g, p, grids, factors)
    assert img.shape == ref.shape and np.all(img >= 0)
    # cells move only where a rounding difference crosses a cell edge
    diff = np.abs(img - ref)
    bad = diff > 1e-5 * np.maximum(ref, 1e-3)
    assert bad.mean() < 1e-4, bad.mean()
    np.testing.assert_allclose(oor, oor_ref, rtol=1e-4, atol=1e-6)
    # conservation per factor: images + out of region = the shower's deposits
    o = 0
    for fi, f in enumerate(factors):
        c = S.supa_layer_images_cells(grids, [f])
        np.testing.assert_allclose(img[:, o:o + c].sum(1) + oor[:, fi], ls.sum(1), rtol=1e-5)
        o += c
    return img, ref


def test_calogan_like_multires_matches_oracle():
    g = inputs.supa_calogan()
    p = inputs.primaries(300, 61, e_lo=1.0, e_hi=100.0)
    img, ref = _check(g, p, 7, inputs.calogan_grids(), [1, 2, 3])
    assert (ref > 0).sum() > 50_000


def test_heterogeneous_grids_axis_roi_inclined():
    g = inputs.supa_d(6, grid=32, roi_mode=inputs.ROI_AXIS)
    p = inputs.primaries(200, 62, e_lo=1.0, e_hi=50.0, theta_max_deg=30.0, entry_halfwidth=0.5)
    grids = [(32, 32, 0.5, 0.5), (16, 8, 1.0, 2.0), (40, 20, 0.4, 0.8), (7, 9, 2.3, 1.7), (64, 3, 0.25, 5.0),
             (12, 12, 1.3333, 1.3333)]
    _check(g, p, 8, grids, [1, 4])
