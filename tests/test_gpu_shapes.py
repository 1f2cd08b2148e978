"""GPU parity of the shower shape variables (Sec. 5.1, App. A.1) against the
FP64 oracle on showers shaped like the 30-layer workload (E U[1,100] GeV,
0-30 deg), and their consistency on the hybrid path
(stepped and surrogate points)."""
import numpy as np
import pytest

import oracle
from oracle import shapes
from paper_2202_05012_gb300 import inputs
from paper_2202_05012_gb300 import supa as S

pytestmark = pytest.mark.gpu


def _gpu_shapes(b, n, L):
    import torch
    lf = torch.full((n, L, 18), np.nan, dtype=torch.float32, device="cuda")
    sf = torch.full((n, 5), np.nan, dtype=torch.float32, device="cuda")
    S.supa_shower_shapes(b, 0, n, lf, sf)
    torch.cuda.synchronize()
    return lf.cpu().numpy().astype(np.float64), sf.cpu().numpy().astype(np.float64)


def test_shapes_match_oracle_30_layer_showers():
    g = inputs.supa_d(30, grid=64, roi_mode=inputs.ROI_AXIS)
    n = 300
    p = inputs.primaries(n, 51, e_lo=1.0, e_hi=100.0, theta_max_deg=30.0, entry_halfwidth=0.25)
    gh = S.supa_init_geometry(g)
    b = S.supa_batch_create([gh], n, {})
    try:
        S.supa_simulate(b, S.primaries_to_device(p), n, 29)
        info = S.supa_batch_get_info(b)
        lf, sf = _gpu_shapes(b, n, info.max_layers)
        counts = S.info_arrays(info)["counts"].cpu().numpy().view(np.uint32).astype(np.int64)
    finally:
        S.supa_destroy_batch(b)
        S.supa_destroy_geometry(gh)
    ora = oracle.simulate(g, p, 29, n_threads=8)
    lo, so = shapes.shower_shapes(g, p, ora)
    assert np.all(np.isfinite(lf)) and np.all(np.isfinite(sf))
    same = counts == np.diff(ora["offsets"])  # showers without a flipped decision
    assert same.mean() > 0.99
    a, o = lf[same], lo[same]
    np.testing.assert_array_equal(a[:, :, 0], o[:, :, 0])                      # points per layer
    np.testing.assert_allclose(a[:, :, 1:3], o[:, :, 1:3], rtol=1e-5, atol=1e-9)  # Ebar, f
    np.testing.assert_allclose(a[:, :, 6], o[:, :, 6], rtol=1e-5, atol=1e-9)      # <E>
    # means and centroids of eta, phi, r: FP32 sums of ~40 points per layer
    for c in (3, 4, 5, 11, 12, 13):
        np.testing.assert_allclose(a[:, :, c], o[:, :, c], rtol=1e-4, atol=2e-5)
    # spreads: FP32 second moments about the means (sqrt amplifies near 0)
    for c in (7, 8, 9, 10, 14, 15, 16):
        np.testing.assert_allclose(a[:, :, c], o[:, :, c], rtol=1e-3, atol=3e-4)
    np.testing.assert_allclose(a[:, :, 17], o[:, :, 17], rtol=0, atol=2e-5)      # E_ratio
    np.testing.assert_allclose(sf[same][:, [0, 2]], so[same][:, [0, 2]], rtol=1e-6)
    np.testing.assert_array_equal(sf[same][:, 1], so[same][:, 1])
    np.testing.assert_allclose(sf[same][:, 3:], so[same][:, 3:], rtol=0, atol=1e-5)
    assert (o[:, :, 0] > 1).sum() > 1000 and np.any(o[:, :, 8] > 0.2)  # non-trivial content


def test_shapes_on_the_hybrid_path_count_every_point():
    import torch
    g = inputs.supa_d(30)
    n = 200
    p = inputs.primaries(n, 8, e_lo=5.0, e_hi=50.0, theta_max_deg=20.0)
    gh = S.supa_init_geometry(g)
    sur = S.supa_surrogate_create(1024, S.pack_mlp_params(inputs.mlp_init(2)))
    b = S.supa_batch_create([gh], n, {})
    try:
        S.supa_batch_set_surrogate(b, sur, 1.0, 1_000_000, S.SUPA_SURROGATE_MEAN)
        S.supa_simulate(b, S.primaries_to_device(p), n, 3)
        info = S.supa_batch_get_info(b)
        assert info.n_diverted > 0
        lf, sf = _gpu_shapes(b, n, info.max_layers)
        arr = S.info_arrays(info)
        counts = arr["counts"].cpu().numpy().view(np.uint32).astype(np.int64)
        ls = arr["layer_sum"].cpu().numpy()
    finally:
        S.supa_destroy_batch(b)
        S.supa_surrogate_destroy(sur)
        S.supa_destroy_geometry(gh)
    np.testing.assert_array_equal(lf[:, :, 0].sum(1), counts)
    np.testing.assert_allclose(lf[:, :, 1], ls, rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(sf[:, 0], ls.sum(1), rtol=1e-6)
    f = lf[:, :, 2].sum(1)
    np.testing.assert_allclose(f[ls.sum(1) > 0], 1.0, rtol=1e-5)
