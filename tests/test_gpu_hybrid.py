"""Sub-shower starts, the surrogate's training set, and the hybrid path
(plain stepping above E_s, network deposits below it)."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2202_05012_gb300 import inputs
from paper_2202_05012_gb300 import supa as S

from gpu_helpers import compare, run_gpu

pytestmark = pytest.mark.gpu

E_S = 1.0


def _features_ref(prims, start, geom, e_s):
    """The 6 network inputs written out from their definition: log(E/E_s),
    direction cosines, position of the start slice in its layer, layers left
    (over 30, capped at 1)."""
    th = prims["theta"].astype(np.float64)
    ph = prims["phi"].astype(np.float64)
    lay = geom.slice_to_layer[start]
    kfirst = np.array([np.nonzero(geom.slice_to_layer == l)[0].min() for l in lay])
    nsl = np.array([np.count_nonzero(geom.slice_to_layer == l) for l in lay])
    return np.stack([np.log(prims["E"].astype(np.float64) / e_s), np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph),
                     np.cos(th), (start - kfirst) / nsl, np.minimum(1.0, (geom.n_layers - lay) / 30.0)], 1), lay


def test_subshower_starts_match_oracle():
    g = inputs.supa_d(30)
    p, start = inputs.subshower_primaries(2000, 5, e_lo=0.05, e_hi=5.0)
    compare(run_gpu([g], p, seed=3), oracle.simulate(g, p, 3, n_threads=8), [g], p)


def test_training_set_matches_oracle_targets():
    import torch
    g = inputs.supa_d(30)
    n = 4096
    p, start = inputs.subshower_primaries(n, 6)
    gh = S.supa_init_geometry(g)
    b = S.supa_batch_create([gh], n, {})
    try:
        S.supa_simulate(b, S.primaries_to_device(p), n, 4)
        S.supa_batch_get_info(b)
        x = torch.zeros((n, 6), dtype=torch.float32, device="cuda")
        y = torch.zeros((n, 60), dtype=torch.float32, device="cuda")
        S.supa_build_training_set(b, E_S, x, y)
        X, Y = x.cpu().numpy(), y.cpu().numpy()
    finally:
        S.supa_destroy_batch(b)
        S.supa_destroy_geometry(gh)
    Xr, lay = _features_ref(p, start, g, E_S)
    np.testing.assert_allclose(X, Xr, rtol=1e-5, atol=1e-6)
    from oracle import hybrid
    ora = oracle.simulate(g, p, 4, n_threads=8)
    Yr = hybrid.training_targets(g, p, ora)
    same = np.abs(Y[:, :30] - Yr[:, :30]).max(1) < 1e-4
    assert same.mean() > 0.999
    np.testing.assert_allclose(Y[same, :30], Yr[same, :30], rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(Y[:, :30].sum(1), Yr[:, :30].sum(1), atol=2e-3)
    # mean lateral distances (FP32 sums on the device)
    assert np.any(Yr[:, 30:] > 0.1)
    np.testing.assert_allclose(Y[same, 30:], Yr[same, 30:], rtol=1e-4, atol=1e-5)


def _surrogate(seed=1):
    return S.supa_surrogate_create(1024, S.pack_mlp_params(inputs.mlp_init(seed)))


def test_hybrid_conserves_energy_and_emits_after_stepped_hits():
    import torch
    g = inputs.supa_d(30, grid=64, roi_mode=inputs.ROI_AXIS)
    n = 3000
    p = inputs.primaries(n, 7, e_lo=5.0, e_hi=60.0, theta_max_deg=30.0)
    gh = S.supa_init_geometry(g)
    sur = _surrogate()
    b = S.supa_batch_create([gh], n, {"record_tags": 1})
    try:
        S.supa_batch_set_surrogate(b, sur, E_S, 4_000_000)
        d = S.primaries_to_device(p)
        S.supa_simulate(b, d, n, 9)
        info = S.supa_batch_get_info(b)
        assert info.n_diverted > 0
        arr = {k: v.cpu().numpy() for k, v in S.info_arrays(info).items()}
        sleak = S.device_view(info.sur_leak_dev, (n,), torch.float64).cpu().numpy()
        tot = arr["layer_sum"].sum(1) + arr["dead"] + arr["leak"] + arr["escape"] + sleak
        np.testing.assert_allclose(tot, p["E"].astype(np.float64), rtol=1e-5)
        hits = torch.zeros((info.n_hits, 4), dtype=torch.float32, device="cuda")
        assert S.supa_fetch_hits(b, 0, info.n_hits, hits) == info.n_hits
        h = hits.cpu().numpy().astype(np.float64)
        sh = np.repeat(np.arange(n), np.diff(arr["offsets"]))
        np.testing.assert_allclose(np.bincount(sh, weights=h[:, 3], minlength=n), arr["layer_sum"].sum(1), rtol=1e-5)
        tags = torch.zeros(info.n_hits, dtype=torch.int64, device="cuda")
        S.supa_fetch_hit_tags(b, 0, info.n_hits, tags)
        t = tags.cpu().numpy()
        assert (t == 0).sum() > 0 and (t != 0).sum() > 0  # surrogate hits carry tag 0
        # within each shower the stepped hits come first
        first_zero = np.array([np.argmax(t[a:c] == 0) if (t[a:c] == 0).any() else c - a
                               for a, c in zip(arr["offsets"][:-1], arr["offsets"][1:])])
        for s in range(0, n, 97):
            seg = t[arr["offsets"][s]:arr["offsets"][s + 1]]
            assert np.all(seg[first_zero[s]:] == 0)
        grid = torch.zeros((n, 30, 64, 64), dtype=torch.float32, device="cuda")
        oor = torch.zeros(n, dtype=torch.float64, device="cuda")
        S.supa_voxelize(b, 0, n, grid, oor)
        np.testing.assert_allclose(grid.double().sum((1, 2, 3)).cpu().numpy() + oor.cpu().numpy(),
                                   arr["layer_sum"].sum(1), rtol=1e-4)
        # replay gives the same showers
        S.supa_simulate(b, d, n, 9)
        info2 = S.supa_batch_get_info(b)
        arr2 = {k: v.cpu().numpy() for k, v in S.info_arrays(info2).items()}
        assert info2.n_hits == info.n_hits and info2.n_diverted == info.n_diverted
        np.testing.assert_allclose(arr2["layer_sum"], arr["layer_sum"], rtol=1e-9, atol=1e-12)
    finally:
        S.supa_destroy_batch(b)
        S.supa_surrogate_destroy(sur)
        S.supa_destroy_geometry(gh)


@pytest.mark.parametrize("mode", [S.SUPA_SURROGATE_SAMPLE, S.SUPA_SURROGATE_MEAN])
def test_hybrid_matches_oracle(mode):
    """Same set-aside decisions and stepped hits as the FP64 oracle; the
    network's deposits agree within BF16 tolerance (per shower, per layer)."""
    import torch
    from oracle import hybrid
    g = inputs.supa_d(30, grid=64, roi_mode=inputs.ROI_AXIS)
    n = 300
    p = inputs.primaries(n, 11, e_lo=5.0, e_hi=60.0, theta_max_deg=30.0)
    vec = S.pack_mlp_params(inputs.mlp_init(3))
    params64 = [(W.astype(np.float64), b.astype(np.float64)) for W, b in S.unpack_mlp_params(vec)]
    gh = S.supa_init_geometry(g)
    sur = S.supa_surrogate_create(1024, vec)
    b = S.supa_batch_create([gh], n, {"record_tags": 1})
    try:
        S.supa_batch_set_surrogate(b, sur, E_S, 1_000_000, mode)
        S.supa_simulate(b, S.primaries_to_device(p), n, 13)
        info = S.supa_batch_get_info(b)
        arr = {k: v.cpu().numpy() for k, v in S.info_arrays(info).items()}
        hits = torch.zeros((info.n_hits, 4), dtype=torch.float32, device="cuda")
        tags = torch.zeros(info.n_hits, dtype=torch.int64, device="cuda")
        S.supa_fetch_hits(b, 0, info.n_hits, hits)
        S.supa_fetch_hit_tags(b, 0, info.n_hits, tags)
        h, t = hits.cpu().numpy(), tags.cpu().numpy().view(np.uint64)
    finally:
        S.supa_destroy_batch(b)
        S.supa_surrogate_destroy(sur)
        S.supa_destroy_geometry(gh)
    ora = oracle.simulate(g, p, 13, n_threads=8, e_s=E_S)
    div = ora["div"]
    dep = hybrid.deposits(div, params64, g, E_S, 13, mode=mode)
    # the same particles are set aside (float32 decisions on both sides)
    assert abs(info.n_diverted - len(div["E"])) <= max(2, 1e-3 * len(div["E"]))
    # stepped hits: same (slice, lineage) keys per shower
    sh = np.repeat(np.arange(n), np.diff(arr["offsets"]))
    stepped = t != 0
    same = 0
    for s in range(n):
        m = (sh == s) & stepped
        a = sorted(zip(np.rint(h[m, 2]).astype(int).tolist(), t[m].tolist()))
        o = ora["offsets"]
        bkeys = sorted(zip(ora["slice"][o[s]:o[s + 1]].tolist(), ora["lineage"][o[s]:o[s + 1]].tolist()))
        same += a == bkeys
    assert same >= n - 2
    # layer sums: oracle stepped part + network deposits
    ls = ora["layer_sum"].copy()
    for j in range(30):
        ok = div["layer"] + j < g.n_layers
        np.add.at(ls, (div["shower"][ok], div["layer"][ok] + j), dep["d"][ok, j])
    E0 = p["E"].astype(np.float64)
    err = np.abs(arr["layer_sum"] - ls).sum(1) / E0
    assert np.quantile(err, 0.99) < 3e-2, np.quantile(err, 0.99)
    np.testing.assert_allclose(arr["layer_sum"].sum(1), ls.sum(1), rtol=2e-2)
    assert abs((~stepped).sum() - len(dep["hits"])) <= 0.03 * len(dep["hits"])
    # surrogate hits (tag 0): per shower, energy-weighted centre and spread
    # around it (the displacements follow the network's rho_j and Philox)
    oh = dep["hits"]
    assert np.any(oh[:, 1:3] != 0)

    def moments(s_idx, x, y, e):
        W = np.bincount(s_idx, weights=e, minlength=n)
        mx = np.bincount(s_idx, weights=e * x, minlength=n) / np.maximum(W, 1e-30)
        my = np.bincount(s_idx, weights=e * y, minlength=n) / np.maximum(W, 1e-30)
        q = np.bincount(s_idx, weights=e * ((x - mx[s_idx]) ** 2 + (y - my[s_idx]) ** 2), minlength=n)
        return W, mx, my, q / np.maximum(W, 1e-30)

    sur = ~stepped
    Wg, mxg, myg, qg = moments(sh[sur], h[sur, 0].astype(np.float64), h[sur, 1].astype(np.float64),
                               h[sur, 3].astype(np.float64))
    Wo, mxo, myo, qo = moments(oh[:, 0].astype(int), oh[:, 1], oh[:, 2], oh[:, 4])
    has = Wo > 0.05 * E0
    assert has.sum() > n // 2
    # deposits carry the BF16 network's error (a few per cent, more for the
    # small ones near mu = 0), which moves an energy-weighted centre by about
    # that error times the spread over the square root of the hits
    dc = np.hypot(mxg - mxo, myg - myo)[has] / np.sqrt(qo[has])
    dq = np.abs(qg - qo)[has] / qo[has]
    assert np.quantile(dc, 0.99) < 5e-2, (np.quantile(dc, [0.5, 0.99]), np.median(np.sqrt(qo[has])))
    assert np.quantile(dq, 0.99) < 5e-2, np.quantile(dq, [0.5, 0.99])


def test_hybrid_queue_overflow_is_an_error():
    g = inputs.supa_d(30)
    p = inputs.primaries(200, 8, e_lo=50.0, e_hi=60.0)
    gh = S.supa_init_geometry(g)
    sur = _surrogate()
    b = S.supa_batch_create([gh], 200, {})
    try:
        S.supa_batch_set_surrogate(b, sur, E_S, 128)
        S.supa_simulate(b, S.primaries_to_device(p), 200, 1)
        with pytest.raises(S.SupaError) as ei:
            S.supa_batch_get_info(b)
        assert ei.value.code == S.SUPA_ERR_OVERFLOW
    finally:
        S.supa_destroy_batch(b)
        S.supa_surrogate_destroy(sur)
        S.supa_destroy_geometry(gh)


def test_exported_diverted_particles_match_the_oracles_set_aside():
    """supa_export_diverted: every particle the hybrid run queued, as a
    sub-shower primary (entry slice, energy, position, direction), equals the
    oracle's set-aside record of the same shower (matched by slice and
    energy; the queue order is not defined)."""
    import torch
    g = inputs.supa_d(30)
    n = 150
    p = inputs.primaries(n, 17, e_lo=5.0, e_hi=40.0, theta_max_deg=30.0)
    gh = S.supa_init_geometry(g)
    sur = _surrogate()
    b = S.supa_batch_create([gh], n, {})
    try:
        S.supa_batch_set_surrogate(b, sur, E_S, 1_000_000, S.SUPA_SURROGATE_MEAN)
        S.supa_simulate(b, S.primaries_to_device(p), n, 9)
        info = S.supa_batch_get_info(b)
        m = S.supa_export_diverted(b)
        assert m == info.n_diverted > 0
        buf = torch.zeros(m * 24, dtype=torch.uint8, device="cuda")
        assert S.supa_export_diverted(b, buf) == m
        ex = buf.cpu().numpy().view(inputs.PRIMARY_DTYPE)
    finally:
        S.supa_destroy_batch(b)
        S.supa_surrogate_destroy(sur)
        S.supa_destroy_geometry(gh)
    div = oracle.simulate(g, p, 9, n_threads=8, e_s=E_S)["div"]
    assert abs(len(div["E"]) - m) <= max(2, 1e-3 * m)
    k_ex = ex["geom"] >> 16
    assert np.all(ex["geom"] & 0xFFFF == 0)
    assert np.all(ex["E"] < E_S) and np.all(g.slice_to_layer[k_ex] >= 0)
    # match each exported particle to the oracle record of nearest energy
    # (energies are continuous: distinct up to float32 rounding)
    ux = np.sin(ex["theta"].astype(np.float64)) * np.cos(ex["phi"].astype(np.float64))
    uz = np.cos(ex["theta"].astype(np.float64))
    oe = np.argsort(div["E"])
    Eo = div["E"][oe]
    j = np.clip(np.searchsorted(Eo, ex["E"].astype(np.float64)), 1, len(Eo) - 1)
    j = np.where(np.abs(Eo[j - 1] - ex["E"]) < np.abs(Eo[j] - ex["E"]), j - 1, j)
    o = oe[j]
    # float32 stepping keeps an energy within ~1e-6 of FP64 after the ~8
    # splits from E0 down to E_s
    close = np.abs(div["E"][o] - ex["E"]) <= 3e-6 * ex["E"]
    assert close.mean() > 0.999
    # a nearest-energy pair is unambiguous where no other oracle energy is
    # within twice that
    gap = np.minimum(np.abs(np.diff(Eo, prepend=-1.0)), np.abs(np.diff(Eo, append=1e30)))[j]
    ok = close & (gap > 6e-6 * ex["E"])
    assert ok.mean() > 0.8
    assert np.array_equal(k_ex[ok], div["k"][o][ok])
    np.testing.assert_allclose(ex["x0"][ok], div["x"][o][ok], rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(ex["y0"][ok], div["y"][o][ok], rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(ux[ok], div["ux"][o][ok], atol=1e-5)
    np.testing.assert_allclose(uz[ok], div["uz"][o][ok], atol=1e-5)
