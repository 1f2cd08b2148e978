"""Sub-shower starts, the surrogate's training set, and the hybrid path
(plain stepping above E_s, network deposits below it)."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2202_05012_gb300 import inputs
from paper_2202_05012_gb300 import supa as S

from gpu_helpers import RTOL, compare, run_gpu

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
        t = tags.cpu().numpy().view(np.uint64)
        sur_hit = (t >> np.uint64(63)) == 1  # surrogate hits: lineage | 2^63
        assert sur_hit.sum() > 0 and (~sur_hit).sum() > 0
        assert np.all(t[~sur_hit] > 0)
        # within each shower the stepped hits come first
        first_sur = np.array([np.argmax(sur_hit[a:c]) if sur_hit[a:c].any() else c - a
                              for a, c in zip(arr["offsets"][:-1], arr["offsets"][1:])])
        for s in range(0, n, 97):
            seg = sur_hit[arr["offsets"][s]:arr["offsets"][s + 1]]
            assert np.all(seg[first_sur[s]:])
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


def bf16_forward_bound(params, X):
    """FP64 network outputs for X and an element-wise bound on how far the
    BF16 tensor-core network can be from them.  Each layer multiplies BF16
    inputs by BF16 weights (each rounded to nearest: relative error <= 2^-9,
    so a product is off by <= 2^-8 + 2^-18 of its magnitude) and accumulates
    at most 256 products in FP32 (<= 256 * 2^-24 of the sum of magnitudes,
    covered by the 2e-5 below); an error already in the inputs passes through
    |W|.  GELU changes an error by at most its largest slope, 1.13, and the
    kernel's tanh (tanh.approx.f32, relative error below 2^-10.9) moves
    GELU(z) = z (1 + tanh) / 2 by less than 2.5e-4 |z|.  The result is a
    worst case (all roundings aligned)."""
    u = 2.0 ** -8 + 2e-5
    h, dh = X, np.zeros_like(X)
    for i, (W, b) in enumerate(params):
        aW = np.abs(W)
        z = h @ W.T + b
        dz = u * (np.abs(h) @ aW.T) + dh @ aW.T
        if i == len(params) - 1:
            return z, dz
        h, dh = mlp.gelu(z), 1.13 * dz + 2.5e-4 * np.abs(z)


def _state_of_records(rec):
    """The diverted particles of exported records as the oracle's set-aside
    dict (directions from the stored slopes)."""
    tx, ty = rec["tx"].astype(np.float64), rec["ty"].astype(np.float64)
    nrm = np.sqrt(1.0 + tx * tx + ty * ty)
    return dict(shower=rec["shower"].astype(np.int64), k=rec["slice"].astype(np.int64),
                lineage=rec["lineage"].astype(np.int64), layer=rec["layer"].astype(np.int64),
                E=rec["E"].astype(np.float64), x=rec["x"].astype(np.float64), y=rec["y"].astype(np.float64),
                ux=tx / nrm, uy=ty / nrm, uz=1.0 / nrm)


@pytest.mark.parametrize("mode", [S.SUPA_SURROGATE_SAMPLE, S.SUPA_SURROGATE_MEAN])
def test_hybrid_matches_oracle_particle_by_particle(mode):
    """Element-wise parity of the surrogate side.  Every particle the GPU
    set aside is matched to the oracle's by (shower, slice, lineage); then
    for each one: its state against the FP64 stepping, the network's 90
    outputs against the FP64 network within the derived BF16 bound, its 30
    deposits against the oracle's deposit rule applied to those outputs, and
    each of its hits (tagged with its lineage) against the oracle's hit
    rule; finally every layer sum against the oracle's stepped deposits plus
    the surrogate deposits."""
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
        m = S.supa_export_surrogate(b)
        assert m == info.n_diverted > 1000
        buf = torch.zeros(m * S.DIVERTED_RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        assert S.supa_export_surrogate(b, buf) == m
        rec = buf.cpu().numpy().view(S.DIVERTED_RECORD_DTYPE)
        hits = torch.zeros((info.n_hits, 4), dtype=torch.float32, device="cuda")
        tags = torch.zeros(info.n_hits, dtype=torch.int64, device="cuda")
        S.supa_fetch_hits(b, 0, info.n_hits, hits)
        S.supa_fetch_hit_tags(b, 0, info.n_hits, tags)
        h, t = hits.cpu().numpy().astype(np.float64), tags.cpu().numpy().view(np.uint64)
    finally:
        S.supa_destroy_batch(b)
        S.supa_surrogate_destroy(sur)
        S.supa_destroy_geometry(gh)
    ora = oracle.simulate(g, p, 13, n_threads=8, e_s=E_S)
    div = ora["div"]
    # 1. the same particles are set aside (a float32 decision can flip one)
    okey = {(int(a), int(k), int(l)): i for i, (a, k, l) in enumerate(zip(div["shower"], div["k"], div["lineage"]))}
    gkey = [(int(a), int(k), int(l)) for a, k, l in zip(rec["shower"], rec["slice"], rec["lineage"])]
    assert len(set(gkey)) == m  # one record per particle
    both = np.array([k in okey for k in gkey])
    assert (~both).sum() <= max(2, 1e-3 * m) and abs(len(okey) - m) <= max(2, 1e-3 * m)
    gi = np.nonzero(both)[0]
    oi = np.array([okey[gkey[i]] for i in gi])
    # 2. their state: FP32 stepping against FP64
    np.testing.assert_allclose(rec["E"][gi], div["E"][oi], rtol=1e-5)
    assert np.array_equal(rec["layer"][gi], div["layer"][oi])
    assert np.all(np.abs(rec["x"][gi] - div["x"][oi]) <= RTOL * np.maximum(np.abs(div["x"][oi]), g.dz))
    assert np.all(np.abs(rec["y"][gi] - div["y"][oi]) <= RTOL * np.maximum(np.abs(div["y"][oi]), g.dz))
    np.testing.assert_allclose(rec["tx"][gi], div["ux"][oi] / div["uz"][oi], atol=2e-5)
    # 3. network outputs against the FP64 network on the features of the
    #    GPU's own state, within the derived BF16 bound
    st = _state_of_records(rec)
    ref, bound = bf16_forward_bound(params64, hybrid.features(st, g, E_S))
    got = np.concatenate([rec["lmu"], rec["s"], rec["rho"]], 1).astype(np.float64)
    err = np.abs(got - ref)
    assert np.all(err <= bound), (err / bound).max()
    assert np.sqrt(np.mean((err / bound) ** 2)) < 0.25  # far inside the worst case
    # 4. deposits: the oracle's rule applied to the GPU's outputs and state
    dep = hybrid.deposits(st, None, g, E_S, 13, mode=mode, out=got)
    E = st["E"][:, None]
    bad = np.any(np.abs(rec["dep"] - dep["d"]) > 1e-4 * dep["d"] + 1e-6 * E, axis=1)
    # a SAMPLE accept test evaluated within rounding of its boundary may flip
    assert bad.sum() <= (0 if mode == S.SUPA_SURROGATE_MEAN else max(1, 1e-3 * m)), np.nonzero(bad)[0][:5]
    assert np.array_equal(rec["n_hits"][~bad], (dep["d"][~bad] > 0).sum(1))
    if mode == S.SUPA_SURROGATE_SAMPLE:  # the draws do move the deposits away from the means
        mean = hybrid.deposits(st, None, g, E_S, 13, mode=S.SUPA_SURROGATE_MEAN, out=got)
        assert np.median(np.abs(dep["d"] - mean["d"]).sum(1) / st["E"]) > 1e-3
    # 5. surrogate hits: tagged with lineage | 2^63, keyed (shower, lineage, depth)
    sh = np.repeat(np.arange(n), np.diff(arr["offsets"]))
    is_sur = (t >> np.uint64(63)) == 1
    assert is_sur.sum() == rec["n_hits"].sum()
    lin = (t & np.uint64((1 << 63) - 1)).astype(np.int64)
    ghit = {(int(sh[i]), int(lin[i]), float(h[i, 2])): i for i in np.nonzero(is_sur)[0]}
    assert len(ghit) == is_sur.sum()
    oh = dep["hits"]
    clean = ~bad[oh[:, 6].astype(int)]
    keys = [(int(r[0]), int(st["lineage"][int(r[6])]), float(r[3])) for r in oh[clean]]
    assert all(k in ghit for k in keys)
    idx = np.array([ghit[k] for k in keys])
    ohc = oh[clean]
    pos_scale = np.maximum(np.abs(ohc[:, 1:3]), g.dz)
    assert np.all(np.abs(h[idx, 0:2] - ohc[:, 1:3]) <= 1e-5 * pos_scale)
    E_part = st["E"][ohc[:, 6].astype(int)]
    assert np.all(np.abs(h[idx, 3] - ohc[:, 4]) <= 1e-4 * ohc[:, 4] + 1e-6 * E_part)
    # 6. layer sums: the oracle's stepped deposits plus the GPU's surrogate
    #    deposits (exact fixed-point sums of float32 on the device)
    ls = ora["layer_sum"].copy()
    for j in range(30):
        ok = rec["layer"] + j < g.n_layers
        np.add.at(ls, (rec["shower"][ok], rec["layer"][ok] + j), rec["dep"][ok, j].astype(np.float64))
    E0 = p["E"].astype(np.float64)
    off = np.abs(arr["layer_sum"] - ls).max(1) > 1e-5 * E0
    assert off.sum() <= 2


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
