"""Helpers for the GPU parity tests: run the library through its C ABI and
match its hits to the oracle's by (shower, slice, lineage id)."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2202_05012_gb300 import supa as S

# Tolerances (FP32 stepping against the FP64 oracle): positions within 1e-5
# relative to max(|x|, dz), energies within 1e-5 relative, FP64 layer sums of
# FP32 deposits within 1e-5 relative.  Decisions that a rounding difference
# can flip (the energy cut, the escape cut) are counted, not compared.
RTOL = 1e-5
MAX_FLIP_RATE = 1e-4


def run_gpu(geoms, prims, seed, *, shower_id_base=0, cfg=None, tags=True):
    import torch
    gh = [S.supa_init_geometry(g) for g in geoms]
    n = len(prims)
    c = {"record_tags": 1 if tags else 0}
    c.update(cfg or {})
    b = None
    try:
        d = S.primaries_to_device(prims)
        b = S.supa_batch_create(gh, max(n, 1), c)
        S.supa_simulate(b, d, n, seed, shower_id_base)
        info = S.supa_batch_get_info(b)
        nh = info.n_hits
        hits = torch.zeros((max(nh, 1), 4), dtype=torch.float32, device="cuda")
        assert S.supa_fetch_hits(b, 0, nh, hits) == nh
        out = {k: v.cpu().numpy().copy() for k, v in S.info_arrays(info).items()}
        out["counts"] = out["counts"].view(np.uint32)
        out["steps"] = out["steps"].view(np.uint32)
        h = hits[:nh].cpu().numpy()
        out.update(x=h[:, 0], y=h[:, 1], z=h[:, 2], E=h[:, 3], n_hits=nh, n_steps=info.n_steps)
        if tags:
            t = torch.zeros(max(nh, 1), dtype=torch.int64, device="cuda")
            assert S.supa_fetch_hit_tags(b, 0, nh, t) == nh
            out["lineage"] = t[:nh].cpu().numpy().view(np.uint64)
        torch.cuda.synchronize()
        return out
    finally:
        if b is not None:
            S.supa_destroy_batch(b)
        for g in gh:
            S.supa_destroy_geometry(g)


def _shower_ids(offsets):
    return np.repeat(np.arange(len(offsets) - 1), np.diff(offsets))


def compare(gpu, ora, geoms, prims, pos_rtol=RTOL):
    """Per-shower comparison; returns a dict of statistics and asserts the
    tolerances on every shower whose decisions all agree.

    pos_rtol: position tolerance.  A step moves x by dz * u_x / u_z, so an
    FP32 error e in the direction becomes e / u_z in the slope: near grazing
    incidence (u_z down to the escape cut) callers pass a looser bound."""
    n = len(prims)
    gidx = prims["geom"].astype(np.int64) & 0xFFFF  # high bits: start slice
    dz = np.array([geoms[i].dz for i in gidx])
    # canonical order within each shower: (slice, lineage)
    g_sh = _shower_ids(gpu["offsets"])
    g_slice = np.rint(gpu["z"] / dz[g_sh]).astype(np.int64)
    g_ord = np.lexsort((gpu["lineage"], g_slice, g_sh))
    o_sh = _shower_ids(ora["offsets"])
    g_cnt = np.diff(gpu["offsets"])
    o_cnt = np.diff(ora["offsets"])
    assert np.array_equal(g_cnt, gpu["counts"].astype(np.int64))
    # showers whose hit keys agree exactly
    clean = g_cnt == o_cnt
    gs = dict(sh=g_sh[g_ord], k=g_slice[g_ord], lin=gpu["lineage"][g_ord], x=gpu["x"][g_ord], y=gpu["y"][g_ord],
              E=gpu["E"][g_ord])
    # vectorised key comparison over showers with equal counts
    same_len = np.repeat(clean, o_cnt)
    g_same = np.repeat(clean, g_cnt)
    ok_keys = np.ones(n, dtype=bool)
    ok_keys[~clean] = False
    ko = (ora["slice"][same_len], ora["lineage"][same_len])
    kg = (gs["k"][g_same], gs["lin"][g_same])
    diff = (ko[0] != kg[0]) | (ko[1] != kg[1])
    bad_sh = np.unique(o_sh[same_len][diff])
    ok_keys[bad_sh] = False
    n_flip_showers = int((~ok_keys).sum())
    # symmetric difference of keys over flipped showers (decisions that differ)
    sym = 0
    for s in np.nonzero(~ok_keys)[0]:
        a = set(zip(ora["slice"][ora["offsets"][s]:ora["offsets"][s + 1]].tolist(),
                    ora["lineage"][ora["offsets"][s]:ora["offsets"][s + 1]].tolist()))
        m = gs["sh"] == s
        b = set(zip(gs["k"][m].tolist(), gs["lin"][m].tolist()))
        sym += len(a ^ b)
    total_steps = int(ora["steps"].sum())
    # values on clean showers
    sel_o = np.repeat(ok_keys, o_cnt)
    sel_g = np.repeat(ok_keys, g_cnt)
    xo, yo, Eo = ora["x"][sel_o], ora["y"][sel_o], ora["E"][sel_o]
    xg, yg, Eg = gs["x"][sel_g].astype(np.float64), gs["y"][sel_g].astype(np.float64), gs["E"][sel_g].astype(np.float64)
    dzh = dz[o_sh[sel_o]]
    zo = ora["z"][sel_o]
    zg = gpu["z"][g_ord][sel_g].astype(np.float64)
    err_x = np.abs(xg - xo) / np.maximum(np.abs(xo), dzh)
    err_y = np.abs(yg - yo) / np.maximum(np.abs(yo), dzh)
    err_E = np.abs(Eg - Eo) / np.abs(Eo)
    stats = dict(
        n_showers=n, n_flip_showers=n_flip_showers, flipped_keys=sym, total_steps=total_steps,
        flip_rate=sym / max(total_steps, 1),
        max_err_x=float(err_x.max(initial=0)), max_err_y=float(err_y.max(initial=0)),
        max_err_E=float(err_E.max(initial=0)),
    )
    assert np.array_equal(zg, zo), "hit depths must be the slice planes exactly"
    assert stats["max_err_x"] <= pos_rtol and stats["max_err_y"] <= pos_rtol, stats
    assert stats["max_err_E"] <= RTOL, stats
    assert stats["flip_rate"] < MAX_FLIP_RATE, stats
    # per-shower bookkeeping on clean showers
    np.testing.assert_array_equal(gpu["steps"][ok_keys].astype(np.int64), ora["steps"][ok_keys])
    L = ora["layer_sum"].shape[1]
    np.testing.assert_allclose(gpu["layer_sum"][ok_keys][:, :L], ora["layer_sum"][ok_keys], rtol=RTOL, atol=1e-12)
    for key in ("dead", "leak", "escape"):
        np.testing.assert_allclose(gpu[key][ok_keys], ora[key][ok_keys], rtol=RTOL, atol=1e-9)
    # energy bookkeeping on every shower: FP32 rounding bound per split
    E0 = prims["E"].astype(np.float64)
    tot = gpu["layer_sum"].sum(1) + gpu["dead"] + gpu["leak"] + gpu["escape"]
    bound = (ora["n_splits"] + 1) * 2.0 ** -22 * E0 + 1e-12
    assert np.all(np.abs(tot - E0) <= bound), np.max(np.abs(tot - E0) / bound)
    lo, lg = ora["layer_sum"][ok_keys], gpu["layer_sum"][ok_keys][:, :L]
    nz = lo > 0
    stats.update(
        max_err_layer_sum=float((np.abs(lg - lo)[nz] / lo[nz]).max(initial=0)),
        max_err_conservation=float((np.abs(tot - E0) / E0).max(initial=0)),
        hit_counts_equal=float(np.mean(g_cnt == o_cnt)),
        steps_equal=float(np.mean(gpu["steps"].astype(np.int64) == ora["steps"])),
    )
    return stats


def oracle_multi(geoms, prims, seed, base):
    """Oracle for a batch mixing geometries: each shower with its own geometry
    and its global id (the random stream depends on nothing else)."""
    parts = []
    for i in range(len(prims)):
        g = geoms[int(prims["geom"][i])]
        parts.append(oracle.simulate(g, prims[i:i + 1], seed, shower_id_base=base + i))
    Lmax = max(g.n_layers for g in geoms)
    out = {}
    for key in ("x", "y", "z", "E", "slice", "lineage"):
        out[key] = np.concatenate([p[key] for p in parts])
    out["offsets"] = np.concatenate([[0], np.cumsum([p["offsets"][-1] for p in parts])]).astype(np.int64)
    for key in ("steps", "dead", "leak", "escape", "n_splits", "max_depth"):
        out[key] = np.concatenate([p[key] for p in parts])
    ls = np.zeros((len(prims), Lmax))
    for i, p in enumerate(parts):
        ls[i, :p["layer_sum"].shape[1]] = p["layer_sum"][0]
    out["layer_sum"] = ls
    return out
