"""Surrogate workflow on top of the C ABI (orchestration only: every step
runs in the library's kernels).

  data = training_set(n, e_s, seed)            # plain-method sub-showers
  data = training_set_matched(geom, prims, e_s, n, seed)   # ... started from
                                               # the particles a workload diverts
  net, log = train(data, epochs, batch, lr)    # tcgen05 training epochs
  ... supa_batch_set_surrogate(batch, net, e_s, capacity) ...

Sub-showers start below E_s (energy log-uniform in [e_min, E_s], polar angle
U[0, 45 deg], start layer uniform, start slice uniform within it) in the
30-layer detector -- or, matched to a workload, from the particles its
showers divert; targets are their per-layer deposit fractions from the start
layer on and the mean lateral distances of those deposits from the
sub-shower's axis.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs
from . import supa as S

# Algorithmic FLOPs per sample of one training step of 6-256-256-256-90:
# forward 2 * sum(in * out), backward twice that (data and weight gradients,
# minus the unused input gradient of the first layer).
_LAYERS = [(6, 256), (256, 256), (256, 256), (256, 90)]
FWD_FLOPS = sum(2 * a * b for a, b in _LAYERS)
TRAIN_FLOPS = FWD_FLOPS + 2 * FWD_FLOPS - 2 * 6 * 256


def training_set(n: int, e_s: float, seed: int, n_layers: int = 30, device="cuda"):
    """Simulate n sub-showers with the plain kernel and build (X, Y) on the GPU."""
    import torch
    g = inputs.supa_d(n_layers)
    prims, _ = inputs.subshower_primaries(n, seed, e_lo=g.e_min, e_hi=e_s, n_layers=n_layers)
    gh = S.supa_init_geometry(g)
    b = S.supa_batch_create([gh], n, {"max_hits": n * 80 + (4 << 20), "lpt_order": 1})
    try:
        d = S.primaries_to_device(prims, device)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.supa_simulate(b, d, n, seed)
        info = S.supa_batch_get_info(b)
        x = torch.empty((n, 6), dtype=torch.float32, device=device)
        y = torch.empty((n, 60), dtype=torch.float32, device=device)
        S.supa_build_training_set(b, e_s, x, y)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        return dict(x=x, y=y, n=n, e_s=e_s, seconds=dt, steps=info.n_steps)
    finally:
        S.supa_destroy_batch(b)
        S.supa_destroy_geometry(gh)


def training_set_matched(geom, prims, e_s: float, n_max: int, seed: int, device="cuda",
                         shower_batch: int = 50_000):
    """A training set matched to what the network replaces: the showers
    `prims` of a workload run in hybrid mode (any network: only the queue of
    particles diverted below e_s is used), those particles become sub-shower
    primaries (supa_export_diverted), and each is simulated by the plain
    method in the same geometry.  At most n_max samples; the set does not
    depend on the order the particles were diverted in."""
    import torch
    gh = S.supa_init_geometry(geom)
    net = S.supa_surrogate_create(128, S.pack_mlp_params(inputs.mlp_init(0)))
    d = S.primaries_to_device(prims, device)
    mean_e = float(prims["E"].mean())
    cap = int(4.0 * mean_e / e_s * shower_batch) + (1 << 20)
    hb = S.supa_batch_create([gh], shower_batch,
                             {"max_hits": int(shower_batch * max(400, 40 * mean_e)) + (8 << 20), "lpt_order": 1})
    chunks, got = [], 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    try:
        S.supa_batch_set_surrogate(hb, net, e_s, cap, S.SUPA_SURROGATE_MEAN)
        for j in range(0, len(prims), shower_batch):
            m = min(shower_batch, len(prims) - j)
            S.supa_simulate(hb, d[j * 24:(j + m) * 24], m, seed, j)
            S.supa_batch_get_info(hb)
            k_all = S.supa_export_diverted(hb)
            buf = torch.empty(k_all * 24, dtype=torch.uint8, device=device)
            S.supa_export_diverted(hb, buf)
            # the queue's order depends on which warp diverted first: sort the
            # records by their bytes, so that the set (and the Philox streams of
            # its plain simulation, keyed by position) is the same every run,
            # then keep a seeded random subset where the set is full
            rec = buf.view(torch.int32).view(k_all, 6)
            for col in range(5, -1, -1):
                rec = rec[torch.sort(rec[:, col], stable=True).indices]
            k = min(k_all, n_max - got)
            if k < k_all:
                gen = torch.Generator().manual_seed(seed * 7919 + j)
                rec = rec[torch.randperm(k_all, generator=gen)[:k].to(device)]
            chunks.append(rec.contiguous().view(torch.uint8).view(-1))
            got += k
            if got >= n_max:
                break
    finally:
        S.supa_destroy_batch(hb)
        S.supa_surrogate_destroy(net)
    del d
    sub = torch.cat(chunks)
    del chunks
    n = sub.numel() // 24
    b = S.supa_batch_create([gh], n, {"max_hits": n * 80 + (4 << 20), "lpt_order": 1})
    try:
        S.supa_simulate(b, sub, n, seed + 1)
        info = S.supa_batch_get_info(b)
        x = torch.empty((n, 6), dtype=torch.float32, device=device)
        y = torch.empty((n, 60), dtype=torch.float32, device=device)
        S.supa_build_training_set(b, e_s, x, y)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        return dict(x=x, y=y, n=n, e_s=e_s, seconds=dt, steps=info.n_steps, matched=True)
    finally:
        S.supa_destroy_batch(b)
        S.supa_destroy_geometry(gh)


def train(data: dict, epochs: int = 20, batch: int = 16384, lr: float = 1e-3, seed: int = 0, init_seed: int = 1,
          lr_final: float | None = None, average_from: int | None = None):
    """Adam epochs on the GPU; returns (network handle, log).  With lr_final
    the learning rate decays geometrically from lr to lr_final over the
    epochs; with average_from the network's final parameters are the average
    of the parameters after every Adam step from that epoch on (iterate
    averaging)."""
    import torch
    net = S.supa_surrogate_create(batch, S.pack_mlp_params(inputs.mlp_init(init_seed)))
    n = data["n"]
    steps = n // batch
    losses = []
    acc = torch.zeros(1, dtype=torch.float64, device="cuda")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    for ep in range(epochs):
        acc.zero_()
        lr_ep = lr if lr_final is None or epochs < 2 else lr * (lr_final / lr) ** (ep / (epochs - 1))
        if average_from is not None and ep == average_from:
            S.supa_surrogate_average(net, S.SUPA_AVERAGE_START)
        S.supa_surrogate_train_epoch(net, data["x"], data["y"], n, seed * 1000 + ep, lr_ep, acc)
        losses.append(acc)  # read after the loop (no synchronisation per epoch)
        acc = torch.zeros(1, dtype=torch.float64, device="cuda")
    if average_from is not None and average_from < epochs:
        S.supa_surrogate_average(net, S.SUPA_AVERAGE_APPLY)
        S.supa_surrogate_average(net, S.SUPA_AVERAGE_STOP)
    ev1.record()
    torch.cuda.synchronize()
    S.supa_surrogate_check(net)
    ms = ev0.elapsed_time(ev1)
    per_epoch = [float(l.item()) / steps for l in losses]
    flops = TRAIN_FLOPS * steps * batch * epochs
    return net, dict(epochs=epochs, batch=batch, lr=lr, lr_final=lr_final, average_from=average_from,
                     steps_per_epoch=steps, seconds=ms / 1000.0,
                     seconds_per_epoch=ms / 1000.0 / epochs, loss_per_epoch=per_epoch,
                     tflops=flops / (ms / 1000.0) / 1e12, samples_per_s=steps * batch * epochs / (ms / 1000.0))


# Profile comparison of a hybrid run against the plain run on the same
# showers.  Lateral profiles are taken in PROFILE_BINS rings of width
# PROFILE_RMAX / PROFILE_BINS around the incidence axis, the last ring open
# to infinity, so that every deposit is counted.
PROFILE_BINS, PROFILE_RMAX = 129, 16.0
PROFILE_GROUP = 0.02


def energy_groups(ref, frac: float = PROFILE_GROUP):
    """Consecutive bins of the reference profile merged into groups that each
    hold at least `frac` of its total (greedily from the first bin; the
    remainder joins the last group): returns the group index of every bin.
    The groups cover every bin, so an error taken over them covers all the
    energy."""
    ref = np.asarray(ref, dtype=np.float64)
    tot = ref.sum()
    gid = np.zeros(len(ref), dtype=np.int64)
    g, acc = 0, 0.0
    for i, v in enumerate(ref):
        gid[i] = g
        acc += v
        if acc >= frac * tot and i < len(ref) - 1:
            g, acc = g + 1, 0.0
    if acc < frac * tot and g > 0:  # the remainder joins the last full group
        gid[gid == g] = g - 1
    return gid


def profile_errors(ref, got, frac: float = PROFILE_GROUP) -> dict:
    """Largest relative deviation of a profile from the reference over groups
    of consecutive bins holding >= frac of the reference's energy each (all
    bins, all the energy), for the longitudinal (per layer) and the lateral
    (per ring, last ring open) mean profiles; the relative deviation of the
    mean total deposit; and, for reference, the largest per-bin deviation
    over single layers holding >= 0.5 % of the energy."""
    (rl, rr), (gl, gr) = ref, got

    def grouped(a, b):
        gid = energy_groups(a, frac)
        sa = np.bincount(gid, weights=a)
        sb = np.bincount(gid, weights=b)
        return float(np.max(np.abs(sb - sa) / sa)), int(gid.max() + 1)

    lo, n_lo = grouped(rl, gl)
    la, n_la = grouped(rr, gr)
    m = rl >= 0.005 * rl.sum()
    return {"longitudinal": lo, "lateral": la, "total_deposit": float(abs(gl.sum() - rl.sum()) / rl.sum()),
            "group_fraction": frac, "groups": [n_lo, n_la], "energy_covered": 1.0,
            "longitudinal_per_layer": float(np.max(np.abs(gl[m] - rl[m]) / rl[m]))}
