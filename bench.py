#!/usr/bin/env python
"""Benchmark of the SUPA hot path on GB300: showers/s through
simulate -> downsample -> fetch of the point clouds.

Workload (default): 1,000,000 showers, E ~ U[1,100], polar angle U[0,30 deg],
entry within +-1 cell, 30 layers x 3 slices, 30 x 64 x 64 images centred on
the shower axis, hits handed out in 64M-hit chunks.  One step = one pass of
the whole path over the batch with inputs resident in HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl supa|reference]

Under torchrun each rank develops its own batch (weak scaling, no data-path
collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "showers/s"
FETCH_CHUNK = 64 << 20  # hits per supa_fetch_hits call (1 GiB of float4)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="supa", choices=["supa", "reference"])
    ap.add_argument("--workload", default="plain30",
                    choices=["plain10", "plain30", "mixed4", "plain50", "surrogate", "hybrid", "forward", "train"])
    ap.add_argument("--e-s-sweep", type=float, nargs="+", default=[0.2, 0.5, 1.0, 2.0, 5.0])
    ap.add_argument("--showers", type=int, default=0, help="override the batch size")
    ap.add_argument("--voxel-chunk", type=int, default=32768)
    ap.add_argument("--fetch-chunk", type=int, default=FETCH_CHUNK)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-hybrid", action="store_true", help="skip the plain-vs-surrogate comparison")
    ap.add_argument("--e-s", type=float, default=2.0, help="surrogate cutoff energy E_s")
    ap.add_argument("--train-samples", type=int, default=10_000_000)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--lr", type=float, default=2e-3, help="initial learning rate")
    ap.add_argument("--batch", type=int, default=16384, help="training minibatch rows (a multiple of 128)")
    ap.add_argument("--lr-final", type=float, default=5e-5, help="learning rate of the last epoch (geometric decay)")
    ap.add_argument("--average-from", type=int, default=-1,
                    help="epoch from which the network is the average of the steps' parameters (-1: off)")
    ap.add_argument("--train-showers", type=int, default=0,
                    help="showers of the workload (another seed) whose diverted particles seed the training set")
    ap.add_argument("--train-set", default="matched", choices=["matched", "generic"],
                    help="hybrid workload: sub-showers from diverted particles, or generic starts (smaller)")
    ap.add_argument("--c5-showers", type=int, default=10_000_000,
                    help="showers of the 50-layer hybrid comparison in the default run (0: skip it)")
    ap.add_argument("--c5-e-s-low", type=float, default=1.5,
                    help="second, lower E_s of the 50-layer hybrid comparison (0: only --e-s)")
    ap.add_argument("--no-mixed4", action="store_true", help="skip the uneven-batch measurement in the default run")
    ap.add_argument("--pipeline", type=int, default=1,
                    help="sub-batches per step; >1 overlaps simulation of one with downsampling of the previous")
    return ap.parse_args()


def workload(name: str, n: int):
    from paper_2202_05012_gb300 import inputs
    if name == "plain10":
        g, p = inputs.workload_plain10(n or 1000)
        return g, p, 0, dict(workload="plain SUPA, 1k showers, E U[1,10], 10 layers, 10x32x32", seed=0)
    if name == "plain50":
        g, p = inputs.workload_plain50(n or 200_000)
        return g, p, 4, dict(workload="plain SUPA, E log-U[10,1000], 0-45 deg, 50 layers, 50x128x128", seed=4)
    g, p = inputs.workload_plain30(n or 1_000_000)
    return g, p, 1, dict(workload="plain SUPA, 1M showers, E U[1,100], 0-30 deg, +-1 cell entry, 30 layers, "
                                  "30x64x64 axis-centred images, point cloud written by the image pass", seed=1)


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", delete=False, suffix=".csv")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        rows = [l.split(",") for l in open(self.f.name).read().strip().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for name, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def stored_traffic(kernel: str, workload_key: str, showers_per_launch: int):
    """DRAM bytes per launch from a committed ncu capture, valid only while the
    kernel source is unchanged (sha256 of its translation unit), scaled from
    the captured launch to one of `showers_per_launch` showers (the traffic
    grows in proportion to the showers processed)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))[kernel][workload_key]
    except (OSError, ValueError, KeyError):
        return None
    src = os.path.join(ROOT, "paper_2202_05012_gb300", "csrc", rec["source"])
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    if sha != rec["sha256"]:
        return None
    return rec["bytes_per_launch"] * showers_per_launch / rec["showers_per_launch"]


# ------------------------------------------------------------------ oracle ---

def oracle_sample(geom, prims, seed, seconds, chunk=500):
    """Time the FP64 oracle (simulate on all host cores, then downsample) on
    consecutive chunks of the workload until `seconds` have passed."""
    import oracle
    threads = os.cpu_count() or 1
    done, t0 = 0, time.perf_counter()
    steps = 0
    while done < len(prims):
        p = prims[done:done + chunk]
        r = oracle.simulate(geom, p, seed, shower_id_base=done, n_threads=threads)
        rx, ry = oracle.roi_origins(geom, p)
        oracle.voxelize(r["x"], r["y"], r["z"], r["E"], r["offsets"], geom, rx, ry)
        steps += int(r["steps"].sum())
        done += len(p)
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return done / dt, steps / dt, done, dt, threads


def cpu_baseline_fresh(args):
    """The oracle timed as the reference arm times it, in a fresh process: in
    this one the host threads of the GPU run would compete with its threads
    and slow it several-fold."""
    import subprocess
    cmd = [sys.executable, os.path.abspath(__file__), "--impl", "reference", "--workload", args.workload,
           "--steps", "1", "--warmup", "1", "--cpu-seconds", str(args.cpu_seconds)]
    if args.showers:
        cmd += ["--showers", str(args.showers)]
    res = subprocess.run(cmd, capture_output=True, text=True, check=True)
    line = json.loads([l for l in res.stdout.splitlines() if l.startswith("{")][-1])
    cb = dict(line["cpu_baseline"])
    cb["sample"] += f"; {line['ms_per_step'] / 1000.0:.1f} s, timed in a fresh process"
    return cb


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    geom, prims, seed, conf = workload(args.workload, args.showers)
    per_step = max(1, int(args.cpu_seconds / max(args.steps, 1)))
    for _ in range(args.warmup):
        oracle_sample(geom, prims[:200], seed, 0.0, chunk=200)
    vals, n_done, t_tot = [], 0, 0.0
    for k in range(args.steps):
        v, sps, done, dt, threads = oracle_sample(geom, prims, seed, per_step)
        vals.append(v)
        n_done += done
        t_tot += dt
    value = n_done / t_tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "showers/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t_tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": conf,
        "cpu_baseline": {"value": value, "unit": "showers/s", "cores": threads, "kind": "oracle",
                         "sample": f"first {done} showers of the workload per step (simulate on {threads} threads, "
                                   f"downsample single-threaded)"},
        "e2e": {"value": value, "unit": "showers/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm ---

class Pipeline:
    """One step = the whole path over the batch, cut into sub-batches that
    alternate between two library batches: stream A simulates sub-batch j+1
    while stream B downsamples and fetches sub-batch j.  The step kernel is
    ALU-bound and the downsampling kernel HBM-bound, so each SM runs both:
    2 step-kernel blocks (80 registers) and 1 downsampling CTA per SM."""

    def __init__(self, S, gh, d_prim, n, n_sub, seed, base, hits_per_shower_cap, V, L, ny, nx, FC):
        import torch
        self.S, self.seed, self.base, self.n = S, seed, base, n
        self.sub = -(-n // n_sub)
        self.ranges = [(j, min(n, j + self.sub)) for j in range(0, n, self.sub)]
        cfg = {"max_hits": int(self.sub * hits_per_shower_cap) + (8 << 20), "lpt_order": 1,
               "blocks_per_sm": 2, "voxel_ctas_per_sm": 1}
        self.batches = [S.supa_batch_create([gh], self.sub, cfg) for _ in range(2)]
        self.d_prim = d_prim
        self.V = min(V, self.sub)
        self.grid = torch.empty((self.V, L, ny, nx), dtype=torch.float32, device="cuda")
        self.oor = torch.empty(self.V, dtype=torch.float64, device="cuda")
        self.FC = FC
        self.fbuf = torch.empty((FC, 4), dtype=torch.float32, device="cuda")
        self.sA, self.sB = torch.cuda.Stream(), torch.cuda.Stream()
        self.ev_sim = [torch.cuda.Event() for _ in range(2)]
        self.ev_out = [torch.cuda.Event() for _ in range(2)]

    def _sim(self, j, prim_src):
        a, b = self.ranges[j]
        if j >= 2:
            self.sA.wait_event(self.ev_out[j % 2])  # the pool of batch j%2 is free again
        self.S.supa_simulate(self.batches[j % 2], prim_src[a * 24:b * 24], b - a, self.seed, self.base + a,
                             stream=self.sA)
        self.ev_sim[j % 2].record(self.sA)

    def step(self, prim_src=None, host_hits=None, host_ls=None):
        """Returns (particle-steps, hits, kernel launches).  With host buffers
        the hits and layer sums of every sub-batch are read back to them."""
        import torch
        S = self.S
        prim_src = self.d_prim if prim_src is None else prim_src
        cur = torch.cuda.current_stream()
        self.sA.wait_stream(cur)
        self.sB.wait_stream(cur)
        steps = hits = launches = 0
        self._sim(0, prim_src)
        for j, (a, b) in enumerate(self.ranges):
            if j + 1 < len(self.ranges):
                self._sim(j + 1, prim_src)
            bt = self.batches[j % 2]
            self.sB.wait_event(self.ev_sim[j % 2])
            info = S.supa_batch_get_info(bt, stream=self.sB)
            launches += 1 + 3 + 3
            m = b - a
            for c0 in range(0, m, self.V):
                S.supa_voxelize(bt, c0, min(m, c0 + self.V), self.grid, self.oor, stream=self.sB)
                launches += 1
            if host_hits is None:
                for h0 in range(0, info.n_hits, self.FC):
                    S.supa_fetch_hits(bt, h0, self.FC, self.fbuf, stream=self.sB)
                    launches += 1
            else:
                got = 0
                while got < info.n_hits:
                    k = S.supa_fetch_hits(bt, got, self.FC, host_hits[hits + got:], dst_is_device=False,
                                          stream=self.sB)
                    got += k
                    launches += 1
                with torch.cuda.stream(self.sB):
                    host_ls[a:b].copy_(S.info_arrays(info)["layer_sum"], non_blocking=True)
            self.ev_out[j % 2].record(self.sB)
            steps += info.n_steps
            hits += info.n_hits
        cur.wait_stream(self.sA)
        cur.wait_stream(self.sB)
        return steps, hits, launches

    def close(self):
        for b in self.batches:
            self.S.supa_destroy_batch(b)


def run_supa(args):
    """Pipelined step (default): see Pipeline.  The kernels' rooflines and
    phase times come from an isolated, serial pass over one sub-batch."""
    import torch
    import torch.distributed as dist

    from paper_2202_05012_gb300 import supa as S

    if args.pipeline <= 1:
        return run_supa_serial(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    geom, prims, seed, conf = workload(args.workload, args.showers)
    n = len(prims)
    base = rank * n
    if world > 1:
        from paper_2202_05012_gb300 import inputs
        prims = inputs.primaries(n, seed + 1000 * rank, e_lo=float(prims["E"].min()), e_hi=float(prims["E"].max()))
    L, ny, nx = geom.n_layers, geom.ny, geom.nx
    gh = S.supa_init_geometry(geom)
    cap = {"plain10": 400, "plain30": 1500, "plain50": 9000}[args.workload]
    d_prim = S.primaries_to_device(prims)
    pipe = Pipeline(S, gh, d_prim, n, args.pipeline, seed, base, cap, args.voxel_chunk, L, ny, nx, args.fetch_chunk)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        pipe.step()
    torch.cuda.synchronize()

    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    launches = n_steps = n_hits = 0
    for _ in range(args.steps):
        st, hi, nl = pipe.step()
        n_steps, n_hits, launches = st, hi, launches + nl
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    elapsed_ms = t_start.elapsed_time(t_end)
    if world > 1:
        t = torch.tensor([elapsed_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    value = args.steps * n * world / (elapsed_ms / 1000.0)
    hits_per_shower = n_hits / n

    # isolated serial pass on one sub-batch with the full launch shapes:
    # simulate timing and the downsampling kernel's roofline
    a, b = pipe.ranges[0]
    m = b - a
    iso = S.supa_batch_create([gh], pipe.sub, {"max_hits": int(pipe.sub * cap) + (8 << 20), "lpt_order": 1})
    V = pipe.V
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    sim_ms = []
    for rep in range(3):
        e[0].record(stream)
        S.supa_simulate(iso, d_prim[a * 24:b * 24], m, seed, base + a)
        e[1].record(stream)
        S.supa_batch_get_info(iso)
        sim_ms.append(e[0].elapsed_time(e[1]))
    info = S.supa_batch_get_info(iso)
    vox = []
    for rep in range(3):
        for c0 in range(0, m - V + 1, V):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            S.supa_voxelize(iso, c0, c0 + V, pipe.grid, pipe.oor)
            e1.record(stream)
            vox.append((e0, e1))
    torch.cuda.synchronize()
    vox_ms = [x.elapsed_time(y) for x, y in vox]
    S.supa_destroy_batch(iso)
    sim_iso = min(sim_ms)
    avg_vox = sum(vox_ms) / len(vox_ms)
    pk, pk_kind = peaks()
    bytes_per_shower = L * ny * nx * 4 + 16 * (info.n_hits / m) + 8
    achieved = V * bytes_per_shower / (avg_vox / 1000.0) / 1e9
    traffic = stored_traffic("supa_voxel_kernel", args.workload, V)
    roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / pk["hbm_gbs"], "traffic": traffic, "kernel": "supa_voxel_kernel",
            "peak_source": pk_kind, "bytes_per_shower": bytes_per_shower, "showers_per_launch": V,
            "measured": "isolated launches, CUDA events on the launching stream"}
    out = {
        "metric": METRIC, "value": value, "unit": "showers/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(conf, showers=n, layers=L, grid=[L, ny, nx], fetch_chunk_hits=args.fetch_chunk,
                       voxel_chunk_showers=V, sub_batches=len(pipe.ranges),
                       l2="inputs larger than L2 (hit pool and image chunks >> 129 MB)",
                       parallelism=f"replicas x{world}"),
        "particle_steps_per_s": n_steps * args.steps * world / (elapsed_ms / 1000.0),
        "hits_per_shower": hits_per_shower, "steps_per_shower": n_steps / n,
        "phase_ms_isolated": {"simulate_per_1M": sim_iso * 1e6 / m, "voxelize_per_1M": avg_vox * 1e6 / V,
                              "step_total_pipelined": elapsed_ms / args.steps},
        "simulate_showers_per_s": m / (sim_iso / 1000.0),
        "simulate_particle_steps_per_s": info.n_steps / (sim_iso / 1000.0),
        "roofline": roof, "gpu_launches": launches, "clocks": clk,
    }
    if not args.no_e2e:
        h_prim = torch.from_numpy(np.ascontiguousarray(prims).view(np.uint8)).pin_memory()
        d_prim2 = torch.empty_like(h_prim, device="cuda")
        h_hits = torch.empty((int(n_hits * 1.02) + 4096, 4), dtype=torch.float32, pin_memory=True)
        h_ls = torch.empty((n, L), dtype=torch.float64, pin_memory=True)

        def e2e_step():
            d_prim2.copy_(h_prim, non_blocking=True)
            r = pipe.step(prim_src=d_prim2, host_hits=h_hits, host_ls=h_ls)
            torch.cuda.synchronize()
            return r

        for _ in range(max(1, args.warmup)):
            e2e_step()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            st, hi, _ = e2e_step()
        dt = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([dt], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        out["e2e"] = {"value": args.steps * n * world / dt, "unit": "showers/s", "h2d_bytes_per_step": n * 24,
                      "d2h_bytes_per_step": hi * 16 + n * L * 8}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_fresh(args)
    pipe.close()
    S.supa_destroy_geometry(gh)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_supa_serial(args):
    import torch
    import torch.distributed as dist

    from paper_2202_05012_gb300 import supa as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    geom, prims, seed, conf = workload(args.workload, args.showers)
    n = len(prims)
    base = rank * n  # each rank develops its own showers (global ids differ)
    if world > 1:
        from paper_2202_05012_gb300 import inputs
        prims = inputs.primaries(n, seed + 1000 * rank, e_lo=float(prims["E"].min()), e_hi=float(prims["E"].max()))
    L, ny, nx = geom.n_layers, geom.ny, geom.nx
    gh = S.supa_init_geometry(geom)
    max_hits = int(n * {"plain10": 400, "plain30": 1500, "plain50": 9000}[args.workload]) + (8 << 20)
    b = S.supa_batch_create([gh], n, {"max_hits": max_hits, "lpt_order": 1})
    d_prim = S.primaries_to_device(prims)
    V = min(args.voxel_chunk, n)
    grid = torch.empty((V, L, ny, nx), dtype=torch.float32, device="cuda")
    oor = torch.empty(V, dtype=torch.float64, device="cuda")
    FC = args.fetch_chunk
    fbuf = torch.empty((FC, 4), dtype=torch.float32, device="cuda")
    # the point cloud of a step, in shower order (written by the image pass)
    hbuf = torch.empty((max_hits, 4), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step(ev=None):
        if ev is not None:
            ev["sim0"].record(stream)
        S.supa_simulate(b, d_prim, n, seed, base)
        if ev is not None:
            ev["sim1"].record(stream)
        # the images follow the simulation in stream order: no host synchronisation in the step
        launches = 1 + 3 + 3  # step kernel, offset scan, energy-ordered queue
        vox_ms = 0.0
        for c0 in range(0, n, V):
            c1 = min(n, c0 + V)
            if ev is not None:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            # images and point cloud of the chunk in one pass over its hits
            S.supa_voxelize_fetch(b, c0, c1, grid, oor, hbuf)
            launches += 1
            if ev is not None:
                e1.record(stream)
                ev["vox"].append((e0, e1, c1 - c0))
        return launches

    for _ in range(args.warmup):
        step()
    info = S.supa_batch_get_info(b)
    torch.cuda.synchronize()
    n_hits, n_steps = info.n_hits, info.n_steps
    hits_per_shower = n_hits / n

    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    evs = []
    t_start.record(stream)
    launches = 0
    for _ in range(args.steps):
        ev = {"sim0": torch.cuda.Event(enable_timing=True), "sim1": torch.cuda.Event(enable_timing=True), "vox": []}
        launches += step(ev)
        evs.append(ev)
    t_end.record(stream)
    torch.cuda.synchronize()
    info = S.supa_batch_get_info(b)  # status and totals of the last timed step
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    elapsed_ms = t_start.elapsed_time(t_end)
    if world > 1:
        t = torch.tensor([elapsed_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    sim_ms = sum(e["sim0"].elapsed_time(e["sim1"]) for e in evs) / args.steps
    vox_launch = [(a.elapsed_time(c), m) for e in evs for (a, c, m) in e["vox"]]
    vox_ms = sum(x for x, _ in vox_launch) / args.steps
    value = args.steps * n * world / (elapsed_ms / 1000.0)

    # roofline of the dominant kernel (the downsampling kernel, HBM-write bound):
    # algorithmic bytes = images written + hits read + out-of-region sums
    pk, pk_kind = peaks()
    full = [(x, m) for x, m in vox_launch if m == V] or vox_launch
    avg_ms = sum(x for x, _ in full) / len(full)
    # images written + hits read + hits written (point cloud) + out-of-region sum
    bytes_per_shower = L * ny * nx * 4 + 32 * hits_per_shower + 8
    achieved = full[0][1] * bytes_per_shower / (avg_ms / 1000.0) / 1e9
    traffic = stored_traffic("supa_voxel_kernel", args.workload, full[0][1])
    roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / pk["hbm_gbs"], "traffic": traffic, "kernel": "supa_voxel_kernel",
            "peak_source": pk_kind, "bytes_per_shower": bytes_per_shower, "showers_per_launch": full[0][1]}

    out = {
        "metric": METRIC, "value": value, "unit": "showers/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(conf, showers=n, layers=L, grid=[L, ny, nx],
                       voxel_chunk_showers=V, l2="inputs larger than L2 (hit pool and image chunks >> 129 MB)",
                       parallelism=f"replicas x{world}"),
        "particle_steps_per_s": n_steps * args.steps * world / (elapsed_ms / 1000.0),
        "hits_per_shower": hits_per_shower, "steps_per_shower": n_steps / n,
        "phase_ms": {"simulate": sim_ms, "voxelize": vox_ms, "step_total": elapsed_ms / args.steps},
        "simulate_showers_per_s": n / (sim_ms / 1000.0),
        "simulate_particle_steps_per_s": n_steps / (sim_ms / 1000.0),
        "roofline": roof, "gpu_launches": launches, "clocks": clk,
    }

    out["shower_shapes"] = shape_timing(S, b, n, L, hits_per_shower)
    if world == 1:
        out["calogan_multires"] = calogan_timing(S)
    if not args.no_e2e:
        out["e2e"] = e2e(args, S, b, geom, prims, seed, base, n, V, grid, oor, world)
    if world == 1 and args.workload == "plain30" and not args.no_hybrid:
        plain = {"step_ms": elapsed_ms / args.steps, "simulate_ms": sim_ms, "steps": n_steps,
                 "profiles": profiles_of(S, b, n, L)}
        out["hybrid"] = hybrid_compare(args, S, gh, geom, prims, d_prim, n, seed, base, V, grid, oor, fbuf, plain)
    if world == 1 and args.workload == "plain30" and (not args.no_mixed4 or (not args.no_hybrid and args.c5_showers)):
        # free the 1M-shower batch and its buffers for the larger workloads
        S.supa_destroy_batch(b)
        b = None
        del grid, oor, fbuf, hbuf
        torch.cuda.empty_cache()
        if not args.no_mixed4:
            out["mixed4"] = mixed4_measure(S, 4_000_000, steps=3, warmup=1)
        if not args.no_hybrid and args.c5_showers:
            out["hybrid_c5"] = hybrid_c5(args, S)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_fresh(args)
    if b is not None:
        S.supa_destroy_batch(b)
    S.supa_destroy_geometry(gh)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def profiles_of(S, b, n, L):
    """Mean longitudinal (per-layer energy / E0) and lateral (energy / E0 per
    ring around the incidence axis, the last ring open) profiles of the
    batch."""
    import torch
    from paper_2202_05012_gb300.surrogate_train import PROFILE_BINS, PROFILE_RMAX
    lo = torch.zeros(L, dtype=torch.float64, device="cuda")
    la = torch.zeros(PROFILE_BINS, dtype=torch.float64, device="cuda")
    S.supa_profiles(b, 0, n, PROFILE_BINS, PROFILE_RMAX, lo, la)
    return lo.cpu().numpy() / n, la.cpu().numpy() / n


def profile_errors(ref, got):
    """Largest relative profile deviations over groups of bins holding >= 2 %
    of the plain run's energy each, covering all of it (see
    surrogate_train.profile_errors)."""
    from paper_2202_05012_gb300.surrogate_train import profile_errors as pe
    return pe(ref, got)


def profile_binning():
    from paper_2202_05012_gb300.surrogate_train import PROFILE_BINS, PROFILE_GROUP, PROFILE_RMAX
    return {"lateral_rings": PROFILE_BINS, "ring_width": PROFILE_RMAX / PROFILE_BINS,
            "last_ring": f"r >= {PROFILE_RMAX * (PROFILE_BINS - 1) / PROFILE_BINS:g} (open)",
            "error": f"largest relative deviation over groups of consecutive bins holding >= "
                     f"{PROFILE_GROUP:.0%} of the plain run's energy each (all bins: 100 % of the energy)"}


def hybrid_run(S, gh, prims, d_prim, n, seed, base, net, e_s, sub, V, grid, oor, fbuf, L, profiles=False, mode=0,
               voxelize=True):
    """The whole path in hybrid mode over n showers in sub-batches: simulate
    (stepping above E_s, network below), images and point cloud in one pass.  Returns timings
    and (optionally) accumulated profiles."""
    import torch
    mean_e = float(prims["E"][:n].mean())
    cap = int(4.0 * mean_e / e_s * sub) + (1 << 20)
    hb_hits = int(sub * max(400, 40 * mean_e)) + (8 << 20)
    hb = S.supa_batch_create([gh], sub, {"max_hits": hb_hits, "lpt_order": 1})
    S.supa_batch_set_surrogate(hb, net, e_s, cap, mode)
    from paper_2202_05012_gb300.surrogate_train import PROFILE_BINS, PROFILE_RMAX
    lo = torch.zeros(L, dtype=torch.float64, device="cuda")
    la = torch.zeros(PROFILE_BINS, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    sim_ms = 0.0
    steps = diverted = hits = 0
    FC = fbuf.shape[0]
    hbuf = torch.empty((hb_hits, 4), dtype=torch.float32, device="cuda") if voxelize else None  # point cloud
    torch.cuda.synchronize()
    ev[0].record(stream)
    for j in range(0, n, sub):
        m = min(sub, n - j)
        ev[2].record(stream)
        S.supa_simulate(hb, d_prim[j * 24:(j + m) * 24], m, seed, base + j)
        ev[3].record(stream)
        info = S.supa_batch_get_info(hb)
        sim_ms += ev[2].elapsed_time(ev[3])
        steps += info.n_steps
        diverted += info.n_diverted
        hits += info.n_hits
        if voxelize:
            for c0 in range(0, m, V):
                S.supa_voxelize_fetch(hb, c0, min(m, c0 + V), grid, oor, hbuf)
        else:
            for h0 in range(0, info.n_hits, FC):
                S.supa_fetch_hits(hb, h0, FC, fbuf)
        if profiles:
            S.supa_profiles(hb, 0, m, PROFILE_BINS, PROFILE_RMAX, lo, la)
    ev[1].record(stream)
    torch.cuda.synchronize()
    total_ms = ev[0].elapsed_time(ev[1])
    S.supa_destroy_batch(hb)
    out = dict(total_ms=total_ms, simulate_ms=sim_ms, steps=steps, diverted=diverted, hits=hits, queue_capacity=cap)
    if profiles:
        out["profiles"] = (lo.cpu().numpy() / n, la.cpu().numpy() / n)
    return out


def matched_training(args, T, make, e_s, mean_e):
    """Training set from the particles that showers of the same workload
    (another seed) divert below e_s, each simulated as a plain sub-shower;
    then the Adam epochs.  Returns (net, training log)."""
    # at least ~E / E_s diverted particles per shower; the set stops growing
    # once train_samples are in
    n_show = args.train_showers or int(min(2_000_000, max(50_000, 2.5 * args.train_samples * e_s / mean_e)))
    g_t, p_t = make(n_show)
    data = T.training_set_matched(g_t, p_t, e_s, args.train_samples, seed=5)
    net, log = T.train(data, epochs=args.epochs, batch=args.batch, lr=args.lr, lr_final=args.lr_final,
                       average_from=args.average_from if args.average_from >= 0 else None)
    return net, {"samples": data["n"], "data_seconds": data["seconds"], "training_showers": n_show,
                 "set": "matched: diverted particles of the workload's showers (seed 11/14), stepped plainly",
                 **log}


def hybrid_compare(args, S, gh, geom, prims, d_prim, n, seed, base, V, grid, oor, fbuf, plain):
    """Train the surrogate on sub-showers started from the particles the
    workload diverts, run the same showers in hybrid mode, and compare
    throughput and profiles with the plain run."""
    from paper_2202_05012_gb300 import inputs
    from paper_2202_05012_gb300 import surrogate_train as T
    net, tlog = matched_training(args, T, lambda m: inputs.workload_plain30(m, seed=11), args.e_s,
                                 float(prims["E"].mean()))
    sub = 125_000
    L = geom.n_layers
    out = {"e_s": args.e_s, "plain_showers_per_s": n / (plain["step_ms"] / 1000.0),
           "plain_simulate_showers_per_s": n / (plain["simulate_ms"] / 1000.0),
           "plain_particle_steps_per_shower": plain["steps"] / n,
           "profile_binning": profile_binning(),
           "training": tlog,
           "note": "hybrid timed in 125k-shower sub-batches (network over each sub-batch's queue); plain as one "
                   "batch; same showers and seeds"}
    for mode, name in ((1, "mean"), (0, "sample")):
        hybrid_run(S, gh, prims, d_prim, min(n, sub), seed, base, net, args.e_s, sub, V, grid, oor, fbuf, L,
                   mode=mode)  # warm-up
        prof = hybrid_run(S, gh, prims, d_prim, n, seed, base, net, args.e_s, sub, V, grid, oor, fbuf, L, True,
                          mode=mode)
        timed = hybrid_run(S, gh, prims, d_prim, n, seed, base, net, args.e_s, sub, V, grid, oor, fbuf, L, mode=mode)
        out[name] = {"showers_per_s": n / (timed["total_ms"] / 1000.0),
                     "simulate_showers_per_s": n / (timed["simulate_ms"] / 1000.0),
                     "particle_steps_per_shower": timed["steps"] / n, "diverted_per_shower": timed["diverted"] / n,
                     "profile_error": profile_errors(plain["profiles"], prof["profiles"])}
    S.supa_surrogate_destroy(net)
    return out


def run_surrogate(args):
    """Surrogate training (10M plain-method sub-showers below E_s, 20 epochs)
    and the hybrid run of the 50-layer workload (50 layers, E log-uniform
    [10,1000], 0-45 deg) against the plain run on the same seeds, for a sweep
    of E_s: showers/s (simulate only; images excluded to keep the sweep
    short) and profile errors."""
    import torch

    from paper_2202_05012_gb300 import inputs
    from paper_2202_05012_gb300 import supa as S
    from paper_2202_05012_gb300 import surrogate_train as T
    from paper_2202_05012_gb300.surrogate_train import PROFILE_BINS, PROFILE_RMAX

    torch.cuda.set_device(0)
    n5 = args.showers or 100_000
    g5, p5 = inputs.workload_plain50(n5)
    gh = S.supa_init_geometry(g5)
    d5 = S.primaries_to_device(p5)
    L = g5.n_layers
    V = 1024
    grid = torch.empty((V, L, g5.ny, g5.nx), dtype=torch.float32, device="cuda")
    oor = torch.empty(V, dtype=torch.float64, device="cuda")
    fbuf = torch.empty((args.fetch_chunk, 4), dtype=torch.float32, device="cuda")
    sub = 25_000
    # plain reference on the same showers
    pb = S.supa_batch_create([gh], sub, {"max_hits": sub * 30_000 + (8 << 20), "lpt_order": 1})
    lo = torch.zeros(L, dtype=torch.float64, device="cuda")
    la = torch.zeros(PROFILE_BINS, dtype=torch.float64, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plain_ms = 0.0
    plain_steps = 0
    for j in range(0, n5, sub):
        m = min(sub, n5 - j)
        e0.record()
        S.supa_simulate(pb, d5[j * 24:(j + m) * 24], m, 4, j)
        e1.record()
        info = S.supa_batch_get_info(pb)
        plain_ms += e0.elapsed_time(e1)
        plain_steps += info.n_steps
        S.supa_profiles(pb, 0, m, PROFILE_BINS, PROFILE_RMAX, lo, la)
    torch.cuda.synchronize()
    plain_prof = (lo.cpu().numpy() / n5, la.cpu().numpy() / n5)
    S.supa_destroy_batch(pb)
    out = {"metric": METRIC, "workload": "surrogate training (10M samples x 20 epochs) + hybrid 50-layer showers vs plain, E_s sweep",
           "showers": n5, "plain": {"simulate_showers_per_s": n5 / (plain_ms / 1000.0),
                                       "particle_steps_per_shower": plain_steps / n5}, "sweep": []}
    for e_s in args.e_s_sweep:
        net, tlog = matched_training(args, T, lambda m: inputs.workload_plain50(m, seed=14), e_s, float(p5["E"].mean()))
        row = {"e_s": e_s, "training": tlog}
        # sub-batches small enough that the queue (about 4 E / E_s particles
        # per shower, ~1 KB each with outputs, deposits and hits) stays < 32 GB
        sub_h = max(1000, min(sub, int(32e6 * e_s / (4.0 * float(p5["E"].mean())))))
        for mode, name in ((1, "mean"), (0, "sample")):
            prof = hybrid_run(S, gh, p5, d5, n5, 4, 0, net, e_s, sub_h, V, grid, oor, fbuf, L, True, mode=mode,
                              voxelize=False)
            timed = hybrid_run(S, gh, p5, d5, n5, 4, 0, net, e_s, sub_h, V, grid, oor, fbuf, L, mode=mode,
                               voxelize=False)
            row[name] = {"simulate_showers_per_s": n5 / (timed["simulate_ms"] / 1000.0),
                         "particle_steps_per_shower": timed["steps"] / n5,
                         "diverted_per_shower": timed["diverted"] / n5,
                         "profile_error": profile_errors(plain_prof, prof["profiles"])}
        S.supa_surrogate_destroy(net)
        out["sweep"].append(row)
        print(json.dumps(row), flush=True)
    S.supa_destroy_geometry(gh)
    print(json.dumps(out), flush=True)


def calogan_timing(S, n=200_000):
    """Per-layer grids at several resolutions: showers of the CaloGAN-like
    detector (E U[1,100], normal incidence at the origin) imaged at 1x, 2x
    and 3x (3x96 / 12x12 / 12x6 cells at 1x) from one pass over the hits;
    showers/s and the achieved bandwidth of algorithmic bytes (hits read
    once, images written)."""
    import torch

    from paper_2202_05012_gb300 import inputs
    g = inputs.supa_calogan()
    p = inputs.primaries(n, 71, e_lo=1.0, e_hi=100.0)
    gh = S.supa_init_geometry(g)
    b = S.supa_batch_create([gh], n, {"max_hits": n * 1500 + (8 << 20), "lpt_order": 1})
    try:
        S.supa_simulate(b, S.primaries_to_device(p), n, 71)
        info = S.supa_batch_get_info(b)
        grids, factors = inputs.calogan_grids(), [1, 2, 3]
        C = S.supa_layer_images_cells(grids, factors)
        img = torch.empty((n, C), dtype=torch.float32, device="cuda")
        oor = torch.empty((n, len(factors)), dtype=torch.float64, device="cuda")
        S.supa_voxelize_layers(b, 0, n, grids, factors, img, oor)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        e0.record()
        for _ in range(reps):
            S.supa_voxelize_layers(b, 0, n, grids, factors, img, oor)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        per = 4 * C + 16 * info.n_hits / n + 8 * len(factors)
        return {"showers": n, "factors": factors, "cells_per_shower": C, "showers_per_s": n / (ms / 1000.0),
                "ms": ms, "bytes_per_shower": per, "achieved_gbs": n * per / (ms / 1000.0) / 1e9,
                "hits_per_shower": info.n_hits / n, "kernel": "supa_grid_kernel"}
    finally:
        S.supa_destroy_batch(b)
        S.supa_destroy_geometry(gh)


def shape_timing(S, b, n, L, hits_per_shower):
    """The shower shape variables (Sec. 5.1, App. A.1) of every shower of the
    last simulation, outside the timed step: showers/s and the achieved
    bandwidth of algorithmic bytes (hits read once, FP64 layer sums, features
    written)."""
    import torch
    lf = torch.empty((n, L, 18), dtype=torch.float32, device="cuda")
    sf = torch.empty((n, 5), dtype=torch.float32, device="cuda")
    S.supa_shower_shapes(b, 0, n, lf, sf)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    reps = 3
    for _ in range(reps):
        S.supa_shower_shapes(b, 0, n, lf, sf)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    per = 16 * hits_per_shower + 8 * L + 4 * (18 * L + 5)
    return {"showers_per_s": n / (ms / 1000.0), "ms": ms, "bytes_per_shower": per,
            "achieved_gbs": n * per / (ms / 1000.0) / 1e9, "kernel": "supa_shape_kernel"}


def e2e(args, S, b, geom, prims, seed, base, n, V, grid, oor, world):
    """Same metric through the public API with host buffers: primaries copied
    from pinned host memory each step, the point cloud (all hits, written by
    the image pass chunk by chunk) and the per-shower FP64 layer sums read
    back to pinned host memory.  Each chunk's hits travel to the host on a
    second stream (copy engines) as soon as its images are made, while the
    next chunks are made and while the next step simulates; two host
    buffers alternate, so a step's results stay intact while the step after
    it runs.  Images stay on the device, consumed chunk by chunk.  Every copy
    of the timed steps has finished when the clock stops."""
    import torch
    import torch.distributed as dist
    h_prim = torch.from_numpy(np.ascontiguousarray(prims).view(np.uint8)).pin_memory()
    d_prim = torch.empty_like(h_prim, device="cuda")
    info = S.supa_batch_get_info(b)
    cap = int(info.n_hits * 1.05) + 1024
    h_hits = [torch.empty((cap, 4), dtype=torch.float32, pin_memory=True) for _ in range(2)]
    d_hits = torch.empty((cap, 4), dtype=torch.float32, device="cuda")
    h_ls = [torch.empty((n, geom.n_layers), dtype=torch.float64, pin_memory=True) for _ in range(2)]
    cur = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    ls_read = torch.cuda.Event()    # the batch's layer sums are on the host
    hits_read = torch.cuda.Event()  # the device hit buffer is on the host
    ls_read.record(side)
    hits_read.record(side)
    h2d = d2h = 0
    it = 0
    chunk_idx = torch.tensor(list(range(0, n, V)) + [n], dtype=torch.int64, device="cuda")

    def step():
        nonlocal h2d, d2h, it
        hh, hl = h_hits[it % 2], h_ls[it % 2]
        it += 1
        d_prim.copy_(h_prim, non_blocking=True)
        cur.wait_event(ls_read)  # the simulation rewrites the layer sums
        S.supa_simulate(b, d_prim, n, seed, base)
        inf = S.supa_batch_get_info(b)
        side.wait_stream(cur)
        with torch.cuda.stream(side):
            hl.copy_(S.info_arrays(inf)["layer_sum"], non_blocking=True)
            ls_read.record(side)
        # first hit of each image chunk (and the end), for the chunks' copies
        bnd = S.info_arrays(inf)["offsets"][chunk_idx].cpu().tolist()
        cur.wait_event(hits_read)  # the image pass rewrites the device hit buffer
        for j, c0 in enumerate(range(0, n, V)):
            S.supa_voxelize_fetch(b, c0, min(n, c0 + V), grid, oor, d_hits)
            a, z = bnd[j], bnd[j + 1]
            if z > a:
                side.wait_stream(cur)
                with torch.cuda.stream(side):
                    hh[a:z].copy_(d_hits[a:z], non_blocking=True)
        hits_read.record(side)
        h2d = h_prim.numel()
        d2h = inf.n_hits * 16 + hl.numel() * 8

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([dt], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dt = float(t.item())
    return {"value": args.steps * n * world / dt, "unit": "showers/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h}


def tail_metrics(t) -> dict:
    """Load balance of one persistent launch from its warps' (start, end)
    global times: the launch span, the time from the last-but-one warp
    running out of showers to the last one, and the fraction of warp time
    idle in the last 10 % of the span."""
    t = np.asarray(t, dtype=np.int64)
    t0, t1 = int(t[:, 0].min()), int(t[:, 1].max())
    span = max(1, t1 - t0)
    ends = np.sort(t[:, 1])
    w0 = t1 - 0.1 * span
    busy = np.clip(np.minimum(t[:, 1], t1) - np.maximum(t[:, 0], w0), 0, None).sum()
    return {"launch_ms": span / 1e6, "tail_last_but_one_ms": (t1 - int(ends[-2])) / 1e6,
            "idle_fraction_last_10pct": float(1.0 - busy / (len(t) * 0.1 * span)), "warps": int(len(t))}


def mixed4_measure(S, n: int, steps: int, warmup: int, clocks: Clocks | None = None) -> dict:
    """Uneven batch: n showers, E log-uniform [1,1000] (multiplicity spans
    ~1000x), geometries of 10/20/30/50 layers mixed in each persistent
    launch; launch shape chosen by the autotuner; each 1M-shower launch
    replayed from a captured CUDA graph.  Simulation only (hits and FP64
    layer sums).  The tail comes from the warps' start and end times of one
    untimed replay of every launch."""
    import torch

    from paper_2202_05012_gb300 import inputs

    sub = min(n, 1_000_000)
    geoms, prims = inputs.workload_mixed4(n)
    gh = [S.supa_init_geometry(g) for g in geoms]
    d_prim = S.primaries_to_device(prims)
    cfg = {"lpt_order": 1, "max_hits": int(sub * 5000) + (16 << 20)}
    tuned, tune_ms = S.supa_autotune(gh, d_prim, sub, seed=2, cfg=cfg)
    b = S.supa_batch_create(gh, sub, dict(tuned, record_warp_times=1))
    graphs = []
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    for j in range(0, n, sub):
        m = min(sub, n - j)
        view = d_prim[j * 24:(j + m) * 24]
        with torch.cuda.stream(s):
            S.supa_simulate(b, view, m, 2, j)  # warm the launch path before capture
            S.supa_batch_get_info(b)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
                S.supa_simulate(b, view, m, 2, j)
            graphs.append(g)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()

    def step():
        st = hi = 0
        for g in graphs:
            g.replay()
            info = S.supa_batch_get_info(b)
            st += info.n_steps
            hi += info.n_hits
        return st, hi

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.start()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(steps):
        n_steps, n_hits = step()
    t1.record()
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks is not None else None
    ms = t0.elapsed_time(t1)
    tails = []
    for g in graphs:
        g.replay()
        S.supa_batch_get_info(b)
        tails.append(tail_metrics(S.supa_batch_warp_times(b)))
    S.supa_destroy_batch(b)
    for g in gh:
        S.supa_destroy_geometry(g)
    return {"workload": "uneven batch: 4M showers, E log-U[1,1000], 10/20/30/50-layer geometries mixed per "
                        "launch, graph-captured 1M-shower launches, autotuned", "showers": n,
            "showers_per_launch": sub, "steps": steps, "warmup": warmup, "ms_per_step": ms / steps,
            "showers_per_s": steps * n / (ms / 1000.0), "particle_steps_per_s": steps * n_steps / (ms / 1000.0),
            "hits_per_shower": n_hits / n, "steps_per_shower": n_steps / n,
            "launch_config": {k: v for k, v in tuned.items() if k != "record_warp_times"},
            "autotune_sample_ms": tune_ms, "gpu_launches": steps * len(graphs) * (1 + 3 + 3),
            "tail_per_launch": tails,
            "tail_mean": {k: float(np.mean([t[k] for t in tails])) for k in tails[0]}, "clocks": clk}


def run_mixed4(args):
    """The uneven batch (see mixed4_measure) as the JSON line."""
    import torch

    from paper_2202_05012_gb300 import supa as S

    torch.cuda.set_device(0)
    n = args.showers or 4_000_000
    m = mixed4_measure(S, n, args.steps, args.warmup, Clocks(0))
    out = {
        "metric": METRIC, "value": m["showers_per_s"], "unit": "showers/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": m["workload"], "showers": n, "showers_per_launch": m["showers_per_launch"],
                   "launch_config": m["launch_config"], "autotune_sample_ms": m["autotune_sample_ms"]},
        "particle_steps_per_s": m["particle_steps_per_s"], "hits_per_shower": m["hits_per_shower"],
        "steps_per_shower": m["steps_per_shower"], "gpu_launches": m["gpu_launches"], "clocks": m["clocks"],
        "tail_mean": m["tail_mean"],
    }
    print(json.dumps(out), flush=True)


def c5_pass(S, gh, p, d, n, seed, sub, V, grid, oor, hits_per_shower, net=None, e_s=0.0, mode=1):
    """The whole path over n showers of the 50-layer workload in sub-batches
    of `sub`: simulate (plain, or hybrid with `net` below e_s), then images
    and point cloud of every chunk of V showers in one pass.  Each
    sub-batch's work is bracketed by CUDA events (the whole path, and the
    simulation alone); the profiles are accumulated between sub-batches,
    outside the events."""
    import torch

    from paper_2202_05012_gb300.surrogate_train import PROFILE_BINS, PROFILE_RMAX
    L = grid.shape[1]
    mean_e = float(p["E"][:n].mean())
    max_hits = int(sub * hits_per_shower) + (8 << 20)
    hb = S.supa_batch_create([gh], sub, {"max_hits": max_hits, "lpt_order": 1})
    try:
        if net is not None:
            S.supa_batch_set_surrogate(hb, net, e_s, int(4.0 * mean_e / e_s * sub) + (1 << 20), mode)
        hbuf = torch.empty((max_hits, 4), dtype=torch.float32, device="cuda")
        lo = torch.zeros(L, dtype=torch.float64, device="cuda")
        la = torch.zeros(PROFILE_BINS, dtype=torch.float64, device="cuda")
        evs = []
        steps = diverted = hits = 0
        for j in range(0, n, sub):
            m = min(sub, n - j)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record()
            S.supa_simulate(hb, d[j * 24:(j + m) * 24], m, seed, j)
            ev[1].record()
            for c0 in range(0, m, V):
                S.supa_voxelize_fetch(hb, c0, min(m, c0 + V), grid, oor, hbuf)
            ev[2].record()
            evs.append(ev)
            info = S.supa_batch_get_info(hb)
            steps += info.n_steps
            diverted += info.n_diverted
            hits += info.n_hits
            S.supa_profiles(hb, 0, m, PROFILE_BINS, PROFILE_RMAX, lo, la)
        torch.cuda.synchronize()
        total_ms = sum(e[0].elapsed_time(e[2]) for e in evs)
        sim_ms = sum(e[0].elapsed_time(e[1]) for e in evs)
        return {"showers_per_s": n / (total_ms / 1000.0), "simulate_showers_per_s": n / (sim_ms / 1000.0),
                "particle_steps_per_s": steps / (sim_ms / 1000.0), "particle_steps_per_shower": steps / n,
                "diverted_per_shower": diverted / n, "hits_per_shower": hits / n, "ms": total_ms,
                "simulate_ms": sim_ms, "sub_batch_showers": sub,
                "profiles": (lo.cpu().numpy() / n, la.cpu().numpy() / n)}
    finally:
        S.supa_destroy_batch(hb)


def hybrid_c5(args, S) -> dict:
    """The surrogate on its own workload: 10M showers, seed 4, E log-uniform
    [10,1000], 0-45 deg, 50 layers, 50 x 128 x 128 images (written chunk by
    chunk with the point cloud), run plainly and with the network below E_s
    in both modes on the same seeds; the network is trained first on 10M
    sub-showers started from the particles showers of the same workload
    (another seed) divert, 20 epochs.  The same again at the lower cutoff
    --c5-e-s-low (fewer particles diverted: less speed-up, smaller errors)
    under "low_e_s"."""
    import torch

    from paper_2202_05012_gb300 import inputs
    from paper_2202_05012_gb300 import surrogate_train as T
    n = args.c5_showers
    g5, p5 = inputs.workload_plain50(n)
    gh = S.supa_init_geometry(g5)
    d5 = S.primaries_to_device(p5)
    L = g5.n_layers
    V = 2048
    grid = torch.empty((V, L, g5.ny, g5.nx), dtype=torch.float32, device="cuda")
    oor = torch.empty(V, dtype=torch.float64, device="cuda")
    mean_e = float(p5["E"].mean())
    net, tlog = matched_training(args, T, lambda m: inputs.workload_plain50(m, seed=14), args.e_s, mean_e)
    out = {"workload": f"hybrid 50-layer showers: {n} showers, seed 4, E log-U[10,1000], 0-45 deg, 50 layers, "
                       "50x128x128 images and point cloud, plain vs surrogate on the same seeds",
           "showers": n, "e_s": args.e_s, "profile_binning": profile_binning(),
           "training": {k: v for k, v in tlog.items() if k != "loss_per_epoch"},
           "training_loss_last_epoch": tlog["loss_per_epoch"][-1]}
    try:
        # a short pass of each kind first (launch paths, allocations)
        c5_pass(S, gh, p5, d5, 20_000, 4, 20_000, V, grid, oor, 9000)
        plain = c5_pass(S, gh, p5, d5, n, 4, 250_000, V, grid, oor, 9000)
        ref = plain.pop("profiles")
        out["plain"] = plain
        sub_h = 100_000

        def both_modes(net, e_s, dst):
            for mode, name in ((S.SUPA_SURROGATE_MEAN, "mean"), (S.SUPA_SURROGATE_SAMPLE, "sample")):
                c5_pass(S, gh, p5, d5, 20_000, 4, 20_000, V, grid, oor, max(400, 40 * mean_e), net, e_s, mode)
                r = c5_pass(S, gh, p5, d5, n, 4, sub_h, V, grid, oor, max(400, 40 * mean_e), net, e_s, mode)
                r["profile_error"] = profile_errors(ref, r.pop("profiles"))
                r["vs_plain"] = {"showers_per_s": r["showers_per_s"] / plain["showers_per_s"],
                                 "simulate_showers_per_s": r["simulate_showers_per_s"] / plain["simulate_showers_per_s"]}
                dst[name] = r

        both_modes(net, args.e_s, out)
        if args.c5_e_s_low > 0:
            S.supa_surrogate_destroy(net)
            net = None
            net, tlog2 = matched_training(args, T, lambda m: inputs.workload_plain50(m, seed=14), args.c5_e_s_low,
                                          mean_e)
            low = {"e_s": args.c5_e_s_low,
                   "training": {k: v for k, v in tlog2.items() if k != "loss_per_epoch"},
                   "training_loss_last_epoch": tlog2["loss_per_epoch"][-1]}
            both_modes(net, args.c5_e_s_low, low)
            out["low_e_s"] = low
    finally:
        if net is not None:
            S.supa_surrogate_destroy(net)
        S.supa_destroy_geometry(gh)
        del grid, oor, d5
        torch.cuda.empty_cache()
    return out


def run_hybrid(args):
    """Hybrid simulation alone (50-layer showers, stepping above E_s, the network
    and its deposits and hits below it; no images), W warm-up and K timed
    supa_simulate calls: the short workload the hybrid kernels are profiled
    on."""
    import torch

    from paper_2202_05012_gb300 import inputs
    from paper_2202_05012_gb300 import supa as S
    from paper_2202_05012_gb300 import surrogate_train as T

    torch.cuda.set_device(0)
    n = args.showers or 20_000
    g, p = inputs.workload_plain50(n)
    mean_e = float(p["E"].mean())
    if args.train_set == "matched":
        net, tlog = matched_training(args, T, lambda m: inputs.workload_plain50(m, seed=14), args.e_s, mean_e)
    else:
        data = T.training_set(args.train_samples, args.e_s, seed=3, n_layers=30)
        net, tlog = T.train(data, epochs=args.epochs, lr=args.lr, lr_final=args.lr_final,
                            average_from=args.average_from if args.average_from >= 0 else None)
        tlog = {"samples": data["n"], "set": "generic sub-shower starts", **tlog}
        del data
    gh = S.supa_init_geometry(g)
    d = S.primaries_to_device(p)
    b = S.supa_batch_create([gh], n, {"max_hits": int(n * max(400, 40 * mean_e)) + (8 << 20), "lpt_order": 1})
    S.supa_batch_set_surrogate(b, net, args.e_s, int(2.0 * mean_e / args.e_s * n) + (1 << 20),
                               S.SUPA_SURROGATE_MEAN)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.warmup):
        S.supa_simulate(b, d, n, 4)
        S.supa_batch_get_info(b)
    ms = []
    for _ in range(args.steps):
        e0.record()
        S.supa_simulate(b, d, n, 4)
        e1.record()
        info = S.supa_batch_get_info(b)
        ms.append(e0.elapsed_time(e1))
    S.supa_destroy_batch(b)
    S.supa_destroy_geometry(gh)
    S.supa_surrogate_destroy(net)
    t = float(np.mean(ms))
    print(json.dumps({"metric": "hybrid showers/s (simulate only)", "value": n / (t / 1000.0), "unit": "showers/s",
                      "workload": f"50-layer showers (E log-U[10,1000], 0-45 deg) x {n}, E_s = {args.e_s} GeV, MEAN mode", "ms_per_call": ms,
                      "diverted_per_shower": info.n_diverted / n, "particle_steps_per_shower": info.n_steps / n,
                      "training": {k: v for k, v in tlog.items() if k != "loss_per_epoch"}}), flush=True)


def run_forward(args):
    """The surrogate network's inference kernel alone: W warm-up and K timed
    supa_surrogate_forward calls on n random feature rows (default 4.5M, the
    queue of about 40k 50-layer showers at E_s = 1), 96-float output rows as
    the hybrid path writes them; TFLOP/s of algorithmic flops (311,296 per
    row) against the measured BF16 peak."""
    import torch

    from paper_2202_05012_gb300 import inputs
    from paper_2202_05012_gb300 import supa as S
    torch.cuda.set_device(0)
    n = args.showers or 4_500_000
    s = S.supa_surrogate_create(256, S.pack_mlp_params(inputs.mlp_init(8)))
    rng = np.random.default_rng(2)
    X = np.stack([rng.uniform(-3, 0, n), *rng.normal(0, 0.3, (2, n)), rng.uniform(0.7, 1, n), rng.uniform(0, 1, n),
                  rng.uniform(0, 1, n)], 1).astype(np.float32)
    xd = torch.from_numpy(X).cuda()
    out = torch.empty((n, 96), dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        S.supa_surrogate_forward(s, xd, n, out)
    S.supa_surrogate_check(s)
    ms = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        e0.record()
        S.supa_surrogate_forward(s, xd, n, out)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    S.supa_surrogate_check(s)
    S.supa_surrogate_destroy(s)
    flops = 2 * (6 * 256 + 2 * 256 * 256 + 256 * 90) * n
    pk, pk_kind = peaks()
    best = min(ms)
    print(json.dumps({"metric": "surrogate inference TFLOP/s (algorithmic)", "value": flops / (best / 1000) / 1e12,
                      "unit": "TFLOP/s", "rows": n, "ms_per_call": ms, "ms_best": best,
                      "frac_of_bf16_burst": flops / (best / 1000) / 1e12 / pk["bf16_tflops"], "peak_source": pk_kind,
                      "kernel": "sur_mlp_kernel"}), flush=True)


def run_train(args):
    """The surrogate's training alone: a generic training set of
    --train-samples sub-showers (E log-uniform [e_min, E_s], plain method,
    E_s = --e-s), then --epochs Adam epochs in --batch-row minibatches (per
    epoch the targets staged once in the training pass's order; each step the
    training pass, the grouped weight gradients and the Adam update);
    W warm-up epochs first (not timed).  TFLOP/s of algorithmic flops
    (forward + backward, 3 x 311,296 per sample) by CUDA events."""
    import torch

    from paper_2202_05012_gb300 import surrogate_train as T
    torch.cuda.set_device(0)
    data = T.training_set(args.train_samples, args.e_s, 5)
    if args.warmup:
        net, _ = T.train(data, epochs=args.warmup, batch=args.batch, lr=args.lr, lr_final=args.lr_final)
        from paper_2202_05012_gb300 import supa as S
        S.supa_surrogate_destroy(net)
    net, log = T.train(data, epochs=args.epochs, batch=args.batch, lr=args.lr, lr_final=args.lr_final,
                       average_from=args.average_from if args.average_from >= 0 else None)
    from paper_2202_05012_gb300 import supa as S
    S.supa_surrogate_destroy(net)
    steps = log["steps_per_epoch"] * log["epochs"]
    print(json.dumps({"metric": "surrogate training TFLOP/s (algorithmic)", "value": log["tflops"], "unit": "TFLOP/s",
                      "samples": args.train_samples, "epochs": args.epochs, "batch": args.batch,
                      "us_per_step": log["seconds"] / steps * 1e6, "samples_per_s": log["samples_per_s"],
                      "seconds": log["seconds"], "loss_last_epoch": log["loss_per_epoch"][-1],
                      "kernels": ["stage_targets (once an epoch)", "train_mlp_kernel", "wgrad_kernel",
                                  "adam_update"]}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "mixed4":
        run_mixed4(args)
    elif args.workload == "surrogate":
        run_surrogate(args)
    elif args.workload == "hybrid":
        run_hybrid(args)
    elif args.workload == "forward":
        run_forward(args)
    elif args.workload == "train":
        run_train(args)
    else:
        run_supa(args)


if __name__ == "__main__":
    main()
