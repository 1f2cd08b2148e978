"""Scheduling: the autotuner's launch shape and CUDA-graph replay change no
result (the random streams are keyed by shower, slice and lineage)."""
import numpy as np
import pytest

from paper_2202_05012_gb300 import inputs
from paper_2202_05012_gb300 import supa as S

pytestmark = pytest.mark.gpu


def _results(b, n):
    import torch
    info = S.supa_batch_get_info(b)
    arr = {k: v.cpu().numpy().copy() for k, v in S.info_arrays(info).items()}
    torch.cuda.synchronize()
    return info, arr


def test_autotune_returns_a_valid_shape_with_identical_results():
    import torch
    geoms, p = inputs.workload_mixed4(20_000)
    gh = [S.supa_init_geometry(g) for g in geoms]
    try:
        d = S.primaries_to_device(p)
        max_hits = len(p) * 5000  # E up to 1000 GeV: about 2,400 hits per shower on average
        cfg, ms = S.supa_autotune(gh, d, len(p), seed=2, cfg={"lpt_order": 1, "max_hits": max_hits})
        assert ms > 0
        assert 2 <= cfg["blocks_per_sm"] <= 4 and cfg["warps_per_block"] in (4, 8)
        assert cfg["stack_depth"] in (96, 128, 192, 256) and cfg["flush_threshold"] in (-1, 64, 128, 256)
        assert cfg["max_hits"] == max_hits
        out = []
        for c in (cfg, {"blocks_per_sm": 2, "warps_per_block": 4, "stack_depth": 64, "flush_threshold": 32,
                        "max_hits": max_hits}):
            b = S.supa_batch_create(gh, len(p), c)
            try:
                S.supa_simulate(b, d, len(p), 2)
                out.append(_results(b, len(p))[1])
            finally:
                S.supa_destroy_batch(b)
        assert np.array_equal(out[0]["counts"], out[1]["counts"])
        assert np.array_equal(out[0]["steps"], out[1]["steps"])
        # fixed-point sums: exact, so equal whatever the order of additions
        assert np.array_equal(out[0]["layer_sum"], out[1]["layer_sum"])
    finally:
        for g in gh:
            S.supa_destroy_geometry(g)


def test_graph_captured_simulate_and_voxelize_match_eager():
    import torch
    g, p = inputs.workload_plain30(5000)
    gh = S.supa_init_geometry(g)
    b = S.supa_batch_create([gh], len(p), {"lpt_order": 1})
    try:
        d = S.primaries_to_device(p)
        grid_e = torch.zeros((len(p), g.n_layers, g.ny, g.nx), dtype=torch.float32, device="cuda")
        S.supa_simulate(b, d, len(p), 1)
        S.supa_voxelize(b, 0, len(p), grid_e)
        info_e, eager = _results(b, len(p))
        grid_e = grid_e.clone()

        grid_g = torch.zeros_like(grid_e)
        graph = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(graph, stream=s, capture_error_mode="thread_local"):
                S.supa_simulate(b, d, len(p), 1)
                S.supa_voxelize(b, 0, len(p), grid_g)
        torch.cuda.current_stream().wait_stream(s)
        for _ in range(2):
            grid_g.zero_()
            graph.replay()
            torch.cuda.synchronize()
            info_g, rep = _results(b, len(p))
            assert info_g.n_hits == info_e.n_hits and info_g.n_steps == info_e.n_steps
            assert np.array_equal(rep["counts"], eager["counts"])
            assert np.array_equal(rep["layer_sum"], eager["layer_sum"])
            assert torch.equal(grid_g != 0, grid_e != 0)
            assert torch.allclose(grid_g, grid_e, rtol=1e-6, atol=0)
    finally:
        S.supa_destroy_batch(b)
        S.supa_destroy_geometry(gh)


def test_warp_timeline_brackets_the_launch_and_changes_nothing():
    """record_warp_times: one (start, end) pair per warp of the persistent
    launch, every end after its start, all inside the launch as CUDA events
    time it; the results equal those of a batch without the timeline."""
    import torch
    geoms, p = inputs.workload_mixed4(30_000)
    gh = [S.supa_init_geometry(g) for g in geoms]
    try:
        d = S.primaries_to_device(p)
        cfg = {"lpt_order": 1, "max_hits": len(p) * 5000, "blocks_per_sm": 3, "warps_per_block": 8}
        res = []
        for rec in (1, 0):
            b = S.supa_batch_create(gh, len(p), dict(cfg, record_warp_times=rec))
            try:
                S.supa_simulate(b, d, len(p), 2)  # warm
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                S.supa_simulate(b, d, len(p), 2)
                e1.record()
                res.append(_results(b, len(p))[1])
                if rec:
                    t = S.supa_batch_warp_times(b).astype(np.int64)
                    sms = torch.cuda.get_device_properties(0).multi_processor_count
                    assert t.shape == (3 * sms * 8, 2)
                    assert np.all(t[:, 1] >= t[:, 0]) and np.all(t[:, 0] > 0)
                    span_ms = (t[:, 1].max() - t[:, 0].min()) / 1e6
                    assert 0 < span_ms <= e0.elapsed_time(e1) * 1.05 + 0.05
                else:
                    with pytest.raises(S.SupaError) as ei:
                        S.supa_batch_warp_times(b)
                    assert ei.value.code == S.SUPA_ERR_INVALID_ARG
            finally:
                S.supa_destroy_batch(b)
        for k in ("counts", "layer_sum", "steps"):
            assert np.array_equal(res[0][k], res[1][k]), k
    finally:
        for g in gh:
            S.supa_destroy_geometry(g)
