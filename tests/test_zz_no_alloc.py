"""The allocation-free offsets entry point, for callers that may not call
cudaMalloc (their memory belongs to a host framework's pool, or their path
must never wait on the allocator): its output must equal the offsets the
batch computes after a simulation, on two calls in a row that share the
library's fixed scratch array.  Named to be collected last."""
import numpy as np
import pytest

from paper_2202_05012_gb300 import inputs
from paper_2202_05012_gb300 import supa as S

pytestmark = pytest.mark.gpu


def test_noalloc_offsets_equal_batch_offsets_twice():
    import torch
    g, p = inputs.workload_plain10(3000)
    gh = S.supa_init_geometry(g)
    b = S.supa_batch_create([gh], len(p), {})
    try:
        S.supa_simulate(b, S.primaries_to_device(p), len(p), 0)
        info = S.supa_batch_get_info(b)
        n = info.n_showers
        ref = S.device_view(info.offsets_dev, (n + 1,), torch.int64).clone()
        counts = S.device_view(info.counts_dev, (n,), torch.int32).clone()
        for _ in range(2):
            out = torch.full((n + 1,), -1, dtype=torch.int64, device="cuda")
            S.supa_shower_offsets_noalloc(counts, n, out)
            torch.cuda.synchronize()
            assert torch.equal(out, ref)
        assert int(ref[-1].item()) == info.n_hits
    finally:
        S.supa_destroy_batch(b)
        S.supa_destroy_geometry(gh)


def test_noalloc_offsets_reject_sizes_beyond_the_scratch():
    import torch
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    counts = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(S.SupaError) as ei:
        S.supa_shower_offsets_noalloc(counts, 16_769_025, out)
    assert ei.value.code == S.SUPA_ERR_INVALID_ARG
    assert "16769024" in str(ei.value)


def _reference_offsets(counts):
    import torch
    ref = torch.zeros(counts.numel() + 1, dtype=torch.int64, device=counts.device)
    if counts.numel():
        ref[1:] = torch.cumsum(counts.to(torch.int64), 0)
    return ref


@pytest.mark.parametrize("n", [0, 1, 4096, 4097, 2 * 4096 + 17, 5 * 4096 + 4095, 1000 * 4096 + 123, 16_769_024])
def test_noalloc_offsets_across_scan_blocks(n):
    """Synthetic counts of every size class: empty, one scan block, several
    blocks with a ragged last one (the carry between blocks and every block's
    read of its predecessors' totals), and the largest accepted n (4,094
    blocks, all 4,095 entries of the fixed array in use)."""
    import torch
    gen = torch.Generator(device="cpu").manual_seed(n)
    hi = 3 if n > 1_000_000 else 5000
    counts = torch.randint(0, hi, (n,), generator=gen, dtype=torch.int32).cuda()
    out = torch.full((n + 1,), -1, dtype=torch.int64, device="cuda")
    S.supa_shower_offsets_noalloc(counts, n, out)
    torch.cuda.synchronize()
    assert torch.equal(out, _reference_offsets(counts))


def test_noalloc_offsets_two_calls_with_different_sizes():
    """A large call fills many entries of the shared array; a smaller call
    right after it on the same stream must not see any of them, and a large
    call after a small one must not see the small one's."""
    import torch
    gen = torch.Generator(device="cpu").manual_seed(7)
    sizes = [9 * 4096 + 5, 3 * 4096 + 1, 0, 12 * 4096 + 4000]
    outs, refs = [], []
    for n in sizes:
        counts = torch.randint(0, 100_000, (n,), generator=gen, dtype=torch.int32).cuda()
        out = torch.full((n + 1,), -1, dtype=torch.int64, device="cuda")
        S.supa_shower_offsets_noalloc(counts, n, out)
        outs.append(out)
        refs.append(_reference_offsets(counts))
    torch.cuda.synchronize()
    for out, ref in zip(outs, refs):
        assert torch.equal(out, ref)
