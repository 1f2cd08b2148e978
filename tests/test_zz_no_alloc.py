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
