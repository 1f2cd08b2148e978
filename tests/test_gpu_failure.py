"""The failure path of the tensor-core pipelines, without a GPU fault: a
bounded wait on a barrier that nothing completes gives up, reports
SUPA_ERR_TIMEOUT, and the context stays usable."""
import numpy as np
import pytest

from paper_2202_05012_gb300 import inputs
from paper_2202_05012_gb300 import supa as S

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    import torch
    L = S.lib()
    # about a millisecond at the SM clock, twice in a row
    for _ in range(2):
        assert L.supa_check_wait_expiry(2_000_000, None) == S.SUPA_ERR_TIMEOUT
        assert "gave up" in S.supa_last_error()
    g = inputs.supa_d(5)
    p = inputs.primaries(50, 3, e_lo=1.0, e_hi=10.0)
    gh = S.supa_init_geometry(g)
    b = S.supa_batch_create([gh], len(p), {})
    try:
        S.supa_simulate(b, S.primaries_to_device(p), len(p), 1)
        info = S.supa_batch_get_info(b)
        assert info.status == S.SUPA_OK and info.n_hits > 0
        ls = S.info_arrays(info)["layer_sum"].cpu().numpy()
        tot = ls.sum(1) + S.info_arrays(info)["dead"].cpu().numpy() + S.info_arrays(info)["leak"].cpu().numpy() + \
            S.info_arrays(info)["escape"].cpu().numpy()
        np.testing.assert_allclose(tot, p["E"].astype(np.float64), rtol=1e-5)
        torch.cuda.synchronize()
    finally:
        S.supa_destroy_batch(b)
        S.supa_destroy_geometry(gh)
