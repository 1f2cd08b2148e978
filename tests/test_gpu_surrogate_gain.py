"""What the trained surrogate gains over the method without it, on the
30-layer workload (E U[1,100] GeV, 0-30 deg) at E_s = 2 GeV: the hybrid path steps a small fraction of the
particles the plain path steps, and its shower profiles stay close to the
plain ones in both modes: every layer holding >= 0.5 % of the energy within
2 %, and within 3 % the largest deviation over groups of consecutive layers,
or of rings around the shower axis, holding >= 2 % of the energy each (every
layer and ring included) -- which an untrained network of the same shape
does not achieve."""
import pytest

from paper_2202_05012_gb300 import inputs
from paper_2202_05012_gb300 import supa as S
from paper_2202_05012_gb300 import surrogate_train as T

pytestmark = pytest.mark.gpu

E_S = 2.0
N = 20_000
BINS, R_MAX = T.PROFILE_BINS, T.PROFILE_RMAX


def _run(gh, d, mean_e, net, mode=S.SUPA_SURROGATE_MEAN):
    import torch
    b = S.supa_batch_create([gh], N, {"max_hits": int(N * 60 * mean_e) + (8 << 20), "lpt_order": 1})
    try:
        if net is not None:
            S.supa_batch_set_surrogate(b, net, E_S, int(4 * mean_e / E_S * N) + (1 << 20), mode)
        S.supa_simulate(b, d, N, 7)
        info = S.supa_batch_get_info(b)
        lo = torch.zeros(30, dtype=torch.float64, device="cuda")
        la = torch.zeros(BINS, dtype=torch.float64, device="cuda")
        S.supa_profiles(b, 0, N, BINS, R_MAX, lo, la)
        torch.cuda.synchronize()
        return info.n_steps, lo.cpu().numpy() / N, la.cpu().numpy() / N
    finally:
        S.supa_destroy_batch(b)


def test_trained_network_replaces_most_steps_at_small_profile_error():
    g, p = inputs.workload_plain30(N, seed=21)
    gt, pt = inputs.workload_plain30(150_000, seed=22)
    data = T.training_set_matched(gt, pt, E_S, 5_000_000, seed=5)
    net, log = T.train(data, epochs=15, lr=2e-3, lr_final=5e-5)
    del data
    untrained = S.supa_surrogate_create(16384, S.pack_mlp_params(inputs.mlp_init(1)))
    gh = S.supa_init_geometry(g)
    try:
        d = S.primaries_to_device(p)
        mean_e = float(p["E"].mean())
        steps_plain, lo_p, la_p = _run(gh, d, mean_e, None)
        steps_h, lo_h, la_h = _run(gh, d, mean_e, net)
        _, lo_s, la_s = _run(gh, d, mean_e, net, S.SUPA_SURROGATE_SAMPLE)
        _, lo_u, la_u = _run(gh, d, mean_e, untrained)
    finally:
        S.supa_destroy_geometry(gh)
        S.supa_surrogate_destroy(net)
        S.supa_surrogate_destroy(untrained)
    # the network replaces most of the stepping
    assert steps_h < 0.2 * steps_plain, (steps_h, steps_plain)
    # ... at small profile error, in both modes
    for lo, la in ((lo_h, la_h), (lo_s, la_s)):
        e = T.profile_errors((lo_p, la_p), (lo, la))
        assert e["longitudinal_per_layer"] < 0.02 and e["longitudinal"] < 0.03, e
        assert e["lateral"] < 0.03 and e["total_deposit"] < 0.006, e
    # which the same network untrained is far from
    e = T.profile_errors((lo_p, la_p), (lo_u, la_u))
    assert e["longitudinal"] > 0.1 or e["lateral"] > 0.1, e
