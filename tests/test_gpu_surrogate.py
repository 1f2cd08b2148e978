"""The BF16 tensor-core surrogate network against its FP64 oracle: forward
outputs, loss, gradients (relative norm error and cosine per tensor), and a
short Adam trajectory."""
import numpy as np
import pytest

from oracle import mlp
from paper_2202_05012_gb300 import inputs
from paper_2202_05012_gb300 import supa as S

pytestmark = pytest.mark.gpu


def _batch(B, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    X = np.stack([rng.uniform(-3, 0, B), *rng.normal(0, 0.3, (2, B)), rng.uniform(0.7, 1, B), rng.uniform(0, 1, B),
                  rng.uniform(0, 1, B)], 1)
    Y = np.concatenate([np.abs(rng.normal(0.05, 0.05, (B, 30))), rng.uniform(0.0, 2.0, (B, 30))], 1)
    return X, Y


def _f32_params(seed):
    p = inputs.mlp_init(seed)
    rng = np.random.default_rng(seed)
    p = [(W, rng.normal(0, 0.05, b.shape)) for W, b in p]
    vec = S.pack_mlp_params(p)
    return vec, [(W.astype(np.float64), b.astype(np.float64)) for W, b in S.unpack_mlp_params(vec)]


@pytest.mark.parametrize("B", [128, 1024])
def test_gradients_match_fp64_oracle(B):
    """One row tile (128: one CTA, two K-blocks of weight gradients) and eight."""
    import torch
    vec, params = _f32_params(7)
    X, Y = _batch(B, 1)
    s = S.supa_surrogate_create(B, vec)
    try:
        xd = torch.from_numpy(X.astype(np.float32)).cuda()
        yd = torch.from_numpy(Y.astype(np.float32)).cuda()
        g, loss = S.supa_surrogate_gradients(s, xd, yd)
        ref_loss, ref = mlp.loss_and_grads(params, X, Y)
        assert abs(loss - ref_loss) <= 1e-2 * abs(ref_loss) + 1e-4
        gg = S.unpack_mlp_params(g.astype(np.float64))
        for i, ((gW, gb), (rW, rb)) in enumerate(zip(gg, ref)):
            for a, r, name in ((gW, rW, f"W{i + 1}"), (gb, rb, f"b{i + 1}")):
                rel = np.linalg.norm(a - r) / np.linalg.norm(r)
                cos = np.dot(a.ravel(), r.ravel()) / (np.linalg.norm(a) * np.linalg.norm(r))
                assert rel < 2e-2 and cos > 0.999, (name, rel, cos)
    finally:
        S.supa_surrogate_destroy(s)


@pytest.mark.parametrize("n,ld", [(1000, 90), (1000, 96), (1000, 93), (40_013, 96), (40_013, 90)])
def test_forward_matches_fp64_oracle_including_ragged_tail(n, ld):
    """Row pitches of 90 and 93 floats take the plain stores, 96 the TMA
    stores; n = 1000 ends in a tile whose last 32-row block is partial, and
    40,013 rows give every CTA two row tiles in flight and more than one pair.
    The rows past n stay untouched, and so do columns 90.. of the plain
    stores; the TMA stores write the zero padding outputs 90..95."""
    import torch
    vec, params = _f32_params(8)
    X, _ = _batch(n, 2)
    s = S.supa_surrogate_create(256, vec)
    try:
        xd = torch.from_numpy(X.astype(np.float32)).cuda()
        out = torch.full((n + 3, ld), np.nan, dtype=torch.float32, device="cuda")
        S.supa_surrogate_forward(s, xd, n, out)
        S.supa_surrogate_check(s)
        o = out.cpu().numpy()
        assert np.all(np.isnan(o[n:]))
        if ld % 4 == 0:
            assert np.all(o[:n, 90:] == 0)
        else:
            assert np.all(np.isnan(o[:, 90:]))
        got = o[:n, :90].astype(np.float64)
        ref, _ = mlp.forward(params, X)
        scale = np.abs(ref).max()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) < 2e-2 * scale
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-2
        if ld != 90:  # the two store paths give the same numbers
            out90 = torch.empty((n, 90), dtype=torch.float32, device="cuda")
            S.supa_surrogate_forward(s, xd, n, out90)
            S.supa_surrogate_check(s)
            assert np.array_equal(out90.cpu().numpy(), o[:n, :90])
    finally:
        S.supa_surrogate_destroy(s)


def test_adam_trajectory_follows_oracle():
    import torch
    B = 512
    vec, params = _f32_params(9)
    X, Y = _batch(B, 3)
    s = S.supa_surrogate_create(B, vec)
    try:
        xd = torch.from_numpy(X.astype(np.float32)).cuda()
        yd = torch.from_numpy(Y.astype(np.float32)).cuda()
        acc = torch.zeros(1, dtype=torch.float64, device="cuda")
        opt = mlp.Adam(params, lr=3e-4)
        ours, ref = [], []
        for step in range(30):
            acc.zero_()
            S.supa_surrogate_train_step(s, xd, yd, 3e-4, acc)
            ours.append(acc.item())
            loss, grads = mlp.loss_and_grads(params, X, Y)
            ref.append(loss)
            params = opt.step(params, grads)
        S.supa_surrogate_check(s)
        ours, ref = np.array(ours), np.array(ref)
        assert ours[-1] < ours[0] - 0.005  # it learns (the NLL can go negative)
        np.testing.assert_allclose(ours, ref, rtol=3e-2, atol=1e-3)
        p = S.unpack_mlp_params(S.supa_surrogate_get_params(s).astype(np.float64))
        for (W, b), (rW, rb) in zip(p, params):
            assert np.linalg.norm(W - rW) / np.linalg.norm(rW) < 2e-2
    finally:
        S.supa_surrogate_destroy(s)


def test_iterate_average_is_the_mean_of_the_steps_parameters():
    """supa_surrogate_average: after START, every Adam step's parameters
    enter a uniform average; APPLY makes the network that average (checked
    against the mean of the parameters read after each step) and the
    inference kernel then uses it."""
    import torch
    B = 256
    vec, _ = _f32_params(11)
    X, Y = _batch(B, 4)
    s = S.supa_surrogate_create(B, vec)
    try:
        xd = torch.from_numpy(X.astype(np.float32)).cuda()
        yd = torch.from_numpy(Y.astype(np.float32)).cuda()
        for _ in range(2):
            S.supa_surrogate_train_step(s, xd, yd, 1e-3)
        S.supa_surrogate_average(s, S.SUPA_AVERAGE_START)
        seen = []
        for _ in range(5):
            S.supa_surrogate_train_step(s, xd, yd, 1e-3)
            seen.append(S.supa_surrogate_get_params(s).astype(np.float64))
        S.supa_surrogate_average(s, S.SUPA_AVERAGE_STOP)
        S.supa_surrogate_train_step(s, xd, yd, 1e-3)  # not averaged
        last = S.supa_surrogate_get_params(s)
        S.supa_surrogate_average(s, S.SUPA_AVERAGE_APPLY)
        got = S.supa_surrogate_get_params(s).astype(np.float64)
        ref = np.mean(seen, axis=0)
        np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-7)
        assert np.abs(got - last).max() > 1e-6  # the steps did move the parameters
        # the BF16 copies follow: the forward equals a network built from the average
        t = S.supa_surrogate_create(B, got.astype(np.float32))
        try:
            o1 = torch.empty((B, 96), dtype=torch.float32, device="cuda")
            o2 = torch.empty((B, 96), dtype=torch.float32, device="cuda")
            S.supa_surrogate_forward(s, xd, B, o1)
            S.supa_surrogate_forward(t, xd, B, o2)
            torch.cuda.synchronize()
            np.testing.assert_allclose(o1.cpu().numpy()[:, :90], o2.cpu().numpy()[:, :90], rtol=0, atol=1e-6)
        finally:
            S.supa_surrogate_destroy(t)
        with pytest.raises(S.SupaError):
            S.supa_surrogate_average(s, 7)
    finally:
        S.supa_surrogate_destroy(s)


def test_gradients_with_several_tiles_per_cta():
    """A minibatch of 40,960 rows: 320 row tiles, more than the GPU has SMs,
    so CTAs of the training pass take two or three tiles one after another
    (input tile, operand buffers, barriers and TMEM accumulators reused) and
    the weight gradients contract over 640 K-blocks.  Same check as for 1,024
    rows against the FP64 oracle."""
    import torch
    B = 40_960
    vec, params = _f32_params(9)
    X, Y = _batch(B, 6)
    s = S.supa_surrogate_create(B, vec)
    try:
        xd = torch.from_numpy(X.astype(np.float32)).cuda()
        yd = torch.from_numpy(Y.astype(np.float32)).cuda()
        g, loss = S.supa_surrogate_gradients(s, xd, yd)
        ref_loss, ref = mlp.loss_and_grads(params, X, Y)
        assert abs(loss - ref_loss) <= 1e-2 * abs(ref_loss) + 1e-4
        gg = S.unpack_mlp_params(g.astype(np.float64))
        for i, ((gW, gb), (rW, rb)) in enumerate(zip(gg, ref)):
            for a, r, name in ((gW, rW, f"W{i + 1}"), (gb, rb, f"b{i + 1}")):
                rel = np.linalg.norm(a - r) / np.linalg.norm(r)
                cos = np.dot(a.ravel(), r.ravel()) / (np.linalg.norm(a) * np.linalg.norm(r))
                assert rel < 2e-2 and cos > 0.999, (name, rel, cos)
        # the same rows in another order give the same gradients (sums over rows)
        perm = np.random.default_rng(1).permutation(B)
        g2, loss2 = S.supa_surrogate_gradients(s, torch.from_numpy(X[perm].astype(np.float32)).cuda(),
                                               torch.from_numpy(Y[perm].astype(np.float32)).cuda())
        for (a1, b1), (a2, b2) in zip(gg, S.unpack_mlp_params(g2.astype(np.float64))):
            for u, v in ((a1, a2), (b1, b2)):
                assert np.linalg.norm(u - v) <= 1e-4 * np.linalg.norm(u)
        assert abs(loss2 - loss) <= 1e-5 * abs(loss)
    finally:
        S.supa_surrogate_destroy(s)


def _epoch_permutation(seed, n):
    """The rows i -> (a i + c) mod n of an epoch, as supa_surrogate_train_epoch
    picks a and c from the seed (host arithmetic restated)."""
    from math import gcd
    m = 2**64 - 1
    a = ((seed * 0x9E3779B97F4A7C15) & m) + 0x632BE59BD9B4E019
    a = (a & m) % n
    if a == 0:
        a = 1
    while gcd(a, n) != 1:
        a = 1 if (a + 1) % n == 0 else a + 1
    c = (seed ^ 0xD1B54A32D192ED03) % n
    return (a * np.arange(n, dtype=object) + c) % n


def test_epoch_with_staged_targets_equals_its_steps():
    """An epoch (targets staged once in the training pass's order) against
    the same minibatches, gathered on the host, as single Adam steps: the
    same parameters and the same loss, up to the order of float additions."""
    import torch
    B, steps, seed = 256, 3, 11
    n = B * steps + 77  # a ragged remainder the epoch leaves out
    vec, _ = _f32_params(5)
    X, Y = _batch(n, 8)
    perm = np.array(_epoch_permutation(seed, n), dtype=np.int64)
    a = S.supa_surrogate_create(B, vec)
    b = S.supa_surrogate_create(B, vec)
    try:
        xd = torch.from_numpy(X.astype(np.float32)).cuda()
        yd = torch.from_numpy(Y.astype(np.float32)).cuda()
        acc_a = torch.zeros(1, dtype=torch.float64, device="cuda")
        acc_b = torch.zeros(1, dtype=torch.float64, device="cuda")
        S.supa_surrogate_train_epoch(a, xd, yd, n, seed, 1e-3, acc_a)
        for k in range(steps):
            rows = perm[k * B:(k + 1) * B]
            xs = torch.from_numpy(X[rows].astype(np.float32)).cuda()
            ys = torch.from_numpy(Y[rows].astype(np.float32)).cuda()
            S.supa_surrogate_train_step(b, xs, ys, 1e-3, acc_b)
        S.supa_surrogate_check(a)
        S.supa_surrogate_check(b)
        np.testing.assert_allclose(acc_a.item(), acc_b.item(), rtol=1e-5)
        pa, pb = S.supa_surrogate_get_params(a), S.supa_surrogate_get_params(b)
        np.testing.assert_allclose(pa, pb, rtol=0, atol=1e-5 * np.abs(pb).max())
    finally:
        S.supa_surrogate_destroy(a)
        S.supa_surrogate_destroy(b)


def test_misaligned_targets_are_refused():
    import torch
    B = 128
    vec, _ = _f32_params(5)
    X, Y = _batch(B + 1, 8)
    s = S.supa_surrogate_create(B, vec)
    try:
        xd = torch.from_numpy(X.astype(np.float32)).cuda()
        buf = torch.from_numpy(np.concatenate([[0.0], Y.ravel()]).astype(np.float32)).cuda()
        y_odd = buf[1:]  # 4 bytes past an aligned allocation: not 8-byte aligned
        for call in (lambda: S.supa_surrogate_gradients(s, xd, y_odd),
                     lambda: S.supa_surrogate_train_step(s, xd, y_odd, 1e-3),
                     lambda: S.supa_surrogate_train_epoch(s, xd, y_odd, B, 1, 1e-3)):
            with pytest.raises(S.SupaError) as e:
                call()
            assert e.value.code == S.SUPA_ERR_INVALID_ARG
    finally:
        S.supa_surrogate_destroy(s)
