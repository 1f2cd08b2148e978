"""Pins of the FP64 surrogate-network oracle: central finite differences,
the same network written with torch.nn in float64 (library routines), and
torch.optim.Adam."""
import math

import numpy as np
import pytest

from oracle import mlp
from paper_2202_05012_gb300 import inputs


def _data(B, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    X = rng.normal(0, 1, (B, 6))
    Y = np.concatenate([rng.uniform(0, 0.3, (B, 30)), rng.uniform(0, 2.0, (B, 30))], 1)
    return X, Y


def test_gelu_and_its_derivative():
    z = np.linspace(-6, 6, 101)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    np.testing.assert_allclose(mlp.gelu(np.array([8.0])), 8.0, rtol=1e-12)
    np.testing.assert_allclose(mlp.gelu(np.array([-8.0])), 0.0, atol=1e-12)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(z), fd, rtol=1e-7, atol=1e-9)


def test_gelu_is_the_tanh_form():
    """The tanh form of GELU (torch's approximate="tanh", a library routine),
    within 5e-4 of the erf form z Phi(z)."""
    torch = pytest.importorskip("torch")
    from scipy.special import erf
    z = np.linspace(-9, 9, 3601)
    ref = torch.nn.functional.gelu(torch.from_numpy(z), approximate="tanh").numpy()
    np.testing.assert_allclose(mlp.gelu(z), ref, rtol=1e-14, atol=1e-15)
    exact = 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))
    assert 4e-4 < np.abs(mlp.gelu(z) - exact).max() < 5e-4


def test_backward_matches_central_finite_differences():
    params = inputs.mlp_init(3, shapes=((16, 6), (16, 16), (16, 16), (90, 16)))
    params = [(W, np.random.default_rng(i).normal(0, 0.1, b.shape)) for i, (W, b) in enumerate(params)]
    X, Y = _data(7, 1)
    loss, grads = mlp.loss_and_grads(params, X, Y)
    rng = np.random.default_rng(0)
    h = 1e-6
    for li, (W, b) in enumerate(params):
        for which, P, G in ((0, W, grads[li][0]), (1, b, grads[li][1])):
            idx = [tuple(rng.integers(0, s) for s in P.shape) for _ in range(6)]
            for ix in idx:
                def f(delta):
                    Q = [[W_.copy(), b_.copy()] for W_, b_ in params]
                    Q[li][which][ix] += delta
                    return mlp.loss(mlp.forward([tuple(q) for q in Q], X)[0], Y)
                fd = (f(h) - f(-h)) / (2 * h)
                assert abs(fd - G[ix]) <= 1e-6 * max(abs(fd), 1e-3), (li, which, ix, fd, G[ix])


def test_matches_torch_nn_float64():
    torch = pytest.importorskip("torch")
    params = inputs.mlp_init(5)
    params = [(W, np.random.default_rng(9 + i).normal(0, 0.05, b.shape)) for i, (W, b) in enumerate(params)]
    X, Y = _data(64, 2)
    loss, grads = mlp.loss_and_grads(params, X, Y)
    layers = []
    for W, b in params:
        lin = torch.nn.Linear(W.shape[1], W.shape[0], dtype=torch.float64)
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(W))
            lin.bias.copy_(torch.from_numpy(b))
        layers.append(lin)
    h = torch.from_numpy(X)
    for i, lin in enumerate(layers):
        h = lin(h)
        if i < 3:
            h = torch.nn.functional.gelu(h, approximate="tanh")
    mu, s, rho = torch.exp(h[:, :30] - mlp.MU_SHIFT), h[:, 30:60], h[:, 60:]
    yt, rt = torch.from_numpy(Y[:, :30]), torch.from_numpy(Y[:, 30:])
    v = torch.exp(s) + mlp.VAR_FLOOR
    tl = torch.mean(0.5 * (yt - mu) ** 2 / v + 0.5 * torch.log(v) + 0.5 * mlp.LAMBDA_R * yt * (rho - rt) ** 2)
    tl.backward()
    assert abs(tl.item() - loss) < 1e-12
    for (gW, gb), lin in zip(grads, layers):
        np.testing.assert_allclose(gW, lin.weight.grad.numpy(), rtol=1e-9, atol=1e-14)
        np.testing.assert_allclose(gb, lin.bias.grad.numpy(), rtol=1e-9, atol=1e-14)


def test_adam_matches_torch_optim():
    torch = pytest.importorskip("torch")
    params = inputs.mlp_init(6, shapes=((8, 6), (8, 8), (8, 8), (90, 8)))
    X, Y = _data(16, 3)
    opt = mlp.Adam(params, lr=1e-2)
    tparams = [torch.tensor(a, requires_grad=True) for W, b in params for a in (W, b)]
    topt = torch.optim.Adam(tparams, lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for _ in range(4):
        loss, grads = mlp.loss_and_grads(params, X, Y)
        params = opt.step(params, grads)
        topt.zero_grad()
        for t, g in zip(tparams, [a for gW, gb in grads for a in (gW, gb)]):
            t.grad = torch.from_numpy(np.ascontiguousarray(g))
        topt.step()
        # feed torch the oracle's gradients at the oracle's own parameters
        for t, a in zip(tparams, [a for W, b in params for a in (W, b)]):
            np.testing.assert_allclose(t.detach().numpy(), a, rtol=1e-12, atol=1e-15)
