"""FP64 oracle of the shower surrogate network -- TEST INFRASTRUCTURE.

The surrogate has no counterpart in the SUPA paper: it is a small MLP that
stands in for the low-energy tail of a shower (sub-showers below a cutoff
energy E_s).  Architecture: 6 inputs -> 3 hidden layers of 256 with GELU
(the tanh form of Hendrycks and Gimpel, "Gaussian Error Linear Units",
2016: 0.5 z (1 + tanh(sqrt(2 / pi) (z + 0.044715 z^3)))) -> 90 outputs o = 30 log-link outputs o_j of the
means mu_j = exp(o_j - MU_SHIFT) and 30 log-variances s_j of the per-layer
deposit fractions, and 30 mean lateral distances rho_j of each layer's
deposits from the sub-shower's axis, layers counted from the sub-shower's
start layer.  The log link keeps every mean positive and makes a rounding
error of o_j a relative error of mu_j, so layers a sub-shower does not
reach get means that go to zero instead of a rounding-noise floor.  Targets Y = [y_j, R_j]: deposit fractions and
energy-weighted mean distances.  Loss: Gaussian negative log-likelihood of
the fractions plus the fraction-weighted squared error of the distances,
averaged over layers and samples,
  L = mean_b (1/30) sum_j [ (y_j - mu_j)^2 / (2 v_j) + ln(v_j) / 2
                            + LAMBDA_R y_j (rho_j - R_j)^2 / 2 ],
  v_j = exp(s_j) + VAR_FLOOR,
the predicted variance of the fraction with a floor of 10^-8 (a standard
deviation of 10^-4): without it a layer whose target is always 0 drives
mu_j and v_j to 0 together and (y - mu)^2 / v overflows.
Optimiser: Adam (Kingma & Ba 2015) with bias correction.

Plain numpy float64, one matrix formula per step; no fusion or reordering.
"""
from __future__ import annotations

import math

import numpy as np

N_IN, N_HID, N_OUT, N_LAYERS_OUT = 6, 256, 90, 30
MU_SHIFT = 4.0  # mu_j = exp(o_j - MU_SHIFT): outputs near 0 at initialisation give means near 1/55
VAR_FLOOR = 1.0e-8
SHAPES = [(N_HID, N_IN), (N_HID, N_HID), (N_HID, N_HID), (N_OUT, N_HID)]
LAMBDA_R = 1.0  # weight of the lateral term


GELU_C = math.sqrt(2.0 / math.pi)
GELU_A = 0.044715


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(GELU_C * (z + GELU_A * z ** 3)))


def gelu_grad(z):
    # d/dz: 0.5 (1 + t) + 0.5 z (1 - t^2) w'(z), t = tanh(w), w = c (z + a z^3)
    t = np.tanh(GELU_C * (z + GELU_A * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * GELU_C * (1.0 + 3.0 * GELU_A * z * z)


def forward(params, X):
    """params: list of (W [out, in], b [out]); X [B, 6].  Returns the output
    [B, 90] and the cache needed by backward."""
    acts = [X]
    pre = []
    h = X
    for i, (W, b) in enumerate(params):
        z = h @ W.T + b
        pre.append(z)
        h = gelu(z) if i < len(params) - 1 else z
        acts.append(h)
    return h, (acts, pre)


def deposit_means(out):
    """mu_j = exp(o_j - MU_SHIFT) of the first 30 outputs, [B, 30]."""
    return np.exp(out[:, :N_LAYERS_OUT] - MU_SHIFT)


def _split(out, Y):
    J = N_LAYERS_OUT
    return deposit_means(out), out[:, J:2 * J], out[:, 2 * J:3 * J], Y[:, :J], Y[:, J:2 * J]


def loss(out, Y):
    """The loss L above: mean over samples and the 30 layers."""
    mu, s, rho, y, R = _split(out, Y)
    v = np.exp(s) + VAR_FLOOR
    return float(np.mean(0.5 * (y - mu) ** 2 / v + 0.5 * np.log(v) + 0.5 * LAMBDA_R * y * (rho - R) ** 2))


def loss_grad(out, Y):
    """d L / d out, [B, 90] (the first 30 columns through the log link)."""
    B = out.shape[0]
    mu, s, rho, y, R = _split(out, Y)
    r = y - mu
    es = np.exp(s)
    v = es + VAR_FLOOR
    g_mu = -r * mu / v / (B * N_LAYERS_OUT)  # d mu / d o = mu
    g_s = 0.5 * es / v * (1.0 - r * r / v) / (B * N_LAYERS_OUT)  # d v / d s = exp(s)
    g_rho = LAMBDA_R * y * (rho - R) / (B * N_LAYERS_OUT)
    return np.concatenate([g_mu, g_s, g_rho], axis=1)


def backward(params, cache, g_out):
    """Gradients [(dW, db)] of the loss given d loss / d out."""
    acts, pre = cache
    grads = [None] * len(params)
    g = g_out
    for i in range(len(params) - 1, -1, -1):
        W, _ = params[i]
        if i < len(params) - 1:
            g = g * gelu_grad(pre[i])  # through the activation of layer i
        grads[i] = (g.T @ acts[i], g.sum(axis=0))
        g = g @ W  # d loss / d input of layer i
    return grads


def loss_and_grads(params, X, Y):
    out, cache = forward(params, X)
    return loss(out, Y), backward(params, cache, loss_grad(out, Y))


class Adam:
    def __init__(self, params, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.t = 0
        self.m = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        self.v = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]

    def step(self, params, grads):
        self.t += 1
        c1 = 1.0 - self.b1 ** self.t
        c2 = 1.0 - self.b2 ** self.t
        new = []
        for i, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
            out = []
            for j, (p, g) in enumerate(((W, gW), (b, gb))):
                m = self.b1 * self.m[i][j] + (1 - self.b1) * g
                v = self.b2 * self.v[i][j] + (1 - self.b2) * g * g
                self.m[i] = tuple(m if jj == j else self.m[i][jj] for jj in range(2))
                self.v[i] = tuple(v if jj == j else self.v[i][jj] for jj in range(2))
                out.append(p - self.lr * (m / c1) / (np.sqrt(v / c2) + self.eps))
            new.append(tuple(out))
        return new
