"""FP64 reference of the closure network -- TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's conclusion conjectures a closure for the collisional friction in terms of the local
plasma state; the network that carries it is this library's reading: inputs x (9 coarse
moments, or 8 without W_ES), normalised per feature as (x - mu) / sigma, two hidden layers of 64
SiLU units and one linear output,

    z1 = W1 xn + b1,  h1 = silu(z1),  z2 = W2 h1 + b2,  h2 = silu(z2),  y = w3 . h2 + b3,

silu(z) = z / (1 + exp(-z)), trained on the mean squared error L = mean (y - t)^2 with Adam.
The tensor-core path rounds the weights W1, W2 and the activations entering the two matrix
products (xn, h1; and the output gradient entering the backward product) to bfloat16 and
accumulates in FP32; `forward(..., bf16=True)` applies the same roundings so that the
comparison isolates accumulation error.

Parameter vector (4865 values, the order of the library's flat parameter array):
    W1[64][9], b1[64], W2[64][64], b2[64], w3[64], b3
"""
from __future__ import annotations

import numpy as np

NIN, NH = 9, 64
SIZES = (("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("w3", (NH,)),
         ("b3", (1,)))
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(p[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as FP64."""
    f = np.asarray(a, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def init_params(seed=0, nin=NIN):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases (inputs past nin get 0)."""
    rng = np.random.default_rng(seed)
    d = {}
    d["W1"] = rng.uniform(-1, 1, (NH, NIN)) / np.sqrt(nin)
    d["W1"][:, nin:] = 0.0
    d["b1"] = rng.uniform(-1, 1, NH) / np.sqrt(nin)
    d["W2"] = rng.uniform(-1, 1, (NH, NH)) / np.sqrt(NH)
    d["b2"] = rng.uniform(-1, 1, NH) / np.sqrt(NH)
    d["w3"] = rng.uniform(-1, 1, NH) / np.sqrt(NH)
    d["b3"] = np.zeros(1)
    return pack(d).astype(np.float32).astype(np.float64)


def forward(p, x, mu, sigma, bf16_path=False):
    """Network output y (n,) and the intermediate values, FP64."""
    P = unpack(p)
    xn = (np.asarray(x, dtype=np.float64) - mu) / sigma
    W1, W2 = P["W1"], P["W2"]
    if bf16_path:
        xn, W1, W2 = bf16(xn), bf16(W1), bf16(W2)
    z1 = xn @ W1.T + P["b1"]
    h1 = silu(z1)
    h1m = bf16(h1) if bf16_path else h1
    z2 = h1m @ W2.T + P["b2"]
    h2 = silu(z2)
    y = h2 @ P["w3"] + P["b3"][0]
    return y, dict(xn=xn, z1=z1, h1=h1m, z2=z2, h2=h2, W1=W1, W2=W2)


def loss_and_grad(p, x, t, mu, sigma, bf16_path=False):
    """L = mean (y - t)^2 and dL/dp (flat, FP64) by the chain rule."""
    y, c = forward(p, x, mu, sigma, bf16_path)
    P = unpack(p)
    n = y.shape[0]
    r = y - np.asarray(t, dtype=np.float64)
    L = float(np.mean(r * r))
    dy = 2.0 * r / n
    g = {}
    g["w3"] = c["h2"].T @ dy
    g["b3"] = np.array([dy.sum()])
    d2 = (dy[:, None] * P["w3"][None, :]) * dsilu(c["z2"])
    g["W2"] = d2.T @ c["h1"]
    g["b2"] = d2.sum(0)
    d2m = bf16(d2) if bf16_path else d2
    d1 = (d2m @ c["W2"]) * dsilu(c["z1"])
    g["W1"] = d1.T @ c["xn"]
    g["b1"] = d1.sum(0)
    return L, pack(g)


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) of step t >= 1; returns p, m, v."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def feature_norm(x):
    """Per-feature mean and standard deviation (1 where a feature is constant)."""
    x = np.asarray(x, dtype=np.float64)
    mu = x.mean(0)
    sd = x.std(0)
    return mu, np.where(sd > 0, sd, 1.0)
