"""Float64 reference of the proposal encoder (test infrastructure only).

The encoder maps a series of length T to a 64-dim embedding whose Euclidean
distances are trained to follow the DTW distances of pairs of series:

    z1 = conv1(x) + b1,  h1 = GELU(z1)       1 -> 64 channels, kernel 7
    z2 = conv2(h1) + b2, h2 = GELU(z2)      64 -> 64 channels, kernel 7
    z3 = conv3(h2) + b3, h3 = GELU(z3)      64 -> 64 channels, kernel 7
    g  = mean_t h3                          global average pooling
    e  = Wl g + bl                          64 -> 64 linear

convolutions are "same" (zero padding of 3 on both sides), GELU is the exact
x * Phi(x) with Phi the standard normal CDF.  Loss over pairs (a, b) with
targets s_ab:  L = mean_p (||e_a - e_b|| - s_ab)^2.

Parameters travel as one flat float vector in this order (shapes, row major):
W1 [64, 7], b1 [64], W2 [7, 64, 64] (tap, out, in), b2 [64],
W3 [7, 64, 64], b3 [64], Wl [64, 64] (out, in), bl [64].

This module is numpy only and shares nothing with the CUDA encoder.  The
network is not from the paper (the paper has no learned part); it is the
proposal model the project adds, defined here as the reference.
"""

from __future__ import annotations

import math

import numpy as np

C = 64
KW = 7
PAD = 3
SHAPES = [("W1", (C, KW)), ("b1", (C,)), ("W2", (KW, C, C)), ("b2", (C,)),
          ("W3", (KW, C, C)), ("b3", (C,)), ("Wl", (C, C)), ("bl", (C,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)

_erf = np.vectorize(math.erf)


def unpack(theta):
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def pack(params):
    return np.concatenate([np.asarray(params[n], np.float64).ravel() for n, _ in SHAPES])


def init_params(seed: int) -> np.ndarray:
    """He-style normal initialisation (std sqrt(2/fan_in)), biases zero."""
    rng = np.random.default_rng(seed)
    p = {"W1": rng.normal(0, math.sqrt(2.0 / KW), (C, KW)), "b1": np.zeros(C),
         "W2": rng.normal(0, math.sqrt(2.0 / (C * KW)), (KW, C, C)), "b2": np.zeros(C),
         "W3": rng.normal(0, math.sqrt(2.0 / (C * KW)), (KW, C, C)), "b3": np.zeros(C),
         "Wl": rng.normal(0, math.sqrt(1.0 / C), (C, C)), "bl": np.zeros(C)}
    return pack(p).astype(np.float32)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)


def _shift(a, s):
    """a[..., t + s] along axis 1 (time) with zeros outside."""
    out = np.zeros_like(a)
    T = a.shape[1]
    if s >= 0:
        out[:, :T - s] = a[:, s:]
    else:
        out[:, -s:] = a[:, :T + s]
    return out


def conv(h, W):
    """out[b, t, o] = sum_k sum_i W[k, o, i] h[b, t + k - 3, i]."""
    return sum(np.einsum("bti,oi->bto", _shift(h, k - PAD), W[k]) for k in range(KW))


def conv1_taps(x):
    """xs[b, t, k] = x[b, t + k - 3] (zero outside the series)."""
    x = np.asarray(x, np.float64)
    return np.stack([_shift(x[:, :, None], k - PAD)[:, :, 0] for k in range(KW)], -1)


def conv_back(dz, h, W):
    """Gradients of out = conv(h, W) given dL/dout = dz: (dL/dW [7, 64, 64], dL/dh)."""
    dW = np.stack([np.einsum("bto,bti->oi", dz, _shift(h, k - PAD)) for k in range(KW)])
    dh = sum(_shift(np.einsum("bto,oi->bti", dz, W[k]), PAD - k) for k in range(KW))
    return dW, dh


def pair_loss_grad(e, pa, pb, target):
    """(L, dL/de) of L = mean_p (||e_a - e_b|| - s_ab)^2 over the pairs p = (pa, pb)."""
    pa, pb = np.asarray(pa), np.asarray(pb)
    diff = e[pa] - e[pb]
    d = np.linalg.norm(diff, axis=1)
    L = float(np.mean((d - target) ** 2))
    coef = 2.0 * (d - target) / len(pa) / np.maximum(d, 1e-12)
    dE = np.zeros_like(e)
    np.add.at(dE, pa, coef[:, None] * diff)
    np.add.at(dE, pb, -coef[:, None] * diff)
    return L, dE


def forward(theta, x):
    """x: [B, T] -> (e [B, 64], cache)."""
    P = unpack(theta)
    xs = conv1_taps(x)  # [B,T,7]
    z1 = np.einsum("btk,ok->bto", xs, P["W1"]) + P["b1"]
    h1 = gelu(z1)
    z2 = conv(h1, P["W2"]) + P["b2"]
    h2 = gelu(z2)
    z3 = conv(h2, P["W3"]) + P["b3"]
    h3 = gelu(z3)
    g = h3.mean(1)
    e = g @ P["Wl"].T + P["bl"]
    return e, dict(P=P, xs=xs, z1=z1, h1=h1, z2=z2, h2=h2, z3=z3, h3=h3, g=g)


def loss(e, pa, pb, target):
    d = np.linalg.norm(e[pa] - e[pb], axis=1)
    return float(np.mean((d - target) ** 2))


def backward(theta, x, pa, pb, target):
    """(loss, flat gradient) of the pair loss."""
    e, c = forward(theta, x)
    P = c["P"]
    L, dE = pair_loss_grad(e, pa, pb, target)
    G = {"Wl": dE.T @ c["g"], "bl": dE.sum(0)}
    dg = dE @ P["Wl"]
    T = x.shape[1]
    dz3 = (dg[:, None, :] / T) * gelu_grad(c["z3"])
    G["W3"], dh2 = conv_back(dz3, c["h2"], P["W3"])
    G["b3"] = dz3.sum((0, 1))
    dz2 = dh2 * gelu_grad(c["z2"])
    G["W2"], dh1 = conv_back(dz2, c["h1"], P["W2"])
    G["b2"] = dz2.sum((0, 1))
    dz1 = dh1 * gelu_grad(c["z1"])
    G["W1"] = np.einsum("bto,btk->ok", dz1, c["xs"])
    G["b1"] = dz1.sum((0, 1))
    return L, pack(G)


def bf16_round(a):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float32."""
    a = np.ascontiguousarray(np.asarray(a, np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)
