"""Pins of the float64 encoder reference (oracle/encoder_ref.py)."""

import math

import numpy as np
import pytest
import torch

from oracle import encoder_ref as R


def _case(seed=0, B=3, T=16, S=None):
    rng = np.random.default_rng(seed)
    theta = R.init_params(seed).astype(np.float64)
    theta += rng.normal(0, 0.05, theta.shape)  # non-zero biases too
    x = rng.standard_normal((B, T))
    pa, pb = np.triu_indices(B, 1)
    target = rng.uniform(0.2, 2.0, len(pa))
    return theta, x, pa, pb, target


def test_param_count():
    assert R.N_PARAMS == 64 * 7 + 64 + 2 * (7 * 64 * 64 + 64) + 64 * 64 + 64 == 62144


def test_gradient_matches_finite_differences():
    theta, x, pa, pb, target = _case()
    L, g = R.backward(theta, x, pa, pb, target)
    assert L == pytest.approx(R.loss(R.forward(theta, x)[0], pa, pb, target))
    rng = np.random.default_rng(1)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in R.SHAPES])
    idx = np.concatenate([rng.integers(offs[i], offs[i + 1], 6) for i in range(len(R.SHAPES))])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (R.loss(R.forward(tp, x)[0], pa, pb, target)
              - R.loss(R.forward(tm, x)[0], pa, pb, target)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9), i


def test_gelu_and_its_derivative():
    z = np.linspace(-6, 6, 101)
    phi = 0.5 * (1 + np.array([math.erf(v / math.sqrt(2)) for v in z]))
    assert np.allclose(R.gelu(z), z * phi, atol=0, rtol=1e-15)
    h = 1e-6
    fd = (R.gelu(z + h) - R.gelu(z - h)) / (2 * h)
    assert np.allclose(R.gelu_grad(z), fd, atol=1e-8)
    assert np.allclose(R.gelu(z), torch.nn.functional.gelu(torch.tensor(z)).numpy(), atol=1e-12)


def test_conv_matches_library_conv1d():
    theta, x, *_ = _case(seed=2, B=2, T=20)
    P = R.unpack(theta)
    _, c = R.forward(theta, x)
    h1 = torch.tensor(c["h1"]).permute(0, 2, 1)  # [B, C, T]
    w = torch.tensor(P["W2"]).permute(1, 2, 0)   # [out, in, tap]
    ref = torch.nn.functional.conv1d(h1, w, torch.tensor(P["b2"]), padding=3).permute(0, 2, 1)
    assert np.allclose(c["z2"], ref.numpy(), atol=1e-12)
    z1 = torch.nn.functional.conv1d(torch.tensor(x)[:, None, :], torch.tensor(P["W1"])[:, None, :],
                                    torch.tensor(P["b1"]), padding=3).permute(0, 2, 1)
    assert np.allclose(c["z1"], z1.numpy(), atol=1e-12)


def test_bf16_round_matches_torch():
    a = np.random.default_rng(3).standard_normal(10000).astype(np.float32) * 7
    ref = torch.tensor(a).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(R.bf16_round(a), ref)


def test_bias_of_the_embedding_has_zero_gradient():
    # the loss only sees differences of embeddings
    theta, x, pa, pb, target = _case(seed=4, B=5, T=12)
    _, g = R.backward(theta, x, pa, pb, target)
    assert np.abs(g[-64:]).max() < 1e-12
