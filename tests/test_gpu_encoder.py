"""The encoder's CUDA forward/backward against the float64 reference (oracle/encoder_ref.py).

The CUDA network keeps activations in bfloat16 (weights are bfloat16 too; the
reference is given the same bfloat16-rounded weights and input), so values
agree to bfloat16 precision, not bit for bit: embeddings within 3e-2 relative
(L2 over the batch) and every parameter block's gradient within 5e-2 relative
with cosine similarity above 0.999.
"""

import numpy as np
import pytest
import torch

from oracle import encoder_ref as R
from paper_2307_04904_gb300 import api, synth

pytestmark = pytest.mark.gpu


def _quantised_params(seed):
    theta = R.init_params(seed).astype(np.float32)
    P = R.unpack(theta)
    rng = np.random.default_rng(seed + 1)
    for b in ("b1", "b2", "b3", "bl"):
        P[b] = rng.normal(0, 0.05, P[b].shape)
    for w in ("W1", "W2", "W3", "Wl"):
        P[w] = R.bf16_round(P[w].astype(np.float32)).astype(np.float64)
    return R.pack(P).astype(np.float32)


def _series(S, T, seed):
    v, o, _ = synth.five_class_set(S, T, seed=seed)
    return v.reshape(S, T)


_GAMMA = np.uint64(0x9E3779B97F4A7C15)


def _splitmix64_at(seed, c):
    """Output c (1-based) of the splitmix64 stream of `seed` (Steele, Lea & Flood 2014), vectorised."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + c.astype(np.uint64) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def _init_params_replay(seed):
    """The documented device initialisation: parameter i = std * z_i, z_i by Box-Muller (float64)
    from outputs 2i+1 (u1 in (0, 1]) and 2i+2 (u2 in [0, 1)) of the stream, std in float32."""
    n = R.N_PARAMS
    i = np.arange(n, dtype=np.uint64)
    u1 = ((_splitmix64_at(seed, 2 * i + 1) >> np.uint64(11)) + np.uint64(1)).astype(np.float64) * 2.0 ** -53
    u2 = (_splitmix64_at(seed, 2 * i + 2) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    z = (np.sqrt(-2.0 * np.log(u1)) * np.cos(6.283185307179586 * u2)).astype(np.float32)
    sd = {"W1": np.sqrt(np.float32(2) / np.float32(7)), "W2": np.sqrt(np.float32(2) / np.float32(448)),
          "W3": np.sqrt(np.float32(2) / np.float32(448)), "Wl": np.float32(0.125)}
    std = np.zeros(n, np.float32)
    o = 0
    for name, shape in R.SHAPES:
        k = int(np.prod(shape))
        std[o:o + k] = sd.get(name, np.float32(0))
        o += k
    return std * z, std


def test_splitmix64_replay_matches_the_oracle_stream():
    from oracle import proposal_ref as P

    state, outs = 12345, []
    for _ in range(5):
        state, out = P.splitmix64(state)
        outs.append(out)
    got = _splitmix64_at(12345, np.arange(1, 6, dtype=np.uint64))
    assert [int(v) for v in got] == outs


@pytest.mark.parametrize("seed", [0, 7, 2**63 + 5])
def test_device_init_params_follow_their_definition(seed):
    """dtw_encoder_init_params against a float64 replay of its documented draw.  The device's
    float64 log and cos are within a few ulp of numpy's, so (float)z agrees except where z lies
    within ~1e-16 of a float32 rounding boundary: every parameter within two float32 steps
    (5e-7 relative), biases exactly zero; each weight block has mean ~0 and its stated std."""
    enc = api.Encoder(64, 2)
    enc.init_params(seed)
    got = enc.params()
    enc.init_params(seed)
    assert np.array_equal(enc.params(), got)  # deterministic
    enc.init_params(seed + 1)
    assert not np.array_equal(enc.params(), got)
    ref, std = _init_params_replay(seed)
    assert np.all(got[std == 0] == 0.0)
    np.testing.assert_allclose(got, ref, rtol=5e-7, atol=0)
    o = 0
    for name, shape in R.SHAPES:
        k = int(np.prod(shape))
        blk = got[o:o + k].astype(np.float64)
        if name.startswith("W"):
            s = float(std[o])
            assert abs(blk.mean()) < 5 * s / np.sqrt(k)
            assert abs(blk.std() / s - 1) < 5 / np.sqrt(2 * k)
        o += k
    enc.close()


@pytest.mark.parametrize("S", [2, 7, 633])
def test_targets_match_reference(S):
    """dtw_encoder_targets: sqrt(D) over the mean of the off-diagonal sqrt(D), zero diagonal.
    Both sides take the square roots, the sum and the quotient in float64 (correctly rounded);
    only the order of the sum differs (relative 1e-15), so after the rounding to float32 every
    target is within one float32 step (2e-7 relative) of the reference."""
    rng = np.random.default_rng(S)
    A = rng.gamma(2.0, 50.0, (S, S)).astype(np.float32)
    D = np.triu(A, 1)
    D = D + D.T
    if S > 2:
        D[0, 1] = D[1, 0] = 0.0  # two identical series: a zero distance, a zero target
    got = api.Encoder.targets(torch.from_numpy(D).cuda()).cpu().numpy()
    sq = np.sqrt(D.astype(np.float64))
    off = ~np.eye(S, dtype=bool)
    ref = (sq / (sq[off].sum() / (S * (S - 1)))).astype(np.float32)
    assert np.all(np.diag(got) == 0.0)
    np.testing.assert_allclose(got[off], ref[off], rtol=2e-7, atol=0)
    assert abs(got[off].astype(np.float64).mean() - 1.0) < 1e-6  # unit-mean by construction


@pytest.mark.parametrize("B,T", [(12, 128), (5, 192), (300, 64)])
def test_embedding_matches_reference(B, T):
    # T = 192 ends in a partial 128-step tile; 300 series x 64 steps give more
    # tiles than there are CTAs
    theta = _quantised_params(3)
    x = _series(B, T, 4)
    enc = api.Encoder(T, max(B, 2), theta)
    e = enc.embed(torch.from_numpy(x).cuda()).cpu().numpy()
    ref, _ = R.forward(theta.astype(np.float64), R.bf16_round(x).astype(np.float64))
    assert np.linalg.norm(e - ref) / np.linalg.norm(ref) < 3e-2
    enc.close()


@pytest.mark.parametrize("S,T", [(10, 64), (6, 192), (3, 320)])
def test_gradients_match_reference(S, T):
    theta = _quantised_params(5)
    x = _series(S, T, 6)
    rng = np.random.default_rng(7)
    tgt = rng.uniform(0.5, 2.0, (S, S)).astype(np.float32)
    tgt = np.triu(tgt, 1) + np.triu(tgt, 1).T
    enc = api.Encoder(T, S, theta)
    losses = enc.train(torch.from_numpy(x).cuda(), torch.from_numpy(tgt).cuda(), 0.0, 1,
                       graph=False)
    g = enc.grads().astype(np.float64)
    assert np.allclose(enc.params(), theta)  # lr = 0 leaves the parameters alone
    enc.check()
    pa, pb = np.triu_indices(S, 1)
    L, gref = R.backward(theta.astype(np.float64), R.bf16_round(x).astype(np.float64), pa, pb,
                         tgt[pa, pb].astype(np.float64))
    assert float(losses[0]) == pytest.approx(L, rel=2e-2)
    off = 0
    for name, shape in R.SHAPES:
        n = int(np.prod(shape))
        a, b = g[off:off + n], gref[off:off + n]
        off += n
        if name == "bl":
            # pair distances do not change when every embedding moves by the same
            # vector, so the exact gradient of bl is 0: only rounding remains
            assert np.linalg.norm(a) < 1e-4 * np.linalg.norm(g) and np.linalg.norm(b) < 1e-9
            continue
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        cos = a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30)
        assert rel < 5e-2 and cos > 0.999, (name, rel, cos)
    enc.close()


def test_training_lowers_the_loss_and_graph_equals_eager():
    S, T = 64, 128
    x = _series(S, T, 8)
    rng = np.random.default_rng(9)
    pts = rng.standard_normal((S, 4))
    tgt = np.sqrt(((pts[:, None] - pts[None]) ** 2).sum(-1)).astype(np.float32)
    theta = R.init_params(11)
    xs, ts = torch.from_numpy(x).cuda(), torch.from_numpy(tgt).cuda()
    a = api.Encoder(T, S, theta)
    la = a.train(xs, ts, 1e-3, 60, graph=True).cpu().numpy()
    b = api.Encoder(T, S, theta)
    lb = b.train(xs, ts, 1e-3, 60, graph=False).cpu().numpy()
    assert np.array_equal(la, lb) and np.array_equal(a.params(), b.params())
    assert la[-1] < 0.5 * la[0]
    a.close()
    b.close()


def _close(got, ref, rel, atol_frac, what):
    """Element-wise |got - ref| <= rel |ref| + atol_frac * rms(ref)."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    assert got.shape == ref.shape, what
    scale = float(np.sqrt(np.mean(ref * ref))) or 1.0
    err = np.abs(got - ref)
    lim = rel * np.abs(ref) + atol_frac * scale
    worst = np.unravel_index(np.argmax(err - lim), err.shape)
    assert np.all(err <= lim), (what, worst, float(got[worst]), float(ref[worst]), scale)


# bfloat16 keeps 8 significant bits: storing a float32 result rounds it by at most 2^-9
# relative, so 2^-8 leaves a factor of two; the float32 accumulations of at most 448
# products add far less than 1e-3 of a layer's RMS.  A tile-edge, halo or channel error
# moves an element by the order of its own value and fails these bounds.
BF16_REL = 2.0 ** -8
ACC_ATOL = 1e-3


@pytest.mark.parametrize("S,T", [(6, 192), (10, 64), (3, 320), (150, 128)])
def test_layers_elementwise_given_their_inputs(S, T):
    """Every layer of one training step, element by element, against the float64 reference
    fed the layer's own GPU inputs (bfloat16 values widened exactly): z1 and h1 from the
    bf16-rounded series; z_l, h_l from h_{l-1}; e from h3; dL/de from e and the targets;
    dz3 from dL/de and z3; dz2, dz1 through the transposed convolutions and GELU' of the
    stored z; every weight and bias gradient from the stored activations and their
    gradients.  T = 192 and 320 end in partial 128-step tiles (halo rows at the tile and
    series edges); S = 150 gives more tiles than there are persistent CTAs."""
    theta = _quantised_params(S + T)
    P = R.unpack(theta.astype(np.float64))
    x = _series(S, T, S * 3 + 1)
    rng = np.random.default_rng(S + 2 * T)
    tgt = rng.uniform(0.5, 2.0, (S, S)).astype(np.float32)
    tgt = np.triu(tgt, 1) + np.triu(tgt, 1).T
    enc = api.Encoder(T, S, theta)
    enc.train(torch.from_numpy(x).cuda(), torch.from_numpy(tgt).cuda(), 0.0, 1, graph=False)
    enc.check()
    t = {n: enc.tensor(n).astype(np.float64) for n in api.Encoder.TENSORS}
    g = enc.grads().astype(np.float64)
    G = R.unpack(g)
    enc.close()
    xq = R.bf16_round(x).astype(np.float64)
    xs = R.conv1_taps(xq)
    # forward
    z1 = np.einsum("btk,ok->bto", xs, P["W1"]) + P["b1"]
    _close(t["z1"], z1, BF16_REL, ACC_ATOL, "z1")
    _close(t["h1"], R.gelu(z1), BF16_REL, ACC_ATOL, "h1")
    z2 = R.conv(t["h1"], P["W2"]) + P["b2"]
    _close(t["z2"], z2, BF16_REL, ACC_ATOL, "z2")
    _close(t["h2"], R.gelu(z2), BF16_REL, ACC_ATOL, "h2")
    z3 = R.conv(t["h2"], P["W3"]) + P["b3"]
    _close(t["z3"], z3, BF16_REL, ACC_ATOL, "z3")
    _close(t["h3"], R.gelu(z3), BF16_REL, ACC_ATOL, "h3")
    gpool = t["h3"].mean(1)
    _close(t["e"], gpool @ P["Wl"].T + P["bl"], 1e-5, 1e-5, "e")  # float32 arithmetic
    # backward
    pa, pb = np.triu_indices(S, 1)
    _, dE = R.pair_loss_grad(t["e"], pa, pb, tgt[pa, pb].astype(np.float64))
    _close(t["dE"], dE, 1e-4, 1e-4, "dE")
    dz3 = ((t["dE"] @ P["Wl"])[:, None, :] / T) * R.gelu_grad(t["z3"])
    _close(t["dz3"], dz3, BF16_REL, ACC_ATOL, "dz3")
    dW3, dh2 = R.conv_back(t["dz3"], t["h2"], P["W3"])
    _close(t["dz2"], dh2 * R.gelu_grad(t["z2"]), BF16_REL, ACC_ATOL, "dz2")
    dW2, dh1 = R.conv_back(t["dz2"], t["h1"], P["W2"])
    _close(t["dz1"], dh1 * R.gelu_grad(t["z1"]), BF16_REL, ACC_ATOL, "dz1")
    # gradients: float32 sums of exact bf16 products (tensor cores, fixed-order partials)
    _close(G["W3"], dW3, 1e-4, ACC_ATOL, "dW3")
    _close(G["W2"], dW2, 1e-4, ACC_ATOL, "dW2")
    _close(G["W1"], np.einsum("bto,btk->ok", t["dz1"], xs), 1e-4, ACC_ATOL, "dW1")
    _close(G["b3"], t["dz3"].sum((0, 1)), 1e-4, ACC_ATOL, "db3")
    _close(G["b2"], t["dz2"].sum((0, 1)), 1e-4, ACC_ATOL, "db2")
    _close(G["b1"], t["dz1"].sum((0, 1)), 1e-4, ACC_ATOL, "db1")
    _close(G["Wl"], t["dE"].T @ gpool, 1e-4, 1e-4, "dWl")
    # bl's exact gradient is 0 (translation invariance); compare to the rounding level
    assert np.abs(G["bl"]).max() <= 1e-4 * np.abs(G["Wl"]).max()


def test_inference_embedding_equals_the_training_forward():
    """dtw_encoder_embed runs the same kernels as the training forward: its embeddings
    equal the training step's e bit for bit, so the layer checks above cover it."""
    S, T = 40, 192
    theta = _quantised_params(21)
    x = _series(S, T, 22)
    tgt = np.ones((S, S), np.float32)
    enc = api.Encoder(T, S, theta)
    xt = torch.from_numpy(x).cuda()
    enc.train(xt, torch.from_numpy(tgt).cuda(), 0.0, 1, graph=False)
    e_train = enc.tensor("e")
    e_inf = enc.embed(xt).cpu().numpy()
    enc.close()
    assert np.array_equal(e_train.view(np.uint32), e_inf.view(np.uint32))
