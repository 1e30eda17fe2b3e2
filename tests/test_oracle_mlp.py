"""Pins of the oracle's visibility-surrogate MLP (CPU only): bf16 rounding
against torch's conversion, the encoding's closed form, a forward pass whose
output is known in closed form, the BCE gradient p - y, FP64 finite
differences of the whole backward (exact mode), and Adam against
torch.optim.Adam."""
import math

import numpy as np
import pytest
import torch

NP = 128 * 80 + 128 + 3 * (128 * 128 + 128) + 128 + 1
OFF_W1, OFF_B1 = 0, 128 * 80
OFF_W2 = OFF_B1 + 128
OFF_W4 = OFF_W2 + 2 * (128 * 128 + 128)
OFF_W5 = OFF_W4 + 128 * 128 + 128
OFF_B5 = OFF_W5 + 128


def test_param_count(orc):
    assert orc.mlp_nparam() == NP


def test_bf16_rounding_matches_torch(orc):
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(5000) * 10 ** rng.uniform(-8, 8, 5000),
                        [0.0, -0.0, 1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -9, 1 + 2 ** -9]])
    x = x.astype(np.float32).astype(np.float64)
    want = torch.from_numpy(x).float().to(torch.bfloat16).double().numpy()
    np.testing.assert_array_equal(orc.bf16_round(x), want)


def test_encoding_closed_form(orc):
    lo = np.array([-1, -2, 0], np.float32)
    hi = np.array([1, 2, 4], np.float32)
    pos = np.array([[-1, -2, 0], [1, 2, 4], [0.5, 1.0, 3.0]], np.float32)
    dirs = np.array([[0, 0, 1], [1, 0, 0], [0.6, 0.8, 0]], np.float32)
    f = orc.mlp_encode(pos, dirs, lo, hi)
    assert f.shape == (3, 80)
    np.testing.assert_array_equal(f[:, 78:], 0)
    # position normalised to [-1, 1]
    np.testing.assert_allclose(f[0, [0, 13, 26]], -1)
    np.testing.assert_allclose(f[1, [0, 13, 26]], 1)
    np.testing.assert_allclose(f[2, [0, 13, 26]], [0.5, 0.5, 0.5])
    # x = 0.5: sin/cos(2^k pi / 2)
    want = [0.5]
    for k in range(6):
        a = (2 ** k) * math.pi * 0.5
        want += [math.sin(a), math.cos(a)]
    np.testing.assert_allclose(f[2, :13], want, atol=1e-15)
    np.testing.assert_allclose(f[2, [39, 52, 65]], [0.6, 0.8, 0.0], rtol=1e-7)


def test_forward_closed_form(orc):
    """Weights that route feature 0 (normalised x) through the first unit of
    every layer: z5 = c * relu(x) + beta, exactly for bf16-representable x."""
    P = np.zeros(NP, np.float32)
    P[OFF_W1 + 0 * 80 + 0] = 1.0
    for l in range(3):
        P[OFF_W2 + l * (128 * 128 + 128)] = 1.0
    P[OFF_W5] = 2.5
    P[OFF_B5] = -0.75
    lo = np.zeros(3, np.float32)
    hi = np.ones(3, np.float32)
    xs = np.array([0.0, 0.25, 0.625, 0.875, 1.0], np.float32)  # p_n = 2x - 1
    pos = np.stack([xs, xs, xs], 1)
    dirs = np.tile(np.array([[0, 0, 1]], np.float32), (5, 1))
    p, z = orc.mlp_forward(P, orc.mlp_encode(pos, dirs, lo, hi))
    want = 2.5 * np.maximum(2 * xs.astype(np.float64) - 1, 0) - 0.75
    np.testing.assert_array_equal(z, want)
    np.testing.assert_allclose(p, 1 / (1 + np.exp(-want)), rtol=1e-15)


def test_bce_gradient_is_p_minus_y(orc):
    P = np.zeros(NP, np.float32)
    P[OFF_B5] = 0.3
    rng = np.random.default_rng(1)
    feat = rng.uniform(-1, 1, (64, 80))
    y = rng.uniform(0, 1, 64)
    loss, g = orc.mlp_loss_grad(P, feat, y)
    p = 1 / (1 + math.exp(-float(np.float32(0.3))))
    assert g[OFF_B5] == pytest.approx(np.mean(p - y), rel=1e-12)
    want = -np.mean(y * math.log(p) + (1 - y) * math.log(1 - p))
    assert loss == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("w", [1.0, 4.0, 30.0])
def test_weighted_bce_minimiser_and_decoding(orc, w):
    """A network that outputs one constant logit b5: the weighted loss over
    targets y is smallest where p = w ybar / (w ybar + 1 - ybar) (a property
    of the loss, found here by minimising it numerically over b5), its
    gradient there is 0, and the visibility decoding returns ybar."""
    rng = np.random.default_rng(8)
    feat = rng.uniform(-1, 1, (64, 80))
    y = np.where(rng.uniform(0, 1, 64) < 0.1, rng.uniform(0, 1, 64), 0.0)
    ybar = y.mean()

    def loss_at(b):
        P = np.zeros(NP, np.float32)
        P[OFF_B5] = b
        return orc.mlp_loss_grad(P, feat, y, pos_weight=w)

    # golden-section search of the loss over b5 (no use of the closed form)
    a, b = -12.0, 6.0
    g = (math.sqrt(5) - 1) / 2
    for _ in range(80):
        c, d = b - g * (b - a), a + g * (b - a)
        if loss_at(c)[0] < loss_at(d)[0]:
            b = d
        else:
            a = c
    z = 0.5 * (a + b)
    p = 1 / (1 + math.exp(-z))
    assert p == pytest.approx(w * ybar / (w * ybar + 1 - ybar), rel=1e-5)
    P = np.zeros(NP, np.float32)
    P[OFF_B5] = z
    _, grad = orc.mlp_loss_grad(P, feat, y, pos_weight=w)
    assert abs(grad[OFF_B5]) < 1e-6
    T = orc.mlp_visibility(P, feat[:4], pos_weight=w)
    np.testing.assert_allclose(T, ybar, rtol=1e-5)
    if w == 1.0:  # plain loss: the decoding is the sigmoid output itself
        np.testing.assert_allclose(T, orc.mlp_forward(P, feat[:4])[0], rtol=1e-15)


def _rand_params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    P = np.zeros(NP, np.float32)
    off = 0
    for kin in (80, 128, 128, 128):
        b = math.sqrt(6.0 / kin) * scale
        P[off:off + 128 * kin] = rng.uniform(-b, b, 128 * kin)
        off += 128 * kin
        P[off:off + 128] = rng.uniform(-0.1, 0.1, 128)
        off += 128
    P[off:off + 128] = rng.uniform(-0.2, 0.2, 128)
    P[off + 128] = 0.1
    return P


@pytest.mark.parametrize("w", [1.0, 12.0])
def test_backward_finite_differences(orc, w):
    orc.mlp_set_bf16(False)
    try:
        P = _rand_params(2)
        rng = np.random.default_rng(3)
        feat = rng.uniform(-1, 1, (16, 80))
        feat[:, 78:] = 0
        y = rng.uniform(0, 1, 16)
        loss, g = orc.mlp_loss_grad(P, feat, y, pos_weight=w)
        idx = np.concatenate([rng.choice(np.arange(OFF_W1, OFF_B1), 40), rng.choice(np.arange(OFF_B1, OFF_W5), 60),
                              np.arange(OFF_W5, OFF_W5 + 8), [OFF_B5]])
        h = 1e-3  # float32 parameters: perturb by a representable step
        for i in idx:
            vals = []
            for sgn in (1, -1):
                P2 = P.copy()
                P2[i] = np.float32(P[i] + sgn * h)
                vals.append(orc.mlp_loss_grad(P2, feat, y, pos_weight=w)[0])
            step = float(np.float32(P[i] + h)) - float(np.float32(P[i] - h))
            fd = (vals[0] - vals[1]) / step
            assert g[i] == pytest.approx(fd, rel=2e-3, abs=1e-7), i
    finally:
        orc.mlp_set_bf16(True)


def test_adam_matches_torch(orc):
    rng = np.random.default_rng(4)
    w = rng.standard_normal(50)
    m = np.zeros(50)
    v = np.zeros(50)
    tw = torch.tensor(w.copy(), requires_grad=True)
    opt = torch.optim.Adam([tw], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for t in range(1, 6):
        g = rng.standard_normal(50)
        orc.adam_step(w, g, m, v, t, lr=1e-2)
        opt.zero_grad()
        tw.grad = torch.tensor(g)
        opt.step()
    np.testing.assert_allclose(w, tw.detach().numpy(), rtol=1e-12, atol=1e-14)
