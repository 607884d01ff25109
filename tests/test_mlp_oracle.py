"""Pins of the FP64 network oracle (oracle/mlp.py), without a GPU."""
import numpy as np

from oracle import mlp


def _batch(seed, m=37):
    g = np.random.default_rng(seed)
    feat = g.standard_normal((m, mlp.IN)) * 3 + 1
    target = g.standard_normal(m) * 2 - 5
    p = mlp.init_params(seed, in_mu=g.standard_normal(mlp.IN), in_sigma=g.random(mlp.IN) + 0.5,
                        out_mu=-4.0, out_sigma=2.5)
    # non-zero biases so every ReLU sees both signs
    d = mlp.unpack(p)
    for name in ("b1", "b2", "b3"):
        d[name] = g.standard_normal(mlp.HID) * 0.3
    d["b4"] = [0.7]
    return mlp.pack(d), feat, target


def test_gradient_matches_central_differences():
    p, feat, target = _batch(1)
    L, g = mlp.loss_and_grad(p, feat, target)
    assert np.isclose(L, mlp.loss(p, feat, target))
    rng = np.random.default_rng(2)
    idx = np.concatenate([rng.choice(np.arange(mlp.TRAINABLE_FROM, mlp.NPARAM), 60, replace=False),
                          [mlp.NPARAM - 1]])
    fd = mlp.grad_fd(p, feat, target, idx)
    assert np.allclose(g[idx], fd, rtol=1e-5, atol=1e-8)
    assert np.all(g[:mlp.TRAINABLE_FROM] == 0.0)  # normalisation is not trained


def test_planted_mistake_is_caught():
    # a backward pass that forgets the ReLU mask of the second layer disagrees
    p, feat, target = _batch(3)
    d = mlp.unpack(p)
    _, (x, h1, h2, h3) = mlp.forward(p, feat)
    y, _ = mlp.forward(p, feat)
    t = (target - d["out_mu"][0]) / d["out_sigma"][0]
    dy = 2.0 * (y - t) / len(y)
    dz3 = np.outer(dy, d["w4"]) * (h3 > 0)
    dz2_wrong = dz3 @ d["W3"]  # mask dropped
    gW2_wrong = (dz2_wrong.T @ h1).reshape(-1)
    off = sum(s for name, s in mlp.SIZES[:mlp.SIZES.index(("W2", mlp.HID * mlp.HID))])
    idx = off + np.arange(0, 4096, 97)
    fd = mlp.grad_fd(p, feat, target, idx)
    assert not np.allclose(gW2_wrong[idx - off], fd, rtol=1e-3, atol=1e-6)


def test_closed_form_constant_network():
    # all weights zero: the prediction is b4, loss = mean((b4 - t_norm)^2)
    d = mlp.unpack(mlp.init_params(0))
    for name in ("W1", "b1", "W2", "b2", "W3", "b3", "w4"):
        d[name] = np.zeros_like(d[name])
    d["b4"] = [1.5]
    d["out_mu"], d["out_sigma"] = [2.0], [4.0]
    p = mlp.pack(d)
    target = np.array([2.0, 6.0, 10.0])  # normalised: 0, 1, 2
    L, g = mlp.loss_and_grad(p, np.zeros((3, mlp.IN)), target)
    assert np.isclose(L, ((1.5 - 0) ** 2 + (1.5 - 1) ** 2 + (1.5 - 2) ** 2) / 3)
    assert np.isclose(g[-1], 2 * ((1.5 - 0) + (1.5 - 1) + (1.5 - 2)) / 3)
    assert np.all(g[:-1] == 0)


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, -2.5, 3.0e-3])
    got = mlp.bf16(vals)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: to even (1); 1 + 3*2^-8 ties up to 1 + 2^-6
    assert got[0] == 1.0 and got[1] == 1.0 and got[2] == 1.0 + 2 ** -6 and got[3] == 1.0
    assert got[4] == -2.5
    assert abs(got[5] - 3.0e-3) <= 3.0e-3 * 2 ** -8


def test_forward_bf16_close_to_exact_forward():
    p, feat, _ = _batch(4, m=200)
    d = mlp.unpack(p)
    y, _ = mlp.forward(p, feat)
    exact = y * d["out_sigma"][0] + d["out_mu"][0] + d["margin"][0]
    approx = mlp.forward_bf16(p, feat)
    assert np.max(np.abs(exact - approx)) < 0.05 * (np.max(np.abs(exact)) + 1)
