"""Pins for the oracle MLP of the learned schedule."""
import numpy as np

from oracle import mlp as M


def test_backward_matches_central_differences():
    rng = np.random.default_rng(0)
    n_out = 7
    theta = rng.standard_normal(M.n_params(n_out)) * 0.3
    x = rng.standard_normal((9, 4))
    t = rng.standard_normal((9, n_out))
    _, g = M.loss_and_grad(theta, x, t, n_out)
    h = 1e-6
    idx = rng.choice(theta.size, 60, replace=False)
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        lp, _ = M.loss_and_grad(theta + e, x, t, n_out)
        lm, _ = M.loss_and_grad(theta - e, x, t, n_out)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i]))


def test_zero_input_gives_bias_path():
    n_out = 5
    rng = np.random.default_rng(1)
    theta = rng.standard_normal(M.n_params(n_out))
    W1, b1, W2, b2, W3, b3 = M.unpack(theta, n_out)
    y, _ = M.forward(theta, np.zeros((1, 4)), n_out)
    h1 = np.maximum(b1, 0)
    h2 = np.maximum(W2 @ h1 + b2, 0)
    assert np.allclose(y[0], W3 @ h2 + b3)


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, -3.14159, 0.0])
    r = M.bf16_round(x)
    # 8 significant bits: spacing 2^-7 at 1.0; ties go to even
    assert r[0] == 1.0
    assert r[1] == 1.0                       # 1 + 2^-8 is a tie: the even neighbour is 1.0
    assert r[2] == 1.0                       # 1 + 2^-9 is below half a spacing
    assert r[3] == 1.0 + 2 ** -7             # 1 + 3 * 2^-9 rounds up
    assert abs(r[4] - (-3.140625)) < 1e-12
    assert r[5] == 0.0
