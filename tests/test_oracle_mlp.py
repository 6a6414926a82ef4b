"""Pins for the oracle MLP of the learned schedule."""
import numpy as np
import pytest

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


def _torch_network(theta, x, target, n_out):
    """The same 4 -> 64 -> 64 -> n_out ReLU network built from torch's own
    linear layers (CPU, FP64), from the documented parameter layout: W1
    (64 x 4, row-major), b1, W2 (64 x 64), b2, W3 (n_out x 64), b3."""
    import torch
    import torch.nn.functional as F
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    sizes = [(64, 4), (64,), (64, 64), (64,), (n_out, 64), (n_out,)]
    parts, o = [], 0
    for shp in sizes:
        n = int(np.prod(shp))
        parts.append(th[o:o + n].reshape(shp))
        o += n
    assert o == th.numel()
    W1, b1, W2, b2, W3, b3 = parts
    xt = torch.tensor(x, dtype=torch.float64)
    y = F.linear(F.relu(F.linear(F.relu(F.linear(xt, W1, b1)), W2, b2)), W3, b3)
    loss = F.mse_loss(y, torch.tensor(target, dtype=torch.float64))
    loss.backward()
    return y.detach().numpy(), float(loss.detach()), th.grad.numpy()


def test_forward_loss_and_gradient_match_torch_autograd():
    """Forward outputs, the MSE loss and its gradient in the parameter layout
    against torch's linear layers and automatic differentiation: a transposed
    weight, a misplaced bias or a wrong slice of the layout changes them at
    O(1), rounding only at 1e-12."""
    pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    for n_out in (1, 7, 25):
        theta = rng.standard_normal(M.n_params(n_out)) * 0.3
        x = rng.standard_normal((11, 4))
        t = rng.standard_normal((11, n_out))
        y, _ = M.forward(theta, x, n_out)
        loss, g = M.loss_and_grad(theta, x, t, n_out)
        y_t, loss_t, g_t = _torch_network(theta, x, t, n_out)
        assert np.allclose(y, y_t, rtol=1e-12, atol=1e-12)
        assert abs(loss - loss_t) <= 1e-12 * max(1.0, loss_t)
        assert np.allclose(g, g_t, rtol=1e-10, atol=1e-12)


def test_bf16_rounding_matches_torch_conversion():
    """bf16_round against torch's FP32 -> BF16 conversion (round to nearest,
    ties to even) on random FP32 values over the whole exponent range, exact
    ties in both directions and subnormals."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    bits = rng.integers(0, 2**32, size=20000, dtype=np.uint64).astype(np.uint32)
    f = bits.view(np.float32)
    f = f[np.isfinite(f)]
    base = rng.integers(0, 2**16, size=2000, dtype=np.uint64).astype(np.uint32) << np.uint32(16)
    ties = (base | np.uint32(0x8000)).view(np.float32)          # exactly half way
    ties = ties[np.isfinite(ties)]
    sub = (rng.integers(1, 2**23, size=2000, dtype=np.uint64).astype(np.uint32)).view(np.float32)
    vals = np.concatenate([f, ties, sub]).astype(np.float32)
    ours = M.bf16_round(vals)
    ref = torch.from_numpy(vals).to(torch.bfloat16).to(torch.float64).numpy()
    same = (ours == ref) | (np.isnan(ours) & np.isnan(ref))
    assert np.all(same)
