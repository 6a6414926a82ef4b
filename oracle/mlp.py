"""The schedule model's MLP in FP64 (oracle side; test infrastructure).

A 4 -> 64 -> 64 -> n_out multilayer perceptron with ReLU hidden layers
predicts, from four features of a problem, the log10 cost of each candidate
sketch-size schedule; the loss is the mean squared error over the batch and
the outputs.  The forward pass uses the BF16-rounded weights (the network's
deployed precision); gradients are taken with respect to those weights.

Parameter vector layout (the CUDA side uses the same layout, defined here in
words): W1 (64 x 4, row-major), b1 (64), W2 (64 x 64), b2 (64),
W3 (n_out x 64), b3 (n_out).

Pins (tests/test_oracle_mlp.py): the backward pass equals central finite
differences of the loss; a zero-input network reduces to its biases; the
forward outputs, loss and gradient equal those of the same network built from
torch's linear layers with automatic differentiation; the BF16 rounding
equals torch's FP32 -> BF16 conversion.
"""
import numpy as np

H = 64
NIN = 4


def n_params(n_out):
    return H * NIN + H + H * H + H + n_out * H + n_out


def unpack(theta, n_out):
    theta = np.asarray(theta, dtype=np.float64)
    o = 0
    W1 = theta[o:o + H * NIN].reshape(H, NIN); o += H * NIN
    b1 = theta[o:o + H]; o += H
    W2 = theta[o:o + H * H].reshape(H, H); o += H * H
    b2 = theta[o:o + H]; o += H
    W3 = theta[o:o + n_out * H].reshape(n_out, H); o += n_out * H
    b3 = theta[o:o + n_out]; o += n_out
    return W1, b1, W2, b2, W3, b3


def forward(theta, x, n_out):
    W1, b1, W2, b2, W3, b3 = unpack(theta, n_out)
    z1 = x @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3.T + b3
    return y, (x, z1, h1, z2, h2)


def loss_and_grad(theta, x, target, n_out):
    """MSE = mean over batch and outputs of (y - target)^2, and d MSE / d theta."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, n_out)
    y, (x, z1, h1, z2, h2) = forward(theta, x, n_out)
    B = x.shape[0]
    diff = y - target
    loss = float(np.mean(diff ** 2))
    dy = 2.0 * diff / (B * n_out)
    gW3 = dy.T @ h2
    gb3 = dy.sum(0)
    dh2 = dy @ W3
    dz2 = dh2 * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (z1 > 0)
    gW1 = dz1.T @ x
    gb1 = dz1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def bf16_round(a):
    """Round FP32/FP64 values to the nearest BF16 (ties to even), as FP64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64)
