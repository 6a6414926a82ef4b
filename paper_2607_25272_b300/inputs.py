"""Seeded synthetic least-squares problems Y = X beta + zeta (Eq. model).

This module generates inputs only; it holds none of SPCG's arithmetic.  It is
the one module that both the CUDA path's tests/bench and the CPU oracle's
tests read their inputs from.  Every generator is a pure function of its
arguments (numpy PCG64 streams), FP64 on the host.

Problem families:
* ``gaussian_problem``   - X_ij iid N(0,1), beta iid N(0,1), zeta iid N(0, sigma^2).
* ``svd_problem``        - X = U diag(s) V^T with U a random N x d orthonormal
  basis (CholeskyQR2 of a Gaussian matrix, optionally with rows scaled by
  |Student-t(df)| before orthonormalising, which gives heavy-tailed leverage
  scores while keeping kappa(X) exact), V a random d x d orthogonal matrix and
  s geometric from 1 to 1/kappa.
* ``paper_problem``      - the experimental design of Sec. 4: X = G diag(s~),
  s~ geometric from 1 to 1/kappa, beta iid N(0,1), zeta iid N(0, sigma^2).
* ``scaled_columns_problem`` - X_ij iid N(0,1) times per-column scales
  log-uniform in [lo, hi] (the batched workload).
"""
import numpy as np


def _response(X, beta, zeta):
    # Row sums without BLAS so that Y does not depend on the BLAS kernel.
    return (X * beta[None, :]).sum(axis=1) + zeta


def gaussian_problem(N, d, sigma=1.0, seed=1):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((N, d))
    beta = rng.standard_normal(d)
    zeta = sigma * rng.standard_normal(N)
    return X, _response(X, beta, zeta), beta


def orthonormal_basis(G):
    """CholeskyQR2: two rounds of G <- G chol(G^T G)^{-T}."""
    Q = np.array(G, dtype=np.float64, copy=True)
    for _ in range(2):
        L = np.linalg.cholesky(Q.T @ Q)
        # Q <- Q L^{-T}: solve L Q^T = Q^T column block by column block.
        Q = np.linalg.solve(L, Q.T).T
    return np.ascontiguousarray(Q)


def svd_problem(N, d, kappa, sigma, seed=1, leverage_df=None):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((N, d))
    if leverage_df is not None:
        w = np.abs(rng.standard_t(leverage_df, size=N))
        G *= w[:, None]
    U = orthonormal_basis(G)
    del G
    V, _ = np.linalg.qr(rng.standard_normal((d, d)))
    s = kappa ** (-np.arange(d) / max(d - 1, 1))
    U *= s[None, :]
    X = np.ascontiguousarray(U @ V.T)
    del U
    beta = rng.standard_normal(d)
    zeta = sigma * rng.standard_normal(N)
    return X, _response(X, beta, zeta), beta


def paper_problem(N, d, kappa, sigma2, seed=1):
    rng = np.random.default_rng(seed)
    s = kappa ** (-np.arange(d) / max(d - 1, 1))
    X = rng.standard_normal((N, d)) * s[None, :]
    beta = rng.standard_normal(d)
    zeta = np.sqrt(sigma2) * rng.standard_normal(N)
    return X, _response(X, beta, zeta), beta


def scaled_columns_problem(N, d, lo, hi, sigma, seed=1):
    rng = np.random.default_rng(seed)
    c = 10.0 ** rng.uniform(np.log10(lo), np.log10(hi), size=d)
    X = rng.standard_normal((N, d)) * c[None, :]
    beta = rng.standard_normal(d)
    zeta = sigma * rng.standard_normal(N)
    return X, _response(X, beta, zeta), beta


def svd_problem_device(N, d, kappa, sigma, seed=1, leverage_df=None, device="cuda"):
    """The svd_problem recipe drawn on a CUDA device with torch (for sizes
    whose host generation takes minutes).  Same construction, a different
    random stream: G iid N(0,1) (rows optionally scaled by |Student-t(df)|,
    drawn as z / sqrt(chi2_df / df)), U = CholeskyQR2(G), V from the QR of a
    Gaussian d x d matrix, s geometric from 1 to 1/kappa, X = U diag(s) V^T,
    beta iid N(0,1), Y = X beta + sigma zeta.

    Returns (X, Y, beta, U^T Y, s, V) as FP64 device tensors; U itself is
    not kept (N x d), but U^T Y, s and V are what a caller needs to form the
    OLS estimator of this construction in closed form."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    f64 = torch.float64
    G = torch.randn((N, d), dtype=f64, device=device, generator=g)
    if leverage_df is not None:
        z = torch.randn(N, dtype=f64, device=device, generator=g)
        chi = (torch.randn((N, int(leverage_df)), dtype=f64, device=device, generator=g) ** 2).sum(1)
        G *= (z / torch.sqrt(chi / leverage_df)).abs()[:, None]
    for _ in range(2):
        L = torch.linalg.cholesky(G.T @ G)
        G = torch.linalg.solve_triangular(L, G.T, upper=False).T.contiguous()
    V, _ = torch.linalg.qr(torch.randn((d, d), dtype=f64, device=device, generator=g))
    s = float(kappa) ** (-torch.arange(d, dtype=f64, device=device) / max(d - 1, 1))
    X = (G * s[None, :]) @ V.T
    beta = torch.randn(d, dtype=f64, device=device, generator=g)
    Y = X @ beta + sigma * torch.randn(N, dtype=f64, device=device, generator=g)
    uty = G.T @ Y
    del G
    return X.contiguous(), Y, beta, uty, s, V


def scaled_columns_problem_device(N, d, lo, hi, sigma, seed=1, device="cuda",
                                  dtype=None):
    """The scaled_columns_problem recipe drawn on a CUDA device with torch
    (same construction, a different random stream): X_ij iid N(0,1) times
    per-column scales 10^U(log10 lo, log10 hi), beta iid N(0,1),
    Y = X beta + sigma zeta, formed in FP64 and returned in `dtype`
    (default float64)."""
    import math

    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    f64 = torch.float64
    c = 10.0 ** (math.log10(lo) + (math.log10(hi) - math.log10(lo)) *
                 torch.rand(d, dtype=f64, device=device, generator=g))
    X = torch.randn((N, d), dtype=f64, device=device, generator=g) * c[None, :]
    beta = torch.randn(d, dtype=f64, device=device, generator=g)
    Y = X @ beta + sigma * torch.randn(N, dtype=f64, device=device, generator=g)
    if dtype is not None:
        X, Y = X.to(dtype), Y.to(dtype)
    return X, Y, beta
