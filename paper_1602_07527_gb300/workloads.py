"""Seeded synthetic inputs shaped like the workloads the Cholesky derivative
routines are measured on.

This module holds no Cholesky or derivative arithmetic: it only draws random
numbers and evaluates covariance functions, so both the CUDA path and the CPU
oracle can be fed identical inputs from it.  Every array is a NumPy float64
array built with ``numpy.random.default_rng``; each input of a recipe has its
own stream ``default_rng([seed, k])`` so that resizing one input never
changes another.

Recipes
-------
* ``wishart``: A iid N(0,1), Sigma = A A^T + n I (condition number about 5),
  the seeded stand-in for the paper's np.cov(randn(N, 2N)) test matrix.
* ``se``: n points iid U[0,1]^dim, Sigma_ij = exp(-|xi-xj|^2 / (2 ell^2)) +
  jitter delta_ij (squared-exponential covariance).
* ``matern52``: the textbook Matern-5/2 covariance
  (1 + sqrt5 r/ell + 5 r^2/(3 ell^2)) exp(-sqrt5 r/ell) + jitter delta_ij.
* ``lbar``: tril of iid N(0,1) (a reverse-mode seed L_bar).
* ``sigma_dot``: (G + G^T)/2 with G iid N(0,1) (a symmetric forward seed).
"""
import math

import numpy as np


def rng(seed: int, stream: int):
    return np.random.default_rng([int(seed), int(stream)])


def points(n: int, dim: int, seed: int, stream: int = 0):
    return rng(seed, stream).uniform(0.0, 1.0, size=(n, dim))


def _sqdist_rows(X, lo, hi):
    a = X[lo:hi]
    d = (a * a).sum(1)[:, None] + (X * X).sum(1)[None, :] - 2.0 * (a @ X.T)
    np.maximum(d, 0.0, out=d)
    return d


def se_cov(X, ell: float, jitter: float, rows: int = 2048):
    """Squared-exponential covariance of the rows of X plus jitter on the diagonal."""
    n = X.shape[0]
    out = np.empty((n, n))
    for lo in range(0, n, rows):
        hi = min(n, lo + rows)
        out[lo:hi] = np.exp(_sqdist_rows(X, lo, hi) * (-0.5 / (ell * ell)))
    out[np.diag_indices(n)] = 1.0 + jitter
    return out


def matern52_cov(X, ell: float, jitter: float, rows: int = 2048):
    """Matern-5/2 covariance of the rows of X plus jitter on the diagonal."""
    n = X.shape[0]
    out = np.empty((n, n))
    s5 = math.sqrt(5.0)
    for lo in range(0, n, rows):
        hi = min(n, lo + rows)
        r = np.sqrt(_sqdist_rows(X, lo, hi)) / ell
        out[lo:hi] = (1.0 + s5 * r + (5.0 / 3.0) * r * r) * np.exp(-s5 * r)
    out[np.diag_indices(n)] = 1.0 + jitter
    return out


def wishart(n: int, seed: int, stream: int = 0):
    A = rng(seed, stream).standard_normal((n, n))
    return A @ A.T + n * np.eye(n)


def lbar(n: int, seed: int, stream: int = 7):
    return np.tril(rng(seed, stream).standard_normal((n, n)))


def sigma_dot(n: int, seed: int, stream: int = 8):
    G = rng(seed, stream).standard_normal((n, n))
    return 0.5 * (G + G.T)


def se(n: int, seed: int, dim: int = 3, ell: float = 0.3, jitter: float = 1e-4):
    return se_cov(points(n, dim, seed), ell, jitter)


def matern52(n: int, seed: int, dim: int = 4, ell: float = 0.2, jitter: float = 1e-3):
    return matern52_cov(points(n, dim, seed), ell, jitter)


# Named workload recipes -----------------------------------------------------

def plain_case(n: int = 256, seed: int = 1):
    """Single plain-method case: Wishart-like Sigma, L_bar, Sigma_dot."""
    return wishart(n, seed), lbar(n, seed), sigma_dot(n, seed)


def large_se_case(n: int, seed: int = 2, jitter: float = 1e-4):
    """Large FP64 case: SE covariance on [0,1]^3, ell 0.3, plus L_bar."""
    return se(n, seed, 3, 0.3, jitter), lbar(n, seed)


def mixed_matern_case(n: int, seed: int = 3):
    """Mixed-precision case: Matern-5/2 on [0,1]^4, ell 0.2, jitter 1e-3, plus L_bar."""
    return matern52(n, seed, 4, 0.2, 1e-3), lbar(n, seed)


def gp_case(n: int, seed: int = 4):
    """GP likelihood case: inputs on [0,1]^4 and targets y iid N(0,1)."""
    return points(n, 4, seed), rng(seed, 9).standard_normal(n)


def serving_stream(seed: int = 5, rate: float = 2000.0, duration: float = 10.0,
                   n_lo: int = 32, n_hi: int = 4096, mixed_frac: float = 0.5):
    """Poisson arrivals: list of (t_arrival_s, n, mixed: bool, request seed).

    n = round(exp(U[ln n_lo, ln n_hi])) (log-uniform); each request's own
    matrices are drawn on the device from its request seed by the serving
    loop.
    """
    g = rng(seed, 11)
    t, out, k = 0.0, [], 0
    while True:
        t += g.exponential(1.0 / rate)
        if t >= duration:
            break
        n = int(round(math.exp(g.uniform(math.log(n_lo), math.log(n_hi)))))
        out.append((t, n, bool(g.uniform() < mixed_frac), int(seed) * 1000003 + k))
        k += 1
    return out

