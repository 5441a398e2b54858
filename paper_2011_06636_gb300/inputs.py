"""Seeded synthetic inputs for the SRJ solver and its oracle.

This module holds no arithmetic of the method itself: it only draws right-hand
sides, coefficient fields and problem lists from ``numpy`` PCG64 generators
(``default_rng(seed)``), so that the CUDA library and the FP64 oracle are fed
identical data.  Arrays follow the library's layout: x varies fastest, so the
numpy shape is the grid sizes reversed, ``(nz, ny, nx)``.

Recipes (the paper uses no dataset; every workload is synthetic):

* 1D Poisson, 16 sine modes: ``f_i = sum_m a_m sin(k_m pi i / (N+1))``,
  i = 1..N, with 16 distinct wavenumbers k_m drawn uniformly from 1..N and
  amplitudes a_m ~ N(0, 1).
* 2D Poisson on a large grid: f i.i.d. uniform[-1, 1].
* 3D variable-coefficient diffusion: log k is a Gaussian random field with
  covariance exp(-r^2 / (2 L^2)), L = 16 cells, sigma = 1: white noise
  convolved along each axis with a Gaussian of standard deviation L/sqrt(2)
  cells (truncated at 4 standard deviations, reflecting edges), rescaled to
  zero mean and unit variance, times sigma.  k = exp(log k) is drawn on the
  interior plus one ghost layer per axis.  f i.i.d. N(0, 1).
* Batched mixed sizes: square 2D grids with sides uniform in [64, 1024]; half
  of the problems (chosen at random) are the constant-coefficient Laplacian,
  the others the anisotropic operator -eps u_xx - u_yy with eps log-uniform in
  [1e-2, 1]; f i.i.d. N(0, 1).
* The paper's own experiments: b = 1 (Sec. 3, Sec. 4.1) and f = 1 (Sec. 4.2.3).
* Random symmetric diagonally dominant tridiagonal matrices (Sec. 4.1):
  diagonal d_i ~ U[0, 1), off-diagonal e_i = -U[0, 1) (the same array above
  and below the diagonal; the sign follows the 1D Poisson matrix, and a
  diagonal +-1 similarity shows it does not change Jacobi or SRJ
  convergence); every row that is not diagonally dominant gets
  |d_i| = |e_(i-1)| + |e_i|; then d_0 = 2 |e_0| and d_(N-1) = 2 |e_(N-2)|.
* Laplace with Neumann boundaries (Sec. 4.2.2): f = 0, u0 i.i.d.
  uniform[-1, 1].
* Learned selector: initial weights He-uniform (limit sqrt(6 / fan_in)), zero
  biases, parameter order W1 (64x12), b1, W2 (64x64), b2, W3 (25x64), b3; the
  minibatch order of training is a seeded permutation per epoch.
"""
from __future__ import annotations

import math

import numpy as np


def shape_of(n):
    """numpy shape of a grid whose interior sizes are ``n`` (x first)."""
    return tuple(int(v) for v in reversed(list(n)))


def poisson1d_sines(N: int, seed: int, modes: int = 16) -> np.ndarray:
    rng = np.random.default_rng(seed)
    ks = rng.choice(np.arange(1, N + 1), size=min(modes, N), replace=False)
    amps = rng.standard_normal(len(ks))
    i = np.arange(1, N + 1, dtype=np.float64)
    f = np.zeros(N)
    for a, k in zip(amps, ks):
        f += a * np.sin(k * math.pi * i / (N + 1))
    return f


def uniform_rhs(n, seed: int, lo: float = -1.0, hi: float = 1.0,
                dtype=np.float64) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=shape_of(n)).astype(dtype)


def normal_rhs(n, seed: int, dtype=np.float64) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=shape_of(n)).astype(dtype)


def ones_rhs(n, dtype=np.float64) -> np.ndarray:
    return np.ones(shape_of(n), dtype=dtype)


def _gauss_kernel(std: float):
    r = int(math.ceil(4.0 * std))
    t = np.arange(-r, r + 1, dtype=np.float64)
    g = np.exp(-0.5 * (t / std) ** 2)
    return g / g.sum()


def _conv_axis_reflect(a: np.ndarray, g: np.ndarray, axis: int) -> np.ndarray:
    """Convolution along one axis with half-sample symmetric extension
    (d c b a | a b c d)."""
    from scipy.ndimage import convolve1d
    return convolve1d(a, g, axis=axis, mode="reflect")


def lognormal_k(n, seed: int, corr: float = 16.0, sigma: float = 1.0,
                dtype=np.float64) -> np.ndarray:
    """Cell coefficient k with one ghost layer: numpy shape (n[::-1] + 2)."""
    rng = np.random.default_rng(seed)
    shp = tuple(v + 2 for v in shape_of(n))
    g = rng.standard_normal(size=shp)
    ker = _gauss_kernel(corr / math.sqrt(2.0))
    for ax in range(g.ndim):
        g = _conv_axis_reflect(g, ker, ax)
    g = (g - g.mean()) / g.std()
    return np.exp(sigma * g).astype(dtype)


def batched_problems(count: int = 256, seed: int = 0, smin: int = 64,
                     smax: int = 1024):
    """List of dicts {n: [side, side], eps: [eps_x, 1.0], seed_f: int}."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(smin, smax + 1, size=count)
    aniso = rng.permutation(count) < count // 2
    logeps = rng.uniform(math.log(1e-2), math.log(1.0), size=count)
    out = []
    for i in range(count):
        e = math.exp(logeps[i]) if aniso[i] else 1.0
        out.append(dict(n=[int(sides[i]), int(sides[i])], eps=[e, 1.0],
                        seed_f=int(seed * 100003 + i)))
    return out


def random_sdd_tridiagonal(N: int, seed: int):
    """(diag, off) of a random symmetric diagonally dominant tridiagonal
    matrix of order N by the recipe of Sec. 4.1 (module docstring): A_ii =
    diag[i], A_(i,i+1) = A_(i+1,i) = off[i] (off has N entries, the last
    unused)."""
    rng = np.random.default_rng(seed)
    d = rng.random(N)
    e = -rng.random(N)
    e[N - 1] = 0.0
    left = np.concatenate([[0.0], np.abs(e[:N - 1])])
    right = np.abs(e)
    need = left + right
    d = np.where(np.abs(d) < need, need, d)
    if N >= 2:
        d[0] = 2.0 * abs(e[0])
        d[N - 1] = 2.0 * abs(e[N - 2])
    return d, e


MLP_SHAPES = [(64, 12), (64,), (64, 64), (64,), (25, 64), (25,)]


def mlp_init(seed: int) -> np.ndarray:
    """Initial selector parameters (FP32 vector of 6617 values)."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in MLP_SHAPES:
        if len(s) == 2:
            lim = math.sqrt(6.0 / s[1])
            parts.append(rng.uniform(-lim, lim, size=s).ravel())
        else:
            parts.append(np.zeros(s))
    return np.concatenate(parts).astype(np.float32)


def minibatch_order(n: int, epochs: int, seed: int) -> np.ndarray:
    """Sample order for training: one seeded permutation of range(n) per epoch."""
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.permutation(n) for _ in range(epochs)]).astype(np.int32)
