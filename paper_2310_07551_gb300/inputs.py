"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module holds no arithmetic of the split exponential integrator itself:
only the counter-based random generator, the grids, the finite-difference
matrices A_mu that are *inputs* of the method (the paper's algorithms take
A_1..A_d as given, Algorithms 1 and 2) and the initial states.

Layout convention (paper Section 2, column-stacking ``vec``): an order-d
tensor with sizes (n_1, ..., n_d) is stored with mode 1 fastest, i.e. as a
C-contiguous numpy/torch array of shape (n_d, ..., n_1).  A two-component
state is stored as shape (2, n_d, ..., n_1).
"""
from __future__ import annotations

import numpy as np

_MASK64 = (1 << 64) - 1


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014), vectorised on uint64."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)).astype(np.uint64)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, stream: int, count: int) -> np.ndarray:
    """Counter-based U[0,1) doubles: top 53 bits of splitmix64 of
    (seed, stream, linear index).  Deterministic on any host."""
    key = np.uint64(((seed & 0xFFFFFFFF) << 32 | (stream & 0xFFFFFFFF)) & _MASK64)
    base = splitmix64(np.array([key], dtype=np.uint64))[0]
    idx = np.arange(count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        r = splitmix64(idx ^ base)
    return (r >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def fd_neumann(n: int, lo: float, hi: float) -> np.ndarray:
    """Second-order centred finite-difference Laplacian on the vertex grid
    x_j = lo + j h, h = (hi - lo)/(n - 1), j = 0..n-1, with homogeneous
    Neumann conditions closed by ghost-point reflection (rows 0 and n-1 read
    [-2, 2] / h^2).  Returned as a dense (n, n) array, entry [i, j] = row i,
    column j."""
    if n < 2:
        raise ValueError("need n >= 2")
    h = (hi - lo) / (n - 1)
    D = np.zeros((n, n))
    i = np.arange(n)
    D[i, i] = -2.0
    D[i[1:], i[1:] - 1] = 1.0
    D[i[:-1], i[:-1] + 1] = 1.0
    D[0, 1] = 2.0
    D[n - 1, n - 2] = 2.0
    return D / (h * h)


def schnakenberg_equilibrium(a: float, b: float) -> tuple[float, float]:
    """Homogeneous steady state of the Schnakenberg kinetics."""
    return a + b, b / (a + b) ** 2


def initial_state(model: str, dims: tuple[int, ...], seed: int,
                  a: float = 0.1, b: float = 0.9, amp: float = 1e-3) -> np.ndarray:
    """Seeded initial data, shape (2, n_d, ..., n_1), float64.

    * ``schnakenberg``: equilibrium + amp * U[0,1) per component and point.
    * ``fhn``: U[-1,1) per component and point.
    """
    n = int(np.prod(dims))
    shape = (2,) + tuple(reversed(dims))
    out = np.empty((2, n))
    for c in range(2):
        r = uniform01(seed, c, n)
        if model == "schnakenberg":
            ue = schnakenberg_equilibrium(a, b)[c]
            out[c] = ue + amp * r
        elif model == "fhn":
            out[c] = 2.0 * r - 1.0
        else:
            raise ValueError(model)
    return out.reshape(shape)


def random_tensor(dims: tuple[int, ...], seed: int, stream: int = 0,
                  lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Uniform seeded tensor of shape (n_d, ..., n_1)."""
    n = int(np.prod(dims))
    r = uniform01(seed, stream, n)
    return (lo + (hi - lo) * r).reshape(tuple(reversed(dims)))


def random_matrix(n: int, seed: int, stream: int = 0, scale: float = 1.0) -> np.ndarray:
    """Dense seeded (n, n) matrix with entries scale * U[-1,1)."""
    r = uniform01(seed, stream, n * n)
    return scale * (2.0 * r - 1.0).reshape(n, n)
