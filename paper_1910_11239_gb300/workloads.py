"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
checks.  Random draws only: nothing here computes any part of the method.

Recipes (numpy default_rng):
* widths_uniform(n): n cells of width 1/n per direction (unit box).
* widths_random(n, seed): per-direction widths drawn U[0.5, 1.5] / n.
* rhs_uniform(ndofs, seed): entries U[-1, 1].
"""
import numpy as np


def widths_uniform(n, dim):
    return [np.full(n, 1.0 / n) for _ in range(dim)]


def widths_random(n, dim, seed):
    rng = np.random.default_rng(seed)
    return [rng.uniform(0.5, 1.5, n) / n for _ in range(dim)]


def rhs_uniform(ndofs, seed, nrhs=1):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, ndofs * nrhs)


def rhs_batch(ndofs, seeds):
    return np.concatenate([rhs_uniform(ndofs, s) for s in seeds])
