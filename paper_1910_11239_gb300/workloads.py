"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
checks.  Random draws only: nothing here computes any part of the method.

Recipes (numpy default_rng):
* widths_uniform(n): n cells of width 1/n per direction (unit box).
* widths_random(n, seed): per-direction widths drawn U[0.5, 1.5] / n.
* rhs_uniform(ndofs, seed): entries U[-1, 1].
* vertices_cartesian(wx, wy): vertex array (ny+1, nx+1, 2) of the Cartesian
  mesh with column widths wx and row widths wy.
* vertices_distorted(n, seed, alpha): the distorted mesh of Sec. 4 -- the
  uniform n x n grid of the unit square with every interior vertex moved by
  alpha h_v (alpha = 0.25 in the paper) in a direction drawn U[0, 2 pi),
  h_v the shortest edge at the vertex (1/n on the uniform grid).
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


def vertices_cartesian(wx, wy):
    xs = np.concatenate(([0.0], np.cumsum(wx)))
    ys = np.concatenate(([0.0], np.cumsum(wy)))
    V = np.zeros((len(ys), len(xs), 2))
    V[:, :, 0] = xs[None, :]
    V[:, :, 1] = ys[:, None]
    return V


def vertices_distorted(n, seed, alpha=0.25):
    V = vertices_cartesian(np.full(n, 1.0 / n), np.full(n, 1.0 / n))
    rng = np.random.default_rng(seed)
    theta = rng.uniform(0.0, 2.0 * np.pi, (n + 1, n + 1))
    out = V.copy()
    for j in range(1, n):
        for i in range(1, n):
            nb = [V[j, i - 1], V[j, i + 1], V[j - 1, i], V[j + 1, i]]
            hv = min(np.linalg.norm(V[j, i] - w) for w in nb)
            out[j, i] = V[j, i] + alpha * hv * np.array([np.cos(theta[j, i]), np.sin(theta[j, i])])
    return out
