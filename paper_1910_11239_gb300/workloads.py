"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
checks.  Random draws only: nothing here computes any part of the method.

Recipes (numpy default_rng):
* widths_uniform(n): n cells of width 1/n per direction (unit box).
* widths_random(n, seed): per-direction widths drawn U[0.5, 1.5] / n.
* rhs_uniform(ndofs, seed): entries U[-1, 1].
* vertices_cartesian(*widths): vertex array ((nz+1,) ny+1, nx+1, d) of the
  Cartesian mesh with the given widths per direction.
* vertices_distorted(n, seed, alpha, dim): the distorted mesh of Sec. 4 --
  the uniform n^dim grid of the unit square / cube with every interior
  vertex moved by alpha h_v (alpha = 0.25 in the paper) in a random
  direction (2D: angle U[0, 2 pi); 3D: uniform on the sphere), h_v the
  shortest edge at the vertex (1/n on the uniform grid).
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


def vertices_cartesian(*widths):
    """Vertex array of the Cartesian mesh with the given widths per direction
    (2 or 3 directions; axes reversed, x fastest, last axis the coordinates)."""
    d = len(widths)
    grids = [np.concatenate(([0.0], np.cumsum(w))) for w in widths]
    V = np.zeros(tuple(len(g) for g in reversed(grids)) + (d,))
    for t in range(d):
        shape = [1] * d
        shape[d - 1 - t] = len(grids[t])
        V[..., t] = grids[t].reshape(shape)
    return V


def vertices_distorted(n, seed, alpha=0.25, dim=2):
    """Uniform n^dim grid of the unit square / cube, every interior vertex moved
    by alpha h_v (h_v = 1/n, its shortest edge) in a random direction: angle
    U[0, 2 pi) in 2D, a normalized standard normal vector (uniform on the
    sphere) in 3D."""
    V = vertices_cartesian(*[np.full(n, 1.0 / n)] * dim)
    rng = np.random.default_rng(seed)
    out = V.copy()
    if dim == 2:
        theta = rng.uniform(0.0, 2.0 * np.pi, (n + 1, n + 1))
        for j in range(1, n):
            for i in range(1, n):
                nb = [V[j, i - 1], V[j, i + 1], V[j - 1, i], V[j + 1, i]]
                hv = min(np.linalg.norm(V[j, i] - w) for w in nb)
                out[j, i] = V[j, i] + alpha * hv * np.array([np.cos(theta[j, i]), np.sin(theta[j, i])])
        return out
    g = rng.standard_normal((n + 1, n + 1, n + 1, 3))
    for l in range(1, n):
        for j in range(1, n):
            for i in range(1, n):
                nb = [V[l, j, i - 1], V[l, j, i + 1], V[l, j - 1, i], V[l, j + 1, i], V[l - 1, j, i], V[l + 1, j, i]]
                hv = min(np.linalg.norm(V[l, j, i] - w) for w in nb)
                out[l, j, i] = V[l, j, i] + alpha * hv * g[l, j, i] / np.linalg.norm(g[l, j, i])
    return out
