"""Level transfers for nested meshes.

Test infrastructure only (see the package docstring).

Sec. 2.2: the prolongation I^up: V_{l-1} -> V_l is the embedding of the nested
spaces, and the restriction I^down is its transpose in the coefficient spaces.
The embedding is written out by definition: the fine coefficient at a fine
support point is the coarse function's value there, i.e. the parent cell's
Lagrange basis evaluated at the child's Gauss-Lobatto points (mapped into the
parent's reference coordinates).

Pins (tests/test_oracle_transfer.py): prolongation of any coarse Q_k function
equals the fine interpolant of the same function; restriction is the exact
transpose.
"""
import itertools

import numpy as np
import scipy.sparse as sp

from .basis import gauss_lobatto_nodes, lagrange_values
from .mesh import local_multi_indices


def prolongation_matrix(coarse, fine, k):
    """Sparse P with fine = P @ coarse, for fine = coarse.refine()."""
    d = coarse.d
    nodes = gauss_lobatto_nodes(k)
    multi = local_multi_indices(k, d)
    nloc = len(multi)
    rows, cols, vals = [], [], []
    for cf in range(fine.num_cells):
        fm = fine.cell_multi(cf)
        pm = [m // 2 for m in fm]
        cp = coarse.cell_index(pm)
        flo, fh = fine.cell_box(cf)
        clo, ch = coarse.cell_box(cp)
        # physical fine support points -> parent reference coordinates
        for I, im in enumerate(multi):
            xhat = [(flo[t] + fh[t] * nodes[im[t]] - clo[t]) / ch[t] for t in range(d)]
            vals_1d = [lagrange_values(nodes, [xhat[t]])[0] for t in range(d)]
            for J, jm in enumerate(multi):
                v = 1.0
                for t in range(d):
                    v *= vals_1d[t][jm[t]]
                if v != 0.0:
                    rows.append(cf * nloc + I)
                    cols.append(cp * nloc + J)
                    vals.append(v)
    shape = (fine.num_cells * nloc, coarse.num_cells * nloc)
    return sp.coo_matrix((vals, (rows, cols)), shape=shape).tocsr()


def prolongate(P, coarse_vec):
    return P @ coarse_vec


def restrict(P, fine_vec):
    """Restriction = transpose of the prolongation (Sec. 2.2)."""
    return P.T @ fine_vec
