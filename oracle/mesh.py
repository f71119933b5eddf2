"""Cartesian tensor meshes and the DG DoF layout.

Test infrastructure only (see the package docstring).

A mesh is the tensor product of d 1D subdivisions (Sec. 3.2: a Cartesian cell
is a product of intervals I_1 x ... x I_d).  Cells are numbered
lexicographically with the first coordinate running fastest.  The DoF vector is
the direct sum over cells (eq. discFEspace): cell c owns the contiguous block
[c (k+1)^d, (c+1) (k+1)^d), ordered by the lexicographic multi-index of
eq. multiindex, i = sum_tau i_tau (k+1)^(tau-1) (first direction fastest).
Refinement splits every cell at its midpoint into 2^d children (Sec. 2.1).

Pins: the numbering is checked in tests/test_oracle_mesh.py (round trips,
refinement keeps the domain and halves every width).
"""
import itertools

import numpy as np


class TensorMesh:
    def __init__(self, widths):
        self.widths = [np.asarray(w, dtype=np.float64).copy() for w in widths]
        self.d = len(self.widths)
        if self.d not in (1, 2, 3):
            raise ValueError("dimension must be 1, 2 or 3")
        for w in self.widths:
            if len(w) < 1 or np.any(w <= 0):
                raise ValueError("widths must be positive and non-empty")
        self.ncells = tuple(len(w) for w in self.widths)
        # left end point of every 1D interval, per direction
        self.origins = [np.concatenate(([0.0], np.cumsum(w)[:-1])) for w in self.widths]

    @property
    def num_cells(self):
        return int(np.prod(self.ncells))

    def cell_multi(self, c):
        """Linear cell index -> multi-index (first direction fastest)."""
        out = []
        for n in self.ncells:
            out.append(c % n)
            c //= n
        return tuple(out)

    def cell_index(self, multi):
        c, stride = 0, 1
        for m, n in zip(multi, self.ncells):
            if not 0 <= m < n:
                raise IndexError("cell multi-index out of range")
            c += m * stride
            stride *= n
        return c

    def cell_box(self, c):
        """(lower corner, widths) of cell c as length-d arrays."""
        m = self.cell_multi(c)
        lo = np.array([self.origins[t][m[t]] for t in range(self.d)])
        h = np.array([self.widths[t][m[t]] for t in range(self.d)])
        return lo, h

    def refine(self):
        """Bisect every cell in every direction (Sec. 2.1)."""
        return TensorMesh([np.repeat(w, 2) * 0.5 for w in self.widths])

    def all_cells(self):
        return range(self.num_cells)


def local_multi_indices(k, d):
    """All local multi-indices (i_1, ..., i_d) of a Q_k cell in DoF order
    (eq. multiindex: the first index runs fastest)."""
    return [tuple(reversed(t)) for t in itertools.product(range(k + 1), repeat=d)]


def dofs_per_cell(k, d):
    return (k + 1) ** d


def num_dofs(mesh, k):
    return mesh.num_cells * dofs_per_cell(k, mesh.d)


def cell_dofs(mesh, k, c):
    n = dofs_per_cell(k, mesh.d)
    return np.arange(c * n, (c + 1) * n)


def unit_hierarchy(d, nlevels, coarse_cells=2):
    """Meshes T_0 .. T_{nlevels-1} of [0,1]^d, T_0 with coarse_cells cells per
    direction (the paper's T_0 has 2^d congruent cells, Sec. 2.4)."""
    w = np.full(coarse_cells, 1.0 / coarse_cells)
    meshes = [TensorMesh([w] * d)]
    for _ in range(nlevels - 1):
        meshes.append(meshes[-1].refine())
    return meshes
