"""Schwarz subspaces, colorings and smoothers.

Test infrastructure only (see the package docstring).

Subspaces (Sec. 2.3): a cell subspace holds the DoFs of one cell; a vertex
patch subspace holds the DoFs of the 2^d cells around one *interior* vertex.
The local solver is the Ritz projection of eq. ritzproj, i.e. the local matrix
A_j = R_j A R_j^T, which is inverted here by dense LU with partial pivoting
(scipy.linalg.lu_factor) -- the standard, non-tensor approach the paper calls
sACS.  The smoothers follow Alg. 2 (additive: one residual, then all local
solves, damped by omega as in eq. additiveschwarz) and Alg. 3 (multiplicative:
a fresh residual before each color, eq. coloredschwarz).

Colorings (Sec. 2.3, Fig. coloring): vertex v = (v_1, ..., v_d) with interior
indices 1 <= v_t <= n_t - 1.
  * additive vertex patches: color = parity bits (v_t mod 2), 2^d colors, no
    two patches of one color share a cell;
  * multiplicative vertex patches: the parity bits plus the bit
    (sum_t floor(v_t / 2)) mod 2, 2^(d+1) colors, no two patches of one color
    share a cell or a face (A-orthogonal);
  * multiplicative cells: red-black, (sum_t c_t) mod 2.
Colors are visited in increasing order, and in reverse order when
`reverse=True` (used for the post-smoother so that the V-cycle is symmetric).
The paper does not fix the color order; this is the reading taken.

Pins (tests/test_oracle_schwarz.py): on the single vertex patch of the coarse
mesh T_0 the additive vertex patch smoother with omega = 1 is an exact solve;
on a one-cell mesh the cell smoother is an exact solve; the colored
multiplicative smoother equals the literal product of eq. multschwarz1 taken in
the same patch order (which holds only if same-color patches are A-orthogonal);
the coloring is checked for shared cells and shared faces by brute force;
additive_local_sum equals omega times the densely assembled
sum_j R_j^T (R_j A R_j^T)^{-1} R_j (tests/test_oracle_checkers.py).
"""
import itertools

import numpy as np
import scipy.linalg as sla


def vertex_patches(mesh):
    """All vertex patches: list of (vertex multi-index v, cells).  The cells of
    the patch around vertex v are those with c_t in {v_t - 1, v_t}, listed
    lexicographically (first direction fastest).  Vertices are interior only
    (Sec. 2.3), enumerated lexicographically."""
    d = mesh.d
    ranges = [range(1, n) for n in mesh.ncells]
    out = []
    for vrev in itertools.product(*reversed(ranges)):
        v = tuple(reversed(vrev))
        cells = []
        for srev in itertools.product((0, 1), repeat=d):
            s = tuple(reversed(srev))
            cells.append(mesh.cell_index([v[t] - 1 + s[t] for t in range(d)]))
        out.append((v, cells))
    return out


def cell_patches(mesh):
    """One subspace per cell: list of (cell multi-index, [cell])."""
    return [(mesh.cell_multi(c), [c]) for c in range(mesh.num_cells)]


def patch_dofs(cells, nloc):
    return np.concatenate([np.arange(c * nloc, (c + 1) * nloc) for c in cells])


def color_additive_vertex(v):
    return sum((v[t] % 2) << t for t in range(len(v)))


def color_multiplicative_vertex(v):
    d = len(v)
    extra = sum(v[t] // 2 for t in range(d)) % 2
    return color_additive_vertex(v) + (extra << d)


def color_multiplicative_cell(c):
    return sum(c) % 2


class LocalSolvers:
    """Dense LU factorizations of A_j = R_j A R_j^T for a list of subspaces.

    `local_matrix(cells)` must return R_j A R_j^T for the listed cells (e.g.
    SIPG.assemble(cells) or a slice of an assembled global matrix)."""

    def __init__(self, patches, nloc, local_matrix):
        self.patches = patches
        self.nloc = nloc
        self.dofs = [patch_dofs(cells, nloc) for _, cells in patches]
        self.lu = []
        for _, cells in patches:
            Aj = local_matrix(cells)
            Aj = Aj.toarray() if hasattr(Aj, "toarray") else np.asarray(Aj)
            self.lu.append(sla.lu_factor(Aj))

    def solve(self, j, rj):
        return sla.lu_solve(self.lu[j], rj)


def additive_smoother(A, b, x, solvers, omega):
    """Alg. 2: r = b - A x; x + omega * sum_j R_j^T A_j^{-1} R_j r."""
    r = b - A @ x
    y = np.zeros_like(x)
    for j, idx in enumerate(solvers.dofs):
        y[idx] += solvers.solve(j, r[idx])
    return x + omega * y


def additive_local_sum(r, solvers, omega, which=None):
    """omega * sum_j R_j^T A_j^{-1} R_j r over the subspaces in `which` (all
    when None): the additive smoother applied with x = 0, b = r."""
    y = np.zeros_like(r)
    for j in (range(len(solvers.dofs)) if which is None else which):
        idx = solvers.dofs[j]
        y[idx] += solvers.solve(j, r[idx])
    return omega * y


def multiplicative_smoother(A, b, x, solvers, colors, omega, reverse=False):
    """Alg. 3: for every color c (in order, or reversed): r = b - A x, then
    x += omega * sum_{j in J_c} R_j^T A_j^{-1} R_j r."""
    x = x.copy()
    order = sorted(set(colors), reverse=reverse)
    for c in order:
        r = b - A @ x
        y = np.zeros_like(x)
        for j, idx in enumerate(solvers.dofs):
            if colors[j] == c:
                y[idx] += solvers.solve(j, r[idx])
        x = x + omega * y
    return x


def product_form_smoother(A, b, x, solvers, order, omega):
    """eq. multschwarz1 applied literally, one subspace at a time in `order`:
    x <- x + omega R_j^T A_j^{-1} R_j (b - A x)."""
    x = x.copy()
    for j in order:
        idx = solvers.dofs[j]
        r = b - A @ x
        x[idx] += omega * solvers.solve(j, r[idx])
    return x
