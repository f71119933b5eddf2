"""Pins for the two oracle helpers that the GPU parity tests use as checkers:

* schwarz.additive_local_sum -- Alg. 2 with x = 0 and b = r, i.e. eq.
  additiveschwarz omega * sum_j R_j^T A_j^{-1} R_j r (the x = 0 smoother
  parity, smoke() and the 2D cell-smoother case);
* SIPG.apply_rows -- rows of the matrix of eq. bfsipg applied to a global
  vector (the sampled operator and residual checks at full size).

Each is compared with a brute-force quantity built densely here (inverses of
the dense blocks R_j A R_j^T by np.linalg.inv, the full assembled matrix), and
each comparison is shown to catch a planted mistake (a wrong omega, a dropped
subspace, a dropped neighbour block)."""
import numpy as np
import pytest

from oracle import schwarz
from oracle.mesh import TensorMesh
from oracle.sipg import SIPG


def _mesh(d, ncells, seed):
    rng = np.random.default_rng(seed)
    return TensorMesh([rng.uniform(0.5, 1.5, n) / n for n in ncells])


def _dense_B(Ad, dofs, which=None):
    """sum_j R_j^T (R_j A R_j^T)^{-1} R_j as a dense matrix, by brute force."""
    N = Ad.shape[0]
    B = np.zeros((N, N))
    for j in (range(len(dofs)) if which is None else which):
        idx = dofs[j]
        B[np.ix_(idx, idx)] += np.linalg.inv(Ad[np.ix_(idx, idx)])
    return B


def _solvers(S, A, kind):
    patches = schwarz.vertex_patches(S.mesh) if kind == "vertex" else schwarz.cell_patches(S.mesh)

    def local(cells):
        idx = schwarz.patch_dofs(cells, S.nloc)
        return A[idx][:, idx]
    return schwarz.LocalSolvers(patches, S.nloc, local)


CASES = [(2, (4, 3), 2, "vertex"), (2, (3, 5), 1, "cell"), (3, (3, 2, 3), 1, "vertex"), (3, (2, 3, 2), 2, "cell")]


@pytest.mark.parametrize("d,ncells,k,kind", CASES)
def test_additive_local_sum_is_omega_B_r(d, ncells, k, kind):
    S = SIPG(_mesh(d, ncells, 31 + d + k), k)
    A = S.assemble().tocsr()
    sol = _solvers(S, A, kind)
    r = np.random.default_rng(32).uniform(-1, 1, A.shape[0])
    omega = 0.7
    y = schwarz.additive_local_sum(r, sol, omega)
    B = _dense_B(A.toarray(), sol.dofs)
    ref = omega * B @ r
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    # guards: a wrong damping factor or one dropped subspace is caught
    assert np.abs(schwarz.additive_local_sum(r, sol, omega * 1.01) - ref).max() > 1e-6 * np.abs(ref).max()
    partial = schwarz.additive_local_sum(r, sol, omega, which=range(1, len(sol.dofs)))
    assert np.abs(partial - ref).max() > 1e-6 * np.abs(ref).max()


@pytest.mark.parametrize("d,ncells,k,kind", CASES[:3])
def test_additive_local_sum_subset_form(d, ncells, k, kind):
    S = SIPG(_mesh(d, ncells, 41 + d), k)
    A = S.assemble().tocsr()
    sol = _solvers(S, A, kind)
    r = np.random.default_rng(42).uniform(-1, 1, A.shape[0])
    which = list(range(0, len(sol.dofs), 2))
    y = schwarz.additive_local_sum(r, sol, 0.5, which=which)
    ref = 0.5 * _dense_B(A.toarray(), sol.dofs, which) @ r
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    # the subsets of a partition add up to the full sum
    rest = [j for j in range(len(sol.dofs)) if j not in which]
    full = schwarz.additive_local_sum(r, sol, 0.5)
    both = y + schwarz.additive_local_sum(r, sol, 0.5, which=rest)
    assert np.abs(both - full).max() <= 1e-13 * np.abs(full).max()


def test_additive_local_sum_equals_smoother_from_zero():
    S = SIPG(_mesh(2, (4, 4), 51), 2)
    A = S.assemble().tocsr()
    sol = _solvers(S, A, "vertex")
    r = np.random.default_rng(52).uniform(-1, 1, A.shape[0])
    y = schwarz.additive_local_sum(r, sol, 0.3)
    z = schwarz.additive_smoother(A, r, np.zeros_like(r), sol, 0.3)
    assert np.abs(y - z).max() <= 1e-14 * np.abs(z).max()


def _boundary_class(mesh, c):
    """Number of directions in which cell c touches the boundary (0 interior,
    1 face, 2 edge, 3 corner in 3D)."""
    m = mesh.cell_multi(c)
    return sum(1 for t in range(mesh.d) if m[t] == 0 or m[t] == mesh.ncells[t] - 1)


@pytest.mark.parametrize("d,ncells,k", [(2, (4, 3), 2), (3, (3, 4, 3), 1), (3, (3, 3, 3), 2)])
def test_apply_rows_equals_assembled_rows(d, ncells, k):
    S = SIPG(_mesh(d, ncells, 61 + k), k)
    A = S.assemble().tocsr()
    x = np.random.default_rng(62).uniform(-1, 1, A.shape[0])
    Ax = A @ x
    mesh = S.mesh
    classes = {_boundary_class(mesh, c) for c in range(mesh.num_cells)}
    assert classes == set(range(d + 1))   # interior, face, edge (and corner) cells all present
    cells = list(range(mesh.num_cells))[::-1]          # every cell, in a non-trivial order
    y = S.apply_rows(cells, x)
    ref = np.concatenate([Ax[c * S.nloc:(c + 1) * S.nloc] for c in cells])
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    sub = [c for c in range(mesh.num_cells) if c % 3 == 1]
    y = S.apply_rows(sub, x)
    ref = np.concatenate([Ax[c * S.nloc:(c + 1) * S.nloc] for c in sub])
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()


def test_apply_rows_guard_dropped_neighbour_block():
    # planted mistake: cell_rows loses the first neighbour (off-diagonal) block
    S = SIPG(_mesh(3, (3, 3, 3), 71), 2)
    A = S.assemble().tocsr()
    x = np.random.default_rng(72).uniform(-1, 1, A.shape[0])
    centre = S.mesh.cell_index((1, 1, 1))
    good = S.apply_rows([centre], x)
    ref = (A @ x)[centre * S.nloc:(centre + 1) * S.nloc]
    assert np.abs(good - ref).max() <= 1e-12 * np.abs(ref).max()
    rows = S.cell_rows
    def dropped(c):
        blocks = list(rows(c))
        first_nb = next(i for i, (nb, _) in enumerate(blocks) if nb != c)
        return blocks[:first_nb] + blocks[first_nb + 1:]
    S.cell_rows = dropped
    bad = S.apply_rows([centre], x)
    assert np.abs(bad - ref).max() > 1e-6 * np.abs(ref).max()
