"""Pins for oracle.schwarz (Sec. 2.3, Alg. 2, Alg. 3)."""
import itertools

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import schwarz
from oracle.mesh import TensorMesh
from oracle.sipg import SIPG


def setup(d, n, k, seed, uniform=False):
    rng = np.random.default_rng(seed)
    widths = [np.full(n, 1.0 / n) if uniform else rng.uniform(0.5, 1.5, n) / n for _ in range(d)]
    S = SIPG(TensorMesh(widths), k)
    A = S.assemble().tocsr()
    return S, A


def local_from(A, nloc):
    def f(cells):
        idx = schwarz.patch_dofs(cells, nloc)
        return A[idx][:, idx]
    return f


@pytest.mark.parametrize("d,k", [(2, 2), (3, 1), (3, 2)])
def test_single_vertex_patch_is_exact_solve(d, k):
    # T_0 with 2^d cells is one vertex patch (Sec. 2.4): AVS with omega = 1 solves exactly
    S, A = setup(d, 2, k, 1)
    patches = schwarz.vertex_patches(S.mesh)
    assert len(patches) == 1
    sol = schwarz.LocalSolvers(patches, S.nloc, local_from(A, S.nloc))
    b = np.random.default_rng(2).uniform(-1, 1, A.shape[0])
    x = schwarz.additive_smoother(A, b, np.zeros_like(b), sol, 1.0)
    assert np.abs(x - spla.spsolve(A.tocsc(), b)).max() < 1e-11 * np.abs(x).max()


def test_one_cell_mesh_cell_smoother_is_exact():
    S, A = setup(3, 1, 3, 3)
    sol = schwarz.LocalSolvers(schwarz.cell_patches(S.mesh), S.nloc, local_from(A, S.nloc))
    b = np.random.default_rng(4).uniform(-1, 1, A.shape[0])
    x = schwarz.additive_smoother(A, b, np.zeros_like(b), sol, 1.0)
    assert np.abs(A @ x - b).max() < 1e-11


def test_additive_smoother_definition_with_nonzero_x():
    S, A = setup(2, 4, 2, 5)
    sol = schwarz.LocalSolvers(schwarz.vertex_patches(S.mesh), S.nloc, local_from(A, S.nloc))
    rng = np.random.default_rng(6)
    b, x = rng.uniform(-1, 1, A.shape[0]), rng.uniform(-1, 1, A.shape[0])
    y = schwarz.additive_smoother(A, b, x, sol, 0.3)
    # brute force: sum_j R_j^T A_j^{-1} R_j assembled as a dense matrix
    N = A.shape[0]
    B = np.zeros((N, N))
    Ad = A.toarray()
    for idx in sol.dofs:
        B[np.ix_(idx, idx)] += np.linalg.inv(Ad[np.ix_(idx, idx)])
    assert np.allclose(y, x + 0.3 * B @ (b - Ad @ x), atol=1e-11)


def _faces_or_cells_shared(mesh, cells_a, cells_b):
    ma = [mesh.cell_multi(c) for c in cells_a]
    mb = [mesh.cell_multi(c) for c in cells_b]
    share_cell = bool(set(cells_a) & set(cells_b))
    share_face = any(sum(abs(x - y) for x, y in zip(p, q)) == 1 for p in ma for q in mb)
    return share_cell, share_face


@pytest.mark.parametrize("d,n", [(2, 7), (3, 6)])
def test_colorings_by_brute_force(d, n):
    mesh = TensorMesh([np.ones(n)] * d)
    patches = schwarz.vertex_patches(mesh)
    add = [schwarz.color_additive_vertex(v) for v, _ in patches]
    mul = [schwarz.color_multiplicative_vertex(v) for v, _ in patches]
    assert len(set(add)) == 2 ** d and len(set(mul)) == 2 ** (d + 1)
    for (i, (va, ca)), (j, (vb, cb)) in itertools.combinations(enumerate(patches), 2):
        cell, face = _faces_or_cells_shared(mesh, ca, cb)
        if add[i] == add[j]:
            assert not cell
        if mul[i] == mul[j]:
            assert not cell and not face
    cells = schwarz.cell_patches(mesh)
    rb = [schwarz.color_multiplicative_cell(m) for m, _ in cells]
    for (i, (ma, ca)), (j, (mb, cb)) in itertools.combinations(enumerate(cells), 2):
        if rb[i] == rb[j]:
            assert sum(abs(x - y) for x, y in zip(ma, mb)) != 1


@pytest.mark.parametrize("kind", ["vertex", "cell"])
def test_colored_multiplicative_equals_product_form(kind):
    # eq. coloredschwarz equals eq. multschwarz1 in color order when the
    # subspaces of one color are A-orthogonal (Sec. 2.3)
    S, A = setup(2, 5, 2, 8)
    if kind == "vertex":
        patches = schwarz.vertex_patches(S.mesh)
        colors = [schwarz.color_multiplicative_vertex(v) for v, _ in patches]
    else:
        patches = schwarz.cell_patches(S.mesh)
        colors = [schwarz.color_multiplicative_cell(m) for m, _ in patches]
    sol = schwarz.LocalSolvers(patches, S.nloc, local_from(A, S.nloc))
    rng = np.random.default_rng(9)
    b, x = rng.uniform(-1, 1, A.shape[0]), rng.uniform(-1, 1, A.shape[0])
    for reverse in (False, True):
        y = schwarz.multiplicative_smoother(A, b, x, sol, colors, 0.9, reverse=reverse)
        order = sorted(range(len(patches)), key=lambda j: colors[j], reverse=reverse)
        z = schwarz.product_form_smoother(A, b, x, sol, order, 0.9)
        assert np.abs(y - z).max() < 1e-11


def test_additive_coloring_would_break_multiplicative_equivalence():
    # guard: with the additive (cell-disjoint but face-sharing) coloring the
    # colored multiplicative sweep is NOT the product form
    S, A = setup(2, 5, 2, 8)
    patches = schwarz.vertex_patches(S.mesh)
    colors = [schwarz.color_additive_vertex(v) for v, _ in patches]
    sol = schwarz.LocalSolvers(patches, S.nloc, local_from(A, S.nloc))
    rng = np.random.default_rng(9)
    b, x = rng.uniform(-1, 1, A.shape[0]), rng.uniform(-1, 1, A.shape[0])
    y = schwarz.multiplicative_smoother(A, b, x, sol, colors, 0.9)
    order = sorted(range(len(patches)), key=lambda j: colors[j])
    z = schwarz.product_form_smoother(A, b, x, sol, order, 0.9)
    assert np.abs(y - z).max() > 1e-6
