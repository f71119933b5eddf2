"""Pins for oracle.fastdiag (Sec. 3.2: eq. KDseparable, eq. generalizedEVP,
eq. fastinverse) and its C sweep oracle/fd_smoother.c, the CPU baseline."""
import itertools

import numpy as np
import pytest

from oracle import fastdiag, schwarz
from oracle.mesh import TensorMesh
from oracle.sipg import SIPG


def _widths(ncells, seed):
    rng = np.random.default_rng(seed)
    return [rng.uniform(0.5, 1.5, n) / n for n in ncells]


@pytest.mark.parametrize("k", [1, 2, 5])
def test_mass_1d_integrates_exactly(k):
    h = 0.37
    M = fastdiag.mass_1d(k, h)
    one = np.ones(k + 1)
    assert abs(one @ M @ one - h) < 1e-14                  # int_0^h 1 = h
    from oracle.basis import gauss_lobatto_nodes
    x = gauss_lobatto_nodes(k) * h                          # nodal values of the coordinate
    assert abs(one @ M @ x - h * h / 2) < 1e-14             # int_0^h x = h^2 / 2
    assert abs(x @ M @ x - h ** 3 / 3) < 1e-14              # int_0^h x^2 = h^3 / 3


def _tensor_to_patch_perm(d, k, vertex, S, cells):
    """perm[e] = position in schwarz.patch_dofs(cells) order of tensor entry e
    (local index i_t = s_t (k+1) + a_t, first direction fastest)."""
    n1 = k + 1
    n = 2 * n1 if vertex else n1
    cell_pos = {c: q for q, c in enumerate(cells)}
    base = S.mesh.cell_multi(cells[0])
    perm = []
    for rev in itertools.product(range(n), repeat=d):
        it = tuple(reversed(rev))
        s = [i // n1 for i in it]
        a = [i % n1 for i in it]
        c = S.mesh.cell_index([base[t] + s[t] for t in range(d)])
        dof = sum(a[t] * n1 ** t for t in range(d))
        perm.append(cell_pos[c] * S.nloc + dof)
    return np.array(perm)


def _kron_sum(factors):
    """sum_t M_d (x) .. (x) A_t (x) .. (x) M_1 (first direction fastest)."""
    d = len(factors)
    out = 0.0
    for t in range(d):
        term = np.ones((1, 1))
        for s in reversed(range(d)):
            A, M = factors[s]
            term = np.kron(term, A if s == t else M)
        out = out + term
    return out


@pytest.mark.parametrize("d,ncells,k,vertex", [(2, (4, 3), 2, True), (2, (3, 4), 3, False),
                                               (3, (3, 3, 4), 1, True), (3, (2, 3, 2), 2, False)])
def test_kronecker_sum_equals_assembled_local_matrix(d, ncells, k, vertex):
    widths = _widths(ncells, 5 + d + k)
    S = SIPG(TensorMesh(widths), k)
    per_dir = [fastdiag.factors_1d(w, k, vertex) for w in widths]
    patches = schwarz.vertex_patches(S.mesh) if vertex else schwarz.cell_patches(S.mesh)
    for j, (pos, cells) in enumerate(patches):
        p = [pos[t] - 1 for t in range(d)] if vertex else list(pos)
        K = _kron_sum([per_dir[t][p[t]] for t in range(d)])
        perm = _tensor_to_patch_perm(d, k, vertex, S, cells)
        Aj = S.assemble(cells).toarray()[np.ix_(perm, perm)]
        assert np.abs(K - Aj).max() <= 1e-12 * np.abs(Aj).max(), (j, pos)


def test_eigendata_diagonalizes():
    widths = _widths((4, 3), 9)
    for vertex in (True, False):
        Zs, lams = fastdiag.eigendata(widths, 3, vertex)
        for t, w in enumerate(widths):
            for p, (A, M) in enumerate(fastdiag.factors_1d(w, 3, vertex)):
                Z = Zs[t][p]
                assert np.abs(Z.T @ M @ Z - np.eye(len(Z))).max() < 1e-12
                assert np.abs(Z.T @ A @ Z - np.diag(lams[t][p])).max() < 1e-10 * np.abs(lams[t][p]).max()


def _lu_reference(widths, k, vertex, r, omega):
    S = SIPG(TensorMesh(widths), k)
    A = S.assemble().tocsr()
    patches = schwarz.vertex_patches(S.mesh) if vertex else schwarz.cell_patches(S.mesh)

    def local(cells):
        idx = schwarz.patch_dofs(cells, S.nloc)
        return A[idx][:, idx]
    sol = schwarz.LocalSolvers(patches, S.nloc, local)
    return schwarz.additive_local_sum(r, sol, omega)


@pytest.mark.parametrize("d,ncells,k,vertex,nrhs", [(2, (5, 4), 2, True, 2), (2, (4, 5), 3, False, 1),
                                                    (3, (3, 4, 3), 1, True, 2), (3, (4, 3, 3), 2, True, 1),
                                                    (3, (3, 2, 3), 2, False, 2)])
def test_c_sweep_equals_dense_lu(d, ncells, k, vertex, nrhs):
    widths = _widths(ncells, 21 + d + k)
    N = int(np.prod(ncells)) * (k + 1) ** d
    r = np.random.default_rng(22).uniform(-1, 1, (nrhs, N))
    y = fastdiag.additive_local_sum(widths, k, vertex, r.ravel(), 0.7, nrhs=nrhs).reshape(nrhs, N)
    for q in range(nrhs):
        ref = _lu_reference(widths, k, vertex, r[q], 0.7)
        assert np.abs(y[q] - ref).max() <= 1e-12 * np.abs(ref).max()
    # one thread gives the same numbers (each entry sums its patches in color order)
    y1 = fastdiag.additive_local_sum(widths, k, vertex, r.ravel(), 0.7, nrhs=nrhs, threads=1).reshape(nrhs, N)
    assert np.array_equal(y, y1)


def test_c_sweep_guard_wrong_eigenvalue():
    # planted mistake: one eigenvalue of one position perturbed by 1%
    widths = _widths((4, 4, 3), 31)
    N = 48 * 27
    r = np.random.default_rng(32).uniform(-1, 1, N)
    Zs, lams = fastdiag.eigendata(widths, 2, True)
    lams[1] = lams[1].copy()
    lams[1][1, 2] *= 1.01
    y = fastdiag.additive_local_sum(widths, 2, True, r, 0.7, eig=(Zs, lams))
    ref = _lu_reference(widths, 2, True, r, 0.7)
    assert np.abs(y - ref).max() > 1e-6 * np.abs(ref).max()


def test_c_sweep_rejects_bad_arguments():
    with pytest.raises(ValueError):
        fastdiag.additive_local_sum([np.ones(1)] * 3, 2, True, np.zeros(27), 0.7)   # 1 cell: no vertex patch


def test_c_sweep_color_subsets_add_up():
    # the per-color sweeps are the patch subsets of the dense-LU sum
    widths = _widths((4, 5, 3), 41)
    ncells = (4, 5, 3)
    N = 60 * 8
    r = np.random.default_rng(42).uniform(-1, 1, N)
    S = SIPG(TensorMesh(widths), 1)
    A = S.assemble().tocsr()
    patches = schwarz.vertex_patches(S.mesh)

    def local(cells):
        idx = schwarz.patch_dofs(cells, S.nloc)
        return A[idx][:, idx]
    sol = schwarz.LocalSolvers(patches, S.nloc, local)
    total = np.zeros(N)
    for c in range(8):
        which = [j for j, (v, _) in enumerate(patches) if schwarz.color_additive_vertex(v) == c]
        assert len(which) == fastdiag.count_color(ncells, c)
        y = fastdiag.additive_local_sum(widths, 1, True, r, 0.5, colors=[c])
        ref = schwarz.additive_local_sum(r, sol, 0.5, which=which)
        assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
        total += y
    full = fastdiag.additive_local_sum(widths, 1, True, r, 0.5)
    assert np.abs(total - full).max() <= 1e-13 * np.abs(full).max()
