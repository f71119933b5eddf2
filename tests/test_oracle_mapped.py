"""Pins of the oracle on bilinear quadrilateral meshes (oracle/mapped.py):
the literal SIPG assembly with mapped gradients and normals, the distorted
mesh of Sec. 4, its refinement, the Cartesian-surrogate local solvers and the
multigrid hierarchy built on them."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import multigrid, schwarz
from oracle.mapped import (MappedHierarchy, MappedSIPG, dlinear_map, exact_solvers, jacobians, refine,
                           surrogate_cell_matrix, surrogate_solvers, surrogate_widths)
from oracle.mesh import TensorMesh
from oracle.sipg import SIPG
from paper_1910_11239_gb300.workloads import vertices_cartesian as cartesian_vertices
from paper_1910_11239_gb300.workloads import vertices_distorted as distorted_vertices


@pytest.mark.parametrize("k,gamma_hat", [(1, 1.0), (3, 4.0), (4, 2.5)])
def test_cartesian_vertices_give_the_tensor_assembly(k, gamma_hat):
    rng = np.random.default_rng(10 + k)
    wx, wy = rng.uniform(0.5, 1.5, 3), rng.uniform(0.5, 1.5, 2)
    A = MappedSIPG(cartesian_vertices(wx, wy), k, gamma_hat).assemble()
    B = SIPG(TensorMesh([wx, wy]), k, gamma_hat).assemble()
    assert abs(A - B).max() <= 1e-11 * abs(B).max()


def _affine_vertices(n, seed):
    V = cartesian_vertices(np.full(n, 1.0 / n), np.full(n, 1.0 / n))
    F = np.array([[1.1, 0.35], [-0.2, 0.9]])
    return V @ F.T + np.array([0.3, -0.1])


@pytest.mark.parametrize("k", [1, 2, 3])
def test_polynomials_are_reproduced_on_parallelograms(k):
    """SIPG consistency: for u in P_k (contained in the mapped Q_k space of an
    affine mesh), A u_I = b(f = -Laplace u, g = u) up to rounding."""
    S = MappedSIPG(_affine_vertices(3, 0), k, gamma_hat=4.0)
    A = S.assemble()
    # u = sum of monomials x^a y^b with a + b <= k
    coef = {(a, b): (-1) ** (a + b) * (0.5 + 0.1 * a + 0.07 * b) for a in range(k + 1) for b in range(k + 1 - a)}
    u = lambda p: sum(c * p[:, 0] ** a * p[:, 1] ** b for (a, b), c in coef.items())

    def lap(p):
        out = np.zeros(len(p))
        for (a, b), c in coef.items():
            if a >= 2:
                out += c * a * (a - 1) * p[:, 0] ** (a - 2) * p[:, 1] ** b
            if b >= 2:
                out += c * b * (b - 1) * p[:, 0] ** a * p[:, 1] ** (b - 2)
        return out

    uI = S.interpolate(u)
    b = S.rhs(lambda p: -lap(p), u)
    assert np.abs(A @ uI - b).max() <= 1e-10 * np.abs(b).max()
    assert np.abs(spla.spsolve(A.tocsc(), b) - uI).max() <= 1e-9


@pytest.mark.parametrize("k", [1, 3])
def test_linear_functions_are_reproduced_on_distorted_meshes(k):
    """A linear u is bilinear in every cell's reference coordinates, so it lies
    in the space of any bilinear mesh and the SIPG solution reproduces it (the
    boundary terms of the right-hand side with the operator's k+1 point rule)."""
    S = MappedSIPG(distorted_vertices(4, seed=3), k, gamma_hat=4.0)
    A = S.assemble()
    u = lambda p: 0.7 - 1.3 * p[:, 0] + 0.4 * p[:, 1]
    uI = S.interpolate(u)
    b = S.rhs(lambda p: np.zeros(len(p)), u, nq=k + 1)
    assert np.abs(A @ uI - b).max() <= 1e-10 * np.abs(b).max()


def test_l2_convergence_on_distorted_meshes():
    """O(h^(k+1)) L2 convergence for u = sin(pi x) sin(pi y) on the 25%-distorted
    mesh and two bilinear refinements of it (k = 2: rate 3)."""
    u = lambda p: np.sin(np.pi * p[:, 0]) * np.sin(np.pi * p[:, 1])
    f = lambda p: 2 * np.pi ** 2 * u(p)
    V = distorted_vertices(4, seed=5)
    errs = []
    for _ in range(3):
        S = MappedSIPG(V, 2, gamma_hat=4.0)
        x = spla.spsolve(S.assemble().tocsc(), S.rhs(f, u))
        errs.append(S.l2_error(x, u))
        V = refine(V)
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > 2.7, (errs, rates)


def test_symmetric_positive_definite_with_the_papers_penalty():
    """Sec. 4: 25% distortion with gamma_hat = 4 keeps the form positive definite."""
    S = MappedSIPG(distorted_vertices(4, seed=1), 3, gamma_hat=4.0)
    A = S.assemble().toarray()
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(A)[0] > 0.0


def test_distorted_vertices_follow_the_recipe():
    n, alpha = 6, 0.25
    V = distorted_vertices(n, seed=2, alpha=alpha)
    U = cartesian_vertices(np.full(n, 1.0 / n), np.full(n, 1.0 / n))
    shift = np.linalg.norm(V - U, axis=2)
    assert np.all(shift[0, :] == 0) and np.all(shift[-1, :] == 0)
    assert np.all(shift[:, 0] == 0) and np.all(shift[:, -1] == 0)
    # uniform grid: the shortest edge at every interior vertex is 1/n
    assert np.allclose(shift[1:-1, 1:-1], alpha / n, rtol=1e-13)


def test_refinement_nests_the_bilinear_maps():
    V = distorted_vertices(3, seed=4)
    F = refine(V)
    xi = np.random.default_rng(0).uniform(0, 1, (7, 2))
    for j in range(3):
        for i in range(3):
            for sy in range(2):
                for sx in range(2):
                    child = dlinear_map(F, (2 * i + sx, 2 * j + sy), xi)
                    parent = dlinear_map(V, (i, j), (xi + np.array([sx, sy])) / 2)
                    assert np.allclose(child, parent, atol=1e-15)


def test_surrogate_widths_are_the_mean_edge_lengths():
    V = np.array([[[0.0, 0.0], [2.0, 0.0]], [[0.0, 1.0], [3.0, 5.0]]])
    h0, h1 = surrogate_widths(V, (0, 0))
    assert h0 == pytest.approx((2.0 + 5.0) / 2) and h1 == pytest.approx((1.0 + np.hypot(1.0, 5.0)) / 2)


def test_surrogate_of_a_cartesian_cell_is_the_exact_local_matrix():
    rng = np.random.default_rng(6)
    wx, wy = rng.uniform(0.5, 1.5, 4), rng.uniform(0.5, 1.5, 3)
    V = cartesian_vertices(wx, wy)
    S = MappedSIPG(V, 3, 4.0)
    A = S.assemble().tocsr()
    for (i, j) in [(0, 0), (1, 1), (3, 2), (2, 0)]:
        idx = schwarz.patch_dofs([S.cell_index((i, j))], S.nloc)
        assert np.allclose(surrogate_cell_matrix(V, (i, j), 3, 4.0), A[idx][:, idx].toarray(), rtol=1e-12, atol=1e-10)


def test_surrogate_is_the_rectangle_of_mean_widths_on_a_distorted_cell():
    """The surrogate block is the Cartesian block of the cell with widths
    (hbar_0, hbar_1) and its neighbours' surrogate widths: its cell-integral part
    is hbar_1/hbar_0 Lhat x Mhat + hbar_0/hbar_1 Mhat x Lhat, so two cells with
    equal mean widths have equal surrogates wherever their neighbours agree."""
    V = distorted_vertices(4, seed=8)
    B = surrogate_cell_matrix(V, (1, 2), 2, 4.0)
    h0, h1 = surrogate_widths(V, (1, 2))
    wx = [surrogate_widths(V, (i, 2))[0] for i in (0, 1, 2)]
    wy = [surrogate_widths(V, (1, j))[1] for j in (1, 2, 3)]
    assert wx[1] == h0 and wy[1] == h1
    C = SIPG(TensorMesh([np.array(wx), np.array(wy)]), 2, 4.0).assemble([4]).toarray()
    assert np.allclose(B, C, rtol=1e-13, atol=1e-12)
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max() and np.linalg.eigvalsh(B)[0] > 0


@pytest.mark.parametrize("smoother,omega", [("ACS", 0.7), ("MCS", 1.0)])
def test_hierarchy_on_cartesian_vertices_is_the_cartesian_vcycle(smoother, omega):
    """On a Cartesian vertex array the surrogate is exact and the transfers are the
    Cartesian ones: the V-cycle equals the (pinned) Cartesian hierarchy's."""
    rng = np.random.default_rng(7)
    widths = [rng.uniform(0.5, 1.5, 2), rng.uniform(0.5, 1.5, 2)]
    H = MappedHierarchy(cartesian_vertices(*widths), 2, 3, smoother, omega, steps=1, gamma_hat=4.0)
    C = multigrid.Hierarchy(widths, 2, 3, smoother, omega, gamma_hat=4.0)
    r = rng.uniform(-1, 1, H.A[-1].shape[0])
    assert np.allclose(H.precondition(r), C.precondition(r), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("smoother,steps", [("ACS", 2), ("MCS", 1)])
def test_vcycle_is_symmetric_on_distorted_meshes(smoother, steps):
    H = MappedHierarchy(distorted_vertices(2, seed=9), 2, 3, smoother, 0.5, steps=steps)
    n = H.A[-1].shape[0]
    rng = np.random.default_rng(1)
    x, y = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    assert abs(x @ H.precondition(y) - y @ H.precondition(x)) <= 1e-11 * abs(x @ H.precondition(x))


def test_inexact_solvers_converge_with_damping_below_one():
    """Sec. 4: with surrogate local solvers, ACS at omega = 0.5 gives a convergent
    preconditioned CG on a distorted mesh, and exact local solvers need fewer steps."""
    V0 = distorted_vertices(4, seed=11)
    its = {}
    for local in ("surrogate", "exact"):
        H = MappedHierarchy(V0, 2, 3, "ACS", 0.5 if local == "surrogate" else 0.7, steps=1, local=local)
        b = np.random.default_rng(2).uniform(-1, 1, H.A[-1].shape[0])
        x, _, hist, ok = multigrid.pcg(H.A[-1], b, H.precondition, rtol=1e-8, maxit=100)
        assert ok
        assert np.linalg.norm(b - H.A[-1] @ x) <= 1e-8 * np.linalg.norm(b) * 1.01
        its[local] = multigrid.fractional_iterations(hist, 1e-8)
    assert its["exact"] < its["surrogate"] < 1.8 * its["exact"], its


# ------------------------------------------------------------------- 3D
@pytest.mark.parametrize("k,gamma_hat", [(1, 1.0), (2, 4.0)])
def test_cartesian_vertices_give_the_tensor_assembly_3d(k, gamma_hat):
    rng = np.random.default_rng(20 + k)
    w = [rng.uniform(0.5, 1.5, 2), rng.uniform(0.5, 1.5, 3), rng.uniform(0.5, 1.5, 2)]
    A = MappedSIPG(cartesian_vertices(*w), k, gamma_hat).assemble()
    B = SIPG(TensorMesh(w), k, gamma_hat).assemble()
    assert abs(A - B).max() <= 1e-11 * abs(B).max()


@pytest.mark.parametrize("k", [1, 2])
def test_polynomials_are_reproduced_on_affine_hexahedra(k):
    V = cartesian_vertices(*[np.full(2, 0.5)] * 3)
    F = np.array([[1.1, 0.3, -0.2], [0.1, 0.9, 0.25], [-0.15, 0.2, 1.05]])
    S = MappedSIPG(V @ F.T + np.array([0.2, -0.1, 0.3]), k, gamma_hat=4.0)
    A = S.assemble()
    coef = {(a, b, c): (-1) ** (a + b + c) * (0.5 + 0.1 * a + 0.07 * b - 0.05 * c)
            for a in range(k + 1) for b in range(k + 1 - a) for c in range(k + 1 - a - b)}
    u = lambda p: sum(v * p[:, 0] ** a * p[:, 1] ** b * p[:, 2] ** c for (a, b, c), v in coef.items())

    def lap(p):
        out = np.zeros(len(p))
        for (a, b, c), v in coef.items():
            if a >= 2:
                out += v * a * (a - 1) * p[:, 0] ** (a - 2) * p[:, 1] ** b * p[:, 2] ** c
            if b >= 2:
                out += v * b * (b - 1) * p[:, 0] ** a * p[:, 1] ** (b - 2) * p[:, 2] ** c
            if c >= 2:
                out += v * c * (c - 1) * p[:, 0] ** a * p[:, 1] ** b * p[:, 2] ** (c - 2)
        return out

    b = S.rhs(lambda p: -lap(p), u)
    assert np.abs(A @ S.interpolate(u) - b).max() <= 1e-10 * np.abs(b).max()


def test_linear_functions_are_reproduced_on_distorted_hexahedra():
    """A linear u is trilinear in the reference coordinates of every cell: it lies
    in the mapped Q_1 space and is reproduced (operator's rule for the boundary terms)."""
    S = MappedSIPG(distorted_vertices(3, seed=4, dim=3), 1, gamma_hat=4.0)
    A = S.assemble()
    u = lambda p: 0.3 - 1.1 * p[:, 0] + 0.6 * p[:, 1] + 0.9 * p[:, 2]
    b = S.rhs(lambda p: np.zeros(len(p)), u, nq=2)
    assert np.abs(A @ S.interpolate(u) - b).max() <= 1e-10 * np.abs(b).max()


def test_symmetric_positive_definite_3d():
    S = MappedSIPG(distorted_vertices(2, seed=5, dim=3), 2, gamma_hat=4.0)
    A = S.assemble().toarray()
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(A)[0] > 0.0


def test_refinement_nests_the_trilinear_maps():
    V = distorted_vertices(2, seed=6, dim=3)
    F = refine(V)
    xi = np.random.default_rng(1).uniform(0, 1, (5, 3))
    for c in range(8):
        m = (c & 1, (c >> 1) & 1, c >> 2)
        for s in range(8):
            o = np.array([s & 1, (s >> 1) & 1, s >> 2])
            child = dlinear_map(F, tuple(2 * np.array(m) + o), xi)
            assert np.allclose(child, dlinear_map(V, m, (xi + o) / 2), atol=1e-15)


def test_face_normals_and_measures_of_a_sheared_cube():
    """Nanson's formula on an affine cell: the face of the parallelepiped spanned by
    the columns of F at xi_2 = 1 has the normal (F e_0 x F e_1)/|..| and area |F e_0 x F e_1|."""
    F = np.array([[1.0, 0.4, 0.1], [0.2, 1.3, -0.3], [0.0, 0.25, 0.8]])
    V = cartesian_vertices(*[np.ones(1)] * 3) @ F.T
    S = MappedSIPG(V, 2)
    xi, W, n, area = S._face((0, 0, 0), 2, 1)
    cr = np.cross(F[:, 0], F[:, 1])
    assert np.allclose(n, cr / np.linalg.norm(cr)) and area == pytest.approx(np.linalg.norm(cr))
    assert np.allclose(jacobians(V, (0, 0, 0), xi), F)


def test_surrogate_of_a_cartesian_hexahedron_is_the_exact_block():
    rng = np.random.default_rng(9)
    w = [rng.uniform(0.5, 1.5, 3), rng.uniform(0.5, 1.5, 2), rng.uniform(0.5, 1.5, 2)]
    V = cartesian_vertices(*w)
    S = MappedSIPG(V, 2, 4.0)
    A = S.assemble().tocsr()
    for m in [(0, 0, 0), (1, 1, 0), (2, 0, 1)]:
        idx = schwarz.patch_dofs([S.cell_index(m)], S.nloc)
        assert np.allclose(surrogate_cell_matrix(V, m, 2, 4.0), A[idx][:, idx].toarray(), rtol=1e-12, atol=1e-10)
    h = surrogate_widths(distorted_vertices(2, seed=3, dim=3), (1, 0, 1))
    assert len(h) == 3 and all(0.3 < x < 0.8 for x in h)


def test_hierarchy_on_cartesian_vertices_is_the_cartesian_vcycle_3d():
    rng = np.random.default_rng(8)
    widths = [rng.uniform(0.5, 1.5, 2) for _ in range(3)]
    H = MappedHierarchy(cartesian_vertices(*widths), 1, 2, "MCS", 1.0, steps=1, gamma_hat=4.0)
    C = multigrid.Hierarchy(widths, 1, 2, "MCS", 1.0, gamma_hat=4.0)
    r = rng.uniform(-1, 1, H.A[-1].shape[0])
    assert np.allclose(H.precondition(r), C.precondition(r), rtol=1e-10, atol=1e-12)


def test_l2_convergence_on_distorted_hexahedra():
    """O(h^(k+1)) L2 convergence on the 25%-distorted cube and two trilinear
    refinements (k = 1: rate 2) for u = sin(pi x) sin(pi y) sin(pi z)."""
    u = lambda p: np.sin(np.pi * p[:, 0]) * np.sin(np.pi * p[:, 1]) * np.sin(np.pi * p[:, 2])
    f = lambda p: 3 * np.pi ** 2 * u(p)
    V = distorted_vertices(2, seed=12, dim=3)
    errs = []
    for _ in range(3):
        S = MappedSIPG(V, 1, gamma_hat=4.0)
        x = spla.spsolve(S.assemble().tocsc(), S.rhs(f, u))
        errs.append(S.l2_error(x, u))
        V = refine(V)
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > 1.8, (errs, rates)


def test_mcs_vcycle_is_symmetric_on_distorted_hexahedra():
    H = MappedHierarchy(distorted_vertices(2, seed=13, dim=3), 1, 2, "MCS", 0.9, steps=1)
    n = H.A[-1].shape[0]
    rng = np.random.default_rng(4)
    x, y = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    assert abs(x @ H.precondition(y) - y @ H.precondition(x)) <= 1e-11 * abs(x @ H.precondition(x))


def test_local_stability_of_the_surrogate_solvers():
    """eq. localstab: a(u, u) <= eta a~(u, u) on every cell subspace with eta
    independent of the cell.  The spectrum of (A~_j)^{-1} A_j is exactly {1} on
    a Cartesian mesh, stays in a fixed interval on distorted meshes, narrows as
    the distortion shrinks, and hardly depends on the degree."""
    import scipy.linalg as sla

    def spectrum(V, k):
        S = MappedSIPG(V, k, 4.0)
        A = S.assemble().tocsr()
        lo, hi = np.inf, 0.0
        for c in range(S.ncells):
            idx = schwarz.patch_dofs([c], S.nloc)
            ev = sla.eigh(A[idx][:, idx].toarray(), surrogate_cell_matrix(V, S.cell_multi(c), k, 4.0),
                          eigvals_only=True)
            lo, hi = min(lo, ev[0]), max(hi, ev[-1])
        return lo, hi

    lo, hi = spectrum(cartesian_vertices(np.full(5, 0.2), np.full(5, 0.2)), 3)
    assert abs(lo - 1) < 1e-10 and abs(hi - 1) < 1e-10
    eta = {}
    for k in (1, 3):
        lo25, hi25 = spectrum(distorted_vertices(6, seed=3), k)
        lo10, hi10 = spectrum(distorted_vertices(6, seed=3, alpha=0.1), k)
        assert 0.4 < lo25 < lo10 < 1.0 < hi10 < hi25 < 2.5, (k, lo25, lo10, hi10, hi25)
        eta[k] = hi25
    assert eta[3] < 1.2 * eta[1], eta
