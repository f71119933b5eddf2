"""Pins for oracle.sipg (eq. bfsipg, eq. penalty, eq. sipg): symmetry, SPD,
consistency (exact reproduction of Q_k solutions) and L2 convergence order."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.mesh import TensorMesh
from oracle.sipg import SIPG


def random_mesh(d, n, seed):
    rng = np.random.default_rng(seed)
    return TensorMesh([rng.uniform(0.5, 1.5, n) / n for _ in range(d)])


@pytest.mark.parametrize("d,n,k", [(2, 3, 1), (2, 4, 3), (3, 2, 2), (3, 3, 1)])
@pytest.mark.parametrize("penalty", ["paper", "kp1sq"])
def test_symmetric_positive_definite(d, n, k, penalty):
    S = SIPG(random_mesh(d, n, 10 * d + n + k), k, penalty_poly=penalty)
    A = S.assemble().toarray()
    assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max()
    np.linalg.cholesky(A)  # raises if not SPD
    assert np.linalg.eigvalsh(A).min() > 0


def test_row_sums_of_pure_bulk_vanish_on_constants():
    # A applied to a constant: bulk terms and interior jumps vanish, only boundary
    # terms remain -> rows of interior cells (no boundary face) sum to zero.
    S = SIPG(random_mesh(2, 4, 1), 2)
    A = S.assemble()
    y = A @ np.ones(A.shape[0])
    mesh = S.mesh
    for c in range(mesh.num_cells):
        m = mesh.cell_multi(c)
        if all(0 < m[t] < mesh.ncells[t] - 1 for t in range(2)):
            assert np.abs(y[c * S.nloc:(c + 1) * S.nloc]).max() < 1e-11


def _solve(S, f, g):
    A = S.assemble().tocsc()
    b = S.rhs(f, g)
    return spla.spsolve(A, b)


@pytest.mark.parametrize("penalty", ["paper", "kp1sq"])
def test_polynomial_solution_reproduced_2d(penalty):
    # u = x^2 y + y^2 in Q_2: the SIPG solution equals the interpolant of u
    u = lambda p: p[:, 0] ** 2 * p[:, 1] + p[:, 1] ** 2
    f = lambda p: -(2 * p[:, 1] + 2.0)
    S = SIPG(random_mesh(2, 3, 5), 2, penalty_poly=penalty)
    x = _solve(S, f, u)
    assert np.abs(x - S.interpolate(u)).max() < 1e-11


def test_polynomial_solution_reproduced_3d():
    u = lambda p: p[:, 0] ** 2 * p[:, 1] + p[:, 2] ** 3 - p[:, 0] * p[:, 1] * p[:, 2]
    f = lambda p: -(2 * p[:, 1] + 6 * p[:, 2])
    S = SIPG(random_mesh(3, 2, 6), 3)
    x = _solve(S, f, u)
    assert np.abs(x - S.interpolate(u)).max() < 1e-10


def test_non_polynomial_not_reproduced():
    # guard against a vacuous consistency test: a Q_3 function is not reproduced by Q_2
    u = lambda p: p[:, 0] ** 3
    f = lambda p: -6 * p[:, 0]
    S = SIPG(random_mesh(2, 3, 5), 2)
    x = _solve(S, f, u)
    assert np.abs(x - S.interpolate(u)).max() > 1e-6


@pytest.mark.parametrize("k", [1, 2])
def test_l2_convergence_order(k):
    u = lambda p: np.sin(np.pi * p[:, 0]) * np.sin(np.pi * p[:, 1])
    f = lambda p: 2 * np.pi ** 2 * u(p)
    errs = []
    for n in (4, 8):
        S = SIPG(TensorMesh([np.full(n, 1.0 / n)] * 2), k)
        x = _solve(S, f, None)
        errs.append(S.l2_error(x, u))
    rate = np.log2(errs[0] / errs[1])
    assert rate > k + 1 - 0.25, rate


def test_penalty_formula_matches_eq_penalty():
    S = SIPG(TensorMesh([np.ones(2)]), 3)
    assert np.isclose(S.gamma(0.5, 0.25), 3 * 4 * (2 + 4))
    S2 = SIPG(TensorMesh([np.ones(2)]), 3, gamma_hat=4.0, penalty_poly="kp1sq")
    assert np.isclose(S2.gamma(0.5, 0.5), 4.0 * 16 * 4)
