"""Pins for oracle.multigrid (Alg. 1, Sec. 2.4)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.multigrid import Hierarchy, fgmres, fractional_iterations, gmres_left, pcg


def coarse(d, n=2):
    return [np.full(n, 1.0 / n)] * d


@pytest.mark.parametrize("smoother", ["ACS", "AVS", "MCS", "MVS"])
def test_pcg_solution_matches_direct_solve(smoother):
    H = Hierarchy(coarse(2), k=2, nlevels=3, smoother=smoother)
    rng = np.random.default_rng(11)
    A = H.A[-1]
    b = rng.uniform(-1, 1, A.shape[0])
    x, it, hist, ok = pcg(A, b, H.precondition, rtol=1e-10, maxit=200)
    assert ok
    xd = spla.spsolve(A.tocsc(), b)
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
    assert it < 40


@pytest.mark.parametrize("smoother", ["ACS", "AVS", "MCS", "MVS"])
def test_vcycle_is_symmetric(smoother):
    H = Hierarchy(coarse(2), k=1, nlevels=3, smoother=smoother)
    N = H.A[-1].shape[0]
    B = np.column_stack([H.precondition(e) for e in np.eye(N)])
    assert np.abs(B - B.T).max() <= 1e-11 * np.abs(B).max()
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0


def test_vcycle_on_coarse_level_is_exact():
    H = Hierarchy(coarse(3), k=2, nlevels=1, smoother="AVS")
    b = np.random.default_rng(3).uniform(-1, 1, H.A[0].shape[0])
    x = H.precondition(b)
    assert np.abs(H.A[0] @ x - b).max() < 1e-11


def test_fractional_iterations_hand_values():
    # e = 1, 0.1, 0.01, 1e-3 ... ; rtol = 10^-2.5 -> nu = 3, frac = 2 + log(1e-2/10^-2.5)/log(10) = 2.5
    hist = [1.0, 0.1, 0.01, 1e-3, 1e-4]
    assert np.isclose(fractional_iterations(hist, 10 ** -2.5), 2.5)
    assert np.isclose(fractional_iterations(hist, 1e-3), 3.0)


def test_gmres_unpreconditioned_finite_termination_and_true_residuals():
    rng = np.random.default_rng(4)
    n = 12
    A = rng.standard_normal((n, n)) + 4 * np.eye(n)      # non-symmetric
    b = rng.standard_normal(n)
    # record the iterates through a restart length of 1 (hist = true residuals)
    x, it, hist, ok = fgmres(A, b, lambda v: v, rtol=1e-12, maxit=n, restart=n)
    assert ok and it <= n
    assert np.linalg.norm(A @ x - b) <= 1e-10 * np.linalg.norm(b)
    # the least-squares residuals are non-increasing
    assert all(hist[i + 1] <= hist[i] * (1 + 1e-12) for i in range(len(hist) - 1))
    # GMRES(1) residual after one step equals the true residual of x_1 = alpha b
    x1, _, h1, _ = fgmres(A, b, lambda v: v, rtol=1e-300, maxit=1, restart=1)
    assert np.isclose(h1[1], np.linalg.norm(b - A @ x1), rtol=1e-10)


@pytest.mark.parametrize("smoother", ["MCS", "MVS"])
def test_fgmres_with_nonsymmetric_vcycle_matches_direct_solve(smoother):
    H = Hierarchy(coarse(2), k=2, nlevels=3, smoother=smoother, symmetric=False)
    A = H.A[-1]
    b = np.random.default_rng(5).uniform(-1, 1, A.shape[0])
    x, it, hist, ok = fgmres(A, b, H.precondition, rtol=1e-10, maxit=60)
    assert ok
    xd = spla.spsolve(A.tocsc(), b)
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
    assert it < 20


def test_nonsymmetric_vcycle_is_not_symmetric():
    H = Hierarchy(coarse(2), k=1, nlevels=3, smoother="MVS", symmetric=False)
    N = H.A[-1].shape[0]
    B = np.column_stack([H.precondition(e) for e in np.eye(N)])
    assert np.abs(B - B.T).max() > 1e-6 * np.abs(B).max()


def test_left_gmres_history_is_the_preconditioned_residual():
    rng = np.random.default_rng(11)
    n = 14
    A = rng.standard_normal((n, n)) + 5 * np.eye(n)
    Mmat = np.diag(rng.uniform(0.5, 2.0, n)) + 0.1 * rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    M = lambda v: Mmat @ v
    x, it, hist, ok = gmres_left(A, b, M, rtol=1e-12, maxit=n, restart=n)
    assert ok and it <= n
    assert np.linalg.norm(A @ x - b) <= 1e-9 * np.linalg.norm(b)
    # GMRES(1) steps one at a time: each history entry is ||M (b - A x_k)|| of
    # the iterate the restart recomputes
    xs, hs = np.zeros(n), [np.linalg.norm(M(b))]
    for _ in range(4):
        xk, _, hk, _ = gmres_left(A, b - A @ xs, M, rtol=1e-300, maxit=1, restart=1)
        xs = xs + xk
        hs.append(hk[1])
        assert np.isclose(hk[1], np.linalg.norm(M(b - A @ xs)), rtol=1e-10)
    # a dropped preconditioner on the restart residual would break this
    assert all(hs[i + 1] <= hs[i] * (1 + 1e-12) for i in range(len(hs) - 1))


def test_left_gmres_with_identity_is_unpreconditioned_gmres():
    rng = np.random.default_rng(12)
    n = 10
    A = rng.standard_normal((n, n)) + 4 * np.eye(n)
    b = rng.standard_normal(n)
    _, it1, h1, _ = gmres_left(A, b, lambda v: v, rtol=1e-10, maxit=n, restart=n)
    _, it2, h2, _ = fgmres(A, b, lambda v: v, rtol=1e-10, maxit=n, restart=n)
    assert it1 == it2 and np.allclose(h1, h2, rtol=1e-8)


def test_left_gmres_with_nonsymmetric_vcycle_matches_direct_solve():
    H = Hierarchy(coarse(2), k=2, nlevels=3, smoother="MVS", symmetric=False)
    A = H.A[-1]
    b = np.random.default_rng(13).uniform(-1, 1, A.shape[0])
    x, it, hist, ok = gmres_left(A, b, H.precondition, rtol=1e-10, maxit=60)
    assert ok and it < 20
    xd = spla.spsolve(A.tocsc(), b)
    assert np.linalg.norm(x - xd) <= 1e-7 * np.linalg.norm(xd)
