"""Pins of the oracle's Chebyshev coarse solver (oracle/chebyshev.py)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import schwarz
from oracle.chebyshev import (chebyshev, iteration_count, lanczos_from_cg, spectral_bounds, splitmix64,
                              start_vector)
from oracle.mesh import TensorMesh
from oracle.sipg import SIPG


def test_splitmix64_reference_outputs():
    # first outputs of SplitMix64 from state 0 (the generator's published test values)
    assert [splitmix64(i) for i in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    s = start_vector(1000)
    assert s.min() >= -1.0 and s.max() < 1.0 and abs(s.mean()) < 0.1


def test_error_is_the_chebyshev_polynomial():
    """Diagonal A, P = I: e_m = p_m(lambda) e_0 with p_m(t) = T_m((theta - t)/delta) / T_m(theta/delta)."""
    lam = np.linspace(1.0, 30.0, 17)
    A = np.diag(lam)
    f = np.random.default_rng(1).uniform(-1, 1, lam.size)
    a, b = 0.9, 33.0
    theta, delta = (a + b) / 2, (b - a) / 2
    xs = f / lam
    for m in (1, 2, 5, 12):
        x = chebyshev(A, f, lambda v: v, a, b, m)
        # (theta - lam)/delta lies in [-1, 1] for lam in [a, b]
        p = np.cos(m * np.arccos((theta - lam) / delta)) / np.cosh(m * np.arccosh(theta / delta))
        assert np.allclose(x - xs, p * (0 - xs), atol=1e-13, rtol=1e-11)


def test_ritz_values_match_explicit_lanczos():
    rng = np.random.default_rng(2)
    n = 40
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.linspace(1.0, 50.0, n)) @ Q.T
    Pd = rng.uniform(0.5, 2.0, n)                  # SPD diagonal preconditioner
    prec = lambda v: Pd * v
    s = rng.uniform(-1, 1, n)
    m = 12
    T = lanczos_from_cg(A, prec, s, m)
    # explicit Lanczos, full reorthogonalization, for P^{1/2} A P^{1/2} (similar to
    # P A) started from P^{-1/2} z_0 = P^{1/2} s, the image of CG's first direction
    S = np.sqrt(Pd)
    B = (S[:, None] * A) * S[None, :]
    V = np.zeros((n, m + 1))
    V[:, 0] = S * s
    V[:, 0] /= np.linalg.norm(V[:, 0])
    al, be = [], []
    for j in range(m):
        w = B @ V[:, j]
        al.append(V[:, j] @ w)
        w -= V[:, :j + 1] @ (V[:, :j + 1].T @ w)
        w -= V[:, :j + 1] @ (V[:, :j + 1].T @ w)
        be.append(np.linalg.norm(w))
        V[:, j + 1] = w / be[-1]
    Tl = np.diag(al) + np.diag(be[:-1], 1) + np.diag(be[:-1], -1)
    assert np.allclose(np.linalg.eigvalsh(T), np.linalg.eigvalsh(Tl), rtol=1e-9)
    # Ritz values lie inside the spectrum of P A
    ev = np.sort(np.linalg.eigvals(Pd[:, None] * A).real)
    assert ev[0] - 1e-9 <= np.linalg.eigvalsh(T)[0] and np.linalg.eigvalsh(T)[-1] <= ev[-1] + 1e-9


def test_iteration_count_reaches_the_bound():
    rng = np.random.default_rng(3)
    n = 60
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.geomspace(1.0, 200.0, n)
    A = Q @ np.diag(lam) @ Q.T
    f = rng.uniform(-1, 1, n)
    a, b = lam[0], lam[-1]
    m = iteration_count(a, b, 1e-8)
    x = chebyshev(A, f, lambda v: v, a, b, m)
    xs = np.linalg.solve(A, f)
    eA = lambda e: np.sqrt(e @ A @ e)
    assert eA(x - xs) <= 1e-8 * eA(xs)
    # one step fewer no longer guarantees it in general; the count is minimal for the bound
    q = (np.sqrt(b / a) - 1) / (np.sqrt(b / a) + 1)
    assert 2 * q ** (m - 1) / (1 + q ** (2 * m - 2)) > 1e-8


@pytest.mark.parametrize("d,k", [(2, 3), (3, 2)])
def test_coarse_solve_with_cell_smoother_reaches_1e8(d, k):
    """T_0 = 2^d cells with the additive cell smoother (omega = 1) as
    preconditioner: the A-norm error falls below 1e-8."""
    mesh = TensorMesh([np.array([0.4, 0.6])] * d)
    S = SIPG(mesh, k)
    A = S.assemble().toarray()
    patches = schwarz.cell_patches(mesh)
    sol = schwarz.LocalSolvers(patches, S.nloc, lambda cells: S.assemble(cells))
    prec = lambda r: schwarz.additive_local_sum(r, sol, 1.0)
    n = A.shape[0]
    a, b = spectral_bounds(A, prec, n)
    ev = np.sort(sla.eigh(A, np.linalg.inv(np.column_stack([prec(e) for e in np.eye(n)])),
                          eigvals_only=True))
    assert b >= ev[-1]                           # the widened upper bound covers the spectrum of P A
    f = np.random.default_rng(4).uniform(-1, 1, n)
    x = chebyshev(A, f, prec, a, b, iteration_count(a, b, 1e-8))
    xs = np.linalg.solve(A, f)
    eA = lambda e: np.sqrt(e @ A @ e)
    assert eA(x - xs) <= 1e-8 * eA(xs)
