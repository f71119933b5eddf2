"""Pin the oracle's d-dimensional SIPG assembly against the Kronecker-sum
structure of Sec. 3.2, built here directly from the paper's 1D matrices:

* eq. 1Dstiffnessmass: M and L on an interval of width h;
* eq. 1Dconsistencypenalty / eq. 1Dnitsche / eq. 1Dsipg for a cell, with
  eta = 1/2 on interior faces and 1 on boundary faces applied to the penalty
  term as well (the reading that follows eq. bfsipg with 1/sqrt(2) averages);
* eq. 1DsipgVP for a vertex patch, with the interface block derived from
  eq. bfsipg: A_{+-}[i, j] = -gamma/2 phi_j(0) phi_i(1)
  - 1/(2 h_-) phi_j'(0) phi_i(1) + 1/(2 h_+) phi_j(0) phi_i'(1)  (test i in the
  left cell "+", trial j in the right cell "-"), A_{-+} = A_{+-}^T;
* eq. KDseparable for the d-dimensional sum.

The same tests also pin the fast diagonalization identities (eq.
generalizedEVP, eq. localsolverEVP, eq. fastinverse) against the dense inverse
of the assembled local matrix.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.basis import gauss_legendre, gauss_lobatto_nodes, lagrange_derivatives, lagrange_values
from oracle.mesh import TensorMesh
from oracle.schwarz import vertex_patches
from oracle.sipg import SIPG, penalty_factor


class OneD:
    def __init__(self, k, gamma_hat, penalty):
        self.k = k
        nodes = gauss_lobatto_nodes(k)
        self.xq, self.wq = gauss_legendre(k + 1)
        self.V = lagrange_values(nodes, self.xq)
        self.D = lagrange_derivatives(nodes, self.xq)
        self.v = lagrange_values(nodes, [0.0, 1.0])
        self.dv = lagrange_derivatives(nodes, [0.0, 1.0])
        self.pk = gamma_hat * penalty_factor(k, penalty)

    def gamma(self, hm, hp):
        return self.pk * (1.0 / hm + 1.0 / hp)

    def mass(self, h):
        return h * (self.V.T * self.wq) @ self.V

    def lap(self, h):
        return (self.D.T * self.wq) @ self.D / h

    def nitsche(self, h, p, gamma, eta):
        # G[i, j] = (-1)^(p+1) eta/h phi_j'(p) phi_i(p);  M_p[i, j] = phi_j(p) phi_i(p)
        G = (-1.0) ** (p + 1) * eta / h * np.outer(self.v[p], self.dv[p])
        Mp = np.outer(self.v[p], self.v[p])
        return eta * gamma * Mp - G - G.T

    def cell(self, widths, c):
        """A^(t) of eq. 1Dsipg for cell c of a 1D subdivision `widths`."""
        h = widths[c]
        A = self.lap(h)
        for p, nb in ((0, c - 1), (1, c + 1)):
            if 0 <= nb < len(widths):
                A = A + self.nitsche(h, p, self.gamma(h, widths[nb]), 0.5)
            else:
                A = A + self.nitsche(h, p, self.gamma(h, h), 1.0)
        return A

    def interface(self, hp, hm):
        g = self.gamma(hp, hm)
        return (-0.5 * g * np.outer(self.v[1], self.v[0])
                - 0.5 / hm * np.outer(self.v[1], self.dv[0])
                + 0.5 / hp * np.outer(self.dv[1], self.v[0]))

    def patch(self, widths, c0):
        """A^(t), M^(t) of eq. 1DsipgVP for the patch of cells c0, c0+1."""
        Ap, Am = self.cell(widths, c0), self.cell(widths, c0 + 1)
        Apm = self.interface(widths[c0], widths[c0 + 1])
        A = np.block([[Ap, Apm], [Apm.T, Am]])
        n = self.k + 1
        M = np.zeros((2 * n, 2 * n))
        M[:n, :n] = self.mass(widths[c0])
        M[n:, n:] = self.mass(widths[c0 + 1])
        return A, M


def kron_sum(As, Ms):
    """eq. KDseparable: sum_t M^(d) x ... x A^(t) x ... x M^(1), first direction
    fastest (np.kron puts its first factor slowest)."""
    d = len(As)
    total = 0
    for t in range(d):
        f = None
        for s in reversed(range(d)):
            m = As[s] if s == t else Ms[s]
            f = m if f is None else np.kron(f, m)
        total = total + f
    return total


def patch_perm(k, d):
    """perm[p] = cell-major position of patch tensor index p, p_t = c_t (k+1) + i_t."""
    n1, n = k + 1, 2 * (k + 1)
    perm = np.zeros(n ** d, dtype=int)
    for p in range(n ** d):
        pm = [(p // n ** t) % n for t in range(d)]
        c = [pm[t] // n1 for t in range(d)]
        i = [pm[t] % n1 for t in range(d)]
        cpos = sum(c[t] << t for t in range(d))
        loc = sum(i[t] * n1 ** t for t in range(d))
        perm[p] = cpos * n1 ** d + loc
    return perm


CASES = [(2, 1, 4), (2, 3, 4), (3, 2, 3), (3, 3, 4)]


@pytest.mark.parametrize("d,k,n", CASES)
@pytest.mark.parametrize("penalty", ["paper", "kp1sq"])
def test_cell_matrix_is_kronecker_sum(d, k, n, penalty):
    rng = np.random.default_rng(100 + d * 10 + k)
    widths = [rng.uniform(0.5, 1.5, n) / n for _ in range(d)]
    mesh = TensorMesh(widths)
    S = SIPG(mesh, k, gamma_hat=1.0, penalty_poly=penalty)
    one = OneD(k, 1.0, penalty)
    for c in range(mesh.num_cells):
        m = mesh.cell_multi(c)
        As = [one.cell(widths[t], m[t]) for t in range(d)]
        Ms = [one.mass(widths[t][m[t]]) for t in range(d)]
        K = kron_sum(As, Ms)
        Aj = S.assemble([c]).toarray()
        assert np.abs(K - Aj).max() <= 1e-12 * np.abs(Aj).max()


@pytest.mark.parametrize("d,k,n", CASES)
@pytest.mark.parametrize("penalty", ["paper", "kp1sq"])
def test_vertex_patch_matrix_is_kronecker_sum(d, k, n, penalty):
    rng = np.random.default_rng(200 + d * 10 + k)
    widths = [rng.uniform(0.5, 1.5, n) / n for _ in range(d)]
    mesh = TensorMesh(widths)
    S = SIPG(mesh, k, gamma_hat=1.0, penalty_poly=penalty)
    one = OneD(k, 1.0, penalty)
    perm = patch_perm(k, d)
    for v, cells in vertex_patches(mesh):
        As, Ms = zip(*[one.patch(widths[t], v[t] - 1) for t in range(d)])
        K = kron_sum(As, Ms)
        Aj = S.assemble(cells).toarray()[np.ix_(perm, perm)]
        assert np.abs(K - Aj).max() <= 1e-12 * np.abs(Aj).max()


def test_interface_sign_matters():
    # a dropped minus sign on the interface penalty must break the agreement
    rng = np.random.default_rng(7)
    k, d = 2, 2
    widths = [rng.uniform(0.5, 1.5, 3) / 3 for _ in range(d)]
    mesh = TensorMesh(widths)
    S = SIPG(mesh, k)
    one = OneD(k, 1.0, "paper")
    v, cells = vertex_patches(mesh)[0]
    As, Ms = [], []
    for t in range(d):
        A, M = one.patch(widths[t], v[t] - 1)
        n1 = k + 1
        A = A.copy()
        A[:n1, n1:] = -A[:n1, n1:]
        A[n1:, :n1] = -A[n1:, :n1]
        As.append(A)
        Ms.append(M)
    Aj = S.assemble(cells).toarray()[np.ix_(patch_perm(k, d), patch_perm(k, d))]
    assert np.abs(kron_sum(As, Ms) - Aj).max() > 1e-3


@pytest.mark.parametrize("d,k", [(2, 2), (3, 2), (3, 3)])
def test_fast_diagonalization_inverse_equals_dense_inverse(d, k):
    rng = np.random.default_rng(300 + d + k)
    n = 3
    widths = [rng.uniform(0.5, 1.5, n) / n for _ in range(d)]
    mesh = TensorMesh(widths)
    S = SIPG(mesh, k)
    one = OneD(k, 1.0, "paper")
    perm = patch_perm(k, d)
    v, cells = vertex_patches(mesh)[-1]
    Zs, lams = [], []
    for t in range(d):
        A, M = one.patch(widths[t], v[t] - 1)
        lam, Z = sla.eigh(A, M)               # generalized symmetric eigenproblem
        assert np.allclose(Z.T @ M @ Z, np.eye(len(lam)), atol=1e-12)
        assert np.allclose(Z.T @ A @ Z, np.diag(lam), atol=1e-10 * lam.max())
        assert lam.min() > 0
        Zs.append(Z)
        lams.append(lam)
    # Z = Z^(d) x ... x Z^(1), Lambda = Kronecker sum of the lambda^(t)
    Z = Zs[-1]
    for t in reversed(range(d - 1)):
        Z = np.kron(Z, Zs[t])
    lam = np.zeros(1)
    for t in reversed(range(d)):
        lam = np.add.outer(lam, lams[t]).ravel()
    inv_fd = Z @ np.diag(1.0 / lam) @ Z.T
    Aj = S.assemble(cells).toarray()[np.ix_(perm, perm)]
    inv_lu = np.linalg.inv(Aj)
    assert np.abs(inv_fd - inv_lu).max() <= 1e-10 * np.abs(inv_lu).max()
