"""1D finite element primitives on the reference interval [0, 1].

Test infrastructure only (see the package docstring).

The shape functions are the Lagrange interpolation polynomials of degree k in
the k+1 Gauss-Lobatto points (Sec. 2.1 and Sec. 3, eq. tppoly / basisref).  The
1D quadrature rule is Gauss-Legendre; the paper only says the number of points
is "almost" k (Sec. 3.1), and the reading taken here is k+1 points, which
integrates products of two degree-k polynomials exactly (no mass lumping).

Pins (tests/test_oracle_basis.py): closed-form Gauss-Lobatto nodes for k = 2, 3,
exactness of the Gauss rule on monomials up to degree 2 nq - 1, the Kronecker
delta property, partition of unity and exact differentiation of interpolated
polynomials.
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def gauss_lobatto_nodes(k):
    """The k+1 Gauss-Lobatto points on [0, 1]: both end points plus the roots
    of P_k' (derivative of the Legendre polynomial of degree k), ascending."""
    if k < 1:
        raise ValueError("degree must be >= 1")
    inner = npleg.Legendre.basis(k).deriv().roots() if k >= 2 else np.array([])
    t = np.concatenate(([-1.0], np.sort(np.real(inner)), [1.0]))
    return 0.5 * (t + 1.0)


def gauss_legendre(nq):
    """nq-point Gauss-Legendre rule mapped to [0, 1]: (points, weights)."""
    t, w = npleg.leggauss(nq)
    return 0.5 * (t + 1.0), 0.5 * w


def lagrange_values(nodes, x):
    """V[q, i] = phi_i(x_q), phi_i the Lagrange polynomial with phi_i(nodes_j) =
    delta_ij, evaluated by the product formula."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    V = np.ones((len(x), n))
    for i in range(n):
        for j in range(n):
            if j != i:
                V[:, i] *= (x - nodes[j]) / (nodes[i] - nodes[j])
    return V


def lagrange_derivatives(nodes, x):
    """D[q, i] = phi_i'(x_q) by the product rule applied to the product formula:
    phi_i' = sum_{m != i} 1/(x_i - x_m) prod_{j != i, m} (x - x_j)/(x_i - x_j)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    D = np.zeros((len(x), n))
    for i in range(n):
        for m in range(n):
            if m == i:
                continue
            term = np.full(len(x), 1.0 / (nodes[i] - nodes[m]))
            for j in range(n):
                if j != i and j != m:
                    term *= (x - nodes[j]) / (nodes[i] - nodes[j])
            D[:, i] += term
    return D
