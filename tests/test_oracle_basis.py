"""Pins for oracle.basis: closed forms and exactness properties (Sec. 2.1, Sec. 3)."""
import numpy as np
import pytest

from oracle.basis import gauss_legendre, gauss_lobatto_nodes, lagrange_derivatives, lagrange_values


def test_gauss_lobatto_closed_forms():
    # k = 1: end points; k = 2: {0, 1/2, 1}; k = 3: {0, 1/2 -+ sqrt(5)/10, 1}
    assert np.allclose(gauss_lobatto_nodes(1), [0.0, 1.0], atol=1e-15)
    assert np.allclose(gauss_lobatto_nodes(2), [0.0, 0.5, 1.0], atol=1e-15)
    r = np.sqrt(5.0) / 10.0
    assert np.allclose(gauss_lobatto_nodes(3), [0.0, 0.5 - r, 0.5 + r, 1.0], atol=1e-15)
    # k = 4: interior roots of P_4' on [-1,1] are 0, +-sqrt(3/7)
    s = np.sqrt(3.0 / 7.0)
    assert np.allclose(gauss_lobatto_nodes(4), [0.0, 0.5 * (1 - s), 0.5, 0.5 * (1 + s), 1.0], atol=1e-15)


@pytest.mark.parametrize("k", range(1, 16))
def test_gauss_lobatto_symmetric_sorted(k):
    x = gauss_lobatto_nodes(k)
    assert len(x) == k + 1
    assert np.all(np.diff(x) > 0)
    assert np.allclose(x + x[::-1], 1.0, atol=1e-14)


@pytest.mark.parametrize("nq", range(1, 18))
def test_gauss_rule_exact_on_monomials(nq):
    x, w = gauss_legendre(nq)
    for m in range(2 * nq):
        assert abs(np.sum(w * x ** m) - 1.0 / (m + 1)) < 1e-14
    # degree 2 nq is not exact; the error is the textbook Gauss remainder
    # (n!)^4 / ((2n+1) ((2n)!)^2) for x^(2n) on [0, 1]
    from math import factorial
    remainder = factorial(nq) ** 4 / ((2 * nq + 1) * factorial(2 * nq) ** 2)
    err = 1.0 / (2 * nq + 1) - np.sum(w * x ** (2 * nq))
    assert abs(err - remainder) < 1e-15 + 1e-9 * remainder


@pytest.mark.parametrize("k", range(1, 16))
def test_lagrange_delta_and_partition_of_unity(k):
    nodes = gauss_lobatto_nodes(k)
    V = lagrange_values(nodes, nodes)
    assert np.allclose(V, np.eye(k + 1), atol=1e-13)
    xs = np.linspace(0, 1, 37)
    assert np.allclose(lagrange_values(nodes, xs).sum(axis=1), 1.0, atol=1e-12)
    assert np.allclose(lagrange_derivatives(nodes, xs).sum(axis=1), 0.0, atol=1e-9)


@pytest.mark.parametrize("k", [1, 2, 3, 5, 7])
def test_interpolation_of_polynomials_is_exact_with_derivative(k):
    nodes = gauss_lobatto_nodes(k)
    xs = np.linspace(0, 1, 23)
    V = lagrange_values(nodes, xs)
    D = lagrange_derivatives(nodes, xs)
    for m in range(k + 1):
        coef = nodes ** m
        assert np.allclose(V @ coef, xs ** m, atol=1e-12)
        dexact = m * xs ** (m - 1) if m > 0 else np.zeros_like(xs)
        assert np.allclose(D @ coef, dexact, atol=1e-9)
