"""Pins for oracle.transfer (Sec. 2.2): embedding exactness and transpose."""
import numpy as np
import pytest

from oracle.mesh import TensorMesh
from oracle.sipg import SIPG
from oracle.transfer import prolongation_matrix


@pytest.mark.parametrize("d,k", [(2, 1), (2, 3), (3, 2)])
def test_prolongation_embeds_coarse_polynomials_exactly(d, k):
    rng = np.random.default_rng(d * 10 + k)
    coarse = TensorMesh([rng.uniform(0.5, 1.5, 3) for _ in range(d)])
    fine = coarse.refine()
    P = prolongation_matrix(coarse, fine, k)
    Sc, Sf = SIPG(coarse, k), SIPG(fine, k)
    # a discontinuous coarse function: random coefficients; its value at fine
    # support points, evaluated directly, must equal P @ coef
    coef = rng.standard_normal(P.shape[1])
    # smooth polynomial of degree k in each variable
    poly = lambda p: np.prod([1 + p[:, t] ** k - 0.5 * p[:, t] for t in range(d)], axis=0)
    assert np.abs(P @ Sc.interpolate(poly) - Sf.interpolate(poly)).max() < 1e-11
    # a Q_{k+1} function is not embedded exactly (guard)
    poly2 = lambda p: p[:, 0] ** (k + 1)
    assert np.abs(P @ Sc.interpolate(poly2) - Sf.interpolate(poly2)).max() > 1e-6
    # rows of P sum to one (constants are embedded)
    assert np.allclose(np.asarray(P.sum(axis=1)).ravel(), 1.0, atol=1e-13)
    del coef


def test_restriction_is_transpose():
    coarse = TensorMesh([np.ones(2), np.ones(3)])
    P = prolongation_matrix(coarse, coarse.refine(), 2)
    rng = np.random.default_rng(1)
    u, v = rng.standard_normal(P.shape[1]), rng.standard_normal(P.shape[0])
    assert np.isclose((P @ u) @ v, u @ (P.T @ v))
