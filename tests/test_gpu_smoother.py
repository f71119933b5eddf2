"""GPU parity of the Schwarz smoothers (Alg. 2, Alg. 3) against the oracle's
dense-LU local solvers, element by element, FP64 relative 1e-12."""
import numpy as np
import pytest
import torch

from gpu_helpers import TOL64, dev, make, oracle_solvers, oracle_sipg, rel_err
from oracle import schwarz
from paper_1910_11239_gb300 import workloads

pytestmark = pytest.mark.gpu

# (dim, k, cells per direction): several tiles and a ragged (odd) count
CASES = [(2, 1, 7), (2, 2, 6), (2, 5, 5), (2, 7, 3), (3, 1, 5), (3, 2, 4), (3, 3, 3), (3, 5, 3)]


@pytest.mark.parametrize("dim,k,n", CASES)
@pytest.mark.parametrize("kind", ["vertex", "cell"])
def test_additive_smoother_matches_oracle(dim, k, n, kind):
    from paper_1910_11239_gb300 import tpss
    widths = workloads.widths_random(n, dim, seed=7 + n + k)
    widths[0] = widths[0][:n]  # keep n per direction
    if dim == 3:
        widths[2] = workloads.widths_random(n + 1, 1, seed=99)[0]  # ragged: n+1 cells along z
    prob = make(dim, k, widths)
    P = prob.setup_patches(0, tpss.VERTEX_PATCH if kind == "vertex" else tpss.CELL)
    S = oracle_sipg(widths, k)
    A = S.assemble().tocsr()
    _, sol = oracle_solvers(S, A, kind)
    N = A.shape[0]
    nrhs = 2
    b = workloads.rhs_uniform(N, seed=1, nrhs=nrhs)
    x0 = workloads.rhs_uniform(N, seed=2, nrhs=nrhs)
    omega = 0.7
    # x = 0 form (smoother only)
    xg = torch.empty(N * nrhs, dtype=torch.float64, device="cuda")
    P.smooth_additive(omega, dev(b), xg, x_is_zero=True, nrhs=nrhs)
    for r in range(nrhs):
        ref = schwarz.additive_local_sum(b[r * N:(r + 1) * N], sol, omega)
        assert rel_err(xg[r * N:(r + 1) * N], ref) < TOL64
    # general form with residual
    xg = dev(x0)
    P.smooth_additive(omega, dev(b), xg, x_is_zero=False, nrhs=nrhs)
    for r in range(nrhs):
        ref = schwarz.additive_smoother(A, b[r * N:(r + 1) * N], x0[r * N:(r + 1) * N], sol, omega)
        assert rel_err(xg[r * N:(r + 1) * N], ref) < TOL64
    prob.close()


@pytest.mark.parametrize("dim,k,n", [(2, 2, 6), (2, 4, 5), (3, 1, 5), (3, 2, 4), (3, 3, 3)])
@pytest.mark.parametrize("kind", ["vertex", "cell"])
@pytest.mark.parametrize("reverse", [False, True])
def test_multiplicative_smoother_matches_oracle(dim, k, n, kind, reverse):
    from paper_1910_11239_gb300 import tpss
    widths = workloads.widths_random(n, dim, seed=17 + n + k)
    prob = make(dim, k, widths)
    P = prob.setup_patches(0, tpss.VERTEX_PATCH if kind == "vertex" else tpss.CELL)
    S = oracle_sipg(widths, k)
    A = S.assemble().tocsr()
    patches, sol = oracle_solvers(S, A, kind)
    if kind == "vertex":
        colors = [schwarz.color_multiplicative_vertex(v) for v, _ in patches]
    else:
        colors = [schwarz.color_multiplicative_cell(m) for m, _ in patches]
    N = A.shape[0]
    b = workloads.rhs_uniform(N, seed=3)
    x0 = workloads.rhs_uniform(N, seed=4)
    xg = dev(x0)
    P.smooth_multiplicative(1.0, dev(b), xg, reverse_colors=reverse)
    ref = schwarz.multiplicative_smoother(A, b, x0, sol, colors, 1.0, reverse=reverse)
    assert rel_err(xg, ref) < TOL64
    assert P.info()["ncolors_mult"] == (2 ** (dim + 1) if kind == "vertex" else 2)
    prob.close()


def test_config1_2d_acs_against_per_cell_lu():
    """2D, 8x8 uniform cells, Q_2 (576 DoFs), gamma_e = (k+1)^2 (1/h+ + 1/h-) =
    2(k+1)^2/h, ACS omega = 0.7 applied once to one seeded U[-1,1] vector."""
    from paper_1910_11239_gb300 import tpss
    widths = workloads.widths_uniform(8, 2)
    prob = make(2, 2, widths, penalty="kp1sq")
    P = prob.setup_patches(0, tpss.CELL)
    S = oracle_sipg(widths, 2, penalty="kp1sq")
    A = S.assemble().tocsr()
    _, sol = oracle_solvers(S, A, "cell")
    b = workloads.rhs_uniform(576, seed=1)
    xg = torch.empty(576, dtype=torch.float64, device="cuda")
    P.smooth_additive(0.7, dev(b), xg, x_is_zero=True)
    ref = schwarz.additive_local_sum(b, sol, 0.7)
    assert rel_err(xg, ref) < TOL64
    prob.close()


def test_deterministic_repeat():
    from paper_1910_11239_gb300 import tpss
    widths = workloads.widths_random(6, 3, seed=5)
    prob = make(3, 2, widths)
    P = prob.setup_patches(0, tpss.VERTEX_PATCH)
    N = prob.ndofs(0)
    b = dev(workloads.rhs_uniform(N, seed=6))
    x1 = torch.empty(N, dtype=torch.float64, device="cuda")
    x2 = torch.empty(N, dtype=torch.float64, device="cuda")
    P.smooth_additive(0.7, b, x1, x_is_zero=True)
    P.smooth_additive(0.7, b, x2, x_is_zero=True)
    assert torch.equal(x1, x2)
    prob.close()


def test_single_vertex_patch_is_exact_solve():
    # T_0 = 2^d cells is one vertex patch: AVS with omega = 1 is A^{-1} b (Sec. 2.4)
    from paper_1910_11239_gb300 import tpss
    widths = workloads.widths_uniform(2, 3)
    prob = make(3, 3, widths)
    P = prob.setup_patches(0, tpss.VERTEX_PATCH)
    S = oracle_sipg(widths, 3)
    A = S.assemble().toarray()
    b = workloads.rhs_uniform(A.shape[0], seed=8)
    xg = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
    P.smooth_additive(1.0, dev(b), xg, x_is_zero=True)
    assert rel_err(xg, np.linalg.solve(A, b)) < 1e-11
    prob.close()
