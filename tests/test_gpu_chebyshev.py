"""The paper's coarse solver (Sec. 2.4): Chebyshev iteration preconditioned by
the additive cell smoother, to a relative accuracy of 1e-8, against the
oracle (oracle/chebyshev.py): the spectral interval and step count the GPU
derives, the coarse solve itself, and the multigrid iteration counts with it
(which stay at the exact-coarse-solve values)."""
import numpy as np
import pytest
import torch

from gpu_helpers import dev, make, oracle_sipg, paper_value, rel_err
from oracle import schwarz
from oracle.chebyshev import chebyshev, iteration_count, spectral_bounds
from paper_1910_11239_gb300 import perf, tpss, workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,k", [(2, 3), (3, 2), (3, 4)])
def test_chebyshev_coarse_solve_matches_oracle(dim, k):
    widths = [workloads.widths_random(2, 1, seed=500 + k + t)[0] for t in range(dim)]
    prob = make(dim, k, widths, nlevels=2)
    prob.mg_setup("ACS", 0.7, tpss.FP64, coarse_solver=tpss.COARSE_CHEBYSHEV)
    info = prob.coarse_chebyshev_info()
    S = oracle_sipg(widths, k)
    A = S.assemble().tocsr()
    patches = schwarz.cell_patches(S.mesh)
    sol = schwarz.LocalSolvers(patches, S.nloc, lambda cells: S.assemble(cells))
    prec = lambda r: schwarz.additive_local_sum(r, sol, 1.0)
    n = A.shape[0]
    a, b = spectral_bounds(A, prec, n)
    assert abs(info["a"] - a) <= 1e-7 * a and abs(info["b"] - b) <= 1e-7 * b, (info, a, b)
    assert info["steps"] == iteration_count(info["a"], info["b"], 1e-8)
    f = workloads.rhs_uniform(n, seed=7)
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    prob.coarse_solve(dev(f), x)
    ref = chebyshev(A, f, prec, info["a"], info["b"], info["steps"])
    assert rel_err(x, ref) < 1e-10
    xs = np.linalg.solve(A.toarray(), f)
    e = x.cpu().numpy() - xs
    assert np.sqrt(e @ (A @ e)) <= 1e-8 * np.sqrt(xs @ (A @ xs))
    prob.close()


@pytest.mark.parametrize("smoother,k,paper,left", [("ACS", 3, paper_value("acs3d_k3_L3"), False),
                                                   ("MCS", 3, paper_value("mcs3d_k3_L3"), True)])
def test_paper_counts_with_chebyshev_coarse_solver(smoother, k, paper, left):
    """tab:cubecp, 3D, L = 3 with the paper's coarse solver: the fractional
    counts equal those with the exact coarse solve (a 1e-8 coarse accuracy is
    below what a 1e-8 outer tolerance resolves) and the paper's."""
    nus = []
    for coarse in (tpss.COARSE_DENSE, tpss.COARSE_CHEBYSHEV):
        prob = tpss.Problem(3, k, workloads.widths_uniform(2, 3), nlevels=4)
        N = prob.ndofs(3)
        b = torch.empty(N, dtype=torch.float64, device="cuda")
        prob.assemble_rhs(3, 1, b)
        x = torch.empty_like(b)
        if smoother == "ACS":
            prob.mg_setup("ACS", 0.7, tpss.FP64, coarse_solver=coarse)
            res = prob.pcg_solve(b, x, rtol=1e-8, maxit=100, history=True)
        else:
            prob.mg_setup(smoother, 1.0, tpss.FP64, nonsymmetric=1, coarse_solver=coarse)
            res = prob.gmres_solve(b, x, rtol=1e-8, maxit=100, restart=30, history=True, left=left)
        nus.append(perf.fractional_iterations(res["history"], 1e-8))
        prob.close()
    assert abs(nus[1] - nus[0]) < 0.05, nus
    assert abs(nus[1] - paper) < (0.2 if left else 0.5), nus


def test_chebyshev_coarse_rejected_for_mixed_precision():
    prob = make(3, 2, workloads.widths_uniform(2, 3), nlevels=2)
    with pytest.raises(tpss.TpssError, match="Chebyshev"):
        prob.mg_setup("ACS", 0.7, tpss.FP32, coarse_solver=tpss.COARSE_CHEBYSHEV)
    with pytest.raises(tpss.TpssError):
        prob.coarse_chebyshev_info()
    prob.close()
