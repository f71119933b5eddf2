"""Pin the whole solver stack to the paper's iteration counts
(tab:cubecp, 3D, L = 3, additive cell smoother with omega = 0.7 inside CG,
V-cycle(1,1), Gaussian-bell solution, relative residual 1e-8): the paper
prints nu_frac = 17.1 (k = 3) and 21.9 (k = 7).  Our coarse solve is exact
(the paper's is Chebyshev to 1e-8) and nu_frac is residual based, so the pin
allows half an iteration."""
import pytest
import torch

from paper_1910_11239_gb300 import perf, tpss, workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k,paper", [(3, 17.1), (7, 21.9)])
def test_acs_fractional_iterations_match_tab_cubecp(k, paper):
    prob = tpss.Problem(3, k, workloads.widths_uniform(2, 3), nlevels=4)
    N = prob.ndofs(3)
    b = torch.empty(N, dtype=torch.float64, device="cuda")
    prob.assemble_rhs(3, 1, b)
    prob.mg_setup("ACS", 0.7, tpss.FP64)
    x = torch.empty_like(b)
    res = prob.pcg_solve(b, x, rtol=1e-8, maxit=100, history=True)
    nu = perf.fractional_iterations(res["history"], 1e-8)
    assert abs(nu - paper) < 0.5, nu
    prob.close()
