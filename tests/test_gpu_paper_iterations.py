"""Pin the whole solver stack to the paper's iteration counts
(tab:cubecp, 3D, L = 3, additive cell smoother with omega = 0.7 inside CG,
V-cycle(1,1), Gaussian-bell solution, relative residual 1e-8): the paper
prints nu_frac = 17.1 (k = 3) and 21.9 (k = 7).  Our coarse solve is exact
(the paper's is Chebyshev to 1e-8) and nu_frac is residual based, so the pin
allows half an iteration.

The k = 15 columns (tab:cubecp and tab:cubemvpminimal; ACS with CG, MCS and
MVS with GMRES and the non-symmetric V-cycle, omega = 1): 3D on L = 1
(T_0 = 2^3 cells, whose exact coarse solve is one vertex patch's fast
diagonalization) and 2D on L = 6; MCS with left-preconditioned GMRES (pinned
to 0.2), MVS with right preconditioning."""
import pytest
import torch

from gpu_helpers import paper_value
from paper_1910_11239_gb300 import perf, tpss, workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k,L", [(3, 3), (7, 2)])
def test_acs_energy_norm_fractional_iterations(k, L):
    """Sec. 2.4 states that CG is measured by the energy norm of the error.
    The A-norm errors ||x* - x_k||_A (x* by PCG to 1e-14) decrease
    monotonically, as CG guarantees; their nu_frac (17.70 at k = 3) lies
    above the residual-based one (17.13), which is the one that matches the
    printed 17.1 / 21.9 -- so the pins above use the residual reading."""
    prob = tpss.Problem(3, k, workloads.widths_uniform(2, 3), nlevels=L + 1)
    N = prob.ndofs(L)
    b = torch.empty(N, dtype=torch.float64, device="cuda")
    prob.assemble_rhs(L, 1, b)
    prob.mg_setup("ACS", 0.7, tpss.FP64)
    errs = perf.cg_energy_errors(prob, b)
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1))   # CG decreases the A-norm error
    x = torch.empty_like(b)
    res = prob.pcg_solve(b, x, rtol=1e-8, maxit=100, history=True)
    nu_r = perf.fractional_iterations(res["history"], 1e-8)
    nu_e = perf.fractional_iterations(errs, 1e-8)
    assert nu_r - 0.2 < nu_e < nu_r + 2.0, (nu_e, nu_r)
    prob.close()


@pytest.mark.parametrize("k,paper", [(3, paper_value("acs3d_k3_L3")), (7, paper_value("acs3d_k7_L3"))])
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


# MCS with left-preconditioned GMRES (the monitored residual is M(b - A x)):
# that reading reproduces every MCS count the paper prints (k = 3, 7, 15 in
# 2D and 3D) within 0.05, while right preconditioning gives 14.41 against
# 15.7 here; MVS is closer to the printed values with right preconditioning.
K15_CASES = [(3, 1, "ACS", paper_value("acs3d_k15_L1"), False), (3, 1, "MCS", paper_value("mcs3d_k15_L1"), True),
             (3, 1, "MVS", paper_value("mvs3d_k15_L1"), False), (2, 6, "ACS", paper_value("acs2d_k15_L6"), False),
             (2, 6, "MCS", paper_value("mcs2d_k15_L6"), True), (2, 6, "MVS", paper_value("mvs2d_k15_L6"), False)]


@pytest.mark.parametrize("dim,L,smoother,paper,left", K15_CASES)
def test_k15_fractional_iterations_match_paper(dim, L, smoother, paper, left):
    prob = tpss.Problem(dim, 15, workloads.widths_uniform(2, dim), nlevels=L + 1)
    N = prob.ndofs(L)
    b = torch.empty(N, dtype=torch.float64, device="cuda")
    prob.assemble_rhs(L, 1, b)
    x = torch.empty_like(b)
    if smoother == "ACS":
        prob.mg_setup("ACS", 0.7, tpss.FP64)
        res = prob.pcg_solve(b, x, rtol=1e-8, maxit=100, history=True)
    else:
        prob.mg_setup(smoother, 1.0, tpss.FP64, nonsymmetric=1)
        res = prob.gmres_solve(b, x, rtol=1e-8, maxit=100, restart=30, history=True, left=left)
    nu = perf.fractional_iterations(res["history"], 1e-8)
    assert abs(nu - paper) < (0.2 if left else 0.6), nu
    prob.close()


# The 2D columns of tab:cubecp / tab:cubemvpminimal at k = 3 (L = 8) and
# k = 7 (L = 7), 4.2 M DoFs each; 8 colors for MVS in 2D.
TWO_D_CASES = [(3, 8, "ACS", paper_value("acs2d_k3_L8"), False), (7, 7, "ACS", paper_value("acs2d_k7_L7"), False),
               (3, 8, "MCS", paper_value("mcs2d_k3_L8"), True), (7, 7, "MCS", paper_value("mcs2d_k7_L7"), True),
               (3, 8, "MVS", paper_value("mvs2d_k3_L8"), False), (7, 7, "MVS", paper_value("mvs2d_k7_L7"), False)]


@pytest.mark.parametrize("k,L,smoother,paper,left", TWO_D_CASES)
def test_2d_fractional_iterations_match_paper(k, L, smoother, paper, left):
    prob = tpss.Problem(2, k, workloads.widths_uniform(2, 2), nlevels=L + 1)
    N = prob.ndofs(L)
    b = torch.empty(N, dtype=torch.float64, device="cuda")
    prob.assemble_rhs(L, 1, b)
    x = torch.empty_like(b)
    if smoother == "ACS":
        prob.mg_setup("ACS", 0.7, tpss.FP64)
        res = prob.pcg_solve(b, x, rtol=1e-8, maxit=100, history=True)
    else:
        prob.mg_setup(smoother, 1.0, tpss.FP64, nonsymmetric=1)
        res = prob.gmres_solve(b, x, rtol=1e-8, maxit=100, restart=30, history=True, left=left)
    nu = perf.fractional_iterations(res["history"], 1e-8)
    assert abs(nu - paper) < (0.2 if left else 0.6), nu
    prob.close()


@pytest.mark.parametrize("mapped", [False, True])
def test_energy_errors_in_one_run_equal_the_reruns(mapped):
    """tpss_pcg_energy_errors records ||x_k - x*||_A inside one PCG run; PCG from
    x_0 = 0 is deterministic, so the k-th value equals that of a separate run
    stopped after k steps (the way it is computed without the entry point)."""
    if mapped:
        prob = tpss.Problem.mapped(3, workloads.vertices_distorted(4, 3), nlevels=3, gamma_hat=4.0)
        prob.mg_setup("ACS", 0.5, tpss.FP64)
    else:
        prob = tpss.Problem(3, 2, workloads.widths_uniform(2, 3), nlevels=3)
        prob.mg_setup("ACS", 0.7, tpss.FP64)
    L = prob.nlevels - 1
    b = torch.empty(prob.ndofs(L), dtype=torch.float64, device="cuda")
    prob.assemble_rhs(L, 0, b)
    xs, x = torch.empty_like(b), torch.empty_like(b)
    prob.pcg_solve(b, xs, rtol=1e-14, maxit=200)
    errs = prob.pcg_energy_errors(b, xs, x, rtol=1e-8, maxit=200)
    Ae = torch.empty_like(b)
    for k in range(len(errs)):
        if k == 0:
            e = xs.clone()
        else:
            prob.pcg_solve(b, x, rtol=1e-300, maxit=k)
            e = xs - x
        prob.apply_operator(L, e, Ae)
        ref = float(torch.dot(e, Ae).clamp_min(0.0).sqrt())
        assert abs(errs[k] - ref) <= 1e-9 * errs[0], (k, errs[k], ref)
    assert errs[-1] <= 1e-8 * errs[0] < errs[-2]
    prob.close()
