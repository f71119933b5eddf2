"""GPU parity of the coarse solve, the V-cycle (Alg. 1) and PCG against the
oracle hierarchy (exact coarse solve, LU local solvers)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

from gpu_helpers import dev, make, rel_err
from oracle.multigrid import Hierarchy, pcg
from paper_1910_11239_gb300 import workloads

pytestmark = pytest.mark.gpu

SMOOTHERS = {"ACS": 0.7, "AVS": 0.125, "MCS": 1.0, "MVS": 1.0}


@pytest.mark.parametrize("dim,k,nlevels", [(2, 2, 3), (2, 4, 2), (3, 1, 2), (3, 2, 2)])
@pytest.mark.parametrize("smoother", ["ACS", "AVS", "MCS", "MVS"])
def test_vcycle_matches_oracle(dim, k, nlevels, smoother):
    omega = SMOOTHERS[smoother] if dim == 3 else {"AVS": 0.25}.get(smoother, SMOOTHERS[smoother])
    coarse = workloads.widths_random(2, dim, seed=3)
    H = Hierarchy(coarse, k, nlevels, smoother=smoother, omega=omega)
    prob = make(dim, k, coarse, nlevels=nlevels)
    prob.mg_setup(smoother, omega)
    N = H.A[-1].shape[0]
    assert prob.ndofs(nlevels - 1) == N
    b = workloads.rhs_uniform(N, seed=11)
    x = torch.empty(N, dtype=torch.float64, device="cuda")
    prob.vcycle(dev(b), x)
    assert rel_err(x, H.precondition(b)) < 1e-11
    # coarse solve
    n0 = H.A[0].shape[0]
    b0 = workloads.rhs_uniform(n0, seed=12)
    x0 = torch.empty(n0, dtype=torch.float64, device="cuda")
    prob.coarse_solve(dev(b0), x0)
    assert rel_err(x0, np.linalg.solve(H.A[0].toarray(), b0)) < 1e-11
    prob.close()


@pytest.mark.parametrize("smoother", ["ACS", "AVS", "MVS"])
def test_pcg_matches_oracle_and_direct_solve(smoother):
    dim, k, nlevels = 3, 2, 2
    omega = SMOOTHERS[smoother]
    coarse = workloads.widths_uniform(2, dim)
    H = Hierarchy(coarse, k, nlevels, smoother=smoother, omega=omega)
    prob = make(dim, k, coarse, nlevels=nlevels)
    prob.mg_setup(smoother, omega)
    A = H.A[-1]
    N = A.shape[0]
    b = torch.empty(N, dtype=torch.float64, device="cuda")
    prob.assemble_rhs(nlevels - 1, 0, b)
    bh = b.cpu().numpy()
    x = torch.empty_like(b)
    res = prob.pcg_solve(b, x, rtol=1e-10, maxit=100, history=True)
    assert res["converged"]
    xo, it, hist, ok = pcg(A, bh, H.precondition, rtol=1e-10, maxit=100)
    assert ok and abs(res["iters"] - it) <= 1
    xd = spla.spsolve(A.tocsc(), bh)
    assert np.linalg.norm(x.cpu().numpy() - xd) <= 1e-8 * np.linalg.norm(xd)
    # residual histories agree while well above rounding
    m = min(len(hist), len(res["history"])) - 2
    assert np.allclose(res["history"][:m], hist[:m], rtol=1e-6)
    prob.close()


def test_pcg_reports_not_converged():
    prob = make(2, 1, workloads.widths_uniform(2, 2), nlevels=2)
    prob.mg_setup("ACS", 0.7)
    N = prob.ndofs(1)
    b = dev(workloads.rhs_uniform(N, seed=1))
    x = torch.empty_like(b)
    res = prob.pcg_solve(b, x, rtol=1e-30, maxit=2)
    assert not res["converged"] and res["iters"] == 2
    prob.close()


def test_invalid_arguments_are_rejected_on_host():
    from paper_1910_11239_gb300 import tpss
    with pytest.raises(tpss.TpssError):
        tpss.Problem(3, 16, workloads.widths_uniform(2, 3))      # degree out of range (1..15)
    prob = make(3, 2, workloads.widths_uniform(2, 3))
    with pytest.raises(tpss.TpssError):
        prob.setup_patches(0, 5)                                 # unknown kind
    with pytest.raises(tpss.TpssError):
        prob.vcycle(torch.zeros(prob.ndofs(0), dtype=torch.float64, device="cuda"),
                    torch.zeros(prob.ndofs(0), dtype=torch.float64, device="cuda"))  # no mg_setup
    prob.close()
