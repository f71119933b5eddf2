"""Failure detection without any GPU fault: errors are data on the host side
(non-finite input, an indefinite discretization, an iteration limit), reported
as status codes."""
import numpy as np
import pytest
import torch

from gpu_helpers import dev, make
from paper_1910_11239_gb300 import tpss, workloads

pytestmark = pytest.mark.gpu


def test_nonfinite_rhs_is_reported_as_breakdown():
    prob = make(3, 2, workloads.widths_uniform(2, 3), nlevels=2)
    prob.mg_setup("AVS", 0.125)
    N = prob.ndofs(1)
    b = np.ones(N)
    b[7] = np.nan
    x = torch.empty(N, dtype=torch.float64, device="cuda")
    with pytest.raises(tpss.TpssError) as e:
        prob.pcg_solve(dev(b), x, rtol=1e-8, maxit=10)
    assert e.value.status == -4  # TPSS_EBREAKDOWN
    prob.close()


def test_indefinite_penalty_is_reported_by_setup():
    # gamma_hat far below the coercivity threshold: the 1D problems are indefinite
    prob = make(3, 3, workloads.widths_uniform(3, 3), gamma_hat=1e-3)
    with pytest.raises(tpss.TpssError) as e:
        prob.setup_patches(0, tpss.VERTEX_PATCH)
    assert e.value.status == -6  # TPSS_ENUMERIC
    prob.close()


def test_iteration_limit_is_a_soft_status():
    prob = make(3, 2, workloads.widths_uniform(2, 3), nlevels=2)
    prob.mg_setup("ACS", 0.7)
    N = prob.ndofs(1)
    x = torch.empty(N, dtype=torch.float64, device="cuda")
    res = prob.pcg_solve(dev(workloads.rhs_uniform(N, 5)), x, rtol=1e-14, maxit=3)
    assert res["converged"] is False and res["iters"] == 3
    prob.close()


def test_context_usable_after_errors():
    prob = make(3, 2, workloads.widths_uniform(2, 3), nlevels=2)
    with pytest.raises(tpss.TpssError):
        prob.apply_operator(5, torch.zeros(1, dtype=torch.float64, device="cuda"),
                            torch.zeros(1, dtype=torch.float64, device="cuda"))
    N = prob.ndofs(1)
    u = dev(workloads.rhs_uniform(N, 1))
    out = torch.empty_like(u)
    prob.apply_operator(1, u, out)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
    prob.close()


def test_tcgen05_wait_expiry_is_reported_and_the_context_recovers():
    # the tcgen05 smoother's bounded MMA wait, made to run out by the test
    # hook (a phase no MMA completes): the call after reports TPSS_ETIMEOUT,
    # the next one runs normally
    from gpu_helpers import rel_err
    from oracle import fastdiag
    widths = workloads.widths_random(4, 3, seed=7)
    prob = make(3, 4, widths)
    P = prob.setup_patches(0, tpss.VERTEX_PATCH, tpss.BF16)
    P.set_additive_schedule(tpss.ADDITIVE_TCGEN05)
    N = prob.ndofs(0)
    b = workloads.rhs_uniform(N, seed=8)
    bd = dev(b, torch.float32)
    x = torch.empty(N, dtype=torch.float32, device="cuda")
    P.test_wait_expiry()
    P.smooth_additive(0.7, bd, x, x_is_zero=True)
    torch.cuda.synchronize()
    with pytest.raises(tpss.TpssError) as e:
        P.smooth_additive(0.7, bd, x, x_is_zero=True)
    assert e.value.status == -5  # TPSS_ETIMEOUT
    P.smooth_additive(0.7, bd, x, x_is_zero=True)
    torch.cuda.synchronize()
    ref = fastdiag.additive_local_sum(widths, 4, True, b.astype(np.float32).astype(np.float64), 0.7)
    assert rel_err(x.double(), ref) < 5e-2
    P.close()
    prob.close()
