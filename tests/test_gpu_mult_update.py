"""The multiplicative sweep with per-color residual updates (one residual
per sweep, then r <- (1 - omega) r on the color's cells and the face
couplings of the update next to them) against the oracle's sweep, which
recomputes r = b - A x before every color as Alg. 3 prints it.  The two are
equal in exact arithmetic; the bar is the FP64 parity bar."""
import numpy as np
import pytest
import torch

from gpu_helpers import TOL64, dev, make, oracle_sipg, oracle_solvers, rel_err
from oracle import schwarz
from paper_1910_11239_gb300 import workloads

pytestmark = pytest.mark.gpu

CASES = [(2, 2, (6, 5), "vertex"), (2, 3, (5, 4), "cell"), (3, 1, (5, 4, 4), "vertex"), (3, 2, (4, 4, 3), "vertex"),
         (3, 3, (3, 3, 4), "cell"), (3, 8, (3, 2, 2), "vertex"), (3, 9, (2, 1, 2), "cell")]


@pytest.mark.parametrize("dim,k,counts,kind", CASES)
@pytest.mark.parametrize("omega,reverse", [(1.0, False), (0.8, True)])
def test_update_sweep_matches_oracle(dim, k, counts, kind, omega, reverse):
    from paper_1910_11239_gb300 import tpss
    widths = [workloads.widths_random(c, 1, seed=300 + k + 7 * t)[0] for t, c in enumerate(counts[:dim])]
    prob = make(dim, k, widths)
    P = prob.setup_patches(0, tpss.VERTEX_PATCH if kind == "vertex" else tpss.CELL)
    P.set_mult_residual(tpss.MULT_RESIDUAL_UPDATE)
    S = oracle_sipg(widths, k)
    A = S.assemble().tocsr()
    patches, sol = oracle_solvers(S, A, kind)
    if kind == "vertex":
        colors = [schwarz.color_multiplicative_vertex(v) for v, _ in patches]
    else:
        colors = [schwarz.color_multiplicative_cell(m) for m, _ in patches]
    N = A.shape[0]
    nrhs = 2
    b = workloads.rhs_uniform(N, seed=21, nrhs=nrhs)
    x0 = workloads.rhs_uniform(N, seed=22, nrhs=nrhs)
    xg = dev(x0)
    P.smooth_multiplicative(omega, dev(b), xg, reverse_colors=reverse, nrhs=nrhs)
    for r in range(nrhs):
        sl = slice(r * N, (r + 1) * N)
        ref = schwarz.multiplicative_smoother(A, b[sl], x0[sl], sol, colors, omega, reverse=reverse)
        assert rel_err(xg[sl], ref) < TOL64
    prob.close()


@pytest.mark.parametrize("dim,k,n,kind", [(3, 4, 9, "vertex"), (3, 7, 6, "cell"), (2, 6, 17, "vertex"),
                                          (3, 15, 3, "vertex")])
def test_update_equals_full_residual_on_gpu(dim, k, n, kind):
    """Larger meshes than the oracle handles: the two GPU modes agree."""
    from paper_1910_11239_gb300 import tpss
    widths = workloads.widths_random(n, dim, seed=40 + k)
    prob = make(dim, k, widths)
    P = prob.setup_patches(0, tpss.VERTEX_PATCH if kind == "vertex" else tpss.CELL)
    N = prob.ndofs(0)
    b = dev(workloads.rhs_uniform(N, seed=5))
    x0 = workloads.rhs_uniform(N, seed=6)
    xs = {}
    for mode in (tpss.MULT_RESIDUAL_FULL, tpss.MULT_RESIDUAL_UPDATE):
        P.set_mult_residual(mode)
        x = dev(x0)
        P.smooth_multiplicative(1.0, b, x)
        P.smooth_multiplicative(1.0, b, x, reverse_colors=True)
        xs[mode] = x.cpu().numpy()
    assert rel_err(xs[tpss.MULT_RESIDUAL_UPDATE], xs[tpss.MULT_RESIDUAL_FULL]) < TOL64
    prob.close()


def test_face_conflicting_coloring_keeps_full_residual():
    """With the 2^d-color vertex coloring same-color patches share faces, so
    the update would be wrong; the sweep recomputes the residual there."""
    from paper_1910_11239_gb300 import tpss
    widths = workloads.widths_random(5, 3, seed=9)
    prob = make(3, 2, widths)
    P = prob.setup_patches(0, tpss.VERTEX_PATCH)
    P.set_mult_colors(8)
    N = prob.ndofs(0)
    b = dev(workloads.rhs_uniform(N, seed=1))
    xs = []
    for mode in (tpss.MULT_RESIDUAL_FULL, tpss.MULT_RESIDUAL_UPDATE):
        P.set_mult_residual(mode)
        x = torch.zeros(N, dtype=torch.float64, device="cuda")
        P.smooth_multiplicative(1.0, b, x)
        xs.append(x)
    assert torch.equal(xs[0], xs[1])
    prob.close()


@pytest.mark.parametrize("smoother,precision,tol", [("MVS", "fp64", 1e-11), ("MCS", "fp64", 1e-11),
                                                    ("MVS", "fp32", 1e-4), ("MVS", "tf32", 2e-2),
                                                    ("MVS", "bf16", 2e-1)])
def test_vcycle_and_pcg_with_updates(smoother, precision, tol):
    """FP64: the V-cycle and the PCG iterates agree with the full-residual
    sweep.  Mixed precisions: the carried residual omits the local solves'
    rounding, so the V-cycles differ at that level (FP32 ~1e-6, TF32 ~1e-3,
    BF16 ~1e-2 relative local errors) and the iteration counts may differ by
    one."""
    from paper_1910_11239_gb300 import tpss
    prob = tpss.Problem(3, 3, workloads.widths_uniform(2, 3), nlevels=4)
    N = prob.ndofs(3)
    b = torch.empty(N, dtype=torch.float64, device="cuda")
    prob.assemble_rhs(3, 1, b)
    out = {}
    for mode in (tpss.MULT_RESIDUAL_FULL, tpss.MULT_RESIDUAL_UPDATE):
        prob.mg_setup(smoother, 1.0, tpss.PRECISIONS[precision], flexible_cg=int(precision != "fp64"),
                      mult_residual=mode)
        z = torch.empty_like(b)
        prob.vcycle(b, z)
        x = torch.empty_like(b)
        res = prob.pcg_solve(b, x, rtol=1e-8, maxit=50)
        out[mode] = (z.cpu().numpy(), res["iters"], res["converged"])
    zf, itf, okf = out[tpss.MULT_RESIDUAL_FULL]
    zu, itu, oku = out[tpss.MULT_RESIDUAL_UPDATE]
    assert okf and oku and abs(itf - itu) <= (0 if precision == "fp64" else 1)
    assert rel_err(zu, zf) < tol
    prob.close()
