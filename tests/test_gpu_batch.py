"""Batched uneven problems (not in the paper): one persistent smoother launch
per level across problems of different degree and size, FP32 V-cycle,
CUDA-graph capture, autotuned work items, FP64 outer PCG per system.
Checked against the per-problem library path and the FP64 oracle."""
import numpy as np
import pytest
import torch

from gpu_helpers import dev, make, rel_err
from oracle.multigrid import Hierarchy
from paper_1910_11239_gb300 import tpss, workloads

pytestmark = pytest.mark.gpu

OMEGA = 0.125
# (degree, coarse cells per direction, nlevels, seed): uneven sizes, degrees and depths
SPECS = [(2, 2, 2, 11), (3, 3, 2, 12), (1, 2, 3, 13), (4, 2, 2, 14)]


def problems():
    return [(k, workloads.widths_random(c, 3, seed), nl) for k, c, nl, seed in SPECS]


def rhs_for(batch, seed):
    b = np.zeros(batch.total)
    rng = np.random.default_rng(seed)
    b[:] = rng.uniform(-1, 1, batch.total)
    return b


@pytest.fixture(scope="module")
def stream():
    return torch.cuda.Stream()


@pytest.mark.parametrize("use_graph,prec", [(True, "fp32"), (False, "fp32"), (True, "bf16")])
def test_batch_smoother_matches_per_problem(use_graph, prec, stream):
    tol = 1e-5 if prec == "fp32" else 2e-2
    with torch.cuda.stream(stream):
        B = tpss.Batch(problems(), nrhs=2, omega=OMEGA, use_graph=use_graph, stream=stream,
                       precision=tpss.PRECISIONS[prec])
        assert B.uses_graph == use_graph
        b = rhs_for(B, 1)
        x = torch.empty(B.total, dtype=torch.float32, device="cuda")
        B.smooth_additive(dev(b, torch.float32), x)
        torch.cuda.synchronize()
        for p, (k, widths, nl) in enumerate(problems()):
            info = B.info(p)
            prob = make(3, k, widths, nlevels=nl)
            P = prob.setup_patches(nl - 1, tpss.VERTEX_PATCH, tpss.PRECISIONS[prec])
            n = info["ndofs"]
            seg = slice(info["offset"], info["offset"] + 2 * n)
            xr = torch.empty(2 * n, dtype=torch.float32, device="cuda")
            P.smooth_additive(OMEGA, dev(b[seg], torch.float32), xr, x_is_zero=True, nrhs=2)
            torch.cuda.synchronize()
            assert rel_err(x[seg].double(), xr.double().cpu().numpy()) < tol
            assert info["ppb"] >= 1
            prob.close()
        B.close()


def test_batch_vcycle_matches_per_problem_and_oracle(stream):
    with torch.cuda.stream(stream):
        B = tpss.Batch(problems(), nrhs=2, omega=OMEGA, stream=stream)
        b = rhs_for(B, 2)
        x = torch.empty(B.total, dtype=torch.float64, device="cuda")
        B.vcycle(dev(b), x)
        x2 = torch.empty_like(x)
        B.vcycle(dev(b), x2)   # replay
        torch.cuda.synchronize()
        assert rel_err(x2, x.cpu().numpy()) < 1e-5
        for p, (k, widths, nl) in enumerate(problems()):
            info = B.info(p)
            n = info["ndofs"]
            prob = make(3, k, widths, nlevels=nl)
            prob.mg_setup("AVS", OMEGA, tpss.FP32)
            for r in range(2):
                seg = slice(info["offset"] + r * n, info["offset"] + (r + 1) * n)
                xr = torch.empty(n, dtype=torch.float64, device="cuda")
                prob.vcycle(dev(b[seg]), xr)
                torch.cuda.synchronize()
                assert rel_err(x[seg], xr.cpu().numpy()) < 1e-4
            if p == 0:
                H = Hierarchy(widths, k, nl, smoother="AVS", omega=OMEGA)
                seg = slice(info["offset"], info["offset"] + n)
                assert rel_err(x[seg], H.precondition(b[seg])) < 1e-4
            prob.close()
        B.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_batch_pcg_converges_every_system(prec, stream):
    with torch.cuda.stream(stream):
        B = tpss.Batch(problems(), nrhs=2, omega=OMEGA, stream=stream, precision=tpss.PRECISIONS[prec])
        b = rhs_for(B, 3)
        x = torch.empty(B.total, dtype=torch.float64, device="cuda")
        res = B.pcg_solve(dev(b), x, rtol=1e-8, maxit=80)
        torch.cuda.synchronize()
        assert res["converged"] and (res["rel_res"] <= 1e-8).all()
        for p, (k, widths, nl) in enumerate(problems()):
            info = B.info(p)
            n = info["ndofs"]
            prob = make(3, k, widths, nlevels=nl)
            prob.mg_setup("AVS", OMEGA, tpss.FP64)
            for r in range(2):
                seg = slice(info["offset"] + r * n, info["offset"] + (r + 1) * n)
                bs = dev(b[seg])
                rr = torch.empty_like(bs)
                prob.residual(nl - 1, bs, x[seg].contiguous(), rr)
                assert (rr.norm() / bs.norm()).item() < 2e-8
                x64 = torch.empty_like(bs)
                prob.pcg_solve(bs, x64, rtol=1e-10, maxit=200)
                assert ((x[seg] - x64).norm() / x64.norm()).item() < 1e-6
            prob.close()
        B.close()


# The batched workload's large patch sizes: k = 5 (n = 12) and k = 7 (n = 16),
# beside a k = 2 problem, each on a 2^3 coarse mesh refined once (4^3 cells).
SPECS_LARGE = [(5, 2, 2, 21), (7, 2, 2, 22), (2, 2, 2, 23)]


def large_problems():
    return [(k, workloads.widths_random(c, 3, seed), nl) for k, c, nl, seed in SPECS_LARGE]


def fine_widths(widths, nlevels):
    """Per-direction widths after nlevels - 1 bisections."""
    out = []
    for w in widths:
        for _ in range(nlevels - 1):
            w = np.repeat(np.asarray(w) / 2.0, 2)
        out.append(np.asarray(w))
    return out


# error bars against the FP64 oracle (as for the single-problem mixed smoothers)
BATCH_TOL = {"fp32": 1e-4, "bf16": 5e-2}


# (precision, columns): FP32 -> batch_group<n>; BF16 without columns ->
# batch_group_bf16<n>; BF16 with columns -> per-problem passes on the side
# streams on every level (tcgen05 columns for n = 12, 16, i.e. k = 5, 7; the
# colored BF16 launches for k = 2)
ROUTES = [("fp32", True), ("bf16", False), ("bf16", True)]


@pytest.mark.parametrize("prec,columns", ROUTES)
def test_batch_smoother_large_patches_match_oracle(prec, columns, stream):
    # each routine is forced by the batch precision and the columns flag
    from oracle import fastdiag
    with torch.cuda.stream(stream):
        B = tpss.Batch(large_problems(), nrhs=2, omega=OMEGA, stream=stream, precision=tpss.PRECISIONS[prec],
                       columns=columns)
        b = rhs_for(B, 4)
        x = torch.full((B.total,), float("nan"), dtype=torch.float32, device="cuda")
        B.smooth_additive(dev(b, torch.float32), x)
        torch.cuda.synchronize()
        xs = x.double().cpu().numpy()
        for p, (k, widths, nl) in enumerate(large_problems()):
            info = B.info(p)
            n = info["ndofs"]
            fw = fine_widths(widths, nl)
            for r in range(2):
                seg = slice(info["offset"] + r * n, info["offset"] + (r + 1) * n)
                ref = fastdiag.additive_local_sum(fw, k, True, b[seg], OMEGA)
                assert rel_err(xs[seg], ref) < BATCH_TOL[prec], (p, k, r)
        B.close()


_LARGE_HIERARCHIES = {}


def _large_hierarchy(p):
    # the oracle hierarchy (dense-LU local solvers, up to 4096 x 4096 at k = 7)
    # is built once per problem and shared by both precisions
    if p not in _LARGE_HIERARCHIES:
        k, widths, nl = large_problems()[p]
        _LARGE_HIERARCHIES[p] = Hierarchy(widths, k, nl, smoother="AVS", omega=OMEGA)
    return _LARGE_HIERARCHIES[p]


@pytest.mark.parametrize("prec,columns", ROUTES)
def test_batch_vcycle_large_patches_match_oracle(prec, columns, stream):
    with torch.cuda.stream(stream):
        B = tpss.Batch(large_problems(), nrhs=2, omega=OMEGA, stream=stream, precision=tpss.PRECISIONS[prec],
                       columns=columns)
        b = rhs_for(B, 5)
        x = torch.empty(B.total, dtype=torch.float64, device="cuda")
        B.vcycle(dev(b), x)
        torch.cuda.synchronize()
        xs = x.cpu().numpy()
        for p, (k, widths, nl) in enumerate(large_problems()):
            info = B.info(p)
            n = info["ndofs"]
            H = _large_hierarchy(p)
            for r in range(2):
                seg = slice(info["offset"] + r * n, info["offset"] + (r + 1) * n)
                assert rel_err(xs[seg], H.precondition(b[seg])) < BATCH_TOL[prec], (p, k, r)
        B.close()


def test_batch_vcycle_every_problem_matches_oracle(stream):
    # the small uneven batch: every problem and right-hand side, not only the first
    with torch.cuda.stream(stream):
        B = tpss.Batch(problems(), nrhs=2, omega=OMEGA, stream=stream)
        b = rhs_for(B, 6)
        x = torch.empty(B.total, dtype=torch.float64, device="cuda")
        B.vcycle(dev(b), x)
        torch.cuda.synchronize()
        xs = x.cpu().numpy()
        for p, (k, widths, nl) in enumerate(problems()):
            info = B.info(p)
            n = info["ndofs"]
            H = Hierarchy(widths, k, nl, smoother="AVS", omega=OMEGA)
            for r in range(2):
                seg = slice(info["offset"] + r * n, info["offset"] + (r + 1) * n)
                assert rel_err(xs[seg], H.precondition(b[seg])) < 1e-4, (p, r)
        B.close()


def test_batch_bf16_columns_deterministic_and_match_single_problem(stream):
    # with the column route, the finest level of every problem of a BF16
    # batch is smoothed by the same deterministic kernels as the problem alone
    # (tcgen05 columns for k >= 4, colored launches below): repeated calls
    # agree bit for bit, and so do the batch and the problem alone
    with torch.cuda.stream(stream):
        B = tpss.Batch(large_problems(), nrhs=2, omega=OMEGA, stream=stream, precision=tpss.BF16)
        b = rhs_for(B, 7)
        x1 = torch.empty(B.total, dtype=torch.float32, device="cuda")
        x2 = torch.empty_like(x1)
        B.smooth_additive(dev(b, torch.float32), x1)
        B.smooth_additive(dev(b, torch.float32), x2)
        torch.cuda.synchronize()
        for p, (k, widths, nl) in enumerate(large_problems()):
            info = B.info(p)
            n = info["ndofs"]
            seg = slice(info["offset"], info["offset"] + 2 * n)
            assert torch.equal(x1[seg], x2[seg])
            prob = make(3, k, widths, nlevels=nl)
            P = prob.setup_patches(nl - 1, tpss.VERTEX_PATCH, tpss.BF16)
            xr = torch.empty(2 * n, dtype=torch.float32, device="cuda")
            P.smooth_additive(OMEGA, dev(b[seg], torch.float32), xr, x_is_zero=True, nrhs=2)
            torch.cuda.synchronize()
            assert torch.equal(x1[seg], xr)
            prob.close()
        B.close()
