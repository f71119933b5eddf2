"""GPU parity of the matrix-free SIPG operator, residual, transfers and
right-hand side against the oracle's assembled matrices, FP64 relative 1e-12."""
import numpy as np
import pytest
import torch

from gpu_helpers import TOL64, dev, make, oracle_sipg, rel_err
from oracle.mesh import TensorMesh
from oracle.transfer import prolongation_matrix
from paper_1910_11239_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,k,n", [(2, 1, 9), (2, 3, 5), (2, 7, 3), (3, 1, 6), (3, 2, 5), (3, 4, 3), (3, 7, 2)])
@pytest.mark.parametrize("penalty", ["paper", "kp1sq"])
def test_operator_matches_assembled_matrix(dim, k, n, penalty):
    widths = workloads.widths_random(n, dim, seed=n * 10 + k)
    if dim == 3:
        widths[1] = workloads.widths_random(n + 1, 1, seed=77)[0]
    prob = make(dim, k, widths, penalty=penalty)
    A = oracle_sipg(widths, k, penalty=penalty).assemble().tocsr()
    N = A.shape[0]
    nrhs = 3
    u = workloads.rhs_uniform(N, seed=5, nrhs=nrhs)
    out = torch.empty(N * nrhs, dtype=torch.float64, device="cuda")
    prob.apply_operator(0, dev(u), out, nrhs=nrhs)
    for r in range(nrhs):
        assert rel_err(out[r * N:(r + 1) * N], A @ u[r * N:(r + 1) * N]) < TOL64
    b = workloads.rhs_uniform(N, seed=6, nrhs=nrhs)
    rr = torch.empty_like(out)
    prob.residual(0, dev(b), dev(u), rr, nrhs=nrhs)
    for r in range(nrhs):
        ref = b[r * N:(r + 1) * N] - A @ u[r * N:(r + 1) * N]
        assert rel_err(rr[r * N:(r + 1) * N], ref) < TOL64
    # operator in FP32 (mixed-precision V-cycle): FP32 rounding bound
    out32 = torch.empty(N, dtype=torch.float32, device="cuda")
    prob.apply_operator(0, dev(u[:N], torch.float32), out32)
    assert rel_err(out32.double(), A @ u[:N].astype(np.float32).astype(np.float64)) < 1e-4
    prob.close()


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 4), (3, 2), (3, 5)])
def test_transfers_match_embedding(dim, k):
    coarse_w = workloads.widths_random(3, dim, seed=21 + k)
    prob = make(dim, k, coarse_w, nlevels=2)
    cm = TensorMesh(coarse_w)
    P = prolongation_matrix(cm, cm.refine(), k)
    nc, nf = P.shape[1], P.shape[0]
    assert prob.ndofs(0) == nc and prob.ndofs(1) == nf
    uc = workloads.rhs_uniform(nc, seed=1, nrhs=2)
    uf0 = workloads.rhs_uniform(nf, seed=2, nrhs=2)
    fg = dev(uf0)
    prob.prolongate_add(1, dev(uc), fg, nrhs=2)
    for r in range(2):
        assert rel_err(fg[r * nf:(r + 1) * nf], uf0[r * nf:(r + 1) * nf] + P @ uc[r * nc:(r + 1) * nc]) < TOL64
    cg = torch.empty(2 * nc, dtype=torch.float64, device="cuda")
    prob.restrict(1, dev(uf0), cg, nrhs=2)
    for r in range(2):
        assert rel_err(cg[r * nc:(r + 1) * nc], P.T @ uf0[r * nf:(r + 1) * nf]) < TOL64
    prob.close()


@pytest.mark.parametrize("dim,k,n", [(2, 2, 4), (3, 1, 3), (3, 3, 2)])
def test_rhs_matches_oracle(dim, k, n):
    widths = workloads.widths_uniform(n, dim)
    prob = make(dim, k, widths)
    S = oracle_sipg(widths, k)
    N = prob.ndofs(0)
    b = torch.empty(N, dtype=torch.float64, device="cuda")
    prob.assemble_rhs(0, 0, b)
    f = lambda p: dim * np.pi ** 2 * np.prod(np.sin(np.pi * p), axis=1)
    assert rel_err(b, S.rhs(f, None)) < TOL64
    # Gaussian bells with boundary data
    sig = 1.0 / 3.0
    src = np.array([[0.0, 0.0, 0.0], [0.25, 0.85, 0.85], [0.6, 0.4, 0.4]])[:, :dim]
    c = 1.0 / (np.sqrt(2 * np.pi) * sig)

    def u(p):
        return c * sum(np.exp(-np.sum((p - s) ** 2, axis=1) / sig ** 2) for s in src)

    def mlap(p):
        out = 0.0
        for s in src:
            r2 = np.sum((p - s) ** 2, axis=1)
            out = out + np.exp(-r2 / sig ** 2) * (2 * dim / sig ** 2 - 4 * r2 / sig ** 4)
        return c * out

    prob.assemble_rhs(0, 1, b)
    assert rel_err(b, S.rhs(mlap, u)) < TOL64
    prob.close()
