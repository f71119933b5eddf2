"""Degrees k = 8..15 (subdomains of up to n = 32 points per direction, the
k = 15 columns of the paper's tables): GPU parity against the oracle, FP64.

* operator and residual against the oracle's literal SIPG assembly (eq. bfsipg);
* prolongation by polynomial exactness (Sec. 2.2: the embedding reproduces
  every coarse Q_k function on the fine mesh), restriction by adjointness,
  and both against the oracle's transfer matrix in 2D;
* cell and vertex-patch smoothers (Alg. 2, Alg. 3) against the oracle's
  dense-LU local solvers, including the 3D vertex patches with n = 18 that
  take the plane-by-plane kernel;
* a single vertex patch covering a 2 x 2 x 2 mesh is A^{-1} (Sec. 3.2: the
  fast-diagonalization inverse is exact on Cartesian meshes), up to n = 32;
* the exact coarse solve by fast diagonalization against the dense inverse.
"""
import numpy as np
import pytest
import torch

from gpu_helpers import TOL64, dev, make, oracle_sipg, oracle_solvers, rel_err
from oracle import schwarz
from oracle.mesh import TensorMesh
from oracle.sipg import SIPG
from oracle.transfer import prolongation_matrix
from paper_1910_11239_gb300 import workloads

pytestmark = pytest.mark.gpu

_ASSEMBLED = {}


def assembled(mesh_key, widths, k):
    """Oracle matrix, cached per module (the k = 15 3D assembly takes ~20 s)."""
    key = (mesh_key, k)
    if key not in _ASSEMBLED:
        _ASSEMBLED[key] = oracle_sipg(widths, k).assemble().tocsr()
    return _ASSEMBLED[key]


def widths_case(dim, counts, seed):
    return [workloads.widths_random(c, 1, seed=seed + 13 * t)[0] for t, c in enumerate(counts[:dim])]


OP_CASES = [(3, 9, (2, 1, 2)), (3, 12, (1, 2, 1)), (3, 15, (1, 1, 2)), (2, 10, (3, 2)), (2, 15, (3, 3))]


@pytest.mark.parametrize("dim,k,counts", OP_CASES)
def test_operator_high_degree(dim, k, counts):
    widths = widths_case(dim, counts, seed=40 + k)
    A = assembled((dim, counts), widths, k)
    prob = make(dim, k, widths)
    N = A.shape[0]
    assert prob.ndofs(0) == N
    u = workloads.rhs_uniform(N, seed=3, nrhs=2)
    out = torch.empty(2 * N, dtype=torch.float64, device="cuda")
    prob.apply_operator(0, dev(u), out, nrhs=2)
    for r in range(2):
        assert rel_err(out[r * N:(r + 1) * N], A @ u[r * N:(r + 1) * N]) < TOL64
    b = workloads.rhs_uniform(N, seed=4)
    rr = torch.empty(N, dtype=torch.float64, device="cuda")
    prob.residual(0, dev(b), dev(u[:N]), rr)
    assert rel_err(rr, b - A @ u[:N]) < TOL64
    prob.close()


def random_qk(dim, k, seed):
    """u(x) = prod_t p_t(x_t), p_t a random polynomial of degree k (Legendre
    series on [0, 1]), so u is in Q_k on every cell."""
    rng = np.random.default_rng(seed)
    coefs = [rng.uniform(-1, 1, k + 1) for _ in range(dim)]

    def u(pts):
        v = np.ones(pts.shape[0])
        for t in range(dim):
            v *= np.polynomial.legendre.legval(2 * pts[:, t] - 1, coefs[t])
        return v
    return u


@pytest.mark.parametrize("dim,k,counts", [(3, 9, (1, 2, 1)), (3, 12, (2, 1, 1)), (3, 15, (1, 1, 2)), (2, 15, (2, 3))])
def test_transfers_high_degree(dim, k, counts):
    cw = widths_case(dim, counts, seed=70 + k)
    prob = make(dim, k, cw, nlevels=2)
    cmesh = TensorMesh(cw)
    Sc, Sf = SIPG(cmesh, k), SIPG(cmesh.refine(), k)
    nc, nf = prob.ndofs(0), prob.ndofs(1)
    # prolongation reproduces coarse Q_k functions exactly
    u = random_qk(dim, k, seed=k)
    uc, uf = Sc.interpolate(u), Sf.interpolate(u)
    fg = torch.zeros(nf, dtype=torch.float64, device="cuda")
    prob.prolongate_add(1, dev(uc), fg)
    assert rel_err(fg, uf) < TOL64
    # restriction is the adjoint: <R f, c> = <f, P c> for random f, c
    f = workloads.rhs_uniform(nf, seed=5, nrhs=2)
    c = workloads.rhs_uniform(nc, seed=6, nrhs=2)
    rg = torch.empty(2 * nc, dtype=torch.float64, device="cuda")
    prob.restrict(1, dev(f), rg, nrhs=2)
    pg = torch.zeros(2 * nf, dtype=torch.float64, device="cuda")
    prob.prolongate_add(1, dev(c), pg, nrhs=2)
    rg, pg = rg.cpu().numpy(), pg.cpu().numpy()
    for r in range(2):
        lhs = rg[r * nc:(r + 1) * nc] @ c[r * nc:(r + 1) * nc]
        rhs = f[r * nf:(r + 1) * nf] @ pg[r * nf:(r + 1) * nf]
        assert abs(lhs - rhs) <= 1e-12 * np.abs(f).sum() * np.abs(pg).max()
    if dim == 2:   # the oracle's transfer matrix, element by element
        P = prolongation_matrix(cmesh, cmesh.refine(), k)
        for r in range(2):
            assert rel_err(rg[r * nc:(r + 1) * nc], P.T @ f[r * nf:(r + 1) * nf]) < TOL64
            assert rel_err(pg[r * nf:(r + 1) * nf], P @ c[r * nc:(r + 1) * nc]) < TOL64
    prob.close()


SMOOTH_CASES = [(3, 15, (1, 1, 2), "cell"), (3, 10, (2, 1, 2), "cell"), (2, 15, (3, 3), "cell"),
                (3, 8, (3, 2, 2), "vertex"), (2, 15, (3, 3), "vertex"), (2, 11, (4, 3), "vertex")]


@pytest.mark.parametrize("dim,k,counts,kind", SMOOTH_CASES)
def test_smoothers_high_degree(dim, k, counts, kind):
    from paper_1910_11239_gb300 import tpss
    widths = widths_case(dim, counts, seed=40 + k)
    A = assembled((dim, counts), widths, k)
    S = oracle_sipg(widths, k)
    prob = make(dim, k, widths)
    P = prob.setup_patches(0, tpss.VERTEX_PATCH if kind == "vertex" else tpss.CELL)
    patches, sol = oracle_solvers(S, A, kind)
    N = A.shape[0]
    b = workloads.rhs_uniform(N, seed=11)
    x0 = workloads.rhs_uniform(N, seed=12)
    omega = 0.7 if kind == "cell" else 0.5 ** dim
    xg = torch.empty(N, dtype=torch.float64, device="cuda")
    P.smooth_additive(omega, dev(b), xg, x_is_zero=True)
    assert rel_err(xg, schwarz.additive_local_sum(b, sol, omega)) < TOL64
    xg = dev(x0)
    P.smooth_additive(omega, dev(b), xg, x_is_zero=False)
    assert rel_err(xg, schwarz.additive_smoother(A, b, x0, sol, omega)) < TOL64
    if kind == "vertex":
        colors = [schwarz.color_multiplicative_vertex(v) for v, _ in patches]
    else:
        colors = [schwarz.color_multiplicative_cell(m) for m, _ in patches]
    xg = dev(x0)
    P.smooth_multiplicative(1.0, dev(b), xg, reverse_colors=True)
    ref = schwarz.multiplicative_smoother(A, b, x0, sol, colors, 1.0, reverse=True)
    assert rel_err(xg, ref) < TOL64
    prob.close()


@pytest.mark.parametrize("k", [8, 10, 13, 15])
def test_single_vertex_patch_inverse_high_degree(k):
    """A 2 x 2 x 2 mesh is one vertex patch (n = 2(k+1) up to 32): AVS with
    omega = 1 and x = 0 is x = A^{-1} b, checked through the operator (pinned
    above) as the relative residual.  With LAPACK's generalized eigensolver
    in place of ours the same fast-diagonalization solve leaves relative
    residuals of about 1e-14 here (1D condition numbers below 3e3), so 1e-12
    leaves two orders of magnitude for the Jacobi eigensolver."""
    from paper_1910_11239_gb300 import tpss
    widths = widths_case(3, (2, 2, 2), seed=120 + k)
    prob = make(3, k, widths)
    P = prob.setup_patches(0, tpss.VERTEX_PATCH)
    assert P.info()["n"] == 2 * (k + 1)
    N = prob.ndofs(0)
    b = dev(workloads.rhs_uniform(N, seed=k, nrhs=2))
    x = torch.empty_like(b)
    P.smooth_additive(1.0, b, x, x_is_zero=True, nrhs=2)
    r = torch.empty_like(b)
    prob.residual(0, b, x, r, nrhs=2)
    for s in range(2):
        rel = (r[s * N:(s + 1) * N].norm() / b[s * N:(s + 1) * N].norm()).item()
        assert rel < 1e-12, rel
    if k == 8:   # direct comparison with the oracle's dense solve (5832 unknowns)
        A = oracle_sipg(widths, k).assemble().toarray()
        assert rel_err(x[:N], np.linalg.solve(A, b[:N].cpu().numpy())) < 1e-11
    prob.close()


@pytest.mark.parametrize("dim,k,counts", [(3, 3, (2, 2, 2)), (3, 5, (1, 1, 1)), (2, 6, (2, 2)), (2, 4, (1, 1))])
def test_coarse_fd_matches_dense(dim, k, counts):
    from paper_1910_11239_gb300 import tpss
    widths = widths_case(dim, counts, seed=150 + k)
    res = {}
    for solver in (tpss.COARSE_DENSE, tpss.COARSE_FD):
        prob = make(dim, k, widths, nlevels=2)
        prob.mg_setup("ACS", 0.7, tpss.FP64, coarse_solver=solver)
        n0 = prob.ndofs(0)
        b = dev(workloads.rhs_uniform(n0, seed=2))
        x = torch.empty_like(b)
        prob.coarse_solve(b, x)
        res[solver] = x.cpu().numpy()
        prob.close()
    assert rel_err(res[tpss.COARSE_FD], res[tpss.COARSE_DENSE]) < 1e-11


def test_coarse_fd_rejected_where_it_does_not_apply():
    from paper_1910_11239_gb300 import tpss
    prob = make(3, 2, widths_case(3, (3, 2, 2), seed=1), nlevels=2)
    with pytest.raises(RuntimeError, match="fast-diagonalization"):
        prob.mg_setup("ACS", 0.7, tpss.FP64, coarse_solver=tpss.COARSE_FD)
    prob.close()
    prob = make(3, 2, widths_case(3, (2, 2, 2), seed=1), nlevels=2)
    with pytest.raises(RuntimeError, match="fast-diagonalization"):
        prob.mg_setup("ACS", 0.7, tpss.FP32, coarse_solver=tpss.COARSE_FD)
    prob.close()


def test_auto_coarse_solver_at_high_degree_is_exact():
    """k = 9 on 2^3 coarse cells: 8000 coarse unknowns, so AUTO takes the fast
    diagonalization; A_0 x = b through the operator."""
    from paper_1910_11239_gb300 import tpss
    prob = make(3, 9, widths_case(3, (2, 2, 2), seed=3), nlevels=2)
    prob.mg_setup("ACS", 0.7, tpss.FP64)
    n0 = prob.ndofs(0)
    b = dev(workloads.rhs_uniform(n0, seed=9))
    x = torch.empty_like(b)
    prob.coarse_solve(b, x)
    r = torch.empty_like(b)
    prob.residual(0, b, x, r)
    assert (r.norm() / b.norm()).item() < 1e-10
    prob.close()


def test_mixed_precision_limited_to_degree_7():
    from paper_1910_11239_gb300 import tpss
    prob = make(3, 8, widths_case(3, (2, 2, 2), seed=4), nlevels=2)
    with pytest.raises(RuntimeError, match="up to 7"):
        prob.setup_patches(1, tpss.VERTEX_PATCH, precision=tpss.FP32)
    with pytest.raises(RuntimeError, match="up to 7"):
        prob.mg_setup("AVS", 0.125, tpss.BF16)
    prob.close()


@pytest.mark.parametrize("k,n", [(8, 4), (15, 3), (11, 5)])
def test_large_patch_cluster_sizes_agree(k, n):
    """The 3D large-patch kernel splits a subdomain over a thread-block
    cluster of 1, 2, 4 or 8 CTAs; every line is contracted by the same
    arithmetic, so all cluster sizes (and the automatic choice) give the
    same bits, for the additive and the multiplicative sweep."""
    from paper_1910_11239_gb300 import tpss
    widths = widths_case(3, (n, n, n), seed=200 + k)
    prob = make(3, k, widths)
    P = prob.setup_patches(0, tpss.VERTEX_PATCH)
    N = prob.ndofs(0)
    b = dev(workloads.rhs_uniform(N, seed=k, nrhs=2))
    x0 = workloads.rhs_uniform(N, seed=k + 1, nrhs=2)
    outs = []
    for cs in (0, 1, 2, 4, 8):
        P.set_large_cluster(cs)
        xa = torch.empty_like(b)
        P.smooth_additive(0.125, b, xa, x_is_zero=True, nrhs=2)
        xm = dev(x0)
        P.smooth_multiplicative(1.0, b, xm, nrhs=2)
        outs.append((xa, xm))
    for xa, xm in outs[1:]:
        assert torch.equal(xa, outs[0][0]) and torch.equal(xm, outs[0][1])
    with pytest.raises(RuntimeError):
        P.set_large_cluster(3)
    prob.close()
