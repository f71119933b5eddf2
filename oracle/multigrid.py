"""Geometric multigrid V-cycle and preconditioned CG.

Test infrastructure only (see the package docstring).

V-cycle: Alg. 1 with m_pre = m_post = 1 (Sec. 2.4).  The coarse level is
solved exactly (dense Cholesky); the paper uses a Chebyshev iteration to a
relative accuracy of 1e-8 there (Sec. 2.4), which it does not specify further,
so the exact solve is the reading taken.  Pre-smoothing visits the colors in
order and post-smoothing in reverse order, so that with multiplicative
smoothers the V-cycle is symmetric and CG applies; with symmetric=False the
post-smoother keeps the pre-smoother's order (the non-symmetric V-cycle the
paper combines with GMRES for multiplicative smoothers).

PCG: standard preconditioned conjugate gradients from x_0 = 0, stopped when
||r_k||_2 <= rtol ||r_0||_2 (Sec. 2.4: relative residual reduction 1e-8).

Fractional iterations (Sec. 2.4): nu_frac = nu - 1 + log(e_{nu-1}/tol) /
log(e_{nu-1}/e_nu) with tol = rtol e_0, here with e the residual norm (the
paper uses the energy norm of the error for CG; the residual-based value is
labelled as such where reported).

Flexible GMRES (right preconditioned, restarted) for the non-symmetric
V-cycle of the multiplicative smoothers (the paper's choice for MCS and MVS),
and GMRES with the preconditioner on the left, which monitors the
preconditioned residual (the paper does not say which side it uses).

Pins (tests/test_oracle_multigrid.py): the PCG and FGMRES solutions match a
direct sparse solve to the residual tolerance; unpreconditioned GMRES
terminates in at most n steps on an n x n system and its least-squares
residual history equals the true residual norms; left-preconditioned GMRES
terminates in at most n steps, its history equals the explicitly recomputed
||M (b - A x_k)||, and with M = I it is the unpreconditioned method; the
V-cycle operator is symmetric for
the additive and the symmetrically ordered multiplicative smoothers; on T_0
the V-cycle is the exact coarse solve; the fractional count reproduces
hand-computed values.
"""
import numpy as np
import scipy.linalg as sla

from . import schwarz
from .mesh import TensorMesh
from .sipg import SIPG
from .transfer import prolongation_matrix


class Hierarchy:
    """Levels 0..L of a nested Cartesian mesh hierarchy with SIPG matrices,
    transfers and local solvers.

    smoother: 'ACS' (additive cells), 'AVS' (additive vertex patches),
              'MCS' (multiplicative cells, red-black),
              'MVS' (multiplicative vertex patches, 2^(d+1) colors)."""

    def __init__(self, coarse_widths, k, nlevels, smoother="AVS", omega=None,
                 gamma_hat=1.0, penalty_poly="paper", symmetric=True):
        self.k = k
        # symmetric=False: the post-smoother visits the colors in the same
        # order as the pre-smoother (the non-symmetric V-cycle used with GMRES)
        self.symmetric = symmetric
        self.smoother = smoother
        self.omega = omega if omega is not None else default_omega(smoother, len(coarse_widths))
        self.meshes = [TensorMesh(coarse_widths)]
        for _ in range(nlevels - 1):
            self.meshes.append(self.meshes[-1].refine())
        self.sipg = [SIPG(m, k, gamma_hat, penalty_poly) for m in self.meshes]
        self.A = [s.assemble() for s in self.sipg]
        self.P = [None] + [prolongation_matrix(self.meshes[l - 1], self.meshes[l], k)
                           for l in range(1, nlevels)]
        self.coarse_chol = sla.cho_factor(self.A[0].toarray())
        self.solvers, self.colors = [None], [None]
        for l in range(1, nlevels):
            mesh, A = self.meshes[l], self.A[l]
            nloc = self.sipg[l].nloc
            if smoother in ("ACS", "MCS"):
                patches = schwarz.cell_patches(mesh)
                cols = [schwarz.color_multiplicative_cell(m) for m, _ in patches]
            else:
                patches = schwarz.vertex_patches(mesh)
                f = (schwarz.color_additive_vertex if smoother == "AVS"
                     else schwarz.color_multiplicative_vertex)
                cols = [f(v) for v, _ in patches]
            A_csr = A.tocsr()
            def local(cells, A_csr=A_csr, nloc=nloc):
                idx = schwarz.patch_dofs(cells, nloc)
                return A_csr[idx][:, idx]
            self.solvers.append(schwarz.LocalSolvers(patches, nloc, local))
            self.colors.append(cols)

    @property
    def nlevels(self):
        return len(self.meshes)

    def smooth(self, l, x, b, post):
        if self.smoother in ("ACS", "AVS"):
            return schwarz.additive_smoother(self.A[l], b, x, self.solvers[l], self.omega)
        return schwarz.multiplicative_smoother(self.A[l], b, x, self.solvers[l], self.colors[l],
                                               self.omega, reverse=post and self.symmetric)

    def vcycle(self, l, x, b):
        """Alg. 1, MG_l(x, b)."""
        if l == 0:
            return sla.cho_solve(self.coarse_chol, b)
        x = self.smooth(l, x, b, post=False)
        b_c = self.P[l].T @ (b - self.A[l] @ x)
        e_c = self.vcycle(l - 1, np.zeros_like(b_c), b_c)
        x = x + self.P[l] @ e_c
        x = self.smooth(l, x, b, post=True)
        return x

    def precondition(self, r):
        L = self.nlevels - 1
        return self.vcycle(L, np.zeros_like(r), r)


def default_omega(smoother, d):
    """Relaxation defaults of Sec. 2.4: 0.7 for ACS, 1 for MCS and MVS; the
    additive vertex patch smoother needs omega < 2^-d (Sec. 2.4)."""
    return {"ACS": 0.7, "MCS": 1.0, "MVS": 1.0, "AVS": 0.5 ** d}[smoother]


def pcg(A, b, precondition, rtol=1e-8, maxit=500):
    """Preconditioned CG from x_0 = 0.  Returns (x, iterations, residual norm
    history [||r_0||, ||r_1||, ...], converged)."""
    x = np.zeros_like(b)
    r = b.copy()
    z = precondition(r)
    p = z.copy()
    rz = r @ z
    hist = [np.linalg.norm(r)]
    if hist[0] == 0.0:
        return x, 0, hist, True
    for it in range(1, maxit + 1):
        q = A @ p
        alpha = rz / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        hist.append(np.linalg.norm(r))
        if hist[-1] <= rtol * hist[0]:
            return x, it, hist, True
        z = precondition(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit, hist, False


def fgmres(A, b, precondition, rtol=1e-8, maxit=500, restart=30):
    """Flexible right-preconditioned GMRES(restart) from x_0 = 0 (the Krylov
    method of Sec. 2.4 for the multiplicative smoothers): Arnoldi with modified
    Gram-Schmidt on A z_j, z_j = M v_j, Givens rotations, x = x_0 + Z y.
    Returns (x, iterations, residual norm history, converged); the history
    holds the Euclidean norms of b - A x_k (the least-squares residuals)."""
    n = b.shape[0]
    x = np.zeros(n)
    beta0 = np.linalg.norm(b)
    hist = [beta0]
    if beta0 == 0.0:
        return x, 0, hist, True
    it = 0
    r = b.copy()
    while it < maxit:
        beta = np.linalg.norm(r)
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        g = np.zeros(restart + 1)
        g[0] = beta
        cs, sn = np.zeros(restart), np.zeros(restart)
        j_done = 0
        for j in range(restart):
            it += 1
            z = precondition(V[j])
            Z.append(z)
            w = A @ z
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            V.append(w / H[j + 1, j] if H[j + 1, j] > 0 else w)
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            d = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / d, H[j + 1, j] / d
            H[j, j] = d
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            hist.append(abs(g[j + 1]))
            j_done = j + 1
            if abs(g[j + 1]) <= rtol * beta0 or it >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        for i in range(j_done):
            x = x + y[i] * Z[i]
        r = b - A @ x
        if np.linalg.norm(r) <= rtol * beta0 * (1 + 1e-6) or hist[-1] <= rtol * beta0:
            return x, it, hist, True
    return x, it, hist, False


def gmres_left(A, b, precondition, rtol=1e-8, maxit=500, restart=30):
    """Left-preconditioned GMRES(restart) from x_0 = 0: GMRES applied to
    M A x = M b (M = precondition), Arnoldi with modified Gram-Schmidt on
    M A v_j, Givens rotations, x = x_0 + V y.  The residual it minimizes and
    monitors is the preconditioned one, ||M (b - A x_k)||; stopped when that
    falls to rtol ||M b||.  Returns (x, iterations, history of the
    preconditioned residual norms, converged).  (The Krylov method of Sec. 2.4
    for multiplicative smoothers, with the preconditioner applied from the
    left; `fgmres` applies it from the right.)"""
    n = b.shape[0]
    x = np.zeros(n)
    r = precondition(b)
    beta0 = np.linalg.norm(r)
    hist = [beta0]
    if beta0 == 0.0:
        return x, 0, hist, True
    it = 0
    while it < maxit:
        beta = np.linalg.norm(r)
        V = [r / beta]
        H = np.zeros((restart + 1, restart))
        g = np.zeros(restart + 1)
        g[0] = beta
        cs, sn = np.zeros(restart), np.zeros(restart)
        j_done = 0
        for j in range(restart):
            it += 1
            w = precondition(A @ V[j])
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            V.append(w / H[j + 1, j] if H[j + 1, j] > 0 else w)
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            d = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / d, H[j + 1, j] / d
            H[j, j] = d
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            hist.append(abs(g[j + 1]))
            j_done = j + 1
            if abs(g[j + 1]) <= rtol * beta0 or it >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        for i in range(j_done):
            x = x + y[i] * V[i]
        r = precondition(b - A @ x)
        if hist[-1] <= rtol * beta0:
            return x, it, hist, True
    return x, it, hist, False


def fractional_iterations(hist, rtol):
    """Sec. 2.4: nu_frac = nu - 1 + log(e_{nu-1}/tol) / log(e_{nu-1}/e_nu),
    tol = rtol e_0, nu the first step with e_nu <= tol."""
    tol = rtol * hist[0]
    for nu in range(1, len(hist)):
        if hist[nu] <= tol:
            return nu - 1 + np.log(hist[nu - 1] / tol) / np.log(hist[nu - 1] / hist[nu])
    return float("nan")
