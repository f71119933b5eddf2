"""Symmetric interior penalty (SIPG) discretization of -Laplace(u) = f.

Test infrastructure only (see the package docstring).

This module writes out the bilinear form a_l(u, v) of eq. bfsipg literally:

    a(u, v) = sum_K int_K grad u . grad v
            + sum_e int_e ( gamma_e {u n}.{v n} - {grad u}.{v n} - {u n}.{grad v} )

with the paper's averages {w} = (w^+ + w^-)/sqrt(2) on interior faces
(eq. jumpavgscalar) and {w} = w on boundary faces (eq. avgbdry), and the
penalty gamma_e = gamma_hat P(k) (1/h^+ + 1/h^-) of eq. penalty, where h^+-
are the widths of the two cells normal to the face and h^+ = h^- = h on the
boundary.  P(k) = k(k+1) is the paper's choice; P(k) = (k+1)^2 is the reading
used for the "gamma = 2(k+1)^2/h" workloads (the same formula with a different
polynomial factor).

Every integral is evaluated with the d-dimensional tensor Gauss rule (cells)
or the (d-1)-dimensional rule (faces), with basis functions and gradients
evaluated point by point as products of 1D Lagrange polynomials -- there is no
use of the Kronecker structure of Sec. 3.2 here; that structure is what the
tests check against this assembly.

The right-hand side is eq. sipg: int f v + int_{boundary} (gamma_e g v - g n.grad v),
integrated with k+2 Gauss points per direction.

Pins (tests/test_oracle_sipg.py): symmetry, positive definiteness, exact
reproduction of polynomial solutions in Q_k (SIPG consistency), O(h^(k+1))
L2 convergence, and agreement with the Kronecker-sum form assembled from the
paper's 1D matrices (tests/test_oracle_kron.py); apply_rows equals the rows of
the assembled matrix (tests/test_oracle_checkers.py).
"""
import itertools

import numpy as np
import scipy.sparse as sp

from .basis import gauss_legendre, gauss_lobatto_nodes, lagrange_derivatives, lagrange_values
from .mesh import dofs_per_cell, local_multi_indices

SQRT2 = np.sqrt(2.0)


def _wsum(W, trial, test):
    """B[j, i] = sum_q W[q] sum_r trial[q, i, r] test[q, j, r]: the quadrature
    sum of a bilinear integrand (test index first), as matrix products."""
    out = 0.0
    for r in range(trial.shape[2]):
        out = out + (test[:, :, r].T * W) @ trial[:, :, r]
    return out


def penalty_factor(k, penalty_poly):
    if penalty_poly == "paper":
        return float(k * (k + 1))
    if penalty_poly == "kp1sq":
        return float((k + 1) ** 2)
    raise ValueError("penalty_poly must be 'paper' or 'kp1sq'")


class SIPG:
    """Assembler for a_l(.,.) on one TensorMesh with Q_k elements."""

    def __init__(self, mesh, k, gamma_hat=1.0, penalty_poly="paper"):
        self.mesh, self.k, self.d = mesh, int(k), mesh.d
        self.gamma_hat = float(gamma_hat)
        self.pk = penalty_factor(self.k, penalty_poly)
        self.nodes = gauss_lobatto_nodes(self.k)
        self.nloc = dofs_per_cell(self.k, self.d)
        self.multi = local_multi_indices(self.k, self.d)
        self.qx, self.qw = gauss_legendre(self.k + 1)
        self.V = lagrange_values(self.nodes, self.qx)          # V[q, i] = phi_i(x_q)
        self.D = lagrange_derivatives(self.nodes, self.qx)     # D[q, i] = phi_i'(x_q)
        self.Vend = lagrange_values(self.nodes, [0.0, 1.0])    # Vend[s, i] = phi_i(s)
        self.Dend = lagrange_derivatives(self.nodes, [0.0, 1.0])
        self._cell_cache = {}
        self._face_cache = {}

    # ---------------------------------------------------------------- helpers
    def gamma(self, h_minus, h_plus):
        """Penalty gamma_e of eq. penalty (pass h, h on boundary faces)."""
        return self.gamma_hat * self.pk * (1.0 / h_minus + 1.0 / h_plus)

    def _cell_tables(self, h):
        """Values Phi[Q, I], gradients G[Q, I, t] and weights W[Q] of the
        d-dimensional Gauss rule on a cell with widths h (physical gradients:
        d/dx_t = (1/h_t) d/dxhat_t).  Each entry is the product over the
        directions of 1D values, evaluated point by point (vectorized over the
        points Q and basis functions I)."""
        d, nq = self.d, len(self.qx)
        qm = np.array(list(itertools.product(range(nq), repeat=d)))   # [Q, d]
        im = np.array(self.multi)                                     # [I, d]
        vals = [self.V[np.ix_(qm[:, t], im[:, t])] for t in range(d)]  # [Q, I] per direction
        ders = [self.D[np.ix_(qm[:, t], im[:, t])] / h[t] for t in range(d)]
        Phi = np.ones((len(qm), len(im)))
        for t in range(d):
            Phi = Phi * vals[t]
        G = np.ones((len(qm), len(im), d))
        for s in range(d):
            for t in range(d):
                G[:, :, s] *= ders[t] if t == s else vals[t]
        W = np.ones(len(qm))
        for t in range(d):
            W = W * self.qw[qm[:, t]] * h[t]
        return Phi, G, W

    def _face_tables(self, h, t, side):
        """Traces on the face x_t = side (0 or 1 in reference coordinates) of a
        cell with widths h: values P[Q, I], gradients G[Q, I, s], weights W[Q]
        of the (d-1)-dimensional Gauss rule over the face."""
        d, nq = self.d, len(self.qx)
        others = [s for s in range(d) if s != t]
        if d == 1:   # a face of a 1D cell is a point: one "quadrature point", weight 1
            qm = np.zeros((1, 0), dtype=int)
        else:
            qm = np.array(list(itertools.product(range(nq), repeat=d - 1))).reshape(-1, d - 1)  # [Q, d-1]
        im = np.array(self.multi)
        nQ = len(qm)
        vals, ders = [], []
        for s in range(d):
            if s == t:
                vals.append(np.tile(self.Vend[side, im[:, s]], (nQ, 1)))
                ders.append(np.tile(self.Dend[side, im[:, s]] / h[s], (nQ, 1)))
            else:
                a = others.index(s)
                vals.append(self.V[np.ix_(qm[:, a], im[:, s])])
                ders.append(self.D[np.ix_(qm[:, a], im[:, s])] / h[s])
        P = np.ones((nQ, len(im)))
        for s in range(d):
            P = P * vals[s]
        G = np.ones((nQ, len(im), d))
        for r in range(d):
            for s in range(d):
                G[:, :, r] *= ders[s] if s == r else vals[s]
        W = np.ones(nQ)
        for a, s in enumerate(others):
            W = W * self.qw[qm[:, a]] * h[s]
        return P, G, W

    # ---------------------------------------------------------- local blocks
    def cell_matrix(self, h):
        """Bulk term int_K grad phi_i . grad phi_iota (test index first)."""
        key = tuple(h)
        if key not in self._cell_cache:
            _, G, W = self._cell_tables(h)
            self._cell_cache[key] = _wsum(W, G, G)
        return self._cell_cache[key]

    def interior_face_blocks(self, hL, hR, t):
        """Face terms of eq. bfsipg on the interior face between the lower cell
        L (widths hL) and upper cell R (widths hR) in direction t, split into
        blocks B[(S, T)][iota, i] with test cell S and trial cell T."""
        key = ("i", tuple(hL), tuple(hR), t)
        if key in self._face_cache:
            return self._face_cache[key]
        gam = self.gamma(hL[t], hR[t])
        PL, GL, W = self._face_tables(hL, t, 1)   # lower cell sees the face at x_t = 1
        PR, GR, WR = self._face_tables(hR, t, 0)  # upper cell sees it at x_t = 0
        assert np.allclose(W, WR)
        e = np.zeros(self.d)
        e[t] = 1.0
        normal = {"L": e, "R": -e}
        val = {"L": PL, "R": PR}
        grad = {"L": GL, "R": GR}
        blocks = {}
        for S in "LR":
            for T in "LR":
                # {u n}_P = u_T n_T / sqrt2, {v n}_P = v_S n_S / sqrt2,
                # {grad u}_P = grad u_T / sqrt2, {grad v}_P = grad v_S / sqrt2
                un = val[T][:, :, None] * normal[T][None, None, :] / SQRT2   # [Q, i, r]
                vn = val[S][:, :, None] * normal[S][None, None, :] / SQRT2   # [Q, iota, r]
                gu = grad[T] / SQRT2
                gv = grad[S] / SQRT2
                B = gam * _wsum(W, un, vn) - _wsum(W, gu, vn) - _wsum(W, un, gv)
                blocks[(S, T)] = B
        self._face_cache[key] = blocks
        return blocks

    def boundary_face_block(self, h, t, side):
        """Boundary face x_t = side of a cell with widths h, eq. bfsipg with the
        averages of eq. avgbdry: gamma_e u v - (grad u . n) v - u (n . grad v),
        gamma_e with h^+ = h^- = h_t."""
        key = ("b", tuple(h), t, side)
        if key in self._face_cache:
            return self._face_cache[key]
        gam = self.gamma(h[t], h[t])
        P, G, W = self._face_tables(h, t, side)
        n = np.zeros(self.d)
        n[t] = 1.0 if side == 1 else -1.0
        un = P[:, :, None] * n[None, None, :]
        B = gam * _wsum(W, un, un) - _wsum(W, G, un) - _wsum(W, un, G)
        self._face_cache[key] = B
        return B

    # -------------------------------------------------------------- assembly
    def _neighbor(self, multi, t, side):
        m = list(multi)
        m[t] += 1 if side == 1 else -1
        if 0 <= m[t] < self.mesh.ncells[t]:
            return self.mesh.cell_index(m)
        return None

    def cell_rows(self, c):
        """All blocks of the rows of cell c: list of (trial cell, block)."""
        mesh = self.mesh
        multi = mesh.cell_multi(c)
        _, h = mesh.cell_box(c)
        diag = self.cell_matrix(h).copy()
        out = []
        for t in range(self.d):
            for side in (0, 1):
                nb = self._neighbor(multi, t, side)
                if nb is None:
                    diag += self.boundary_face_block(h, t, side)
                    continue
                _, hn = mesh.cell_box(nb)
                if side == 1:   # c is the lower cell L, nb the upper cell R
                    B = self.interior_face_blocks(h, hn, t)
                    diag += B[("L", "L")]
                    out.append((nb, B[("L", "R")]))
                else:           # c is the upper cell R, nb the lower cell L
                    B = self.interior_face_blocks(hn, h, t)
                    diag += B[("R", "R")]
                    out.append((nb, B[("R", "L")]))
        out.append((c, diag))
        return out

    def assemble(self, cells=None):
        """The SIPG matrix restricted to the DoFs of `cells` (all cells when
        None), i.e. R A R^T with R the restriction to those cells (eq. ritzproj
        gives A_j = R_j A R_j^T).  Local numbering follows the order of
        `cells`, cell by cell, DoFs within a cell in eq. multiindex order."""
        if cells is None:
            cells = list(range(self.mesh.num_cells))
        cells = list(cells)
        pos = {c: p for p, c in enumerate(cells)}
        n = self.nloc
        rows, cols, vals = [], [], []
        li = np.repeat(np.arange(n), n)
        lj = np.tile(np.arange(n), n)
        for p, c in enumerate(cells):
            for nb, B in self.cell_rows(c):
                if nb not in pos:
                    continue
                q = pos[nb]
                rows.append(p * n + li)
                cols.append(q * n + lj)
                vals.append(B.ravel())
        N = len(cells) * n
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(N, N)).tocsr()
        A.sum_duplicates()
        return A

    def apply_rows(self, cells, x):
        """(A x) restricted to the DoFs of `cells`, for a global vector x, using
        only the rows of those cells (for sampled checks on large meshes)."""
        n = self.nloc
        out = np.zeros(len(cells) * n)
        for p, c in enumerate(cells):
            acc = np.zeros(n)
            for nb, B in self.cell_rows(c):
                acc += B @ x[nb * n:(nb + 1) * n]
            out[p * n:(p + 1) * n] = acc
        return out

    # ------------------------------------------------------- right-hand side
    def rhs(self, f, g=None, nq=None):
        """eq. sipg: b_iota = int f phi_iota + int_boundary (gamma_e g phi_iota
        - g n . grad phi_iota).  f(x) and g(x) take an array of points [P, d]."""
        d, k = self.d, self.k
        nq = k + 2 if nq is None else nq
        qx, qw = gauss_legendre(nq)
        V = lagrange_values(self.nodes, qx)
        Dv = lagrange_derivatives(self.nodes, qx)
        mesh = self.mesh
        b = np.zeros(mesh.num_cells * self.nloc)
        qmulti = list(itertools.product(range(nq), repeat=d))
        for c in range(mesh.num_cells):
            lo, h = mesh.cell_box(c)
            pts = np.array([[lo[t] + h[t] * qx[qm[t]] for t in range(d)] for qm in qmulti])
            wts = np.array([np.prod([qw[qm[t]] * h[t] for t in range(d)]) for qm in qmulti])
            fv = f(pts)
            loc = np.zeros(self.nloc)
            for I, im in enumerate(self.multi):
                phi = np.array([np.prod([V[qm[t], im[t]] for t in range(d)]) for qm in qmulti])
                loc[I] = np.sum(wts * fv * phi)
            if g is not None:
                multi = mesh.cell_multi(c)
                for t in range(d):
                    for side in (0, 1):
                        if self._neighbor(multi, t, side) is not None:
                            continue
                        loc += self._boundary_rhs(g, lo, h, t, side, qx, qw, V, Dv)
            b[c * self.nloc:(c + 1) * self.nloc] = loc
        return b

    def _boundary_rhs(self, g, lo, h, t, side, qx, qw, V, Dv):
        d = self.d
        others = [s for s in range(d) if s != t]
        gam = self.gamma(h[t], h[t])
        nsign = 1.0 if side == 1 else -1.0
        qmulti = list(itertools.product(range(len(qx)), repeat=d - 1))
        out = np.zeros(self.nloc)
        for qm in qmulti:
            x = np.array(lo, dtype=np.float64)
            w = 1.0
            for a, s in enumerate(others):
                x[s] = lo[s] + h[s] * qx[qm[a]]
                w *= qw[qm[a]] * h[s]
            x[t] = lo[t] + h[t] * side
            gv = float(g(x[None, :])[0])
            for I, im in enumerate(self.multi):
                val, dn = 1.0, 1.0
                for s in range(d):
                    if s == t:
                        v_s = self.Vend[side, im[s]]
                        d_s = self.Dend[side, im[s]] / h[s]
                    else:
                        a = others.index(s)
                        v_s, d_s = V[qm[a], im[s]], None
                    val *= v_s
                    dn *= d_s if s == t else v_s
                out[I] += w * gv * (gam * val - nsign * dn)
        return out

    # ------------------------------------------------------------ utilities
    def interpolate(self, u):
        """Nodal interpolant of u(x) (points [P, d]) into the Gauss-Lobatto
        Lagrange basis: coefficient = value at the support point."""
        mesh, d = self.mesh, self.d
        out = np.zeros(mesh.num_cells * self.nloc)
        for c in range(mesh.num_cells):
            lo, h = mesh.cell_box(c)
            pts = np.array([[lo[t] + h[t] * self.nodes[im[t]] for t in range(d)] for im in self.multi])
            out[c * self.nloc:(c + 1) * self.nloc] = u(pts)
        return out

    def l2_error(self, coef, u, nq=None):
        """|| u_h - u ||_L2 by Gauss quadrature with k+3 points per direction."""
        d, k, mesh = self.d, self.k, self.mesh
        nq = k + 3 if nq is None else nq
        qx, qw = gauss_legendre(nq)
        V = lagrange_values(self.nodes, qx)
        qmulti = list(itertools.product(range(nq), repeat=d))
        Phi = np.array([[np.prod([V[qm[t], im[t]] for t in range(d)]) for im in self.multi]
                        for qm in qmulti])
        err2 = 0.0
        for c in range(mesh.num_cells):
            lo, h = mesh.cell_box(c)
            pts = np.array([[lo[t] + h[t] * qx[qm[t]] for t in range(d)] for qm in qmulti])
            wts = np.array([np.prod([qw[qm[t]] * h[t] for t in range(d)]) for qm in qmulti])
            uh = Phi @ coef[c * self.nloc:(c + 1) * self.nloc]
            err2 += np.sum(wts * (uh - u(pts)) ** 2)
        return np.sqrt(err2)
