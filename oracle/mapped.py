"""SIPG on meshes of bilinear quadrilaterals (2D) and trilinear hexahedra (3D)
and the inexact local solvers on Cartesian surrogate cells of Sec. 4.

Test infrastructure only (see the package docstring).

Mesh.  A structured vertex array V with one more vertex than cells per
direction, indexed V[j, i] (2D) or V[l, j, i] (3D) with the x index i
fastest, last axis the coordinates.  Cell (i, j[, l]) has the 2^d corners
c = a_0 + 2 a_1 [+ 4 a_2] (a_t in {0, 1}) at vertex (i + a_0, j + a_1[, l + a_2])
and reference corner (a_0, a_1[, a_2]); its map is the d-linear interpolation
x(xi) = sum_c v_c prod_t (a_t xi_t + (1 - a_t)(1 - xi_t)).  Cells are
numbered with i fastest, a cell's DoFs are the GL nodal values with the first
reference index fastest (the layout of the Cartesian case).  The distorted
meshes of Sec. 4 come from the shared input generators
(workloads.vertices_distorted).  `refine` splits every cell at its
reference midpoints: a new vertex is the mean of the 2^m old vertices of the
edge (m = 1), face (m = 2) or cell (m = d) it sits in, the image of the
midpoint under the d-linear map, so every child map is the parent map on a
sub-box of the reference cell; the fine space contains the coarse one and
the transfers are the Cartesian ones.

Bilinear form: eq. bfsipg written literally, as in sipg.py, with physical
gradients grad phi = J^{-T} grad_ref phi and, on the face xi_t = side, the
outward unit normal n = +-J^{-T} e_t / |J^{-T} e_t| and the surface element
|det J| |J^{-T} e_t| dxi (Nanson's formula; on a straight 2D edge this is the
edge's normal and length); the paper's 1/sqrt(2) averages on interior faces;
the penalty gamma_e = gamma_hat P(k) (1/h^+ + 1/h^-) of eq. penalty with
h^+- = |K^+-| / |e|, the mean extent of the cell normal to the face (the
reading for non-rectangular cells; the normal width on a box); boundary
faces: h^+ = h^- = h_K.  Integrals by the tensor Gauss rule with k+1 points
per direction, on cells and faces (|e| as well).  On an interior face both
cells see the same surface; its normal, surface element and |e| are taken
from the cell with the lower index.

Surrogate local solvers (Sec. 4, eq. schwarzproj, eq. avglength): cell K is
replaced by the box whose width along t is the mean length of K's 2^(d-1)
edges along t (vertex distances; in 2D hbar_0 = (l_01 + l_23)/2, hbar_1 =
(l_02 + l_13)/2); its local matrix is the Cartesian SIPG block of that box,
with the penalty on each interior face taken with the neighbour's surrogate
width normal to that face (every cell the local form touches is replaced by
its surrogate).  It is assembled by the Cartesian oracle (sipg.py) on the
tensor mesh of K's and its face neighbours' surrogate widths.

Pins (tests/test_oracle_mapped.py): on a Cartesian vertex array the assembly
equals sipg.SIPG (2D, 3D); on an affine mesh polynomials of degree k are
reproduced exactly (SIPG consistency, 2D, 3D); linear functions on
distorted meshes; L2 order k+1 on distorted meshes (2D, 3D); symmetry and
positive definiteness with gamma_hat = 4 (2D, 3D); the child maps of
`refine` equal the parent maps on the sub-boxes; the surrogate of a
Cartesian cell is its exact block; the mapped V-cycle on a Cartesian vertex
array is the Cartesian V-cycle.
"""
import itertools

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import schwarz
from .basis import gauss_legendre, gauss_lobatto_nodes, lagrange_derivatives, lagrange_values
from .sipg import SIPG, penalty_factor
from .mesh import TensorMesh
from .transfer import prolongation_matrix

SQRT2 = np.sqrt(2.0)


# ------------------------------------------------------------------ meshes
def mesh_dim(V):
    return V.shape[-1]


def mesh_cells(V):
    """Cells per direction (x first)."""
    return tuple(int(s) - 1 for s in reversed(V.shape[:-1]))


def refine(V):
    """Split every cell at its reference midpoints (d-linear images).  A new
    point between old vertices along the directions in `odd` is the mean of
    the 2^m surrounding old vertices, summed in corner order (first
    direction fastest)."""
    d = mesh_dim(V)
    nc = mesh_cells(V)
    F = np.zeros(tuple(2 * n + 1 for n in reversed(nc)) + (d,))
    for odd in itertools.product((0, 1), repeat=d):          # odd[t] = 1: between old vertices along t
        dst = tuple(slice(odd[t], None, 2) for t in reversed(range(d)))
        acc = None
        for c in range(2 ** d):                              # corners, first direction fastest
            a = [(c >> t) & 1 for t in range(d)]
            if any(a[t] and not odd[t] for t in range(d)):
                continue
            src = tuple((slice(1, None) if a[t] else slice(None, -1)) if odd[t] else slice(None)
                        for t in reversed(range(d)))
            acc = V[src] if acc is None else acc + V[src]
        m = sum(odd)
        F[dst] = acc if m == 0 else (0.5 ** m) * acc
    return F


def corner_vertices(V, multi):
    """The 2^d corners of cell `multi`, corner c = sum_t a_t 2^t."""
    d = mesh_dim(V)
    out = []
    for c in range(2 ** d):
        a = [(c >> t) & 1 for t in range(d)]
        out.append(V[tuple(multi[t] + a[t] for t in reversed(range(d)))])
    return out


def _shape(xi, d):
    """N[P, 2^d] and dN[P, 2^d, d] of the d-linear corner functions."""
    P = xi.shape[0]
    N = np.ones((P, 2 ** d))
    dN = np.ones((P, 2 ** d, d))
    for c in range(2 ** d):
        for t in range(d):
            a = (c >> t) & 1
            f = xi[:, t] if a else 1.0 - xi[:, t]
            N[:, c] *= f
            for s in range(d):
                dN[:, c, s] *= (1.0 if a else -1.0) if s == t else f
    return N, dN


def dlinear_map(V, multi, xi):
    """Physical points of reference points xi [P, d] in cell `multi`."""
    N, _ = _shape(xi, mesh_dim(V))
    return N @ np.array(corner_vertices(V, multi))


def jacobians(V, multi, xi):
    """J[P, d, d] with J[:, r, c] = d x_r / d xi_c."""
    _, dN = _shape(xi, mesh_dim(V))
    return np.einsum("pcs,cr->prs", dN, np.array(corner_vertices(V, multi)))


def surrogate_widths(V, multi):
    """eq. avglength: per direction t the mean length of the cell's edges along t."""
    d = mesh_dim(V)
    C = corner_vertices(V, multi)
    out = []
    for t in range(d):
        lens = [np.linalg.norm(C[c + (1 << t)] - C[c]) for c in range(2 ** d) if not (c >> t) & 1]
        out.append(sum(lens) / len(lens))
    return tuple(out)


# ---------------------------------------------------------------- assembly
class MappedSIPG:
    """SIPG matrix and right-hand side on the d-linear mesh V (d = 2, 3)."""

    def __init__(self, V, k, gamma_hat=4.0, penalty_poly="paper"):
        self.V = np.asarray(V, dtype=np.float64)
        self.d = mesh_dim(self.V)
        self.k = int(k)
        self.nc = mesh_cells(self.V)
        self.ncells = int(np.prod(self.nc))
        self.n1 = self.k + 1
        self.nloc = self.n1 ** self.d
        self.gamma_hat = float(gamma_hat)
        self.pk = penalty_factor(self.k, penalty_poly)
        self.nodes = gauss_lobatto_nodes(self.k)
        self.qx, self.qw = gauss_legendre(self.k + 1)
        # local DoF I = i0 + n1 i1 (+ n1^2 i2)
        self.idx = np.array([[(I // self.n1 ** t) % self.n1 for t in range(self.d)] for I in range(self.nloc)])

    def cell_multi(self, c):
        out = []
        for n in self.nc:
            out.append(c % n)
            c //= n
        return tuple(out)

    def cell_index(self, multi):
        c, s = 0, 1
        for t in range(self.d):
            c += multi[t] * s
            s *= self.nc[t]
        return c

    @staticmethod
    def _tensor_points(x, w, m):
        """m-dimensional tensor rule, first coordinate fastest."""
        pts = np.array([p[::-1] for p in itertools.product(x, repeat=m)]).reshape(-1, m)
        wts = np.array([np.prod(p) for p in itertools.product(w, repeat=m)])
        return pts, wts

    def _basis(self, xi):
        """Values P[Q, I] and reference gradients G[Q, I, d] at points xi [Q, d]."""
        P = np.ones((xi.shape[0], self.nloc))
        G = np.ones((xi.shape[0], self.nloc, self.d))
        for t in range(self.d):
            v = lagrange_values(self.nodes, xi[:, t])[:, self.idx[:, t]]
            dv = lagrange_derivatives(self.nodes, xi[:, t])[:, self.idx[:, t]]
            P *= v
            for s in range(self.d):
                G[:, :, s] *= dv if s == t else v
        return P, G

    def _physical_gradients(self, multi, xi, G):
        J = jacobians(self.V, multi, xi)
        Jinv = np.linalg.inv(J)                               # [Q, d, d]
        # grad phi = J^{-T} grad_ref phi: (J^{-T})[r, c] = Jinv[c, r]
        return np.einsum("qcr,qic->qir", Jinv, G, optimize=True), np.abs(np.linalg.det(J))

    def volume(self, multi):
        q, w = self._tensor_points(self.qx, self.qw, self.d)
        return float(np.sum(w * np.abs(np.linalg.det(jacobians(self.V, multi, q)))))

    def cell_matrix(self, multi):
        q, w = self._tensor_points(self.qx, self.qw, self.d)
        _, G = self._basis(q)
        Gp, detj = self._physical_gradients(multi, q, G)
        return np.einsum("q,qir,qjr->ij", w * detj, Gp, Gp, optimize=True)

    def _face(self, multi, t, side, x=None, w=None):
        """Reference points on face (t, side) (the other coordinates a tensor
        rule, lowest direction fastest), surface weights W, outward unit
        normals n [Q, d] and the face measure |e| (k+1 point rule)."""
        other = [s for s in range(self.d) if s != t]

        def points(x, w):
            pts, wts = self._tensor_points(x, w, self.d - 1)
            xi = np.zeros((len(wts), self.d))
            xi[:, t] = float(side)
            for m, s in enumerate(other):
                xi[:, s] = pts[:, m]
            J = jacobians(self.V, multi, xi)
            g = np.linalg.inv(J)[:, t, :]                   # (J^{-T} e_t)_r = Jinv[t, r]
            gn = np.linalg.norm(g, axis=1)
            return xi, wts * np.abs(np.linalg.det(J)) * gn, (1.0 if side else -1.0) * g / gn[:, None]

        _, W0, _ = points(self.qx, self.qw)
        xi, W, n = points(self.qx if x is None else x, self.qw if w is None else w)
        return xi, W, n, float(np.sum(W0))

    def _neighbor(self, multi, t, side):
        m = list(multi)
        m[t] += 1 if side else -1
        return tuple(m) if 0 <= m[t] < self.nc[t] else None

    def interior_face_blocks(self, mL, t):
        """Face between cell L = mL and its upper neighbour R along t:
        blocks[(S, T)][iota, i] (test cell S, trial cell T)."""
        mR = self._neighbor(mL, t, 1)
        xiL, W, nL, area = self._face(mL, t, 1)
        xiR = xiL.copy()
        xiR[:, t] = 0.0
        gam = self.gamma_hat * self.pk * (area / self.volume(mL) + area / self.volume(mR))
        PL, GL = self._basis(xiL)
        PR, GR = self._basis(xiR)
        GLp, _ = self._physical_gradients(mL, xiL, GL)
        GRp, _ = self._physical_gradients(mR, xiR, GR)
        val = {"L": PL, "R": PR}
        grad = {"L": GLp, "R": GRp}
        normal = {"L": nL, "R": -nL}
        blocks = {}
        for S in "LR":
            for T in "LR":
                un = val[T][:, :, None] * normal[T][:, None, :] / SQRT2
                vn = val[S][:, :, None] * normal[S][:, None, :] / SQRT2
                gu, gv = grad[T] / SQRT2, grad[S] / SQRT2
                blocks[(S, T)] = (gam * np.einsum("q,qir,qjr->ji", W, un, vn, optimize=True)
                                  - np.einsum("q,qir,qjr->ji", W, gu, vn, optimize=True)
                                  - np.einsum("q,qir,qjr->ji", W, un, gv, optimize=True))
        return blocks

    def boundary_face_block(self, multi, t, side):
        xi, W, n, area = self._face(multi, t, side)
        gam = self.gamma_hat * self.pk * 2.0 * area / self.volume(multi)
        P, G = self._basis(xi)
        Gp, _ = self._physical_gradients(multi, xi, G)
        un = P[:, :, None] * n[:, None, :]
        return (gam * np.einsum("q,qir,qjr->ji", W, un, un, optimize=True) - np.einsum("q,qir,qjr->ji", W, Gp, un, optimize=True)
                - np.einsum("q,qir,qjr->ji", W, un, Gp, optimize=True))

    def assemble(self):
        n = self.nloc
        rows, cols, vals = [], [], []
        li = np.repeat(np.arange(n), n)
        lj = np.tile(np.arange(n), n)

        def add(p, q, B):
            rows.append(p * n + li)
            cols.append(q * n + lj)
            vals.append(B.ravel())

        for c in range(self.ncells):
            m = self.cell_multi(c)
            add(c, c, self.cell_matrix(m))
            for t in range(self.d):
                for side in range(2):
                    nb = self._neighbor(m, t, side)
                    if nb is None:
                        add(c, c, self.boundary_face_block(m, t, side))
                    elif side == 1:
                        B = self.interior_face_blocks(m, t)
                        r = self.cell_index(nb)
                        add(c, c, B[("L", "L")])
                        add(c, r, B[("L", "R")])
                        add(r, c, B[("R", "L")])
                        add(r, r, B[("R", "R")])
        N = self.ncells * n
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N)).tocsr()
        A.sum_duplicates()
        return A

    def interpolate(self, u):
        """Nodal interpolant of u(points [P, d])."""
        xi = np.stack([self.nodes[self.idx[:, t]] for t in range(self.d)], axis=1)
        out = np.zeros(self.ncells * self.nloc)
        for c in range(self.ncells):
            out[c * self.nloc:(c + 1) * self.nloc] = u(dlinear_map(self.V, self.cell_multi(c), xi))
        return out

    def l2_error(self, coef, u):
        """||u_h - u||_{L2} with k+2 Gauss points per direction on every cell."""
        qx, qw = gauss_legendre(self.k + 2)
        q, w = self._tensor_points(qx, qw, self.d)
        P, _ = self._basis(q)
        err = 0.0
        for c in range(self.ncells):
            m = self.cell_multi(c)
            detj = np.abs(np.linalg.det(jacobians(self.V, m, q)))
            e = P @ coef[c * self.nloc:(c + 1) * self.nloc] - u(dlinear_map(self.V, m, q))
            err += np.sum(w * detj * e * e)
        return np.sqrt(err)

    def rhs(self, f, g, nq=None):
        """eq. sipg: int f phi + sum over boundary faces int (gamma g phi - g n.grad phi),
        nq (default k+2) Gauss points per direction.  On a non-affine cell the
        term g n.grad phi is rational (grad phi carries 1/det J), so a
        consistency check against the operator takes the operator's rule, nq = k+1."""
        qx, qw = gauss_legendre(self.k + 2 if nq is None else nq)
        q, w = self._tensor_points(qx, qw, self.d)
        P, _ = self._basis(q)
        out = np.zeros(self.ncells * self.nloc)
        for c in range(self.ncells):
            m = self.cell_multi(c)
            detj = np.abs(np.linalg.det(jacobians(self.V, m, q)))
            acc = P.T @ (w * detj * f(dlinear_map(self.V, m, q)))
            for t in range(self.d):
                for side in range(2):
                    if self._neighbor(m, t, side) is not None:
                        continue
                    xi, W, n, area = self._face(m, t, side, qx, qw)
                    gam = self.gamma_hat * self.pk * 2.0 * area / self.volume(m)
                    Pe, Ge = self._basis(xi)
                    Gp, _ = self._physical_gradients(m, xi, Ge)
                    gv = g(dlinear_map(self.V, m, xi))
                    acc += Pe.T @ (W * gam * gv) - np.einsum("q,qir,qr->i", W * gv, Gp, n, optimize=True)
            out[c * self.nloc:(c + 1) * self.nloc] = acc
        return out


# -------------------------------------------------- surrogate local solvers
def surrogate_cell_matrix(V, multi, k, gamma_hat=4.0, penalty_poly="paper"):
    """Cartesian SIPG block of the surrogate box of cell `multi`, with the face
    neighbours' surrogate widths normal to each shared face (eq. schwarzproj
    with the surrogate of eq. avglength)."""
    d = mesh_dim(V)
    nc = mesh_cells(V)
    h = surrogate_widths(V, multi)
    widths, centre = [], []
    for t in range(d):
        w, ct = [h[t]], 0
        m = list(multi)
        if multi[t] > 0:
            m[t] = multi[t] - 1
            w.insert(0, surrogate_widths(V, m)[t])
            ct = 1
        if multi[t] + 1 < nc[t]:
            m[t] = multi[t] + 1
            w.append(surrogate_widths(V, m)[t])
        widths.append(np.array(w))
        centre.append(ct)
    mesh = TensorMesh(widths)
    S = SIPG(mesh, k, gamma_hat=gamma_hat, penalty_poly=penalty_poly)
    return S.assemble([mesh.cell_index(tuple(centre))]).toarray()


def cell_patches(V):
    """One subspace per cell of the mapped mesh: list of (cell multi-index, [cell])."""
    nc = mesh_cells(V)
    out = []
    for c in range(int(np.prod(nc))):
        m, r = [], c
        for n in nc:
            m.append(r % n)
            r //= n
        out.append((tuple(m), [c]))
    return out


def surrogate_solvers(V, k, gamma_hat=4.0, penalty_poly="paper"):
    """Cell subspaces with the surrogate local matrices, as schwarz.LocalSolvers (dense LU)."""
    patches = cell_patches(V)
    multi = {cells[0]: m for m, cells in patches}
    nloc = (k + 1) ** mesh_dim(V)
    return schwarz.LocalSolvers(patches, nloc,
                                lambda cells: surrogate_cell_matrix(V, multi[cells[0]], k, gamma_hat, penalty_poly))


def exact_solvers(A, V, k):
    """The exact cell solvers R_j A R_j^T of the mapped matrix (the sACS of Sec. 4)."""
    nloc = (k + 1) ** mesh_dim(V)
    A = A.tocsr()
    return schwarz.LocalSolvers(cell_patches(V), nloc,
                                lambda cells: A[schwarz.patch_dofs(cells, nloc)][:, schwarz.patch_dofs(cells, nloc)])


class MappedHierarchy:
    """Levels 0..L of nested d-linear meshes (level 0 = V0, each further level
    `refine` of the previous) with the mapped SIPG matrices, the Cartesian
    reference-space transfers and cell smoothers with surrogate (inexact) or
    exact local solvers.

    smoother: 'ACS' (additive) or 'MCS' (multiplicative, red-black, reversed
    colors in post-smoothing so that the V-cycle is symmetric, Sec. 4);
    steps: pre- and post-smoothing steps m (ACS_m, MCS_m of Sec. 4); the coarse
    level is solved exactly (Cholesky)."""

    def __init__(self, V0, k, nlevels, smoother="ACS", omega=0.5, steps=1, gamma_hat=4.0,
                 penalty_poly="paper", local="surrogate"):
        self.k, self.smoother, self.omega, self.steps = k, smoother, omega, steps
        self.V = [np.asarray(V0, dtype=np.float64)]
        for _ in range(nlevels - 1):
            self.V.append(refine(self.V[-1]))
        self.ops = [MappedSIPG(V, k, gamma_hat, penalty_poly) for V in self.V]
        self.A = [op.assemble() for op in self.ops]
        # reference-space embedding: the Cartesian transfers of a uniform mesh with the same cells
        unit = [TensorMesh([np.ones(n) for n in mesh_cells(self.V[0])])]
        for _ in range(nlevels - 1):
            unit.append(unit[-1].refine())
        self.P = [None] + [prolongation_matrix(unit[l - 1], unit[l], k) for l in range(1, nlevels)]
        self.coarse_chol = sla.cho_factor(self.A[0].toarray())
        self.solvers, self.colors = [None], [None]
        for l in range(1, nlevels):
            V = self.V[l]
            self.solvers.append(surrogate_solvers(V, k, gamma_hat, penalty_poly) if local == "surrogate"
                                else exact_solvers(self.A[l], V, k))
            self.colors.append([schwarz.color_multiplicative_cell(m) for m, _ in cell_patches(V)])

    @property
    def nlevels(self):
        return len(self.V)

    def smooth(self, l, x, b, post):
        for _ in range(self.steps):
            if self.smoother == "ACS":
                x = schwarz.additive_smoother(self.A[l], b, x, self.solvers[l], self.omega)
            else:
                x = schwarz.multiplicative_smoother(self.A[l], b, x, self.solvers[l], self.colors[l],
                                                    self.omega, reverse=post)
        return x

    def vcycle(self, l, x, b):
        """Alg. 1 with m pre- and post-smoothing steps."""
        if l == 0:
            return sla.cho_solve(self.coarse_chol, b)
        x = self.smooth(l, x, b, post=False)
        b_c = self.P[l].T @ (b - self.A[l] @ x)
        x = x + self.P[l] @ self.vcycle(l - 1, np.zeros_like(b_c), b_c)
        return self.smooth(l, x, b, post=True)

    def precondition(self, r):
        return self.vcycle(self.nlevels - 1, np.zeros_like(r), r)
