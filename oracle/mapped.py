"""SIPG on 2D meshes of bilinear quadrilaterals and the inexact local solvers
on Cartesian surrogate cells of Sec. 4.

Test infrastructure only (see the package docstring).

Mesh.  A structured (nx+1) x (ny+1) array of vertices V[j, i] (x index i
fastest); cell (i, j) has the corners v0 = V[j, i], v1 = V[j, i+1],
v2 = V[j+1, i], v3 = V[j+1, i+1] at the reference corners (0,0), (1,0),
(0,1), (1,1) and the bilinear map x(xi) = v0 (1-xi0)(1-xi1) + v1 xi0 (1-xi1)
+ v2 (1-xi0) xi1 + v3 xi0 xi1.  Cells are numbered with i fastest, the DoFs
of a cell are the GL nodal values ordered with the first reference index
fastest (the layout of the Cartesian case).  The distorted meshes of Sec. 4
come from the shared input generators (workloads.vertices_distorted).
`refine` splits every cell at its
reference midpoints: the new vertices are the images of the edge midpoints
and of the cell centre under the cell's bilinear map, so every child map is
the parent map composed with the affine child map; the fine space contains
the coarse one and the transfers are the Cartesian ones.

Bilinear form: eq. bfsipg written literally, as in sipg.py, with physical
gradients grad phi = J^{-T} grad_ref phi, the physical unit normal of each
(straight) edge, the paper's 1/sqrt(2) averages on interior edges, and the
penalty gamma_e = gamma_hat P(k) (1/h^+ + 1/h^-) of eq. penalty with h^+- =
|K^+-| / |e|, the mean width of the cell normal to the edge (the reading for
non-rectangular cells: area over edge length, which is the normal width on a
rectangle); boundary edges: h^+ = h^- = h_K.  Integrals by the tensor Gauss
rule with k+1 points per direction (cells) and k+1 points (edges).

Surrogate local solvers (Sec. 4, eq. schwarzproj, eq. avglength): cell K is
replaced by the rectangle with the mean lengths of its opposite edges,
hbar_0 = (l_01 + l_23)/2, hbar_1 = (l_02 + l_13)/2 (edge lengths as vertex
distances); its local matrix is the Cartesian SIPG block of that rectangle,
with the penalty on each interior face taken with the neighbour's surrogate
width normal to that face (the reading: the surrogate of a cell subdomain
keeps the face terms of the cell's own faces).  It is assembled by the
Cartesian oracle (sipg.py) on the 3 x 3 (or smaller, at the boundary)
tensor mesh of K's and its neighbours' surrogate widths.

Pins (tests/test_oracle_mapped.py): on a Cartesian vertex array the assembly
equals sipg.SIPG; on an affine (parallelogram) mesh polynomials of degree k
are reproduced exactly (SIPG consistency: A u_I = b(f = -Laplace u, g = u));
symmetry; positive definiteness on a 25%-distorted mesh with gamma_hat = 4;
the child maps of `refine` equal the parent maps on the sub-squares; the
surrogate of a rectangle in a Cartesian mesh is the exact local matrix.
"""
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
def refine(V):
    """Split every cell at its reference midpoints (bilinear images)."""
    ny, nx = V.shape[0] - 1, V.shape[1] - 1
    F = np.zeros((2 * ny + 1, 2 * nx + 1, 2))
    F[::2, ::2] = V
    F[::2, 1::2] = 0.5 * (V[:, :-1] + V[:, 1:])
    F[1::2, ::2] = 0.5 * (V[:-1, :] + V[1:, :])
    F[1::2, 1::2] = 0.25 * (V[:-1, :-1] + V[:-1, 1:] + V[1:, :-1] + V[1:, 1:])
    return F


def cell_corners(V, i, j):
    return V[j, i], V[j, i + 1], V[j + 1, i], V[j + 1, i + 1]


def bilinear_map(V, i, j, xi):
    """Physical points of reference points xi [P, 2] in cell (i, j)."""
    v0, v1, v2, v3 = cell_corners(V, i, j)
    a, b = xi[:, 0:1], xi[:, 1:2]
    return v0 * (1 - a) * (1 - b) + v1 * a * (1 - b) + v2 * (1 - a) * b + v3 * a * b


def jacobians(V, i, j, xi):
    """J[P, 2, 2] with J[:, r, c] = d x_r / d xi_c."""
    v0, v1, v2, v3 = cell_corners(V, i, j)
    a, b = xi[:, 0:1], xi[:, 1:2]
    d0 = (v1 - v0) * (1 - b) + (v3 - v2) * b          # d x / d xi0   [P, 2]
    d1 = (v2 - v0) * (1 - a) + (v3 - v1) * a          # d x / d xi1
    return np.stack([d0, d1], axis=2)


def surrogate_widths(V, i, j):
    """eq. avglength: mean lengths of the opposite edges."""
    v0, v1, v2, v3 = cell_corners(V, i, j)
    h0 = 0.5 * (np.linalg.norm(v1 - v0) + np.linalg.norm(v3 - v2))
    h1 = 0.5 * (np.linalg.norm(v2 - v0) + np.linalg.norm(v3 - v1))
    return h0, h1


# ---------------------------------------------------------------- assembly
class MappedSIPG:
    """SIPG matrix and right-hand side on the bilinear quadrilateral mesh V."""

    def __init__(self, V, k, gamma_hat=4.0, penalty_poly="paper"):
        self.V = np.asarray(V, dtype=np.float64)
        self.k = int(k)
        self.ny, self.nx = self.V.shape[0] - 1, self.V.shape[1] - 1
        self.ncells = self.nx * self.ny
        self.n1 = self.k + 1
        self.nloc = self.n1 ** 2
        self.gamma_hat = float(gamma_hat)
        self.pk = penalty_factor(self.k, penalty_poly)
        self.nodes = gauss_lobatto_nodes(self.k)
        self.qx, self.qw = gauss_legendre(self.k + 1)
        # local DoF i = i0 + n1 i1 (first reference index fastest)
        self.i0 = np.tile(np.arange(self.n1), self.n1)
        self.i1 = np.repeat(np.arange(self.n1), self.n1)

    def cell_index(self, i, j):
        return i + self.nx * j

    def _basis(self, xi):
        """Values P[Q, I] and reference gradients G[Q, I, 2] at points xi [Q, 2]."""
        v0 = lagrange_values(self.nodes, xi[:, 0])
        v1 = lagrange_values(self.nodes, xi[:, 1])
        d0 = lagrange_derivatives(self.nodes, xi[:, 0])
        d1 = lagrange_derivatives(self.nodes, xi[:, 1])
        P = v0[:, self.i0] * v1[:, self.i1]
        G = np.stack([d0[:, self.i0] * v1[:, self.i1], v0[:, self.i0] * d1[:, self.i1]], axis=2)
        return P, G

    def _physical_gradients(self, i, j, xi, G):
        J = jacobians(self.V, i, j, xi)
        Jinv = np.linalg.inv(J)                               # [Q, 2, 2]
        # grad phi = J^{-T} grad_ref phi: (J^{-T})[r, c] = Jinv[c, r]
        return np.einsum("qcr,qic->qir", Jinv, G), np.abs(np.linalg.det(J))

    def area(self, i, j):
        q = np.array([[a, b] for b in self.qx for a in self.qx])
        w = np.array([wa * wb for wb in self.qw for wa in self.qw])
        return float(np.sum(w * np.abs(np.linalg.det(jacobians(self.V, i, j, q)))))

    def cell_matrix(self, i, j):
        q = np.array([[a, b] for b in self.qx for a in self.qx])
        w = np.array([wa * wb for wb in self.qw for wa in self.qw])
        _, G = self._basis(q)
        Gp, detj = self._physical_gradients(i, j, q, G)
        W = w * detj
        return np.einsum("q,qir,qjr->ij", W, Gp, Gp)

    def _edge(self, i, j, t, side):
        """Reference points on edge (t, side) of cell (i, j), edge weights
        (Gauss weight x edge length), the outward unit normal and |e|."""
        s = self.qx
        xi = np.zeros((len(s), 2))
        xi[:, t] = float(side)
        xi[:, 1 - t] = s
        v0, v1, v2, v3 = cell_corners(self.V, i, j)
        if t == 0:   # edge xi0 = side: from (side, 0) to (side, 1)
            a, b = (v0, v2) if side == 0 else (v1, v3)
        else:        # edge xi1 = side: from (0, side) to (1, side)
            a, b = (v0, v1) if side == 0 else (v2, v3)
        tau = b - a
        le = np.linalg.norm(tau)
        # outward normal: for t = 0 the edge runs in +xi1, for t = 1 in +xi0
        if t == 0:
            n = np.array([tau[1], -tau[0]]) / le
        else:
            n = np.array([-tau[1], tau[0]]) / le
        if side == 0:
            n = -n
        return xi, self.qw * le, n, le

    def _h(self, i, j, le):
        return self.area(i, j) / le

    def interior_edge_blocks(self, iL, jL, t):
        """Edge between cell L = (iL, jL) and its upper neighbour R in
        direction t: blocks[(S, T)][iota, i] (test cell S, trial cell T)."""
        iR, jR = (iL + 1, jL) if t == 0 else (iL, jL + 1)
        xiL, W, nL, le = self._edge(iL, jL, t, 1)
        xiR, WR, nR, leR = self._edge(iR, jR, t, 0)
        assert np.allclose(W, WR) and np.allclose(nL, -nR)
        gam = self.gamma_hat * self.pk * (1.0 / self._h(iL, jL, le) + 1.0 / self._h(iR, jR, le))
        PL, GL = self._basis(xiL)
        PR, GR = self._basis(xiR)
        GLp, _ = self._physical_gradients(iL, jL, xiL, GL)
        GRp, _ = self._physical_gradients(iR, jR, xiR, GR)
        val = {"L": PL, "R": PR}
        grad = {"L": GLp, "R": GRp}
        normal = {"L": nL, "R": nR}
        blocks = {}
        for S in "LR":
            for T in "LR":
                un = val[T][:, :, None] * normal[T][None, None, :] / SQRT2
                vn = val[S][:, :, None] * normal[S][None, None, :] / SQRT2
                gu, gv = grad[T] / SQRT2, grad[S] / SQRT2
                blocks[(S, T)] = (gam * np.einsum("q,qir,qjr->ji", W, un, vn)
                                  - np.einsum("q,qir,qjr->ji", W, gu, vn)
                                  - np.einsum("q,qir,qjr->ji", W, un, gv))
        return blocks

    def boundary_edge_block(self, i, j, t, side):
        xi, W, n, le = self._edge(i, j, t, side)
        h = self._h(i, j, le)
        gam = self.gamma_hat * self.pk * (2.0 / h)
        P, G = self._basis(xi)
        Gp, _ = self._physical_gradients(i, j, xi, G)
        un = P[:, :, None] * n[None, None, :]
        return (gam * np.einsum("q,qir,qjr->ji", W, un, un) - np.einsum("q,qir,qjr->ji", W, Gp, un)
                - np.einsum("q,qir,qjr->ji", W, un, Gp))

    def assemble(self):
        n = self.nloc
        rows, cols, vals = [], [], []
        li = np.repeat(np.arange(n), n)
        lj = np.tile(np.arange(n), n)

        def add(p, q, B):
            rows.append(p * n + li)
            cols.append(q * n + lj)
            vals.append(B.ravel())

        for j in range(self.ny):
            for i in range(self.nx):
                c = self.cell_index(i, j)
                add(c, c, self.cell_matrix(i, j))
                for t in range(2):
                    for side in range(2):
                        ii, jj = (i + (1 if side else -1), j) if t == 0 else (i, j + (1 if side else -1))
                        inside = 0 <= ii < self.nx and 0 <= jj < self.ny
                        if not inside:
                            add(c, c, self.boundary_edge_block(i, j, t, side))
                        elif side == 1:
                            B = self.interior_edge_blocks(i, j, t)
                            r = self.cell_index(ii, jj)
                            add(c, c, B[("L", "L")])
                            add(c, r, B[("L", "R")])
                            add(r, c, B[("R", "L")])
                            add(r, r, B[("R", "R")])
        N = self.ncells * n
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N)).tocsr()
        A.sum_duplicates()
        return A

    def interpolate(self, u):
        """Nodal interpolant of u(points [P, 2])."""
        xi = np.stack([self.nodes[self.i0], self.nodes[self.i1]], axis=1)
        out = np.zeros(self.ncells * self.nloc)
        for j in range(self.ny):
            for i in range(self.nx):
                c = self.cell_index(i, j)
                out[c * self.nloc:(c + 1) * self.nloc] = u(bilinear_map(self.V, i, j, xi))
        return out

    def l2_error(self, coef, u):
        """||u_h - u||_{L2} with k+2 Gauss points per direction on every cell."""
        qx, qw = gauss_legendre(self.k + 2)
        q = np.array([[a, b] for b in qx for a in qx])
        w = np.array([wa * wb for wb in qw for wa in qw])
        P, _ = self._basis(q)
        err = 0.0
        for j in range(self.ny):
            for i in range(self.nx):
                c = self.cell_index(i, j)
                detj = np.abs(np.linalg.det(jacobians(self.V, i, j, q)))
                e = P @ coef[c * self.nloc:(c + 1) * self.nloc] - u(bilinear_map(self.V, i, j, q))
                err += np.sum(w * detj * e * e)
        return np.sqrt(err)

    def rhs(self, f, g, nq=None):
        """eq. sipg: int f phi + sum over boundary edges int (gamma g phi - g n.grad phi),
        nq (default k+2) Gauss points per direction.  On a non-affine cell the
        term g n.grad phi is rational (grad phi carries 1/det J), so a
        consistency check against the operator takes the operator's rule, nq = k+1."""
        qx, qw = gauss_legendre(self.k + 2 if nq is None else nq)
        q = np.array([[a, b] for b in qx for a in qx])
        w = np.array([wa * wb for wb in qw for wa in qw])
        out = np.zeros(self.ncells * self.nloc)
        for j in range(self.ny):
            for i in range(self.nx):
                c = self.cell_index(i, j)
                P, G = self._basis(q)
                detj = np.abs(np.linalg.det(jacobians(self.V, i, j, q)))
                acc = P.T @ (w * detj * f(bilinear_map(self.V, i, j, q)))
                for t in range(2):
                    for side in range(2):
                        ii, jj = (i + (1 if side else -1), j) if t == 0 else (i, j + (1 if side else -1))
                        if 0 <= ii < self.nx and 0 <= jj < self.ny:
                            continue
                        xi = np.zeros((len(qx), 2))
                        xi[:, t] = float(side)
                        xi[:, 1 - t] = qx
                        _, _, n, le = self._edge(i, j, t, side)
                        gam = self.gamma_hat * self.pk * (2.0 / self._h(i, j, le))
                        Pe, Ge = self._basis(xi)
                        Gp, _ = self._physical_gradients(i, j, xi, Ge)
                        gv = g(bilinear_map(self.V, i, j, xi))
                        acc += Pe.T @ (qw * le * gam * gv) - np.einsum("q,qir,r->i", qw * le * gv, Gp, n)
                out[c * self.nloc:(c + 1) * self.nloc] = acc
        return out


# -------------------------------------------------- surrogate local solvers
def surrogate_cell_matrix(V, i, j, k, gamma_hat=4.0, penalty_poly="paper"):
    """Cartesian SIPG block of cell (i, j)'s surrogate rectangle, with the
    neighbours' surrogate widths normal to each shared face (eq. schwarzproj
    with the surrogate of eq. avglength)."""
    ny, nx = V.shape[0] - 1, V.shape[1] - 1
    h0, h1 = surrogate_widths(V, i, j)
    wx, wy, cx, cy = [h0], [h1], 0, 0
    if i > 0:
        wx.insert(0, surrogate_widths(V, i - 1, j)[0])
        cx = 1
    if i + 1 < nx:
        wx.append(surrogate_widths(V, i + 1, j)[0])
    if j > 0:
        wy.insert(0, surrogate_widths(V, i, j - 1)[1])
        cy = 1
    if j + 1 < ny:
        wy.append(surrogate_widths(V, i, j + 1)[1])
    mesh = TensorMesh([np.array(wx), np.array(wy)])
    S = SIPG(mesh, k, gamma_hat=gamma_hat, penalty_poly=penalty_poly)
    return S.assemble([mesh.cell_index((cx, cy))]).toarray()


def surrogate_solvers(V, k, gamma_hat=4.0, penalty_poly="paper"):
    """Cell subspaces of the mapped mesh (x index fastest) with the surrogate
    local matrices, as schwarz.LocalSolvers (dense LU)."""
    ny, nx = V.shape[0] - 1, V.shape[1] - 1
    nloc = (k + 1) ** 2
    patches = [((i, j), [i + nx * j]) for j in range(ny) for i in range(nx)]

    def local(cells):
        c = cells[0]
        return surrogate_cell_matrix(V, c % nx, c // nx, k, gamma_hat, penalty_poly)

    return schwarz.LocalSolvers(patches, nloc, local)


def exact_solvers(A, V, k):
    """The exact cell solvers R_j A R_j^T of the mapped matrix (the sACS of Sec. 4)."""
    ny, nx = V.shape[0] - 1, V.shape[1] - 1
    nloc = (k + 1) ** 2
    patches = [((i, j), [i + nx * j]) for j in range(ny) for i in range(nx)]
    A = A.tocsr()
    return schwarz.LocalSolvers(patches, nloc, lambda cells: A[schwarz.patch_dofs(cells, nloc)][:, schwarz.patch_dofs(cells, nloc)])


class MappedHierarchy:
    """Levels 0..L of nested bilinear meshes (level 0 = V0, each further level
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
        unit = [TensorMesh([np.ones(self.V[0].shape[1] - 1), np.ones(self.V[0].shape[0] - 1)])]
        for _ in range(nlevels - 1):
            unit.append(unit[-1].refine())
        self.P = [None] + [prolongation_matrix(unit[l - 1], unit[l], k) for l in range(1, nlevels)]
        self.coarse_chol = sla.cho_factor(self.A[0].toarray())
        self.solvers, self.colors = [None], [None]
        for l in range(1, nlevels):
            V = self.V[l]
            nx = V.shape[1] - 1
            ncell = nx * (V.shape[0] - 1)
            self.solvers.append(surrogate_solvers(V, k, gamma_hat, penalty_poly) if local == "surrogate"
                                else exact_solvers(self.A[l], V, k))
            self.colors.append([schwarz.color_multiplicative_cell((c % nx, c // nx)) for c in range(ncell)])

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
