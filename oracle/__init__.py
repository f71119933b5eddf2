"""Plain FP64 CPU oracle for the fast tensor-product Schwarz smoother method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the CUDA library and its Python binding) never
imports, links or calls it, and this package imports nothing from the product.

Everything here is written from the definitions in the paper (Witte, Arndt,
Kanschat, "Fast tensor product Schwarz smoothers for high-order discontinuous
Galerkin methods"), in FP64, with no Kronecker shortcuts:

* ``basis``     -- Gauss-Lobatto Lagrange basis and Gauss quadrature (Sec. 3,
                   eq. tppoly / basisref; Sec. 2.1).
* ``mesh``      -- Cartesian tensor meshes, nested by bisection (Sec. 2.1),
                   DoF layout as a direct sum over cells (eq. discFEspace,
                   eq. multiindex).
* ``sipg``      -- the interior penalty bilinear form (eq. bfsipg, eq. penalty)
                   and right-hand side (eq. sipg), assembled by d-dimensional
                   quadrature over cells and faces.
* ``schwarz``   -- cell and vertex-patch subspaces (Sec. 2.3), local solvers
                   A_j = R_j A R_j^T (eq. ritzproj) inverted by dense LU,
                   additive (Alg. 2, eq. additiveschwarz) and colored
                   multiplicative (Alg. 3, eq. coloredschwarz) smoothers.
* ``transfer``  -- prolongation as the embedding V_{l-1} in V_l and restriction
                   as its transpose (Sec. 2.2).
* ``multigrid`` -- V-cycle (Alg. 1) with an exact coarse solve, preconditioned
                   CG, flexible and left-preconditioned GMRES and the
                   fractional iteration count (Sec. 2.4).
* ``chebyshev`` -- the Chebyshev coarse solver with the additive cell smoother
                   as preconditioner (Sec. 2.4).
* ``fastdiag``  -- the same local solvers by fast diagonalization (Sec. 3.2,
                   eq. KDseparable, eq. generalizedEVP, eq. fastinverse): 1D
                   factors from the 1D bilinear form, scipy eigh, and the
                   additive sweep in plain C with OpenMP (``fd_smoother.c``),
                   the timed CPU baseline.
* ``mapped``    -- SIPG on distorted meshes of bilinear / trilinear cells and
                   the Cartesian-surrogate local solvers (Sec. 4, eq.
                   schwarzproj, eq. avglength), with their multigrid hierarchy.

Each function below states whether parity for it is pinned by the tests under
``tests/test_oracle_*.py``.  All functions are pinned (no "parity unpinned"
function) except where a docstring says otherwise.
"""
