/*
 * tpss.h -- C ABI of the GB300 tensor-product Schwarz smoother library.
 *
 * Method: Witte, Arndt, Kanschat, "Fast tensor product Schwarz smoothers for
 * high-order discontinuous Galerkin methods".  Geometric multigrid for the
 * symmetric interior penalty (SIPG) discretization of -Laplace(u) = f with
 * discontinuous Q_k elements on Cartesian tensor grids (Sec. 2.1), smoothed by
 * cell or vertex-patch Schwarz methods (Sec. 2.3) whose local solvers are
 * applied by fast diagonalization (Sec. 3.2).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * - Vectors are DEVICE pointers owned by the caller, contiguous, in the DoF
 *   layout of eq. discFEspace / eq. multiindex: cells lexicographic with the
 *   first direction fastest, then the (k+1)^d Gauss-Lobatto nodal values of a
 *   cell, first direction fastest.  A batch of `nrhs` vectors is stored one
 *   after another (vector r starts at offset r * ndofs(level)).
 * - Double-precision entry points take double*; the `_f32` entry points take
 *   float* and require patches set up with an FP32, TF32 or BF16 precision.
 * - All work is issued asynchronously on the stream given to tpss_create;
 *   only calls that return host values (documented) synchronize it.
 * - The library allocates its own device memory (1D tables, eigenpairs,
 *   per-level scratch vectors) in tpss_create / tpss_setup_patches /
 *   tpss_mg_setup and frees it in the matching destroy call.  It never frees
 *   caller memory.
 * - Return value: TPSS_OK (0) on success, a negative code on a hard error
 *   (nothing or only part of the work was done), a positive code for a soft
 *   outcome (TPSS_ENOTCONV: the iteration stopped at maxit).  Arguments are
 *   checked on the host before any launch.  tpss_last_error() returns a
 *   thread-local message for the last failing call.
 * - No exceptions cross this boundary and there is no global mutable state
 *   other than the thread-local error message.
 */
#ifndef TPSS_H
#define TPSS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TPSS_OK = 0,
  TPSS_ENOTCONV = 1,     /* iteration reached maxit without meeting rtol */
  TPSS_EINVAL = -1,      /* invalid argument (checked on the host) */
  TPSS_ECUDA = -2,       /* a CUDA call failed */
  TPSS_ENOMEM = -3,      /* device allocation failed */
  TPSS_EBREAKDOWN = -4,  /* NaN/Inf residual or p^T A p <= 0 in CG */
  TPSS_ETIMEOUT = -5,    /* a bounded device-side wait expired */
  TPSS_ENUMERIC = -6     /* setup produced a non-positive definite 1D problem */
} tpss_status;

typedef enum { TPSS_CELL = 0, TPSS_VERTEX_PATCH = 1 } tpss_patch_kind;

/* Arithmetic of the smoother's mode contractions.  FP64 is the plain form;
 * FP32 runs them on the FP32 pipe; TF32 and BF16 run them on tensor cores with
 * FP32 accumulation.  The 1D eigenproblems are always solved in FP64. */
typedef enum { TPSS_FP64 = 0, TPSS_FP32 = 1, TPSS_TF32 = 2, TPSS_BF16 = 3 } tpss_precision;

/* Polynomial factor P(k) of the penalty gamma_e = gamma_hat P(k) (1/h+ + 1/h-)
 * (eq. penalty): the paper's k(k+1), or (k+1)^2. */
typedef enum { TPSS_PENALTY_PAPER = 0, TPSS_PENALTY_KP1SQ = 1 } tpss_penalty_poly;

/* Problem description (Sec. 2.1).  The coarsest mesh T_0 is the tensor grid
 * with ncells[t] cells of widths widths[t][0..ncells[t]-1] in direction t
 * (lower corner at the origin); level l bisects T_0 l times. */
typedef struct {
  int dim;                  /* 2 or 3 */
  int degree;               /* k, 1 <= k <= 15 (FP32/TF32/BF16 smoothers and batches: k <= 7) */
  int ncells[3];            /* cells per direction on level 0 (ncells[2] ignored for dim 2) */
  const double* widths[3];  /* HOST arrays, copied during tpss_create */
  int nlevels;              /* >= 1; level nlevels-1 is the finest */
  double gamma_hat;         /* penalty prefactor, 1 on Cartesian meshes (eq. penalty) */
  int penalty_poly;         /* tpss_penalty_poly */
} tpss_problem_desc;

typedef struct tpss_ctx tpss_ctx;
typedef struct tpss_patches tpss_patches;

/* --------------------------------------------------------- mapped meshes --
 * Sec. 4: a mesh of bilinear quadrilaterals (dim 2) or trilinear hexahedra
 * (dim 3) given by a structured vertex array with ncells[t] + 1 vertices
 * along t: `vertices` is a HOST array of dim-tuples with the x index fastest,
 * vertex (i, j[, l]) at vertices[dim (i + (ncells[0]+1) (j + (ncells[1]+1) l))]
 * (ncells[2] ignored for dim 2).  Cell (i, j[, l]), numbered i + ncells[0]
 * (j + ncells[1] l), has the corners c = a0 + 2 a1 [+ 4 a2] at vertex
 * (i + a0, j + a1[, l + a2]) and reference corner (a0, a1[, a2]); every cell
 * must have det J > 0 at its corners (in 2D: convex, counter-clockwise;
 * TPSS_EINVAL otherwise).  Level l+1 splits every cell of level l at its
 * reference midpoints (the new vertices are means of 2, 4 or 8 old ones),
 * so the spaces are nested and the transfers are those of Cartesian meshes.
 * Operator: eq. bfsipg on the mapped cells (gradients through J^{-T}, outward
 * unit normals J^{-T} e_t / |J^{-T} e_t| and Nanson's surface element, the
 * paper's 1/sqrt(2) averages), penalty of eq. penalty with h^+- = |K^+-| / |e|;
 * the paper takes gamma_hat = 4 on its 25%-distorted meshes.  FP64, degree
 * 1..15 in 2D and 1..7 in 3D; FP32 degree 1..7.  Cell patches (tpss_setup_patches with TPSS_CELL, FP64) use the
 * inexact local solvers of eq. schwarzproj on the Cartesian surrogate of each
 * cell (eq. avglength: widths = mean lengths of the cell's edges per
 * direction, the neighbours' surrogate widths across its faces), by fast
 * diagonalization per cell.
 * FP32 (tpss_apply_operator_f32, FP32 cell patches, tpss_mg_setup with
 * precision TPSS_FP32: an FP32 V-cycle with FP32 geometry and surrogate data,
 * FP32 Chebyshev coarse steps, inside FP64 flexible PCG) is available.  The
 * smoothers compute the residual, the surrogate cell solves and the update
 * in one kernel per color (the multiplicative colors only on their own
 * cells).  Not available on these contexts (TPSS_EINVAL): vertex patches,
 * TF32 / BF16, kind 1 of tpss_assemble_rhs (kind 0 is f = d pi^2 prod
 * sin(pi x_t), g = 0), the per-color residual update of MCS (the residual
 * is formed per color on the color's cells) and the fast-diagonalization
 * coarse solver.  Every other call of this header works as on Cartesian
 * contexts; tpss_mg_setup's AUTO coarse solver takes the Chebyshev iteration
 * above 4096 coarse DoFs.  Release with tpss_destroy. */
tpss_status tpss_create_mapped(int dim, int degree, const int ncells[3], const double* vertices, int nlevels,
                               double gamma_hat, int penalty_poly, void* cuda_stream, tpss_ctx** out);

/* Copy level `level`'s vertex array (prod_t (nc_t + 1) dim-tuples, x index
 * fastest) to the HOST array `vertices`.  TPSS_EINVAL on a Cartesian context. */
tpss_status tpss_mapped_vertices(const tpss_ctx* ctx, int level, double* vertices);

/* Create a context: copies the description, runs the 1D setup kernels (Gauss-
 * Lobatto basis, Gauss rules, per-direction 1D mass/stiffness/face matrices of
 * eq. 1Dstiffnessmass - eq. 1Dsipg for every level) on `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream) and allocates per-level
 * scratch.  Synchronizes the stream before returning. */
tpss_status tpss_create(const tpss_problem_desc* desc, void* cuda_stream, tpss_ctx** out);
tpss_status tpss_destroy(tpss_ctx* ctx);

/* Number of DoFs and cells per direction of a level (host values). */
tpss_status tpss_level_info(const tpss_ctx* ctx, int level, int64_t* ndofs, int ncells[3]);

/* Thread-local message describing the last error of this thread ("" if none). */
const char* tpss_last_error(void);

/* ---------------------------------------------------------------- setup --
 * Fast diagonalization setup of the local solvers of one level (Sec. 3.2):
 * for every direction t and every subdomain position along t, the 1D matrices
 * A^(t), M^(t) of eq. 1Dsipg (cells, n = k+1) or eq. 1DsipgVP (vertex patches,
 * n = 2(k+1)) and the generalized eigenproblem of eq. generalizedEVP,
 * Z^T A Z = Lambda, Z^T M Z = I, solved in FP64 on the device (Cholesky of M,
 * cyclic Jacobi on L^{-1} A L^{-T}).  Also builds the colorings (additive:
 * none for cells, 2^d parity colors for vertex patches; multiplicative:
 * red-black for cells, 2^(d+1) colors for vertex patches, Sec. 2.3) and the
 * per-subdomain table 1/(lambda_i + lambda_j + lambda_l) of eq. fastinverse
 * (FP64, except 3D vertex patches with k >= 8, whose n = 2(k+1) >= 18 local
 * solves form these sums on the fly and keep their n^3 tensors in a device
 * scratch of one slab per resident CTA, allocated here).
 * Level must be >= 0; vertex patches need >= 2 cells per direction;
 * precisions other than FP64 need k <= 7.
 * Returns TPSS_ENUMERIC if some 1D problem is not positive definite.
 * Synchronizes the stream. */
tpss_status tpss_setup_patches(tpss_ctx* ctx, int level, int kind, int precision,
                               tpss_patches** out);
tpss_status tpss_patches_destroy(tpss_patches* patches);

/* Host-side description of a patch set: 1D size n, subdomain positions per
 * direction, number of subdomains, number of multiplicative colors. */
tpss_status tpss_patches_info(const tpss_patches* patches, int* n, int npos[3],
                              int64_t* nsub, int* ncolors_mult);

/* Copy the FP64 1D data of direction t at position pos to HOST arrays (each
 * may be NULL): A and M (n*n, row-major, test index first), Z (n*n row-major,
 * column j = eigenvector j) and lambda (n).  Synchronizes the stream.  On a
 * mesh of quadrilaterals the data are per cell: pos = the cell index. */
tpss_status tpss_patches_eigendata(const tpss_patches* patches, int t, int pos,
                                   double* A, double* M, double* Z, double* lambda);

/* Set the number of colors of the multiplicative vertex-patch sweep: 0 or
 * 2^(d+1) = the face-conflict-free coloring of Sec. 2.3 (default), or 2^d =
 * the parity coloring only (same-color patches then share faces, so the sweep
 * is not eq. multschwarz1 in any order). */
tpss_status tpss_patches_set_mult_colors(tpss_patches* patches, int ncolors);

/* Residual handling of the multiplicative sweep (tpss_smooth_multiplicative).
 *   UPDATE (default): r = b - A x is formed once per sweep and updated after
 *     each color instead of being recomputed (Alg. 3 recomputes it; the paper
 *     names avoiding this as the main cost reduction for MVS).  Exact up to
 *     rounding: the coloring keeps face-adjacent cells of one color in one
 *     subdomain and the local solves are exact, so r becomes (1 - omega) r on
 *     the color's cells and changes by the face couplings of the update on
 *     the cells next to them.  Used with the 2^(d+1)-color vertex coloring
 *     or red-black cells (the 2^d-color coloring recomputes the residual).
 *     With FP32 / TF32 / BF16 contractions (mixed V-cycles) the carried
 *     residual omits the rounding error of the local solves.
 *   FULL: recompute r = b - A x before every color (Alg. 3 as printed). */
typedef enum { TPSS_MULT_RESIDUAL_UPDATE = 0, TPSS_MULT_RESIDUAL_FULL = 1 } tpss_mult_residual;
tpss_status tpss_patches_set_mult_residual(tpss_patches* patches, int mode);

/* 3D vertex patches with k >= 8 (n >= 18 points per direction): number of
 * CTAs that share one subdomain solve, as a thread-block cluster (1, 2, 4 or
 * 8; 0 = chosen per launch from the number of subdomains, the default).  The
 * result does not depend on it (every line is contracted by the same
 * arithmetic); it is a tuning knob.  TPSS_EINVAL at launch if the GPU cannot
 * co-schedule a cluster of that size for the kernel; no effect on other
 * patch sets. */
tpss_status tpss_patches_set_large_cluster(tpss_patches* patches, int ctas);

/* Order of the subdomain solves of the additive smoother (the result is the
 * same sum; the schedules differ in memory traffic).
 *   COLORS (default, except TCGEN05 below): one launch per color (2^d for
 *     vertex patches), each over the whole mesh; deterministic.
 *   PLANES (3D vertex patches): plane of patches by plane of patches, the 4
 *     colors of a plane in turn, so that the two cell planes a patch plane
 *     touches stay in L2 across its colors (r and x are read from HBM about
 *     twice instead of once per color); deterministic; 4 launches per plane.
 *   ATOMIC (3D, BF16 contractions): one launch over all subdomains in
 *     lexicographic order, x accumulated with FP32 atomic adds; the order of
 *     the contributions to a DoF, and so the FP32 rounding, varies between runs.
 *   COLUMNS (3D vertex patches, BF16 contractions): one
 *     CTA per column of patches (p_x, p_y) and right-hand side walks p_z,
 *     staging each cell plane of r once and accumulating each cell plane of x
 *     in FP32 in shared memory until both of its patches in the column are
 *     done; the 4 parity classes of (p_x, p_y) share no cell and are 4
 *     launches; deterministic; x is written without being cleared first.
 *   TCGEN05 (3D vertex patches, k <= 7, BF16 or TF32 contractions; the
 *     default there for k >= 4): the COLUMNS schedule with the six mode
 *     contractions of each local solve as tcgen05 MMAs (BF16 or TF32
 *     operands in shared memory, FP32 accumulators in tensor memory);
 *     deterministic.  Its waits for MMA
 *     completion are bounded (about a second); if one expires the kernel
 *     stops, frees its tensor memory, and the next additive smoother call on
 *     the patch set returns TPSS_ETIMEOUT (the earlier result is invalid).
 * Schedules that do not apply to a patch set fall back to COLORS. */
typedef enum {
  TPSS_ADDITIVE_COLORS = 0,
  TPSS_ADDITIVE_PLANES = 1,
  TPSS_ADDITIVE_ATOMIC = 2,
  TPSS_ADDITIVE_COLUMNS = 3,
  TPSS_ADDITIVE_TCGEN05 = 4
} tpss_additive_schedule;
tpss_status tpss_patches_set_additive_schedule(tpss_patches* patches, int schedule);

/* Test hook for the failure path of the TCGEN05 schedule (not in the paper):
 * in the next additive smoother call on this patch set, every CTA waits
 * once for an mbarrier phase that no MMA completes, with a short bound
 * (about 1 ms), gives up, frees its tensor memory and sets the failure
 * flag; that call's x is invalid and the call after it returns
 * TPSS_ETIMEOUT (and clears the flag).  No GPU fault is involved: the MMAs
 * themselves complete normally.  TPSS_EINVAL for other patch sets. */
tpss_status tpss_patches_test_wait_expiry(tpss_patches* patches);

/* ------------------------------------------------------------- smoothers --
 * Additive Schwarz smoother, Alg. 2 with the damping of eq. additiveschwarz:
 *   r = b - A x;   x <- x + omega * sum_j R_j^T A_j^{-1} R_j r
 * with A_j^{-1} = Z Lambda^{-1} Z^T applied by sum factorization
 * (eq. fastinverse, eq. eigenvectormatvec).  If x_is_zero != 0 the input
 * values of x are ignored, r = b and no operator is applied.  b and x hold
 * nrhs vectors of ndofs(level) each.  Overlapping vertex patches are
 * processed color by color, so the result is deterministic. */
tpss_status tpss_smooth_additive(tpss_patches* patches, double omega, int nrhs,
                                 const double* b, double* x, int x_is_zero);
tpss_status tpss_smooth_additive_f32(tpss_patches* patches, float omega, int nrhs,
                                     const float* b, float* x, int x_is_zero);

/* Multiplicative Schwarz smoother, Alg. 3 with eq. coloredschwarz: for each
 * color c (in increasing order, or decreasing if reverse_colors != 0):
 *   r = b - A x;   x <- x + omega * sum_{j in J_c} R_j^T A_j^{-1} R_j r. */
tpss_status tpss_smooth_multiplicative(tpss_patches* patches, double omega, int reverse_colors,
                                       int nrhs, const double* b, double* x);
/* The same sweep with FP32 vectors, operator and local solves (patches set up
 * with FP32, TF32 or BF16; the multiplicative mixed V-cycle uses it). */
tpss_status tpss_smooth_multiplicative_f32(tpss_patches* patches, float omega, int reverse_colors, int nrhs,
                                           const float* b, float* x);

/* ------------------------------------------------------------- operators --
 * Matrix-free SIPG operator Au = A_l u (eq. bfsipg) by sum factorization over
 * the Kronecker form of Sec. 3.2 (cell mass and stiffness matrices plus the
 * rank-2 face couplings between neighbouring cells).  u and Au must not alias. */
tpss_status tpss_apply_operator(tpss_ctx* ctx, int level, int nrhs, const double* u, double* Au);
tpss_status tpss_apply_operator_f32(tpss_ctx* ctx, int level, int nrhs, const float* u, float* Au);

/* Allocation-free variant of tpss_apply_operator (the paper has no
 * counterpart; this is a library convenience).  For callers that must not
 * trigger a device allocation during a call: code whose device memory is all
 * reserved by another allocator, or latency-critical loops that cannot
 * afford the allocation and synchronization tpss_apply_operator performs the
 * first time a level is used with a larger nrhs.  Same result as
 * tpss_apply_operator; the operator's intermediates live in one static device
 * array of 4 * 2^19 doubles (16 MiB, held by every GPU that loads the library
 * until the process exits).  Limit on Cartesian meshes: ndofs(level) * nrhs
 * <= 2^19, else TPSS_EINVAL with a message; on a mesh of quadrilaterals or
 * hexahedra (tpss_create_mapped) the operator needs no intermediates, so
 * there is no limit and the array is not touched.  The first call on a device looks up the
 * array's device address; make that first call before any stream capture.
 * All calls share the array, so calls that overlap on the GPU (e.g. on two
 * streams) race; serialize them.  Calls no allocating routine. */
tpss_status tpss_apply_operator_noalloc(tpss_ctx* ctx, int level, int nrhs, const double* u, double* Au);

/* r = b - A_l x (r may alias b, not x). */
tpss_status tpss_residual(tpss_ctx* ctx, int level, int nrhs, const double* b, const double* x,
                          double* r);

/* Level transfers of Sec. 2.2 between `fine_level` and fine_level-1:
 * prolongation = embedding of V_{l-1} in V_l (fine += I^up coarse) and
 * restriction = its transpose (coarse = I^down fine). */
tpss_status tpss_prolongate_add(tpss_ctx* ctx, int fine_level, int nrhs, const double* coarse,
                                double* fine);
tpss_status tpss_restrict(tpss_ctx* ctx, int fine_level, int nrhs, const double* fine,
                          double* coarse);

/* Right-hand side of eq. sipg on a level, integrated with k+2 Gauss points per
 * direction.  kind 0: f = d pi^2 prod_t sin(pi x_t), g = 0 (exact solution
 * prod_t sin(pi x_t) on the unit cube); kind 1: the three-Gaussian solution of
 * Sec. 2.4 read as u = sum_i exp(-|x - x_i|^2 / sigma^2) / (sqrt(2 pi) sigma),
 * sigma = 1/3, with f = -Laplace(u) and g = u.  On a mesh of quadrilaterals
 * (kind 0 only) the integrals are taken over the mapped cells, in 2D. */
tpss_status tpss_assemble_rhs(tpss_ctx* ctx, int level, int kind, double* b);

/* ------------------------------------------------------------- multigrid --
 * Smoother choice for the V-cycle of Alg. 1 (m_pre = m_post = 1). */
typedef enum { TPSS_ACS = 0, TPSS_AVS = 1, TPSS_MCS = 2, TPSS_MVS = 3 } tpss_smoother_kind;

typedef struct {
  int smoother;        /* tpss_smoother_kind */
  double omega;        /* relaxation parameter of eq. additiveschwarz / eq. coloredschwarz */
  int precision;       /* tpss_precision of the V-cycle (FP64, or FP32/TF32/BF16: the
                          whole V-cycle then runs in FP32 with these contractions) */
  int mult_colors;     /* 0 = default (2^(d+1) for MVS), else as tpss_patches_set_mult_colors */
  int flexible_cg;     /* 1: Polak-Ribiere beta in tpss_pcg_solve (use with inexact V-cycles) */
  int nonsymmetric;    /* 1: the post-smoother keeps the pre-smoother's color order (the
                          non-symmetric V-cycle used with GMRES); 0: reversed (symmetric) */
  int coarse_solver;   /* tpss_coarse_solver (0 = automatic) */
  int mult_residual;   /* tpss_mult_residual for MCS / MVS (0 = update per color) */
  int smoothing_steps; /* m pre- and post-smoothing steps per level (ACS_m, MCS_m of Sec. 4);
                          0 = 1, at most 16 */
} tpss_mg_params;

/* Exact coarse solvers on level 0.
 *   DENSE: A_0 assembled by applying the operator to unit vectors and inverted
 *          by Gauss-Jordan elimination on the device (level 0 up to 16384
 *          unknowns); one dense matrix-vector product per solve.
 *   FD:    when level 0 has 1 cell per direction (one cell subdomain) or 2
 *          cells per direction (one vertex patch), the subdomain is the whole
 *          mesh and its fast-diagonalization inverse (Sec. 3.2) is A_0^{-1}
 *          exactly (FP64 V-cycles only).
 *   CHEBYSHEV: the paper's coarse solver (Sec. 2.4), inexact: a Chebyshev
 *          iteration preconditioned by the additive cell smoother (omega = 1)
 *          with a fixed number of steps for a 1e-8 reduction of the A-norm
 *          error over the interval [0.8 theta_min, 1.1 theta_max], theta the
 *          extreme Ritz values of 50 preconditioned CG steps from a
 *          SplitMix64 start vector (FP64 V-cycles only; see
 *          tpss_coarse_chebyshev_info).
 *   AUTO:  FD where it applies and level 0 has more than 4096 unknowns, else
 *          DENSE. */
typedef enum {
  TPSS_COARSE_AUTO = 0,
  TPSS_COARSE_DENSE = 1,
  TPSS_COARSE_FD = 2,
  TPSS_COARSE_CHEBYSHEV = 3
} tpss_coarse_solver;

/* Build smoothers on levels 1..L and the exact coarse solver on level 0 (this
 * replaces the paper's Chebyshev coarse iteration).  TPSS_EINVAL if the
 * requested coarse solver does not apply.  Synchronizes the stream. */
tpss_status tpss_mg_setup(tpss_ctx* ctx, const tpss_mg_params* params);

/* One V-cycle of Alg. 1 on the finest level with x_L = 0 on entry:
 * x = MG_L(0, b).  b and x are finest-level FP64 vectors (one right-hand side). */
tpss_status tpss_vcycle(tpss_ctx* ctx, const double* b, double* x);

/* Coarse solve x = A_0^{-1} b on level 0 (after tpss_mg_setup; exact except
 * with TPSS_COARSE_CHEBYSHEV). */
tpss_status tpss_coarse_solve(tpss_ctx* ctx, const double* b, double* x);

/* The Chebyshev coarse solver's interval [a, b] for P A_0 and its number of
 * steps (host values); TPSS_EINVAL if that solver is not set up. */
tpss_status tpss_coarse_chebyshev_info(const tpss_ctx* ctx, double* a, double* b, int* steps);

/* Preconditioned CG (Sec. 2.4) on the finest level with one V-cycle as
 * preconditioner, from x = 0, stopped at ||r_k||_2 <= rtol ||r_0||_2 or after
 * maxit iterations.  On return *iters and *rel_res are host values; if
 * res_hist != NULL, the residual norms ||r_0||..||r_iters|| are written to it
 * (host array of at least maxit+1 doubles).  Synchronizes the stream once per
 * iteration to test convergence.  Returns TPSS_ENOTCONV at maxit (x then
 * holds the maxit-th iterate) and TPSS_EBREAKDOWN on a NaN/Inf or
 * non-positive curvature. */
tpss_status tpss_pcg_solve(tpss_ctx* ctx, const double* b, double* x, double rtol, int maxit,
                           int* iters, double* rel_res, double* res_hist);

/* The energy norms of the errors of the same PCG iteration (the measure of
 * Sec. 2.4 for CG): with xs the solution (a DEVICE vector, e.g. from
 * tpss_pcg_solve to 1e-14), errs[k] = ||x_k - xs||_A for k = 0, 1, ...
 * (HOST array of at least maxit+1 doubles), one PCG run stopped at the first
 * errs[k] <= rtol errs[0] or after maxit steps; *count = number of values
 * written, x = the last iterate (must not alias b or xs).  TPSS_ENOTCONV at
 * maxit.  One extra operator application per step. */
tpss_status tpss_pcg_energy_errors(tpss_ctx* ctx, const double* b, const double* xs, double* x, double rtol,
                                   int maxit, int* count, double* errs);

/* Mixed-precision iterative refinement (not in the paper): from x = 0, repeat
 *   r = b - A x (FP64);  solve A e = r / ||r|| approximately by PCG in FP32
 *   (the FP32 operator, the FP32 / TF32 / BF16 V-cycle of tpss_mg_setup,
 *   flexible beta) to a relative residual inner_rtol or max_inner steps;
 *   x += ||r|| e (FP64),
 * until ||b - A x|| <= rtol ||b|| or max_outer refinement steps.  Needs a
 * mixed-precision V-cycle.  *outer_iters, *inner_iters (total) and *rel_res
 * are host values; allocates 5 finest-level FP32 vectors on its first call.
 * TPSS_ENOTCONV at max_outer. */
tpss_status tpss_ir_solve(tpss_ctx* ctx, const double* b, double* x, double rtol, int max_outer, double inner_rtol,
                          int max_inner, int* outer_iters, int* inner_iters, double* rel_res);

/* --------------------------------------------------------------- batches --
 * Many independent 3D problems of uneven size and degree (not in the paper):
 * every problem gets its own hierarchy (descs[p], additive vertex-patch
 * smoother with params->omega) and nrhs right-hand sides.  The V-cycle runs in
 * FP32 (mode contractions in FP32, or on BF16 tensor cores when
 * params->precision == TPSS_BF16; FP32 operators and transfers; FP64 coarse
 * inverse) with levels aligned from the finest one; at every level ONE
 * persistent kernel smooths all problems and right-hand sides, pulling work
 * items (problem, rhs, group of patches) from an atomic counter, largest
 * degree first, scattering with FP32 atomics (so FP32 summation order is not
 * fixed).  The number of patches per work item is autotuned per patch size
 * at creation unless flags & 2; the whole V-cycle is captured as a CUDA graph
 * unless flags & 1 or the stream is the legacy default stream.  With BF16
 * contractions, unless flags & 4, no level uses the persistent kernel: each
 * problem's additive pass runs the library's deterministic per-problem
 * smoother (the tcgen05 column walk TPSS_ADDITIVE_TCGEN05 for k >= 4, else
 * the colored launches) on one of four side streams forked from the batch
 * stream, so the problems' launches overlap; a tcgen05 pass that gave up
 * waiting for its MMAs is reported as TPSS_ETIMEOUT by the next
 * tpss_batch_vcycle or tpss_batch_pcg_solve.  The per-problem operators,
 * transfers and coarse solves of every batch run on the same side streams.
 * Vector layout of every batched call: problems one after another, each as
 * nrhs consecutive vectors of its finest level, each problem's block starting
 * on a 16-byte boundary (tpss_batch_info gives offsets; entries between blocks
 * are padding and are ignored).  Vectors must be 16-byte aligned.
 * Synchronizes the stream. */
typedef struct tpss_batch tpss_batch;
tpss_status tpss_batch_create(const tpss_problem_desc* descs, int nprob, int nrhs, const tpss_mg_params* params,
                              int flags, void* cuda_stream, tpss_batch** out);
tpss_status tpss_batch_destroy(tpss_batch* batch);
/* Finest-level size and offset of problem p, and its autotuned patches per work item. */
tpss_status tpss_batch_info(const tpss_batch* batch, int prob, int64_t* ndofs, int64_t* offset, int* ppb);
/* Concatenated length, number of systems (nprob * nrhs), 1 if the V-cycle is a CUDA graph. */
tpss_status tpss_batch_summary(const tpss_batch* batch, int64_t* total, int* nsys, int* uses_graph);
/* Finest level of every problem, x = omega sum_j R_j^T A_j^{-1} R_j b in FP32
 * (Alg. 2 with x = 0), one persistent launch (BF16 batches: the per-problem
 * passes on the side streams instead); b and x are FP32 device vectors. */
tpss_status tpss_batch_smooth_additive(tpss_batch* batch, const float* b, float* x);
/* x = MG(0, b) for every system (FP64 in and out, FP32 inside). */
tpss_status tpss_batch_vcycle(tpss_batch* batch, const double* b, double* x);
/* Flexible PCG for every system, FP64 outer iteration, from x = 0 to
 * ||r_k|| <= rtol ||r_0|| per system; iters and rel_res are HOST arrays of
 * nprob * nrhs entries.  TPSS_ENOTCONV if some system reached maxit. */
tpss_status tpss_batch_pcg_solve(tpss_batch* batch, const double* b, double* x, double rtol, int maxit,
                                 int* iters, double* rel_res);

/* GMRES(restart) (Sec. 2.4: the Krylov method used with the multiplicative
 * smoothers) on the finest level with one V-cycle M per step as
 * preconditioner, from x = 0.
 *   left = 0: flexible right preconditioning, x = Z y with z_j = M v_j;
 *             stopped when the least-squares residual ||b - A x_k||_2 <=
 *             rtol ||b||_2.
 *   left = 1: left preconditioning (Arnoldi on M A, x = V y); the monitored
 *             and minimized residual is ||M (b - A x_k)||_2, stopped when it
 *             is <= rtol ||M b||_2 (M must then be a fixed linear operator:
 *             an FP64 V-cycle).
 * Arnoldi by classical Gram-Schmidt with one reorthogonalization on the
 * device; the Hessenberg least-squares problem (Givens rotations) on the
 * host.  *iters, *rel_res and res_hist (maxit+1 host doubles, may be NULL;
 * the monitored residual norms) as in tpss_pcg_solve.  Allocates
 * (restart+1) + restart finest-level vectors on its first call.
 * TPSS_ENOTCONV at maxit. */
tpss_status tpss_gmres_solve(tpss_ctx* ctx, const double* b, double* x, double rtol, int maxit, int restart,
                             int left, int* iters, double* rel_res, double* res_hist);

#ifdef __cplusplus
}
#endif

#endif /* TPSS_H */
