"""Algorithmic work counts used for roofline reporting (what the method must
do, not what an implementation happens to do).

Local solver of one subdomain with n points per direction in d dimensions
(eq. fastinverse applied by sum factorization, eq. eigenvectormatvec):
  Z^T and Z: 2 d contractions of n^d values with an n x n matrix, 2 n^(d+1)
  flops each -> 4 d n^(d+1); Lambda^{-1}: n^d multiplications; damped
  scatter-add x += omega y: 2 n^d.  In 3D: 12 n^4 + 3 n^3 per subdomain.
The paper's likwid counts of the local solvers (tab:flop-additive) follow
12 n^4 per subdomain within a few percent; tests/test_perf.py checks that.

Minimal HBM traffic of one smoother application in the x = 0 form: read the
right-hand side once and write x once, 16 bytes per DoF in FP64 (8 in FP32).

Peaks: GB300 FP64 DFMA issue rate is 2 FMA per clock per SM (measured
1.20 TFLOP/s with a DFMA throughput probe at ~2.0 GHz); the derived peak at
the 2070 MHz maximum SM clock is 152 * 2 * 2 * 2.07e9 = 1.2586e12 flop/s.
"""

SMS = 152
FP64_FMA_PER_CLK_PER_SM = 2
FP32_FMA_PER_CLK_PER_SM = 128
MAX_SM_HZ = 2.07e9


def fp64_peak_flops(sm_hz=MAX_SM_HZ):
    return SMS * FP64_FMA_PER_CLK_PER_SM * 2 * sm_hz


def fp32_peak_flops(sm_hz=MAX_SM_HZ):
    return SMS * FP32_FMA_PER_CLK_PER_SM * 2 * sm_hz


def local_solver_flops(n, d=3):
    return 4 * d * n ** (d + 1) + 3 * n ** d


def num_vertex_patches(ncells):
    p = 1
    for c in ncells:
        p *= c - 1
    return p


def num_cells(ncells):
    p = 1
    for c in ncells:
        p *= c
    return p


def smoother_flops(ncells, k, d=3, vertex=True, nrhs=1):
    n = 2 * (k + 1) if vertex else k + 1
    nsub = num_vertex_patches(ncells) if vertex else num_cells(ncells)
    return nsub * local_solver_flops(n, d) * nrhs


def ndofs(ncells, k, d=3):
    return num_cells(ncells) * (k + 1) ** d


def smoother_bytes(ncells, k, d=3, nrhs=1, word=8):
    return 2 * word * ndofs(ncells, k, d) * nrhs


def operator_flops(ncells, k, d=3, nrhs=1):
    """Sum-factorized SIPG operator: 3 passes with 7 (k+1)^4 FMAs per cell
    (3D; 4 (k+1)^3 in 2D) plus the rank-2 face couplings, 2 faces per
    direction, each 2 (k+1) FMAs per line."""
    n1 = k + 1
    if d == 3:
        per_cell = 2 * (7 * n1 ** 4 + 3 * 2 * n1 ** 2 * 2 * n1)
    else:
        per_cell = 2 * (4 * n1 ** 3 + 2 * 2 * n1 * 2 * n1)
    return num_cells(ncells) * per_cell * nrhs


def operator_bytes(ncells, k, d=3, nrhs=1, word=8):
    """Minimal HBM traffic of one operator application: read u, write A u."""
    return 2 * word * ndofs(ncells, k, d) * nrhs


def mapped_operator_flops(ncells, k, nrhs=1):
    """Matrix-free SIPG operator on 2D bilinear cells as the kernel computes it,
    per cell (n1 = k+1 Gauss points per direction; geometry precomputed):
    4 sum-factorization stages of 2 n1^3 FMAs (reference gradients and their
    transposes) = 16 n1^3 flops; the metric at n1^2 points (6 each); per edge
    (4, each evaluated from both of its cells) the normal-derivative lines of
    both sides (2 n1^2 FMAs), 3 + 3 interpolations at n1 points (6 n1^2 FMAs)
    and ~17 flops of coefficients per point, the test sums (3 n1^2 FMAs); the
    edge terms' scatter (~10 n1^2): 16 n1^3 + 104 n1^2 + 68 n1."""
    n1 = k + 1
    return num_cells(ncells) * (16 * n1 ** 3 + 104 * n1 ** 2 + 68 * n1) * nrhs


def mapped3_operator_flops(ncells, k, nrhs=1):
    """The 3D kernel on trilinear hexahedra, per cell (n1 = k+1): 6 sum-
    factorization stages of 2 + 3 + 3 (and transposed) arrays of n1^4 FMAs
    (32 n1^4 flops), the metric (15 n1^3); per face (6, both sides each
    evaluated from both cells) the normal-derivative planes (2 n1^3 FMAs),
    two interpolation stages (6 + 8 n1^3 FMAs, both sides), ~30 flops of
    coefficients per point (180 n1^2 in total), two test stages (4 + 3 n1^3
    FMAs); the scatter (12 n1^3): 32 n1^4 + 303 n1^3 + 180 n1^2."""
    n1 = k + 1
    return num_cells(ncells) * (32 * n1 ** 4 + 303 * n1 ** 3 + 180 * n1 ** 2) * nrhs


def mapped3_operator_bytes(ncells, k, nrhs=1, word=8):
    """Read u, write A u, read the per-cell geometry (6 n1^3 + 24 n1^2 + 6 words)."""
    n1 = k + 1
    return num_cells(ncells) * word * (2 * n1 ** 3 * nrhs + 6 * n1 ** 3 + 24 * n1 ** 2 + 6)


def mapped_operator_bytes(ncells, k, nrhs=1, word=8):
    """Minimal HBM traffic: read u, write A u, read the per-cell geometry
    (3 n1^2 + 8 n1 + 8 words)."""
    nx, ny = ncells
    n1 = k + 1
    return nx * ny * word * (2 * n1 ** 2 * nrhs + 3 * n1 ** 2 + 8 * n1 + 8)


def transfer_flops(coarse_ncells, k, d=3, nrhs=1):
    """Embedding of a parent's (k+1)^d values into its 2^d children by sum
    factorization, one direction after another: 2 n1^4 + 4 n1^4 + 8 n1^4
    FMAs in 3D (2 n1^3 + 4 n1^3 in 2D), n1 = k+1; restriction is the
    transpose with the same count."""
    n1 = k + 1
    fmas = 14 * n1 ** 4 if d == 3 else 6 * n1 ** 3
    return num_cells(coarse_ncells) * 2 * fmas * nrhs


def transfer_bytes(coarse_ncells, k, d=3, nrhs=1, word=8, prolong=True):
    """Minimal HBM traffic: prolongate-add reads the coarse vector and reads
    and writes the fine one; restriction reads the fine vector and writes the
    coarse one."""
    nc = ndofs(coarse_ncells, k, d)
    nf = nc * 2 ** d
    return word * (nc + 2 * nf if prolong else nf + nc) * nrhs


def fractional_iterations(hist, rtol):
    """Fractional iteration count of Sec. 2.4:
    nu_frac = nu - 1 + log(e_{nu-1} / tol) / log(e_{nu-1} / e_nu), tol = rtol e_0,
    nu the first step with e_nu <= tol, here with e = residual norm (the
    paper uses the energy norm of the error for CG)."""
    import math
    tol = rtol * hist[0]
    for nu in range(1, len(hist)):
        if hist[nu] <= tol:
            return nu - 1 + math.log(hist[nu - 1] / tol) / math.log(hist[nu - 1] / hist[nu])
    return float("nan")


def cg_energy_errors(prob, b, rtol=1e-8, ref_rtol=1e-14, maxit=200):
    """Energy norms ||x* - x_k||_A of the PCG iterates k = 0, 1, ... on the
    finest level (Sec. 2.4 measures CG by these) until the first one at or
    below rtol ||x*||_A: x* from PCG to ref_rtol, then one PCG run that
    records the errors on the device (tpss_pcg_energy_errors).  The V-cycle
    must be set up (FP64)."""
    import torch
    xs = torch.empty_like(b)
    prob.pcg_solve(b, xs, rtol=ref_rtol, maxit=maxit)
    x = torch.empty_like(b)
    return prob.pcg_energy_errors(b, xs, x, rtol=rtol, maxit=maxit)