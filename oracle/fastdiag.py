"""Fast-diagonalization local solvers on the CPU (Sec. 3.2), FP64.

Test infrastructure only (see the package docstring).  This is the timed CPU
baseline of the smoother; the dense-LU solvers of `schwarz.py` stay the
reference it is checked against.

The separable structure of Sec. 3.2 (eq. KDseparable): on a Cartesian mesh the
local matrix of a cell or vertex patch is the Kronecker sum
    A_j = sum_t M_d (x) .. (x) A_t (x) .. (x) M_1
of 1D factors, where A_t is the 1D SIPG matrix of the subspace's cells along
direction t (the 1D form of eq. bfsipg, face terms with the neighbours
included) and M_t the 1D mass matrix.  Here the 1D SIPG matrix is assembled by
`sipg.SIPG` on the 1D mesh of direction t (so every face term comes from the
bilinear form, not from the paper's 1D formulas), the mass matrix is the
Gauss-quadrature definition int phi_i phi_j, and the generalized eigenproblem
of eq. generalizedEVP, A_t Z = M_t Z Lambda with Z^T M_t Z = I, is solved by
scipy.linalg.eigh.  The local solves (eq. fastinverse) and the additive sum
run in `fd_smoother.c` (plain C with OpenMP over the patches of one color).

Pins (tests/test_oracle_fastdiag.py): the 1D mass matrix integrates constants
and linear functions exactly; the Kronecker sum of the 1D factors equals the
assembled d-dimensional local matrix (cells and vertex patches, 2D and 3D,
boundary and interior positions, random widths); Z^T M Z = I and
Z^T A Z = Lambda; the C sweep equals the dense-LU additive_local_sum of
`schwarz.py` to 1e-12 (and fails with a planted wrong eigenvalue).
"""
import ctypes
import os
import subprocess

import numpy as np
import scipy.linalg as sla

from .basis import gauss_legendre, gauss_lobatto_nodes, lagrange_values
from .mesh import TensorMesh
from .sipg import SIPG

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fd_smoother.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libfdsmoother.so")


def build():
    """Compile fd_smoother.c with gcc and OpenMP (plain -O2, portable flags)."""
    os.makedirs(BUILD, exist_ok=True)
    tmp = LIB + ".tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c99", SRC, "-o", tmp]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"gcc failed for {SRC}:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
            build()
        L = ctypes.CDLL(LIB)
        L.fd_additive_local_sum.restype = ctypes.c_int
        L.fd_additive_local_sum.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                            ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_int, ctypes.c_int]
        L.fd_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def mass_1d(k, h):
    """M[i, j] = int_0^h phi_i phi_j (Gauss rule with k+1 points, exact)."""
    x, w = gauss_legendre(k + 1)
    V = lagrange_values(gauss_lobatto_nodes(k), x)
    return h * (V.T * w) @ V


def factors_1d(widths_t, k, vertex, gamma_hat=1.0, penalty_poly="paper"):
    """The 1D factors (A_t, M_t) of every subspace position along one
    direction with cell widths `widths_t`: positions p = 0 .. c-2 for vertex
    patches (cells p, p+1) and p = 0 .. c-1 for cells."""
    w = np.asarray(widths_t, dtype=np.float64)
    S = SIPG(TensorMesh([w]), k, gamma_hat=gamma_hat, penalty_poly=penalty_poly)
    out = []
    npos = len(w) - 1 if vertex else len(w)
    for p in range(npos):
        cells = [p, p + 1] if vertex else [p]
        A = S.assemble(cells).toarray()
        M = sla.block_diag(*[mass_1d(k, w[c]) for c in cells])
        out.append((A, M))
    return out


def eigendata(widths, k, vertex, gamma_hat=1.0, penalty_poly="paper"):
    """Per direction t: Z[t] (npos, n, n) and lam[t] (npos, n) of eq.
    generalizedEVP, A_t Z = M_t Z Lambda, Z^T M_t Z = I."""
    Zs, lams = [], []
    for wt in widths:
        Z, L = [], []
        for A, M in factors_1d(wt, k, vertex, gamma_hat, penalty_poly):
            lam, z = sla.eigh(A, M)
            Z.append(z)
            L.append(lam)
        Zs.append(np.ascontiguousarray(np.array(Z)))
        lams.append(np.ascontiguousarray(np.array(L)))
    return Zs, lams


def additive_local_sum(widths, k, vertex, r, omega, nrhs=1, threads=0, eig=None, gamma_hat=1.0,
                       penalty_poly="paper", colors=None):
    """omega * sum_j R_j^T A_j^{-1} R_j r with A_j^{-1} applied by fast
    diagonalization (eq. fastinverse), for all cells or all vertex patches of
    the tensor mesh with per-direction widths `widths`; r holds nrhs vectors
    back to back.  threads = 0: OpenMP's default (all cores).  colors: the
    additive vertex-patch colors sum_t (v_t mod 2) 2^t to include (all when
    None; a bounded sample of the patches otherwise)."""
    d = len(widths)
    Zs, lams = eig if eig is not None else eigendata(widths, k, vertex, gamma_hat, penalty_poly)
    r = np.ascontiguousarray(r, dtype=np.float64)
    y = np.empty_like(r)
    nc = (ctypes.c_int * 3)(*([len(w) for w in widths] + [1] * (3 - d)))
    zp = (ctypes.c_void_p * 3)(*([z.ctypes.data for z in Zs] + [None] * (3 - d)))
    lp = (ctypes.c_void_p * 3)(*([l.ctypes.data for l in lams] + [None] * (3 - d)))
    mask = (1 << (1 << d)) - 1 if colors is None else sum(1 << c for c in colors)
    st = lib().fd_additive_local_sum(d, k, 1 if vertex else 0, nc, zp, lp, float(omega), int(nrhs),
                                     r.ctypes.data, y.ctypes.data, int(mask), int(threads))
    if st != 0:
        raise ValueError("fd_additive_local_sum: invalid arguments")
    return y


def count_color(ncells, color):
    """Number of interior vertices v (1 <= v_t <= ncells[t] - 1) of additive
    color sum_t (v_t mod 2) 2^t."""
    out = 1
    for t, n in enumerate(ncells):
        par = (color >> t) & 1
        out *= sum(1 for v in range(1, n) if v % 2 == par)
    return out


def max_threads():
    return int(lib().fd_max_threads())
