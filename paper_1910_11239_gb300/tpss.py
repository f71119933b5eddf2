"""Thin Python binding of the C ABI in include/tpss.h (argument marshalling only).

Every numerical step runs in the CUDA library libtpss.so; this module only
converts torch tensors to device pointers and checks shapes/dtypes.  If the
library is missing, importing works but the first call raises -- there is no
fallback implementation.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtpss.so")

TPSS_OK, TPSS_ENOTCONV = 0, 1
STATUS_NAMES = {0: "TPSS_OK", 1: "TPSS_ENOTCONV", -1: "TPSS_EINVAL", -2: "TPSS_ECUDA", -3: "TPSS_ENOMEM",
                -4: "TPSS_EBREAKDOWN", -5: "TPSS_ETIMEOUT", -6: "TPSS_ENUMERIC"}
CELL, VERTEX_PATCH = 0, 1
FP64, FP32, TF32, BF16 = 0, 1, 2, 3
PENALTY_PAPER, PENALTY_KP1SQ = 0, 1
COARSE_AUTO, COARSE_DENSE, COARSE_FD, COARSE_CHEBYSHEV = 0, 1, 2, 3
MULT_RESIDUAL_UPDATE, MULT_RESIDUAL_FULL = 0, 1
ADDITIVE_COLORS, ADDITIVE_PLANES, ADDITIVE_ATOMIC, ADDITIVE_COLUMNS, ADDITIVE_TCGEN05 = 0, 1, 2, 3, 4
ACS, AVS, MCS, MVS = 0, 1, 2, 3
SMOOTHERS = {"ACS": ACS, "AVS": AVS, "MCS": MCS, "MVS": MVS}
PRECISIONS = {"fp64": FP64, "fp32": FP32, "tf32": TF32, "bf16": BF16}


class TpssError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class ProblemDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("degree", ctypes.c_int), ("ncells", ctypes.c_int * 3),
                ("widths", ctypes.POINTER(ctypes.c_double) * 3), ("nlevels", ctypes.c_int),
                ("gamma_hat", ctypes.c_double), ("penalty_poly", ctypes.c_int)]


class MGParams(ctypes.Structure):
    _fields_ = [("smoother", ctypes.c_int), ("omega", ctypes.c_double), ("precision", ctypes.c_int),
                ("mult_colors", ctypes.c_int), ("flexible_cg", ctypes.c_int), ("nonsymmetric", ctypes.c_int),
                ("coarse_solver", ctypes.c_int), ("mult_residual", ctypes.c_int), ("smoothing_steps", ctypes.c_int)]


_lib = None

# exported symbols and their argument types (c_void_p = device or host pointer)
_VP, _I, _D, _F, _I64P = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_float, ctypes.POINTER(ctypes.c_int64)
SIGNATURES = {
    "tpss_create": [ctypes.POINTER(ProblemDesc), _VP, ctypes.POINTER(_VP)],
    "tpss_create_mapped": [_I, _I, ctypes.POINTER(ctypes.c_int), _VP, _I, _D, _I, _VP, ctypes.POINTER(_VP)],
    "tpss_mapped_vertices": [_VP, _I, _VP],
    "tpss_destroy": [_VP],
    "tpss_level_info": [_VP, _I, _I64P, ctypes.POINTER(ctypes.c_int)],
    "tpss_last_error": [],
    "tpss_setup_patches": [_VP, _I, _I, _I, ctypes.POINTER(_VP)],
    "tpss_patches_destroy": [_VP],
    "tpss_patches_info": [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _I64P,
                          ctypes.POINTER(ctypes.c_int)],
    "tpss_patches_eigendata": [_VP, _I, _I, _VP, _VP, _VP, _VP],
    "tpss_patches_set_mult_colors": [_VP, _I],
    "tpss_patches_set_mult_residual": [_VP, _I],
    "tpss_patches_set_large_cluster": [_VP, _I],
    "tpss_patches_set_additive_schedule": [_VP, _I],
    "tpss_patches_test_wait_expiry": [_VP],
    "tpss_smooth_additive": [_VP, _D, _I, _VP, _VP, _I],
    "tpss_smooth_additive_f32": [_VP, _F, _I, _VP, _VP, _I],
    "tpss_smooth_multiplicative": [_VP, _D, _I, _I, _VP, _VP],
    "tpss_smooth_multiplicative_f32": [_VP, _F, _I, _I, _VP, _VP],
    "tpss_apply_operator": [_VP, _I, _I, _VP, _VP],
    "tpss_apply_operator_f32": [_VP, _I, _I, _VP, _VP],
    "tpss_apply_operator_noalloc": [_VP, _I, _I, _VP, _VP],
    "tpss_residual": [_VP, _I, _I, _VP, _VP, _VP],
    "tpss_prolongate_add": [_VP, _I, _I, _VP, _VP],
    "tpss_restrict": [_VP, _I, _I, _VP, _VP],
    "tpss_assemble_rhs": [_VP, _I, _I, _VP],
    "tpss_mg_setup": [_VP, ctypes.POINTER(MGParams)],
    "tpss_vcycle": [_VP, _VP, _VP],
    "tpss_coarse_solve": [_VP, _VP, _VP],
    "tpss_ir_solve": [_VP, _VP, _VP, _D, _I, _D, _I, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                      ctypes.POINTER(ctypes.c_double)],
    "tpss_coarse_chebyshev_info": [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_int)],
    "tpss_pcg_solve": [_VP, _VP, _VP, _D, _I, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                       _VP],
    "tpss_pcg_energy_errors": [_VP, _VP, _VP, _VP, _D, _I, ctypes.POINTER(ctypes.c_int), _VP],
    "tpss_gmres_solve": [_VP, _VP, _VP, _D, _I, _I, _I, ctypes.POINTER(ctypes.c_int),
                         ctypes.POINTER(ctypes.c_double), _VP],
    "tpss_batch_create": [ctypes.POINTER(ProblemDesc), _I, _I, ctypes.POINTER(MGParams), _I, _VP,
                          ctypes.POINTER(_VP)],
    "tpss_batch_destroy": [_VP],
    "tpss_batch_info": [_VP, _I, _I64P, _I64P, ctypes.POINTER(ctypes.c_int)],
    "tpss_batch_summary": [_VP, _I64P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
    "tpss_batch_smooth_additive": [_VP, _VP, _VP],
    "tpss_batch_vcycle": [_VP, _VP, _VP],
    "tpss_batch_pcg_solve": [_VP, _VP, _VP, _D, _I, _VP, _VP],
}


def lib():
    """Load libtpss.so (built by build_lib.build()); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} not found: build it with paper_1910_11239_gb300.build_lib.build() "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_char_p if name == "tpss_last_error" else ctypes.c_int
        _lib = L
    return _lib


def _check(status, allow=(TPSS_OK,)):
    if status not in allow:
        raise TpssError(status, lib().tpss_last_error().decode())
    return status


def _ptr(t, dtype, numel=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if not t.is_cuda:
        raise ValueError("tensor must live on the GPU")
    if t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


class Problem:
    """tpss_create / tpss_destroy and the level-wise operations of a context."""

    def __init__(self, dim, degree, widths, nlevels=1, gamma_hat=1.0, penalty_poly=PENALTY_PAPER, stream=None):
        self._keep = [(ctypes.c_double * len(w))(*[float(v) for v in w]) for w in widths]
        desc = ProblemDesc()
        desc.dim, desc.degree, desc.nlevels = dim, degree, nlevels
        desc.gamma_hat, desc.penalty_poly = gamma_hat, penalty_poly
        for t in range(3):
            desc.ncells[t] = len(widths[t]) if t < dim else 1
            desc.widths[t] = ctypes.cast(self._keep[t], ctypes.POINTER(ctypes.c_double)) if t < dim else None
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        handle = ctypes.c_void_p()
        _check(lib().tpss_create(ctypes.byref(desc), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(handle)))
        self.h = handle
        self.dim, self.degree, self.nlevels = dim, degree, nlevels
        self._patches = []

    @classmethod
    def mapped(cls, degree, vertices, nlevels=1, gamma_hat=4.0, penalty_poly=PENALTY_PAPER, stream=None):
        """tpss_create_mapped: mesh of bilinear quadrilaterals / trilinear
        hexahedra from a vertex array of shape (ny+1, nx+1, 2) or
        (nz+1, ny+1, nx+1, 3) (x index fastest, Sec. 4)."""
        import numpy as np
        V = np.ascontiguousarray(vertices, dtype=np.float64)
        dim = V.shape[-1]
        if dim not in (2, 3) or V.ndim != dim + 1:
            raise ValueError("vertices must have shape (ny+1, nx+1, 2) or (nz+1, ny+1, nx+1, 3)")
        nc = (ctypes.c_int * 3)(*([s - 1 for s in reversed(V.shape[:-1])] + [1] * (3 - dim)))
        self = cls.__new__(cls)
        self._keep = [V]
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        handle = ctypes.c_void_p()
        _check(lib().tpss_create_mapped(dim, degree, nc, ctypes.c_void_p(V.ctypes.data), nlevels, gamma_hat,
                                        penalty_poly, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(handle)))
        self.h = handle
        self.dim, self.degree, self.nlevels = dim, degree, nlevels
        self._patches = []
        return self

    def mapped_vertices(self, level):
        import numpy as np
        nc = self.level_info(level)[1]
        out = np.empty(tuple(n + 1 for n in reversed(nc[:self.dim])) + (self.dim,))
        _check(lib().tpss_mapped_vertices(self.h, level, ctypes.c_void_p(out.ctypes.data)))
        return out

    def close(self):
        if getattr(self, "h", None):
            for p in self._patches:
                p.close()
            lib().tpss_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def level_info(self, level):
        n = ctypes.c_int64()
        nc = (ctypes.c_int * 3)()
        _check(lib().tpss_level_info(self.h, level, ctypes.byref(n), nc))
        return n.value, tuple(nc)

    def ndofs(self, level):
        return self.level_info(level)[0]

    def setup_patches(self, level, kind, precision=FP64):
        out = ctypes.c_void_p()
        _check(lib().tpss_setup_patches(self.h, level, kind, precision, ctypes.byref(out)))
        p = Patches(self, out, level, kind, precision)
        self._patches.append(p)
        return p

    def apply_operator(self, level, u, out, nrhs=1):
        n = self.ndofs(level) * nrhs
        if u.dtype == torch.float64:
            _check(lib().tpss_apply_operator(self.h, level, nrhs, _ptr(u, torch.float64, n), _ptr(out, torch.float64, n)))
        else:
            _check(lib().tpss_apply_operator_f32(self.h, level, nrhs, _ptr(u, torch.float32, n), _ptr(out, torch.float32, n)))
        return out

    def apply_operator_noalloc(self, level, u, out, nrhs=1):
        """tpss_apply_operator_noalloc: same result as apply_operator, no device
        allocation (intermediates in the library's fixed 16 MiB array;
        ndofs * nrhs <= 2^19 on Cartesian meshes; no limit on mapped meshes)."""
        n = self.ndofs(level) * nrhs
        _check(lib().tpss_apply_operator_noalloc(self.h, level, nrhs, _ptr(u, torch.float64, n),
                                                 _ptr(out, torch.float64, n)))
        return out

    def residual(self, level, b, x, r, nrhs=1):
        n = self.ndofs(level) * nrhs
        _check(lib().tpss_residual(self.h, level, nrhs, _ptr(b, torch.float64, n), _ptr(x, torch.float64, n),
                                   _ptr(r, torch.float64, n)))
        return r

    def prolongate_add(self, fine_level, coarse, fine, nrhs=1):
        _check(lib().tpss_prolongate_add(self.h, fine_level, nrhs,
                                         _ptr(coarse, torch.float64, self.ndofs(fine_level - 1) * nrhs),
                                         _ptr(fine, torch.float64, self.ndofs(fine_level) * nrhs)))
        return fine

    def restrict(self, fine_level, fine, coarse, nrhs=1):
        _check(lib().tpss_restrict(self.h, fine_level, nrhs, _ptr(fine, torch.float64, self.ndofs(fine_level) * nrhs),
                                   _ptr(coarse, torch.float64, self.ndofs(fine_level - 1) * nrhs)))
        return coarse

    def assemble_rhs(self, level, kind, b):
        _check(lib().tpss_assemble_rhs(self.h, level, kind, _ptr(b, torch.float64, self.ndofs(level))))
        return b

    def mg_setup(self, smoother, omega, precision=FP64, mult_colors=0, flexible_cg=0, nonsymmetric=0,
                 coarse_solver=COARSE_AUTO, mult_residual=MULT_RESIDUAL_UPDATE, smoothing_steps=1):
        p = MGParams()
        p.smoothing_steps = smoothing_steps
        p.smoother = SMOOTHERS[smoother] if isinstance(smoother, str) else smoother
        p.omega, p.precision, p.mult_colors, p.flexible_cg = omega, precision, mult_colors, flexible_cg
        p.nonsymmetric = int(bool(nonsymmetric))
        p.coarse_solver = coarse_solver
        p.mult_residual = mult_residual
        _check(lib().tpss_mg_setup(self.h, ctypes.byref(p)))

    def vcycle(self, b, x):
        n = self.ndofs(self.nlevels - 1)
        _check(lib().tpss_vcycle(self.h, _ptr(b, torch.float64, n), _ptr(x, torch.float64, n)))
        return x

    def coarse_solve(self, b, x):
        n = self.ndofs(0)
        _check(lib().tpss_coarse_solve(self.h, _ptr(b, torch.float64, n), _ptr(x, torch.float64, n)))
        return x


    def ir_solve(self, b, x, rtol=1e-8, max_outer=20, inner_rtol=1e-3, max_inner=100):
        """Mixed-precision iterative refinement (FP64 residual, FP32 inner PCG)."""
        n = self.ndofs(self.nlevels - 1)
        o, i, rel = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        st = lib().tpss_ir_solve(self.h, _ptr(b, torch.float64, n), _ptr(x, torch.float64, n), rtol, max_outer,
                                 inner_rtol, max_inner, ctypes.byref(o), ctypes.byref(i), ctypes.byref(rel))
        _check(st, allow=(TPSS_OK, TPSS_ENOTCONV))
        return {"outer": o.value, "inner": i.value, "rel_res": rel.value, "converged": st == TPSS_OK}

    def coarse_chebyshev_info(self):
        a, b, m = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        _check(lib().tpss_coarse_chebyshev_info(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(m)))
        return {"a": a.value, "b": b.value, "steps": m.value}
    def pcg_energy_errors(self, b, xs, x, rtol=1e-8, maxit=200):
        """||x_k - xs||_A of the PCG iterates in one run (tpss_pcg_energy_errors)."""
        n = self.ndofs(self.nlevels - 1)
        cnt = ctypes.c_int()
        errs = (ctypes.c_double * (maxit + 1))()
        st = lib().tpss_pcg_energy_errors(self.h, _ptr(b, torch.float64, n), _ptr(xs, torch.float64, n),
                                          _ptr(x, torch.float64, n), rtol, maxit, ctypes.byref(cnt),
                                          ctypes.cast(errs, ctypes.c_void_p))
        _check(st, allow=(TPSS_OK, TPSS_ENOTCONV))
        return list(errs[:cnt.value])

    def pcg_solve(self, b, x, rtol=1e-8, maxit=200, history=False):
        n = self.ndofs(self.nlevels - 1)
        it, rel = ctypes.c_int(), ctypes.c_double()
        hist = (ctypes.c_double * (maxit + 1))() if history else None
        st = lib().tpss_pcg_solve(self.h, _ptr(b, torch.float64, n), _ptr(x, torch.float64, n), rtol, maxit,
                                  ctypes.byref(it), ctypes.byref(rel),
                                  ctypes.cast(hist, ctypes.c_void_p) if hist is not None else None)
        _check(st, allow=(TPSS_OK, TPSS_ENOTCONV))
        out = {"iters": it.value, "rel_res": rel.value, "converged": st == TPSS_OK}
        if history:
            out["history"] = [hist[i] for i in range(it.value + 1)]
        return out


def _gmres(self, b, x, rtol=1e-8, maxit=200, restart=30, history=False, left=False):
    n = self.ndofs(self.nlevels - 1)
    it, rel = ctypes.c_int(), ctypes.c_double()
    hist = (ctypes.c_double * (maxit + 1))() if history else None
    st = lib().tpss_gmres_solve(self.h, _ptr(b, torch.float64, n), _ptr(x, torch.float64, n), rtol, maxit, restart,
                                int(bool(left)), ctypes.byref(it), ctypes.byref(rel),
                                ctypes.cast(hist, ctypes.c_void_p) if hist is not None else None)
    _check(st, allow=(TPSS_OK, TPSS_ENOTCONV))
    out = {"iters": it.value, "rel_res": rel.value, "converged": st == TPSS_OK}
    if history:
        out["history"] = [hist[i] for i in range(it.value + 1)]
    return out


Problem.gmres_solve = _gmres


class Patches:
    """A tpss_patches handle: fast-diagonalization data of one level."""

    def __init__(self, problem, handle, level, kind, precision):
        self.problem, self.h, self.level, self.kind, self.precision = problem, handle, level, kind, precision

    def close(self):
        if getattr(self, "h", None):
            lib().tpss_patches_destroy(self.h)
            self.h = None

    def info(self):
        n, nsub, nc = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int()
        npos = (ctypes.c_int * 3)()
        _check(lib().tpss_patches_info(self.h, ctypes.byref(n), npos, ctypes.byref(nsub), ctypes.byref(nc)))
        return {"n": n.value, "npos": tuple(npos), "nsub": nsub.value, "ncolors_mult": nc.value}

    def eigendata(self, t, pos):
        import numpy as np
        n = self.info()["n"]
        A, M, Z = (np.zeros((n, n)) for _ in range(3))
        lam = np.zeros(n)
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(lib().tpss_patches_eigendata(self.h, t, pos, p(A), p(M), p(Z), p(lam)))
        return A, M, Z, lam

    def set_mult_colors(self, ncolors):
        _check(lib().tpss_patches_set_mult_colors(self.h, ncolors))

    def set_mult_residual(self, mode):
        _check(lib().tpss_patches_set_mult_residual(self.h, mode))

    def set_large_cluster(self, ctas):
        _check(lib().tpss_patches_set_large_cluster(self.h, ctas))

    def set_additive_schedule(self, schedule):
        _check(lib().tpss_patches_set_additive_schedule(self.h, schedule))

    def test_wait_expiry(self):
        _check(lib().tpss_patches_test_wait_expiry(self.h))

    def smooth_additive(self, omega, b, x, x_is_zero=False, nrhs=1):
        n = self.problem.ndofs(self.level) * nrhs
        if self.precision == FP64:
            _check(lib().tpss_smooth_additive(self.h, omega, nrhs, _ptr(b, torch.float64, n), _ptr(x, torch.float64, n),
                                              int(bool(x_is_zero))))
        else:
            _check(lib().tpss_smooth_additive_f32(self.h, omega, nrhs, _ptr(b, torch.float32, n),
                                                  _ptr(x, torch.float32, n), int(bool(x_is_zero))))
        return x

    def smooth_multiplicative(self, omega, b, x, reverse_colors=False, nrhs=1):
        n = self.problem.ndofs(self.level) * nrhs
        if self.precision == FP64:
            _check(lib().tpss_smooth_multiplicative(self.h, omega, int(bool(reverse_colors)), nrhs,
                                                    _ptr(b, torch.float64, n), _ptr(x, torch.float64, n)))
        else:
            _check(lib().tpss_smooth_multiplicative_f32(self.h, omega, int(bool(reverse_colors)), nrhs,
                                                        _ptr(b, torch.float32, n), _ptr(x, torch.float32, n)))
        return x


class Batch:
    """tpss_batch_*: many independent 3D problems (list of (degree, widths,
    nlevels)) with nrhs right-hand sides each, mixed-precision V-cycle with one
    persistent smoother launch per level, optionally graph-captured."""

    def __init__(self, problems, nrhs, omega=0.125, use_graph=True, autotune=True, stream=None,
                 gamma_hat=1.0, penalty_poly=PENALTY_PAPER, precision=FP32, columns=True):
        self._keep = []
        descs = (ProblemDesc * len(problems))()
        for i, (degree, widths, nlevels) in enumerate(problems):
            arrs = [(ctypes.c_double * len(w))(*[float(v) for v in w]) for w in widths]
            self._keep.append(arrs)
            d = descs[i]
            d.dim, d.degree, d.nlevels, d.gamma_hat, d.penalty_poly = 3, degree, nlevels, gamma_hat, penalty_poly
            for t in range(3):
                d.ncells[t] = len(widths[t])
                d.widths[t] = ctypes.cast(arrs[t], ctypes.POINTER(ctypes.c_double))
        p = MGParams()
        p.smoother, p.omega, p.precision, p.mult_colors, p.flexible_cg = AVS, omega, precision, 0, 1
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        flags = (0 if use_graph else 1) | (0 if autotune else 2) | (0 if columns else 4)
        h = ctypes.c_void_p()
        _check(lib().tpss_batch_create(descs, len(problems), nrhs, ctypes.byref(p), flags,
                                       ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.h, self.nprob, self.nrhs = h, len(problems), nrhs
        t, ns, g = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
        _check(lib().tpss_batch_summary(self.h, ctypes.byref(t), ctypes.byref(ns), ctypes.byref(g)))
        self.total, self.nsys, self.uses_graph = t.value, ns.value, bool(g.value)

    def info(self, p):
        n, o, g = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        _check(lib().tpss_batch_info(self.h, p, ctypes.byref(n), ctypes.byref(o), ctypes.byref(g)))
        return {"ndofs": n.value, "offset": o.value, "ppb": g.value}

    def close(self):
        if getattr(self, "h", None):
            lib().tpss_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def smooth_additive(self, b, x):
        _check(lib().tpss_batch_smooth_additive(self.h, _ptr(b, torch.float32, self.total),
                                                _ptr(x, torch.float32, self.total)))
        return x

    def vcycle(self, b, x):
        _check(lib().tpss_batch_vcycle(self.h, _ptr(b, torch.float64, self.total), _ptr(x, torch.float64, self.total)))
        return x

    def pcg_solve(self, b, x, rtol=1e-8, maxit=100):
        import numpy as np
        it = np.zeros(self.nsys, dtype=np.int32)
        rel = np.zeros(self.nsys)
        st = lib().tpss_batch_pcg_solve(self.h, _ptr(b, torch.float64, self.total), _ptr(x, torch.float64, self.total),
                                        rtol, maxit, it.ctypes.data_as(ctypes.c_void_p),
                                        rel.ctypes.data_as(ctypes.c_void_p))
        _check(st, allow=(TPSS_OK, TPSS_ENOTCONV))
        return {"iters": it, "rel_res": rel, "converged": st == TPSS_OK}
