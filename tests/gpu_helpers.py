"""Helpers shared by the GPU parity tests: build the CUDA problem and the
oracle for the same seeded mesh and compare element by element."""
import numpy as np
import torch

from oracle import schwarz
from oracle.mesh import TensorMesh
from oracle.sipg import SIPG

# FP64 parity bar: relative max-norm error (max |gpu - oracle| / max |oracle|)
TOL64 = 1e-12


def rel_err(gpu, ref):
    gpu = gpu.detach().cpu().numpy() if isinstance(gpu, torch.Tensor) else np.asarray(gpu)
    ref = np.asarray(ref)
    return float(np.abs(gpu - ref).max() / max(np.abs(ref).max(), 1e-300))


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def make(dim, degree, widths, nlevels=1, penalty="paper", gamma_hat=1.0):
    from paper_1910_11239_gb300 import tpss
    pp = tpss.PENALTY_PAPER if penalty == "paper" else tpss.PENALTY_KP1SQ
    prob = tpss.Problem(dim, degree, widths, nlevels=nlevels, gamma_hat=gamma_hat, penalty_poly=pp)
    return prob


def oracle_sipg(widths, degree, penalty="paper", gamma_hat=1.0):
    return SIPG(TensorMesh(widths), degree, gamma_hat=gamma_hat, penalty_poly=penalty)


def oracle_solvers(S, A, kind):
    patches = schwarz.vertex_patches(S.mesh) if kind == "vertex" else schwarz.cell_patches(S.mesh)

    def local(cells):
        idx = schwarz.patch_dofs(cells, S.nloc)
        return A[idx][:, idx]

    return patches, schwarz.LocalSolvers(patches, S.nloc, local)


def paper_value(key):
    """A value printed in the paper, from tests/golden/paper_tables.txt."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.txt")
    for line in open(path):
        parts = line.split()
        if parts and not line.startswith("#") and parts[0] == key:
            return float(parts[1])
    raise KeyError(key)
