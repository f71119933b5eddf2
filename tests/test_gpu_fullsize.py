"""Full-size parity for the benchmark workloads, in the launch configuration
the benchmark times, on outputs the oracle can compute one by one.

3D additive vertex-patch smoother on a 32^3 tensor grid with per-direction
widths U[0.5, 1.5]/32 (seed 2), omega = 0.7, 8 right-hand sides U[-1, 1]
(seeds 100..107) in one batched call, k = 2..7.  For sampled cells K the
oracle evaluates x_K = omega sum_{j containing K} (A_j^{-1} R_j b)_K with
A_j = R_j A R_j^T assembled from the bilinear form and solved by dense LU."""
import numpy as np
import pytest
import scipy.linalg as sla
import torch

from gpu_helpers import TOL64, dev, make, rel_err
from oracle import schwarz
from oracle.mesh import TensorMesh
from oracle.sipg import SIPG
from paper_1910_11239_gb300 import workloads

pytestmark = pytest.mark.gpu

NC = 32
SEEDS = list(range(100, 108))


def patches_containing(mesh, c):
    m = mesh.cell_multi(c)
    out = []
    for s in np.ndindex(*(2,) * mesh.d):
        v = [m[t] + s[t] for t in range(mesh.d)]  # vertex index: cell is at v-1 or v
        if all(1 <= v[t] <= mesh.ncells[t] - 1 for t in range(mesh.d)):
            cells = [mesh.cell_index([v[t] - 1 + q[t] for t in range(mesh.d)])
                     for q in [tuple(reversed(r)) for r in np.ndindex(*(2,) * mesh.d)]]
            out.append(cells)
    return out


@pytest.mark.parametrize("k", [2, 3, 4, 5, 6, 7])
def test_avs_32cubed_sampled(k):
    from paper_1910_11239_gb300 import tpss
    widths = workloads.widths_random(NC, 3, seed=2)
    prob = make(3, k, widths)
    P = prob.setup_patches(0, tpss.VERTEX_PATCH)
    N = prob.ndofs(0)
    b = workloads.rhs_batch(N, SEEDS)
    x = torch.empty(N * len(SEEDS), dtype=torch.float64, device="cuda")
    P.smooth_additive(0.7, dev(b), x, x_is_zero=True, nrhs=len(SEEDS))
    xh = x.cpu().numpy()
    assert np.isfinite(xh).all()
    mesh = TensorMesh(widths)
    S = SIPG(mesh, k)
    nloc = S.nloc
    sample = [mesh.cell_index([13, 17, 9]), mesh.cell_index([0, 0, 0])]
    if k <= 3:
        sample += [mesh.cell_index([31, 5, 0]), mesh.cell_index([16, 31, 20])]
    for c in sample:
        ref = np.zeros((len(SEEDS), nloc))
        for cells in patches_containing(mesh, c):
            lu = sla.lu_factor(S.assemble(cells).toarray())
            idx = schwarz.patch_dofs(cells, nloc)
            pos = cells.index(c)
            for r in range(len(SEEDS)):
                y = sla.lu_solve(lu, b[r * N + idx])
                ref[r] += 0.7 * y[pos * nloc:(pos + 1) * nloc]
        for r in range(len(SEEDS)):
            got = xh[r * N + c * nloc: r * N + (c + 1) * nloc]
            assert rel_err(got, ref[r]) < TOL64, (k, c, r)
    prob.close()
