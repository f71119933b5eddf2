"""The allocation-free operator entry point, tpss_apply_operator_noalloc.

It exists for callers that must not cause a device allocation while they run
(their device memory is all held by another allocator, or they sit in a loop
where an allocation and its implied synchronization are not acceptable).  It
must give the same result as tpss_apply_operator, call after call, from its
fixed 16 MiB device array.  This file is collected last on purpose, and it
also passes when run on its own in a fresh process."""
import numpy as np
import pytest
import torch

from gpu_helpers import TOL64, dev, make, rel_err
from paper_1910_11239_gb300 import tpss, workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,k,cells,nrhs", [(3, 3, (6, 5, 4), 2), (2, 5, (9, 7), 3), (3, 1, (4, 4, 4), 1)])
def test_noalloc_matches_apply_operator_on_two_calls(dim, k, cells, nrhs):
    widths = [workloads.widths_random(n, 1, seed=60 + i)[0] for i, n in enumerate(cells)]
    prob = make(dim, k, widths)
    N = prob.ndofs(0)
    u1 = dev(workloads.rhs_uniform(N, seed=1, nrhs=nrhs))
    u2 = dev(workloads.rhs_uniform(N, seed=2, nrhs=nrhs))
    for u in (u1, u2):  # two calls in a row, the second reusing the array left by the first
        ref = torch.empty_like(u)
        got = torch.full_like(u, np.nan)
        prob.apply_operator(0, u, ref, nrhs=nrhs)
        prob.apply_operator_noalloc(0, u, got, nrhs=nrhs)
        torch.cuda.synchronize()
        assert rel_err(got, ref.cpu().numpy()) < TOL64
    prob.close()


def test_noalloc_does_not_grow_device_memory():
    widths = workloads.widths_random(5, 3, seed=3)
    prob = make(3, 2, widths)
    N = prob.ndofs(0)
    u = dev(workloads.rhs_uniform(N, seed=4, nrhs=4))
    out = torch.empty_like(u)
    prob.apply_operator_noalloc(0, u, out, nrhs=4)   # first call on this device: address lookup
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        prob.apply_operator_noalloc(0, u, out, nrhs=4)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    prob.close()


def test_noalloc_rejects_sizes_beyond_its_limit():
    widths = workloads.widths_uniform(16, 3)
    prob = make(3, 3, widths)                        # 16^3 * 64 = 262144 DoFs
    N = prob.ndofs(0)
    u = torch.zeros(N * 3, dtype=torch.float64, device="cuda")
    out = torch.empty_like(u)
    with pytest.raises(tpss.TpssError) as e:
        prob.apply_operator_noalloc(0, u, out, nrhs=3)   # 786432 > 2^19
    assert "exceeds" in str(e.value)
    prob.apply_operator_noalloc(0, u[:2 * N], out[:2 * N], nrhs=2)  # 524288 == 2^19 is allowed
    prob.close()


@pytest.mark.parametrize("dim,k,n0,nrhs", [(2, 3, 64, 3), (3, 2, 14, 1)])
def test_noalloc_on_mapped_meshes_has_no_scratch_limit(dim, k, n0, nrhs):
    # On a mesh of quadrilaterals / hexahedra the operator is one pass with no
    # intermediates: the call must match tpss_apply_operator even where
    # ndofs * nrhs is above the Cartesian scratch limit of 2^19.
    V0 = workloads.vertices_distorted(n0, 7, dim=dim)
    prob = tpss.Problem.mapped(k, V0, nlevels=2, gamma_hat=4.0)
    N = prob.ndofs(1)
    assert N * nrhs > 2 ** 19
    for seed in (1, 2):   # two calls in a row
        u = dev(workloads.rhs_uniform(N, seed=seed, nrhs=nrhs))
        ref = torch.empty_like(u)
        got = torch.full_like(u, np.nan)
        prob.apply_operator(1, u, ref, nrhs=nrhs)
        prob.apply_operator_noalloc(1, u, got, nrhs=nrhs)
        torch.cuda.synchronize()
        assert rel_err(got, ref.cpu().numpy()) < TOL64
    prob.close()
