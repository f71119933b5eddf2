"""GPU setup parity: the device-computed 1D matrices reproduce the oracle's
assembled local matrices through the Kronecker sum (eq. KDseparable), and the
device eigenpairs satisfy eq. generalizedEVP and invert the oracle's local
matrices (eq. fastinverse)."""
import numpy as np
import pytest

from gpu_helpers import make, oracle_sipg
from oracle import schwarz
from paper_1910_11239_gb300 import workloads

pytestmark = pytest.mark.gpu


def kron_sum(As, Ms):
    d = len(As)
    total = 0
    for t in range(d):
        f = None
        for s in reversed(range(d)):
            m = As[s] if s == t else Ms[s]
            f = m if f is None else np.kron(f, m)
        total = total + f
    return total


def patch_perm(k, d, vertex):
    n1 = k + 1
    n = 2 * n1 if vertex else n1
    perm = np.zeros(n ** d, dtype=int)
    for p in range(n ** d):
        pm = [(p // n ** t) % n for t in range(d)]
        c = [pm[t] // n1 for t in range(d)]
        i = [pm[t] % n1 for t in range(d)]
        perm[p] = sum(c[t] << t for t in range(d)) * n1 ** d + sum(i[t] * n1 ** t for t in range(d))
    return perm


@pytest.mark.parametrize("dim,k,n", [(2, 1, 4), (2, 4, 3), (3, 2, 4), (3, 3, 3), (3, 7, 2)])
@pytest.mark.parametrize("vertex", [True, False])
@pytest.mark.parametrize("penalty", ["paper", "kp1sq"])
def test_kronecker_and_eigenpairs(dim, k, n, vertex, penalty):
    from paper_1910_11239_gb300 import tpss
    widths = workloads.widths_random(n, dim, seed=40 + dim * 10 + k)
    prob = make(dim, k, widths, penalty=penalty)
    P = prob.setup_patches(0, tpss.VERTEX_PATCH if vertex else tpss.CELL)
    S = oracle_sipg(widths, k, penalty=penalty)
    perm = patch_perm(k, dim, vertex)
    subs = schwarz.vertex_patches(S.mesh) if vertex else schwarz.cell_patches(S.mesh)
    rng = np.random.default_rng(0)
    for j in rng.choice(len(subs), size=min(4, len(subs)), replace=False):
        v, cells = subs[j]
        pos = [v[t] - 1 for t in range(dim)] if vertex else list(v)
        As, Ms, Zs, lams = [], [], [], []
        for t in range(dim):
            A, M, Z, lam = P.eigendata(t, pos[t])
            # eq. generalizedEVP
            assert np.abs(Z.T @ M @ Z - np.eye(len(lam))).max() < 1e-12
            assert np.abs(Z.T @ A @ Z - np.diag(lam)).max() < 1e-12 * np.abs(lam).max()
            assert lam.min() > 0
            As.append(A); Ms.append(M); Zs.append(Z); lams.append(lam)
        Aj = S.assemble(cells).toarray()[np.ix_(perm, perm)]
        K = kron_sum(As, Ms)
        assert np.abs(K - Aj).max() <= 1e-12 * np.abs(Aj).max()
        # eq. fastinverse: Z Lambda^{-1} Z^T == A_j^{-1}
        Z = Zs[-1]
        for t in reversed(range(dim - 1)):
            Z = np.kron(Z, Zs[t])
        lam = np.zeros(1)
        for t in reversed(range(dim)):
            lam = np.add.outer(lam, lams[t]).ravel()
        inv_fd = (Z / lam) @ Z.T
        inv = np.linalg.inv(Aj)
        assert np.abs(inv_fd - inv).max() <= 1e-10 * np.abs(inv).max()
    prob.close()
