"""Chebyshev iteration with an SPD preconditioner: the coarse-level solver of
Sec. 2.4 (relative accuracy 1e-8, the additive cell smoother as
preconditioner), written from the textbook method the paper cites (Varga).

Test infrastructure only (see the package docstring).

The paper states neither how the spectral interval of the preconditioned
operator P A is found nor how the iteration is stopped.  Reading taken:
  * start vector: s_i = SplitMix64(i) mapped to [-1, 1) (the generator of
    Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
    OOPSLA 2014: state += 0x9E3779B97F4A7C15, then two xor-shift-multiply
    rounds), the same definition on both sides;
  * bounds: m_L = min(n, 50) steps of preconditioned CG on A y = s from
    y = 0; the Lanczos matrix T of P A follows from the CG coefficients
    (T_00 = 1/alpha_0, T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},
    T_{j,j+1} = sqrt(beta_j)/alpha_j); its extreme eigenvalues (Ritz values,
    inside the spectrum) are widened to [a, b] = [0.8 theta_min,
    1.1 theta_max];
  * iteration count: the smallest m with 2 q^m / (1 + q^(2m)) <= tol,
    q = (sqrt(kappa) - 1) / (sqrt(kappa) + 1), kappa = b / a (the Chebyshev
    bound on the error reduction in the A-norm over [a, b]); no residual is
    monitored.
Recurrence (x_0 = 0):
    theta = (b + a)/2, delta = (b - a)/2, sigma = theta/delta, rho_0 = 1/sigma
    r_0 = f, d_0 = P r_0 / theta
    x_{k+1} = x_k + d_k,  r_{k+1} = f - A x_{k+1}
    rho_{k+1} = 1/(2 sigma - rho_k)
    d_{k+1} = rho_{k+1} rho_k d_k + (2 rho_{k+1} / delta) P r_{k+1}
so that x_m - x* = p_m(P A)(x_0 - x*) with p_m(t) = T_m((theta - t)/delta) /
T_m(theta/delta).

Pins (tests/test_oracle_chebyshev.py): the error after m steps on a diagonal
system equals p_m(lambda_i) e_0 entry by entry (closed form of the Chebyshev
polynomial); the Ritz values from the CG coefficients equal those of an
explicit Lanczos process with full reorthogonalization; the a-priori count
reaches the requested A-norm reduction; SplitMix64 reproduces the published
reference outputs for seed 0.
"""
import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64(i):
    """Output number i (i = 0, 1, ...) of SplitMix64 started from state 0."""
    z = ((i + 1) * 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def start_vector(n):
    """s_i = top 53 bits of SplitMix64(i) as a double in [0, 1), mapped to [-1, 1)."""
    return np.array([2.0 * ((splitmix64(i) >> 11) * 2.0 ** -53) - 1.0 for i in range(n)])


def lanczos_from_cg(A, precondition, s, steps):
    """Run `steps` steps of preconditioned CG on A y = s from y = 0 and return
    the Lanczos tridiagonal matrix of P A built from its coefficients."""
    r = s.copy()
    z = precondition(r)
    p = z.copy()
    rz = r @ z
    alphas, betas = [], []
    for _ in range(steps):
        q = A @ p
        pq = p @ q
        if pq <= 0.0:
            break
        alpha = rz / pq
        r = r - alpha * q
        z = precondition(r)
        rz_new = r @ z
        alphas.append(alpha)
        betas.append(rz_new / rz)
        if rz_new <= 0.0:
            break
        p = z + (rz_new / rz) * p
        rz = rz_new
    m = len(alphas)
    T = np.zeros((m, m))
    for j in range(m):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < m:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(betas[j]) / alphas[j]
    return T


def spectral_bounds(A, precondition, n, steps=50, lo=0.8, hi=1.1):
    steps = min(n, steps)
    T = lanczos_from_cg(A, precondition, start_vector(n), steps)
    ev = np.linalg.eigvalsh(T)
    return lo * ev[0], hi * ev[-1]


def iteration_count(a, b, tol=1e-8):
    kappa = b / a
    q = (np.sqrt(kappa) - 1.0) / (np.sqrt(kappa) + 1.0)
    m = 0
    while 2.0 * q ** m / (1.0 + q ** (2 * m)) > tol:
        m += 1
    return m


def chebyshev(A, f, precondition, a, b, m):
    """m steps of the preconditioned Chebyshev iteration from x_0 = 0."""
    theta, delta = 0.5 * (b + a), 0.5 * (b - a)
    sigma = theta / delta
    rho = 1.0 / sigma
    x = np.zeros_like(f)
    d = precondition(f) / theta
    for _ in range(m):
        x = x + d
        r = f - A @ x
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * precondition(r)
        rho = rho_new
    return x
