/* Additive Schwarz local solves by fast diagonalization on the CPU, FP64.
 *
 * TEST INFRASTRUCTURE ONLY (part of the oracle package): it is the timed CPU
 * baseline of the smoother and is checked against the dense-LU oracle by the
 * tests; the product library never links or calls it.
 *
 * What it computes (Sec. 3.2, eq. fastinverse with eq. generalizedEVP, and the
 * additive sum of eq. additiveschwarz / Alg. 2 with x = 0):
 *
 *     y = omega * sum_j R_j^T  A_j^{-1}  R_j r,
 *     A_j^{-1} = (Z_d (x) ... (x) Z_1) diag(1 / (lambda_1 + ... + lambda_d)) (Z_d (x) ... (x) Z_1)^T,
 *
 * for the subspaces j of a d-dimensional Cartesian tensor mesh: either cells
 * (n = k+1 points per direction) or vertex patches of 2^d cells around an
 * interior vertex (n = 2(k+1)).  Z_t and lambda_t are the 1D generalized
 * eigenpairs A_t z = lambda M_t z (Z_t^T M_t Z_t = I) of the subspace's
 * direction-t factor; they are inputs (computed by oracle/fastdiag.py).
 *
 * Each local solve is written out step by step: gather R_j r into an n^d
 * tensor, apply Z_t^T along every direction t, divide by the eigenvalue
 * sums, apply Z_t along every direction, add omega times the result back.
 * Vertex patches of one parity color (v_t mod 2) share no cell, so the
 * patches of a color are solved in parallel (OpenMP) and the colors one
 * after another; cells never overlap.
 *
 * Layouts: DoF vectors are cell-major, cells lexicographic (first direction
 * fastest), (k+1)^d nodal values per cell (first direction fastest), nrhs
 * vectors back to back.  Z[t] holds npos[t] matrices of n x n, row-major,
 * Z[t][p][i * n + a] = entry (i, a) (column a = eigenvector a); lam[t] holds
 * npos[t] vectors of n eigenvalues.  npos[t] = ncells[t] - 1 (vertex) or
 * ncells[t] (cells).  color_mask selects the subspaces solved: bit c set
 * solves the vertex patches of additive color c = sum_t (v_t mod 2) 2^t
 * (all of them: (1 << 2^d) - 1); for cells any nonzero mask solves all.  y
 * is overwritten (zero where no selected subspace reaches).  Returns 0, or -1
 * on bad arguments.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* u <- (I (x) .. (x) X^(T) (x) .. (x) I) u along direction t of an n^d tensor
 * (index i_0 + n i_1 + n^2 i_2), with X = Z (transpose = 0: out_i = sum_a Z_ia u_a)
 * or X = Z^T (transpose = 1: out_a = sum_i Z_ia u_i). */
static void apply_dir(int d, int n, int t, const double* Z, int transpose, const double* u, double* out) {
  int64_t total = 1;
  for (int s = 0; s < d; ++s) total *= n;
  int64_t stride = 1;
  for (int s = 0; s < t; ++s) stride *= n;
  for (int64_t e = 0; e < total; ++e) {
    const int64_t it = (e / stride) % n;      /* index along t of the output entry */
    const int64_t base = e - it * stride;     /* same entry with index 0 along t */
    double acc = 0.0;
    for (int m = 0; m < n; ++m) {
      const double z = transpose ? Z[m * n + it] : Z[it * n + m];
      acc += z * u[base + m * stride];
    }
    out[e] = acc;
  }
}

int fd_additive_local_sum(int d, int k, int vertex, const int* ncells, const double* const* Z,
                          const double* const* lam, double omega, int nrhs, const double* r, double* y,
                          int color_mask, int nthreads) {
  if (d < 1 || d > 3 || k < 1 || nrhs < 1 || !ncells || !Z || !lam || !r || !y) return -1;
  const int n1 = k + 1;
  const int n = vertex ? 2 * n1 : n1;
  int64_t nloc = 1, ncell_total = 1;
  int npos[3] = {1, 1, 1};
  for (int t = 0; t < d; ++t) {
    if (ncells[t] < (vertex ? 2 : 1)) return -1;
    nloc *= n1;
    ncell_total *= ncells[t];
    npos[t] = vertex ? ncells[t] - 1 : ncells[t];
  }
  const int64_t N = ncell_total * nloc;
  int64_t nsub = 1, tens = 1;
  for (int t = 0; t < d; ++t) {
    nsub *= npos[t];
    tens *= n;
  }
  memset(y, 0, sizeof(double) * (size_t)(N * nrhs));
#ifdef _OPENMP
  const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
#endif
  const int ncolors = vertex ? (1 << d) : 1;
  for (int color = 0; color < ncolors; ++color) {
    if (!(color_mask & (1 << color))) continue;
#pragma omp parallel num_threads(nt)
    {
      double* u = (double*)malloc(sizeof(double) * (size_t)tens);
      double* w = (double*)malloc(sizeof(double) * (size_t)tens);
#pragma omp for schedule(dynamic, 4)
      for (int64_t j = 0; j < nsub; ++j) {
        int p[3] = {0, 0, 0};
        int64_t rest = j;
        for (int t = 0; t < d; ++t) {
          p[t] = (int)(rest % npos[t]);
          rest /= npos[t];
        }
        if (vertex) {   /* vertex v_t = p_t + 1; additive color = parity bits of v */
          int c = 0;
          for (int t = 0; t < d; ++t) c |= ((p[t] + 1) & 1) << t;
          if (c != color) continue;
        }
        for (int rhs = 0; rhs < nrhs; ++rhs) {
          const double* rr = r + rhs * N;
          double* yy = y + rhs * N;
          /* gather R_j r: local index i_t = s_t n1 + a_t (s_t = which cell along t) */
          for (int64_t e = 0; e < tens; ++e) {
            int64_t q = e, cell = 0, cstride = 1, dof = 0, dstride = 1;
            for (int t = 0; t < d; ++t) {
              const int it = (int)(q % n);
              q /= n;
              const int s = it / n1, a = it % n1;
              cell += (int64_t)(p[t] + s) * cstride;
              cstride *= ncells[t];
              dof += a * dstride;
              dstride *= n1;
            }
            u[e] = rr[cell * nloc + dof];
          }
          /* Z^T along every direction */
          for (int t = 0; t < d; ++t) {
            apply_dir(d, n, t, Z[t] + (int64_t)p[t] * n * n, 1, u, w);
            double* tmp = u; u = w; w = tmp;
          }
          /* divide by the eigenvalue sums */
          for (int64_t e = 0; e < tens; ++e) {
            int64_t q = e;
            double s = 0.0;
            for (int t = 0; t < d; ++t) {
              s += lam[t][(int64_t)p[t] * n + (q % n)];
              q /= n;
            }
            u[e] /= s;
          }
          /* Z along every direction */
          for (int t = 0; t < d; ++t) {
            apply_dir(d, n, t, Z[t] + (int64_t)p[t] * n * n, 0, u, w);
            double* tmp = u; u = w; w = tmp;
          }
          /* y += omega R_j^T u */
          for (int64_t e = 0; e < tens; ++e) {
            int64_t q = e, cell = 0, cstride = 1, dof = 0, dstride = 1;
            for (int t = 0; t < d; ++t) {
              const int it = (int)(q % n);
              q /= n;
              const int s = it / n1, a = it % n1;
              cell += (int64_t)(p[t] + s) * cstride;
              cstride *= ncells[t];
              dof += a * dstride;
              dstride *= n1;
            }
            yy[cell * nloc + dof] += omega * u[e];
          }
        }
      }
      free(u);
      free(w);
    }
  }
  return 0;
}

int fd_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
