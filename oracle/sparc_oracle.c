/*
 * CPU oracle for one CheFSI step (test infrastructure only).
 *
 * This file is the plain, slow FP64 reference that the CUDA library is checked
 * against.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline use it; the product path never links or calls it, and it shares no
 * code, header or table with the CUDA sources.
 *
 * Every routine follows the paper's Algorithm 1 (CheFSI-based partial
 * diagonalisation) in its stated order: Chebyshev filtering, projection,
 * subspace diagonalisation, rotation, with the matrix-free Hamiltonian of
 * Sec. II A (finite-difference Laplacian, pointwise Veff, per-atom nonlocal
 * projectors).  Loops are written straight from the definitions; sums run in
 * natural index order; OpenMP only splits independent outputs (orbitals or
 * matrix entries), so results do not depend on the thread count.
 *
 * Readings of points the paper leaves open (documented with the project):
 *  - FD order n0 = 12 (radius 6), central second-derivative weights.
 *  - Periodic axes wrap modulo N; Dirichlet axes have zero ghost values.
 *  - Nonlocal term sum_J chi_J Gamma_J h^3 chi_J^T X (quadrature weight h^3).
 *  - Filter in the scaled three-term form of Zhou et al. (cited by the paper
 *    for CheFSI); it equals the paper's p_m((H - cI)/e) X divided by the scalar
 *    p_m((a0 - c)/e), so the Ritz pairs are identical under either form.
 *  - Lanczos bounds: b = theta_max + |beta_k|, a0 = theta_min, start vector
 *    from the counter-based splitmix64 generator.
 *  - Generalised eigensolve by Cholesky reduction, Householder
 *    tridiagonalisation and implicit-shift QR; eigenvalues ascending, each
 *    eigenvector's largest-magnitude entry made positive.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_NOT_SPD 4
#define OR_ERR_NUMERIC 5

#define FD_RADIUS 6

typedef struct {
  int nx, ny, nz;
  double h;
  int bc[3]; /* 0 periodic, 1 Dirichlet */
  long nd;
  double* veff;
  int natoms;
  long* supp_ptr;
  int* supp_idx;
  int* nproj;
  long* chi_ptr;
  double* chi;
  long* proj_ptr;
  double* gamma;
  double w[FD_RADIUS + 1];
} or_system;

/* ------------------------------------------------------------------------ */
/* FD weights (Sec. II A names the order n0 only; 12th order is used here).  */
/* Central second-derivative weights of radius n:                            */
/*   w_p = 2 (-1)^(p+1) (n!)^2 / (p^2 (n-p)! (n+p)!),  p = 1..n,              */
/*   w_0 = -2 sum_p w_p   (the weights of a derivative sum to zero).          */
/* ------------------------------------------------------------------------ */
void or_fd_weights(int n, double* w) {
  double nf = 1.0;
  for (int i = 2; i <= n; ++i) nf *= i;
  double s = 0.0;
  for (int p = 1; p <= n; ++p) {
    double a = 1.0, b = 1.0;
    for (int i = 2; i <= n - p; ++i) a *= i;
    for (int i = 2; i <= n + p; ++i) b *= i;
    double sign = (p % 2 == 1) ? 1.0 : -1.0;
    w[p] = 2.0 * sign * nf * nf / ((double)p * p * a * b);
    s += w[p];
  }
  w[0] = -2.0 * s;
}

or_system* or_create(int nx, int ny, int nz, double h, const int* bc, const double* veff,
                     int natoms, const long* supp_ptr, const int* supp_idx, const int* nproj,
                     const long* chi_ptr, const double* chi, const long* proj_ptr,
                     const double* gamma) {
  or_system* s = (or_system*)calloc(1, sizeof(or_system));
  s->nx = nx; s->ny = ny; s->nz = nz; s->h = h;
  for (int d = 0; d < 3; ++d) s->bc[d] = bc[d];
  s->nd = (long)nx * ny * nz;
  s->veff = (double*)malloc(sizeof(double) * s->nd);
  memcpy(s->veff, veff, sizeof(double) * s->nd);
  s->natoms = natoms;
  s->supp_ptr = (long*)malloc(sizeof(long) * (natoms + 1));
  s->chi_ptr = (long*)malloc(sizeof(long) * (natoms + 1));
  s->proj_ptr = (long*)malloc(sizeof(long) * (natoms + 1));
  memcpy(s->supp_ptr, supp_ptr, sizeof(long) * (natoms + 1));
  memcpy(s->chi_ptr, chi_ptr, sizeof(long) * (natoms + 1));
  memcpy(s->proj_ptr, proj_ptr, sizeof(long) * (natoms + 1));
  long nsupp = supp_ptr[natoms], nchi = chi_ptr[natoms], nprj = proj_ptr[natoms];
  s->supp_idx = (int*)malloc(sizeof(int) * (nsupp > 0 ? nsupp : 1));
  s->chi = (double*)malloc(sizeof(double) * (nchi > 0 ? nchi : 1));
  s->gamma = (double*)malloc(sizeof(double) * (nprj > 0 ? nprj : 1));
  s->nproj = (int*)malloc(sizeof(int) * (natoms > 0 ? natoms : 1));
  if (nsupp) memcpy(s->supp_idx, supp_idx, sizeof(int) * nsupp);
  if (nchi) memcpy(s->chi, chi, sizeof(double) * nchi);
  if (nprj) memcpy(s->gamma, gamma, sizeof(double) * nprj);
  if (natoms) memcpy(s->nproj, nproj, sizeof(int) * natoms);
  or_fd_weights(FD_RADIUS, s->w);
  return s;
}

void or_destroy(or_system* s) {
  if (!s) return;
  free(s->veff); free(s->supp_ptr); free(s->supp_idx); free(s->nproj);
  free(s->chi_ptr); free(s->chi); free(s->proj_ptr); free(s->gamma);
  free(s);
}

/* Value of orbital column x at grid point (i, j, k) with boundary handling. */
static double or_at(const or_system* s, const double* x, int i, int j, int k) {
  int n[3] = {s->nx, s->ny, s->nz};
  int c[3] = {i, j, k};
  for (int d = 0; d < 3; ++d) {
    if (c[d] < 0 || c[d] >= n[d]) {
      if (s->bc[d] == 1) return 0.0;
      c[d] = ((c[d] % n[d]) + n[d]) % n[d];
    }
  }
  return x[c[0] + (long)s->nx * (c[1] + (long)s->ny * c[2])];
}

/* Y = H X for ns columns: H = -1/2 Lap + Veff + sum_J chi_J Gamma_J h^3 chi_J^T (Sec. II A). */
void or_hpsi(const or_system* s, const double* X, long ldx, double* Y, long ldy, int ns) {
  const double h2 = s->h * s->h, h3 = s->h * s->h * s->h;
#pragma omp parallel for schedule(dynamic, 1)
  for (int n = 0; n < ns; ++n) {
    const double* x = X + (long)n * ldx;
    double* y = Y + (long)n * ldy;
    /* local part: -1/2 Laplacian plus Veff */
    for (int k = 0; k < s->nz; ++k)
      for (int j = 0; j < s->ny; ++j)
        for (int i = 0; i < s->nx; ++i) {
          double lap = 0.0;
          double xc = or_at(s, x, i, j, k);
          for (int d = 0; d < 3; ++d) {
            double acc = s->w[0] * xc;
            for (int p = 1; p <= FD_RADIUS; ++p) {
              int ip = i, jp = j, kp = k, im = i, jm = j, km = k;
              if (d == 0) { ip += p; im -= p; }
              if (d == 1) { jp += p; jm -= p; }
              if (d == 2) { kp += p; km -= p; }
              acc += s->w[p] * (or_at(s, x, ip, jp, kp) + or_at(s, x, im, jm, km));
            }
            lap += acc / h2;
          }
          long g = i + (long)s->nx * (j + (long)s->ny * k);
          y[g] = -0.5 * lap + s->veff[g] * xc;
        }
    /* nonlocal part: per atom, c = h^3 chi^T x, then y += chi Gamma c */
    for (int J = 0; J < s->natoms; ++J) {
      long p0 = s->supp_ptr[J], np_ = s->supp_ptr[J + 1] - p0;
      const double* chi = s->chi + s->chi_ptr[J];
      const double* gam = s->gamma + s->proj_ptr[J];
      for (int q = 0; q < s->nproj[J]; ++q) {
        const double* col = chi + (long)q * np_;
        double c = 0.0;
        for (long t = 0; t < np_; ++t) c += col[t] * x[s->supp_idx[p0 + t]];
        c *= h3 * gam[q];
        for (long t = 0; t < np_; ++t) y[s->supp_idx[p0 + t]] += col[t] * c;
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Chebyshev filter (Algorithm 1, "Filtering"), scaled three-term form.     */
/*   e = (b - a)/2, c = (b + a)/2, sigma_1 = e/(a0 - c), tau = 2/sigma_1     */
/*   Y_1 = (sigma_1/e)(H - c) X                                              */
/*   sigma_{i+1} = 1/(tau - sigma_i)                                         */
/*   Y_{i+1} = (2 sigma_{i+1}/e)(H - c) Y_i - sigma_i sigma_{i+1} Y_{i-1}    */
/* Output Y_m = T_m((H - c)/e) X / T_m((a0 - c)/e), written over X.          */
/* ------------------------------------------------------------------------ */
int or_cheb_filter(const or_system* s, double* X, long ld, int ns, int m, double a, double b,
                   double a0) {
  if (m < 1 || !(a0 < a) || !(a < b)) return OR_ERR_ARG;
  long nd = s->nd;
  double e = (b - a) / 2.0, c = (b + a) / 2.0;
  double sigma = e / (a0 - c), sigma1 = sigma, tau = 2.0 / sigma1;
  double* prev = (double*)malloc(sizeof(double) * nd * ns);
  double* cur = (double*)malloc(sizeof(double) * nd * ns);
  double* hy = (double*)malloc(sizeof(double) * nd * ns);
  for (int n = 0; n < ns; ++n) memcpy(prev + (long)n * nd, X + (long)n * ld, sizeof(double) * nd);
  or_hpsi(s, prev, nd, hy, nd, ns);
  for (long t = 0; t < nd * ns; ++t) cur[t] = (hy[t] - c * prev[t]) * (sigma1 / e);
  for (int i = 2; i <= m; ++i) {
    double sigma_new = 1.0 / (tau - sigma);
    or_hpsi(s, cur, nd, hy, nd, ns);
    for (long t = 0; t < nd * ns; ++t) {
      double next = (hy[t] - c * cur[t]) * (2.0 * sigma_new / e) - sigma * sigma_new * prev[t];
      prev[t] = cur[t];
      cur[t] = next;
    }
    sigma = sigma_new;
  }
  for (int n = 0; n < ns; ++n) memcpy(X + (long)n * ld, cur + (long)n * nd, sizeof(double) * nd);
  free(prev); free(cur); free(hy);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* splitmix64 (Steele, Lea & Flood 2014) as a counter-based generator:       */
/* value i of stream `seed` is the splitmix64 output for state               */
/* seed + (i + 1) * 0x9E3779B97F4A7C15, mapped to [0,1) by its top 53 bits.  */
/* ------------------------------------------------------------------------ */
static uint64_t or_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

double or_uniform(uint64_t seed, uint64_t i) {
  uint64_t z = or_mix64(seed + (i + 1) * 0x9E3779B97F4A7C15ULL);
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

static double or_dot(const double* u, const double* v, long n) {
  double s = 0.0;
  for (long t = 0; t < n; ++t) s += u[t] * v[t];
  return s;
}

/* ------------------------------------------------------------------------ */
/* Implicit-shift symmetric tridiagonal QR (Golub & Van Loan, Sec. 8.3).    */
/* d[0..n-1] diagonal, e[0..n-2] off-diagonal (destroyed).  If z != NULL the */
/* Givens rotations are accumulated into the columns of the n x n column-    */
/* major matrix z (ldz).  Returns 0, or OR_ERR_NUMERIC if it fails to        */
/* converge.  Eigenvalues are left unsorted in d.                            */
/* ------------------------------------------------------------------------ */
int or_tridiag_qr(int n, double* d, double* e, double* z, int ldz, int zrows) {
  const double eps = 2.220446049250313e-16;
  long iters = 0, max_iters = 60L * n + 60;
  int hi = n - 1;
  while (hi > 0) {
    /* deflate negligible off-diagonals */
    for (int i = 0; i < hi; ++i)
      if (fabs(e[i]) <= eps * (fabs(d[i]) + fabs(d[i + 1]))) e[i] = 0.0;
    while (hi > 0 && e[hi - 1] == 0.0) --hi;
    if (hi == 0) break;
    int lo = hi - 1;
    while (lo > 0 && e[lo - 1] != 0.0) --lo;
    if (++iters > max_iters) return OR_ERR_NUMERIC;
    /* Wilkinson shift from the trailing 2x2 block of the unreduced block [lo, hi] */
    double dd = 0.5 * (d[hi - 1] - d[hi]);
    double bb = e[hi - 1];
    double sg = dd >= 0.0 ? 1.0 : -1.0;
    double mu = d[hi] - bb * bb / (dd + sg * hypot(dd, bb));
    double x = d[lo] - mu, y = e[lo], bulge = 0.0;
    for (int k = lo; k < hi; ++k) {
      double r = hypot(x, y);
      double c = r == 0.0 ? 1.0 : x / r;
      double s = r == 0.0 ? 0.0 : -y / r;
      if (k > lo) e[k - 1] = c * e[k - 1] - s * bulge;
      double p = d[k], q = d[k + 1], t = e[k];
      d[k] = c * c * p - 2.0 * c * s * t + s * s * q;
      d[k + 1] = s * s * p + 2.0 * c * s * t + c * c * q;
      e[k] = c * s * (p - q) + (c * c - s * s) * t;
      if (k + 1 < hi) {
        bulge = -s * e[k + 1];
        e[k + 1] = c * e[k + 1];
      }
      if (z) {
        double* zk = z + (long)k * ldz;
        double* zk1 = z + (long)(k + 1) * ldz;
        for (int r2 = 0; r2 < zrows; ++r2) {
          double u = zk[r2], v = zk1[r2];
          zk[r2] = c * u - s * v;
          zk1[r2] = s * u + c * v;
        }
      }
      x = e[k];
      y = bulge;
    }
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Lanczos estimate of the spectrum ends (bounds used by the filter).       */
/*   v_0 random (splitmix64, uniform in [-1/2, 1/2)), normalised;            */
/*   w = H v_j - beta_j v_{j-1}; alpha_j = w.v_j; w -= alpha_j v_j;          */
/*   beta_{j+1} = |w|; v_{j+1} = w / beta_{j+1}.                             */
/* theta_min/theta_max are the extreme eigenvalues of the k x k tridiagonal; */
/* the upper bound is b = theta_max + beta_k.                                */
/* ------------------------------------------------------------------------ */
int or_lanczos(const or_system* s, int k, uint64_t seed, double* alpha, double* beta,
               double* theta_min, double* theta_max, double* b_upper) {
  long nd = s->nd;
  if (k < 1) return OR_ERR_ARG;
  double* v = (double*)malloc(sizeof(double) * nd);
  double* vp = (double*)calloc(nd, sizeof(double));
  double* w = (double*)malloc(sizeof(double) * nd);
  for (long t = 0; t < nd; ++t) v[t] = or_uniform(seed, (uint64_t)t) - 0.5;
  double nrm = sqrt(or_dot(v, v, nd));
  for (long t = 0; t < nd; ++t) v[t] /= nrm;
  double bprev = 0.0;
  for (int j = 0; j < k; ++j) {
    or_hpsi(s, v, nd, w, nd, 1);
    for (long t = 0; t < nd; ++t) w[t] -= bprev * vp[t];
    double al = or_dot(w, v, nd);
    for (long t = 0; t < nd; ++t) w[t] -= al * v[t];
    double bt = sqrt(or_dot(w, w, nd));
    alpha[j] = al;
    beta[j] = bt; /* beta[j] couples v_j and v_{j+1} */
    for (long t = 0; t < nd; ++t) {
      vp[t] = v[t];
      v[t] = bt > 0.0 ? w[t] / bt : 0.0;
    }
    bprev = bt;
  }
  double* d = (double*)malloc(sizeof(double) * k);
  double* e = (double*)malloc(sizeof(double) * (k > 1 ? k : 1));
  memcpy(d, alpha, sizeof(double) * k);
  for (int j = 0; j + 1 < k; ++j) e[j] = beta[j];
  int st = or_tridiag_qr(k, d, e, NULL, 0, 0);
  double lo = d[0], hi = d[0];
  for (int j = 1; j < k; ++j) {
    if (d[j] < lo) lo = d[j];
    if (d[j] > hi) hi = d[j];
  }
  *theta_min = lo;
  *theta_max = hi;
  *b_upper = hi + fabs(beta[k - 1]);
  free(v); free(vp); free(w); free(d); free(e);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Projection (Algorithm 1, "Projection"): Hs = Xt^T Yt, Ms = Xt^T Xt.      */
/* Column-major ns x ns outputs; each entry summed over grid points in order.*/
/* ------------------------------------------------------------------------ */
void or_project(const double* Xt, long ldx, const double* Yt, long ldy, long nd, int ns,
                double* Hs, double* Ms) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int j = 0; j < ns; ++j)
    for (int i = 0; i < ns; ++i) {
      Hs[i + (long)j * ns] = or_dot(Xt + (long)i * ldx, Yt + (long)j * ldy, nd);
      Ms[i + (long)j * ns] = or_dot(Xt + (long)i * ldx, Xt + (long)j * ldx, nd);
    }
}

/* Cholesky M = L L^T (column-major, lower, L over a separate buffer). */
int or_cholesky(int n, const double* M, double* L) {
  memset(L, 0, sizeof(double) * (long)n * n);
  for (int j = 0; j < n; ++j) {
    double s = M[j + (long)j * n];
    for (int k = 0; k < j; ++k) s -= L[j + (long)k * n] * L[j + (long)k * n];
    if (!(s > 0.0)) return OR_ERR_NOT_SPD;
    double ljj = sqrt(s);
    L[j + (long)j * n] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double t = M[i + (long)j * n];
      for (int k = 0; k < j; ++k) t -= L[i + (long)k * n] * L[j + (long)k * n];
      L[i + (long)j * n] = t / ljj;
    }
  }
  return OR_OK;
}

/* Householder reduction A = Q T Q^T of a symmetric column-major n x n A.   */
/* On return d, e hold T and Q (n x n) the accumulated reflectors.           */
void or_householder_tridiag(int n, const double* A_in, double* d, double* e, double* Q) {
  double* A = (double*)malloc(sizeof(double) * (long)n * n);
  memcpy(A, A_in, sizeof(double) * (long)n * n);
  double* v = (double*)malloc(sizeof(double) * n);
  double* p = (double*)malloc(sizeof(double) * n);
  for (long t = 0; t < (long)n * n; ++t) Q[t] = 0.0;
  for (int i = 0; i < n; ++i) Q[i + (long)i * n] = 1.0;
  for (int k = 0; k + 2 < n; ++k) {
    /* reflector H = I - 2 v v^T (|v| = 1) mapping A[k+1:, k] to alpha e_1 */
    double xn = 0.0;
    for (int i = k + 1; i < n; ++i) xn += A[i + (long)k * n] * A[i + (long)k * n];
    xn = sqrt(xn);
    double x0 = A[k + 1 + (long)k * n];
    if (xn == 0.0) continue;
    double alpha = x0 >= 0.0 ? -xn : xn;
    for (int i = 0; i < n; ++i) v[i] = 0.0;
    for (int i = k + 1; i < n; ++i) v[i] = A[i + (long)k * n];
    v[k + 1] -= alpha;
    double vn = 0.0;
    for (int i = k + 1; i < n; ++i) vn += v[i] * v[i];
    vn = sqrt(vn);
    if (vn == 0.0) continue;
    for (int i = k + 1; i < n; ++i) v[i] /= vn;
    /* A <- H A H = A - 2 v q^T - 2 q v^T with p = A v, q = p - (v^T p) v */
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int j = k + 1; j < n; ++j) s += A[i + (long)j * n] * v[j];
      p[i] = s;
    }
    double vp = 0.0;
    for (int i = k + 1; i < n; ++i) vp += v[i] * p[i];
    for (int i = 0; i < n; ++i) p[i] -= vp * v[i];
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i)
        A[i + (long)j * n] -= 2.0 * (v[i] * p[j] + p[i] * v[j]);
    /* Q <- Q H */
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int j = k + 1; j < n; ++j) s += Q[i + (long)j * n] * v[j];
      for (int j = k + 1; j < n; ++j) Q[i + (long)j * n] -= 2.0 * s * v[j];
    }
  }
  for (int i = 0; i < n; ++i) d[i] = A[i + (long)i * n];
  for (int i = 0; i + 1 < n; ++i) e[i] = A[i + 1 + (long)i * n];
  free(A); free(v); free(p);
}

/* Standard symmetric eigenproblem A V = V diag(lam), ascending, sign-fixed. */
int or_sym_eig(int n, const double* A, double* lam, double* V) {
  double* e = (double*)malloc(sizeof(double) * (n > 1 ? n : 1));
  or_householder_tridiag(n, A, lam, e, V);
  int st = or_tridiag_qr(n, lam, e, V, n, n);
  free(e);
  if (st) return st;
  /* selection sort of eigenpairs by ascending eigenvalue */
  double* tmp = (double*)malloc(sizeof(double) * n);
  for (int i = 0; i < n; ++i) {
    int m = i;
    for (int j = i + 1; j < n; ++j)
      if (lam[j] < lam[m]) m = j;
    if (m != i) {
      double t = lam[i]; lam[i] = lam[m]; lam[m] = t;
      memcpy(tmp, V + (long)i * n, sizeof(double) * n);
      memcpy(V + (long)i * n, V + (long)m * n, sizeof(double) * n);
      memcpy(V + (long)m * n, tmp, sizeof(double) * n);
    }
  }
  free(tmp);
  return OR_OK;
}

static void or_fix_signs(int n, int rows, double* Z, int ldz) {
  for (int j = 0; j < n; ++j) {
    double* z = Z + (long)j * ldz;
    int im = 0;
    for (int i = 1; i < rows; ++i)
      if (fabs(z[i]) > fabs(z[im])) im = i;
    if (z[im] < 0.0)
      for (int i = 0; i < rows; ++i) z[i] = -z[i];
  }
}

/* ------------------------------------------------------------------------ */
/* Subspace diagonalisation (Algorithm 1): Hs Z = Ms Z D with Z^T Ms Z = I. */
/*   Ms = L L^T;  A = L^-1 Hs L^-T (symmetrised);  A = V D V^T;  Z = L^-T V */
/* ------------------------------------------------------------------------ */
int or_gen_eig(int n, const double* Hs, const double* Ms, double* lam, double* Z) {
  long nn = (long)n * n;
  double* L = (double*)malloc(sizeof(double) * nn);
  int st = or_cholesky(n, Ms, L);
  if (st) { free(L); return st; }
  double* W = (double*)malloc(sizeof(double) * nn);
  double* A = (double*)malloc(sizeof(double) * nn);
  /* W = L^-1 Hs (forward substitution on each column) */
  for (int c = 0; c < n; ++c)
    for (int i = 0; i < n; ++i) {
      double s = Hs[i + (long)c * n];
      for (int k = 0; k < i; ++k) s -= L[i + (long)k * n] * W[k + (long)c * n];
      W[i + (long)c * n] = s / L[i + (long)i * n];
    }
  /* A = L^-1 W^T  (= L^-1 Hs L^-T since Hs is symmetric) */
  for (int c = 0; c < n; ++c)
    for (int i = 0; i < n; ++i) {
      double s = W[c + (long)i * n];
      for (int k = 0; k < i; ++k) s -= L[i + (long)k * n] * A[k + (long)c * n];
      A[i + (long)c * n] = s / L[i + (long)i * n];
    }
  for (int c = 0; c < n; ++c)
    for (int i = c + 1; i < n; ++i) {
      double s = 0.5 * (A[i + (long)c * n] + A[c + (long)i * n]);
      A[i + (long)c * n] = s;
      A[c + (long)i * n] = s;
    }
  double* V = W;
  st = or_sym_eig(n, A, lam, V);
  if (!st) {
    /* Z = L^-T V (back substitution on each column) */
    for (int c = 0; c < n; ++c)
      for (int i = n - 1; i >= 0; --i) {
        double s = V[i + (long)c * n];
        for (int k = i + 1; k < n; ++k) s -= L[k + (long)i * n] * Z[k + (long)c * n];
        Z[i + (long)c * n] = s / L[i + (long)i * n];
      }
    or_fix_signs(n, n, Z, n);
    for (int i = 0; i < n; ++i)
      if (!isfinite(lam[i])) st = OR_ERR_NUMERIC;
  }
  free(L); free(W); free(A);
  return st;
}

/* Rotation (Algorithm 1): Xout = Xt Z, column-major, Xt has leading dim ld. */
void or_rotate(const double* Xt, long ld, long nd, int ns, const double* Z, double* Xout,
               long ldo) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int j = 0; j < ns; ++j) {
    double* out = Xout + (long)j * ldo;
    for (long t = 0; t < nd; ++t) {
      double s = 0.0;
      for (int k = 0; k < ns; ++k) s += Xt[t + (long)k * ld] * Z[k + (long)j * ns];
      out[t] = s;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* One CheFSI step (Algorithm 1) with given bounds: filter, Yt = H Xt,       */
/* projection, diagonalisation, rotation.  X is replaced by Xt Z and lam    */
/* receives the ns Ritz values in ascending order.                           */
/* ------------------------------------------------------------------------ */
int or_chefsi_step(const or_system* s, double* X, long ld, int ns, int m, double a, double b,
                   double a0, double* lam) {
  long nd = s->nd;
  int st = or_cheb_filter(s, X, ld, ns, m, a, b, a0);
  if (st) return st;
  double* Yt = (double*)malloc(sizeof(double) * nd * ns);
  double* Hs = (double*)malloc(sizeof(double) * (long)ns * ns);
  double* Ms = (double*)malloc(sizeof(double) * (long)ns * ns);
  double* Z = (double*)malloc(sizeof(double) * (long)ns * ns);
  double* Xn = (double*)malloc(sizeof(double) * nd * ns);
  or_hpsi(s, X, ld, Yt, nd, ns);
  or_project(X, ld, Yt, nd, nd, ns, Hs, Ms);
  st = or_gen_eig(ns, Hs, Ms, lam, Z);
  if (!st) {
    or_rotate(X, ld, nd, ns, Z, Xn, nd);
    for (int j = 0; j < ns; ++j) memcpy(X + (long)j * ld, Xn + (long)j * nd, sizeof(double) * nd);
  }
  free(Yt); free(Hs); free(Ms); free(Z); free(Xn);
  return st;
}
