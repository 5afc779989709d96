// FP64 generalised symmetric eigensolver for the subspace problem
// Hs Z = Ms Z D (Algorithm 1, "Diagonalization"; paper Sec. II C solves it
// with a single-GPU sygvd).  Steps, all on the device:
//   1. Cholesky Ms = L L^T (blocked, right-looking; status NOT_SPD on a
//      non-positive pivot);
//   2. A = L^-1 Hs L^-T by two triangular solves (warp per column), symmetrised;
//   3. Householder reduction A = Q T Q^T (T tridiagonal);
//   4. eigenvalues of T by Sturm-count bisection (thread per eigenvalue);
//   5. eigenvectors of T by inverse iteration (thread per eigenvalue; clusters
//      of nearly equal eigenvalues are iterated in sequence with Gram-Schmidt
//      against the earlier members), then one Cholesky-QR pass that restores
//      orthonormality to working precision;
//   6. V = Q V_T by applying the reflectors (warp per column, all reflectors);
//   7. Z = L^-T V, each column's largest-magnitude entry made positive.
// Every reduction runs in a fixed order, so results are bit-reproducible.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "internal.cuh"

namespace sparc {

namespace {

constexpr int kNb = 32;  // Cholesky panel width
constexpr int kTcEigMin = 256;  // smallest n for the tensor-core mode

enum { ST_OK = 0, ST_NOT_SPD = 4, ST_NUMERIC = 5 };

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Cholesky (lower, column-major, in place on A's lower triangle)
// ---------------------------------------------------------------------------
__global__ void k_potrf_diag(double* A, int n, int j0, int jb, int* status) {
  __shared__ double s[kNb][kNb + 1];
  if (*status) return;
  const int t = threadIdx.x;  // 0..kNb-1: row within the block
  for (int c = 0; c < jb; ++c)
    if (t < jb) s[t][c] = A[(j0 + t) + (int64_t)(j0 + c) * n];
  __syncthreads();
  for (int c = 0; c < jb; ++c) {
    if (t == 0) {
      double d = s[c][c];
      if (!(d > 0.0) || !isfinite(d)) {
        *status = ST_NOT_SPD;
        s[c][c] = 1.0;
      } else {
        s[c][c] = sqrt(d);
      }
    }
    __syncthreads();
    if (t > c && t < jb) s[t][c] /= s[c][c];
    __syncthreads();
    if (t > c && t < jb)
      for (int k = c + 1; k <= t; ++k) s[t][k] -= s[t][c] * s[k][c];
    __syncthreads();
  }
  for (int c = 0; c < jb; ++c)
    if (t < jb && t >= c) A[(j0 + t) + (int64_t)(j0 + c) * n] = s[t][c];
}

// rows i >= j0 + jb: L[i, j0:j0+jb] = A[i, j0:j0+jb] L11^-T
__global__ void k_potrf_panel(double* A, int n, int j0, int jb, const int* status) {
  __shared__ double L11[kNb][kNb + 1];
  if (*status) return;
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
    int r = e % jb, c = e / jb;
    L11[r][c] = A[(j0 + r) + (int64_t)(j0 + c) * n];
  }
  __syncthreads();
  int i = j0 + jb + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x[kNb];
#pragma unroll
  for (int c = 0; c < kNb; ++c)
    if (c < jb) x[c] = A[i + (int64_t)(j0 + c) * n];
#pragma unroll
  for (int c = 0; c < kNb; ++c) {
    if (c < jb) {
      double v = x[c];
#pragma unroll
      for (int k = 0; k < kNb; ++k)
        if (k < c) v -= x[k] * L11[c][k];
      x[c] = v / L11[c][c];
    }
  }
#pragma unroll
  for (int c = 0; c < kNb; ++c)
    if (c < jb) A[i + (int64_t)(j0 + c) * n] = x[c];
}

// trailing update A22 -= L21 L21^T on the lower triangle (32 x 32 tiles)
__global__ void k_potrf_update(double* A, int n, int j0, int jb, const int* status) {
  __shared__ double Li[32][kNb + 1];
  __shared__ double Lj[32][kNb + 1];
  if (*status) return;
  const int base = j0 + jb;
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bj > bi) return;
  const int i0 = base + bi * 32, jj0 = base + bj * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 32 x 8 threads
  for (int e = threadIdx.x; e < 32 * jb; e += blockDim.x) {
    int r = e % 32, c = e / 32;
    Li[r][c] = (i0 + r < n) ? A[(i0 + r) + (int64_t)(j0 + c) * n] : 0.0;
    Lj[r][c] = (jj0 + r < n) ? A[(jj0 + r) + (int64_t)(j0 + c) * n] : 0.0;
  }
  __syncthreads();
  for (int rr = ty; rr < 32; rr += 8) {
    int i = i0 + tx, j = jj0 + rr;
    if (i < n && j < n && j <= i) {
      double s = 0.0;
      for (int c = 0; c < jb; ++c) s += Li[tx][c] * Lj[rr][c];
      A[i + (int64_t)j * n] -= s;
    }
  }
}

// lower-triangular copy with zeroed upper part: L = tril(A)
__global__ void k_tril_copy(const double* A, double* L, int n) {
  int64_t nn = (int64_t)n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nn;
       t += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(t % n), j = (int)(t / n);
    L[t] = i >= j ? A[t] : 0.0;
  }
}

__global__ void k_transpose(const double* __restrict__ A, double* __restrict__ B, int n) {
  __shared__ double tile[32][33];
  int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int i = bx + threadIdx.x, j = by + r;
    if (i < n && j < n) tile[r][threadIdx.x] = A[i + (int64_t)j * n];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int i = by + threadIdx.x, j = bx + r;
    if (i < n && j < n) B[i + (int64_t)j * n] = tile[threadIdx.x][r];
  }
}

// B = (A + A^T)/2
__global__ void k_symmetrize(const double* __restrict__ A, double* __restrict__ B, int n) {
  int64_t nn = (int64_t)n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nn;
       t += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(t % n), j = (int)(t / n);
    B[t] = 0.5 * (A[t] + A[j + (int64_t)i * n]);
  }
}

// ---------------------------------------------------------------------------
// Triangular solves, one warp per right-hand-side column (column-major B, X).
// forward:  X = L^-1 B   (Lrm = L stored row-major, i.e. L^T column-major)
// backward: X = L^-T B   (Lcm = L column-major)
// ---------------------------------------------------------------------------
constexpr int kTrsmWarps = 4;

template <bool FORWARD>
__global__ void __launch_bounds__(kTrsmWarps * 32)
    k_trsm(const double* __restrict__ Lt, const double* __restrict__ B, double* __restrict__ X,
           int n, int ncols, const int* status) {
  extern __shared__ double xs_all[];
  if (*status) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + warp;
  if (c >= ncols) return;
  double* xs = xs_all + (int64_t)warp * n;
  const double* b = B + (int64_t)c * n;
  for (int step = 0; step < n; ++step) {
    const int i = FORWARD ? step : n - 1 - step;
    // Lt row i holds L[i, k] (forward, k < i) or L[k, i] (backward, k > i)
    const double* row = Lt + (int64_t)i * n;
    double s = 0.0;
    if (FORWARD) {
      for (int k = lane; k < i; k += 32) s += row[k] * xs[k];
    } else {
      for (int k = i + 1 + lane; k < n; k += 32) s += row[k] * xs[k];
    }
    s = warp_sum_d(s);
    double xi = (b[i] - s) / row[i];
    if (lane == 0) xs[i] = xi;
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) X[(int64_t)c * n + i] = xs[i];
}

// ---------------------------------------------------------------------------
// Householder tridiagonalisation of a symmetric A (column-major == row-major).
// Step k: v from A[k+1:, k]; p = A v on the trailing block; A -= 2(v q^T + q v^T)
// with q = p - (v.p) v.  Reflector k is stored in row k of Hv (entries k+1..n-1).
// ---------------------------------------------------------------------------
__device__ double block_sum_d(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum_d(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  return t;  // every thread gets the same value
}

__global__ void k_house_vec(const double* __restrict__ A, double* __restrict__ Hv, double* d,
                            double* e, int n, int k) {
  __shared__ double sh[32];
  const double* col = A + (int64_t)k * n;  // column k == row k
  double acc = 0.0;
  for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) acc += col[i] * col[i];
  double xn = sqrt(block_sum_d(acc, sh));
  double x0 = col[k + 1];
  double alpha = x0 >= 0.0 ? -xn : xn;
  // v = x - alpha e1, |v|^2 = xn^2 - 2 alpha x0 + alpha^2 = 2 xn^2 + 2 xn |x0|
  double vn2 = 0.0;
  for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) {
    double v = col[i] - (i == k + 1 ? alpha : 0.0);
    vn2 += v * v;
  }
  double vn = sqrt(block_sum_d(vn2, sh));
  double* hv = Hv + (int64_t)k * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double v = 0.0;
    if (i > k && xn > 0.0 && vn > 0.0) v = (col[i] - (i == k + 1 ? alpha : 0.0)) / vn;
    hv[i] = v;
  }
  if (threadIdx.x == 0) {
    d[k] = col[k];
    e[k] = xn > 0.0 ? alpha : 0.0;
  }
}

// p_i = sum_{j>k} A[i][j] v_j for i > k (warp per row)
__global__ void k_house_matvec(const double* __restrict__ A, const double* __restrict__ Hv,
                               double* __restrict__ p, int n, int k) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int i = k + 1 + warp;
  if (i >= n) return;
  const double* row = A + (int64_t)i * n;
  const double* v = Hv + (int64_t)k * n;
  double s = 0.0;
  for (int j = k + 1 + lane; j < n; j += 32) s += row[j] * v[j];
  s = warp_sum_d(s);
  if (lane == 0) p[i] = s;
}

// A[i][j] -= 2 (v_i q_j + q_i v_j), q = p - (v.p) v, on the trailing block
__global__ void k_house_update(double* __restrict__ A, const double* __restrict__ Hv,
                               const double* __restrict__ p, int n, int k) {
  __shared__ double sh[32];
  const double* v = Hv + (int64_t)k * n;
  double acc = 0.0;
  for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) acc += v[i] * p[i];
  const double K = block_sum_d(acc, sh);
  const int m = n - k - 1;
  const int64_t mm = (int64_t)m * m;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < mm;
       t += (int64_t)gridDim.x * blockDim.x) {
    int i = k + 1 + (int)(t % m), j = k + 1 + (int)(t / m);
    double qi = p[i] - K * v[i], qj = p[j] - K * v[j];
    A[i + (int64_t)j * n] -= 2.0 * (v[i] * qj + qi * v[j]);
  }
}

__global__ void k_house_tail(const double* A, double* Hv, double* d, double* e, int n) {
  if (threadIdx.x != 0) return;
  int k0 = n >= 2 ? n - 2 : 0;
  for (int k = k0; k < n; ++k) {
    d[k] = A[k + (int64_t)k * n];
    for (int i = 0; i < n; ++i) Hv[(int64_t)k * n + i] = 0.0;
  }
  if (n >= 2) e[n - 2] = A[(n - 1) + (int64_t)(n - 2) * n];
}

// ---------------------------------------------------------------------------
// Persistent form of the Householder reduction: one cooperative launch runs all
// n - 2 steps, separated by grid barriers (2 per step) instead of 3 kernel
// launches per step.  The barrier waits are bounded: on expiry the kernel
// records SPARC_ERR_TIMEOUT in status[4] and every block leaves the loop.
// ---------------------------------------------------------------------------
struct GridBar {
  unsigned* count;
  unsigned* gen;
  int* status;
  long long cycles;  // bound of each barrier wait (SM clock cycles)
};

constexpr int kHouseThreads = 512;  // largest CTA (one per SM)

// Returns false if the barrier timed out (in any block).
__device__ bool grid_barrier(const GridBar& gb, unsigned nblocks, int* abort_sh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = gb.gen;
    const unsigned g = *vgen;
    __threadfence();
    if (atomicAdd(gb.count, 1u) == nblocks - 1) {
      atomicExch(gb.count, 0u);
      __threadfence();
      atomicAdd(gb.gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == g) {
        if (*(volatile int*)gb.status != 0 || clock64() - t0 > gb.cycles) {
          atomicCAS(gb.status, 0, SPARC_ERR_TIMEOUT);
          *abort_sh = 1;
          break;
        }
      }
    }
    __threadfence();
    if (*(volatile int*)gb.status != 0) *abort_sh = 1;
  }
  __syncthreads();
  return *abort_sh == 0;
}

__global__ void __launch_bounds__(kHouseThreads)
    k_house_persistent(double* __restrict__ A, double* __restrict__ Hv, double* d, double* e,
                       double* __restrict__ p, int n, GridBar gb) {
  // every block forms the step's reflector itself, in shared memory (the
  // column it reads was completed by the previous step's barrier), so a step
  // needs two grid barriers: after p = A v and after the rank-2 update
  extern __shared__ double vsh[];
  __shared__ double sh[32];
  __shared__ int abort_sh;
  if (threadIdx.x == 0) abort_sh = 0;
  __syncthreads();
  const unsigned nb = gridDim.x;
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int k = 0; k + 2 < n; ++k) {
    const double* col = A + (int64_t)k * n;
    double acc = 0.0;
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) acc += col[i] * col[i];
    const double xn = sqrt(block_sum_d(acc, sh));
    const double x0 = col[k + 1];
    const double alpha = x0 >= 0.0 ? -xn : xn;
    double vn2 = 0.0;
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) {
      const double v = col[i] - (i == k + 1 ? alpha : 0.0);
      vn2 += v * v;
    }
    const double vn = sqrt(block_sum_d(vn2, sh));
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x)
      vsh[i] = (xn > 0.0 && vn > 0.0) ? (col[i] - (i == k + 1 ? alpha : 0.0)) / vn : 0.0;
    __syncthreads();  // the whole reflector is in shared memory from here on
    if (blockIdx.x == 0) {
      double* hv = Hv + (int64_t)k * n;
      for (int i = threadIdx.x; i < n; i += blockDim.x) hv[i] = i > k ? vsh[i] : 0.0;
      if (threadIdx.x == 0) {
        d[k] = col[k];
        e[k] = xn > 0.0 ? alpha : 0.0;
      }
    }
    // p = A v on the trailing block (warp per row)
    for (int i = k + 1 + gwarp; i < n; i += nwarps) {
      const double* row = A + (int64_t)i * n;
      double s2 = 0.0;
      for (int j = k + 1 + lane; j < n; j += 32) s2 += row[j] * vsh[j];
      s2 = warp_sum_d(s2);
      if (lane == 0) p[i] = s2;
    }
    if (!grid_barrier(gb, nb, &abort_sh)) return;
    acc = 0.0;
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) acc += vsh[i] * p[i];
    const double K = block_sum_d(acc, sh);
    // element r + m c of the trailing block, stepped by the grid size with
    // (r, c) carried instead of divided out
    const int m = n - k - 1;
    const int nthr = gridDim.x * blockDim.x;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int sq = nthr / m, sr = nthr % m;
    for (int r = gtid % m, c = gtid / m; c < m;) {
      const int i = k + 1 + r, j = k + 1 + c;
      const double vi = vsh[i], vj = vsh[j];
      const double qi = p[i] - K * vi, qj = p[j] - K * vj;
      A[i + (int64_t)j * n] -= 2.0 * (vi * qj + qi * vj);
      r += sr;
      c += sq;
      if (r >= m) {
        r -= m;
        ++c;
      }
    }
    if (!grid_barrier(gb, nb, &abort_sh)) return;
  }
}

// ---------------------------------------------------------------------------
// Tridiagonal eigenvalues by bisection.  scal[0..1] = Gershgorin interval,
// scal[2] = pivmin.
// ---------------------------------------------------------------------------
__global__ void k_gersh(const double* d, const double* e, int n, double* e2, double* scal) {
  double lo = 1e300, hi = -1e300, emax = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
    lo = fmin(lo, d[i] - r);
    hi = fmax(hi, d[i] + r);
    if (i + 1 < n) {
      e2[i] = e[i] * e[i];
      emax = fmax(emax, e2[i]);
    }
  }
  // block min / max via shared memory
  __shared__ double slo[1024], shi[1024], sem[1024];
  slo[threadIdx.x] = lo;
  shi[threadIdx.x] = hi;
  sem[threadIdx.x] = emax;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int t = 1; t < (int)blockDim.x; ++t) {
      lo = fmin(lo, slo[t]);
      hi = fmax(hi, shi[t]);
      emax = fmax(emax, sem[t]);
    }
    double tnorm = fmax(fabs(lo), fabs(hi));
    double pad = 2.2e-16 * tnorm * n + 1e-300;
    scal[0] = lo - pad;
    scal[1] = hi + pad;
    scal[2] = fmax(2.2250738585072014e-308 * fmax(1.0, emax), 1e-300);
    scal[3] = tnorm;
  }
}

__device__ int sturm(const double* __restrict__ d, const double* __restrict__ e2, int n,
                     double x, double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0.0) ++cnt;
  for (int i = 1; i < n; ++i) {
    q = d[i] - x - e2[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// Eigenvalue j of the tridiagonal matrix by multisection: the L lanes of a
// group evaluate Sturm counts at L interior points of [lo, hi] at once, and the
// interval shrinks (L + 1)-fold per round (bisection's 2-fold per count, with
// L times the parallelism for the latency-bound count recurrence).  Stops at
// the same relative width as plain bisection: 2 eps max(|lo|, |hi|).  The
// whole-GPU eigensolver takes this form: with few eigenvalues per SM the
// count recurrence's latency bounds the step (L = 8); with many, the FP64
// pipe does, and fewer counts per eigenvalue win (L = 4 from n = 2048).
template <int L>
__global__ void k_bisect(const double* __restrict__ d, const double* __restrict__ e2, int n,
                         const double* __restrict__ scal, double* __restrict__ lam) {
  constexpr int kMsLanes = L;
  const int g = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kMsLanes);
  const int l = threadIdx.x % kMsLanes;
  const unsigned gmask = ((1u << kMsLanes) - 1u) << ((threadIdx.x & 31) & ~(kMsLanes - 1));
  const int j = min(g, n - 1);  // surplus groups repeat the last eigenvalue, unwritten
  double lo = scal[0], hi = scal[1];
  const double pivmin = scal[2];
  for (int it = 0; it < 64; ++it) {
    if (hi - lo <= 2.0 * 2.2e-16 * fmax(fabs(lo), fabs(hi))) break;
    const double step = (hi - lo) / (kMsLanes + 1);
    const double x = lo + (l + 1) * step;
    const bool above = sturm(d, e2, n, x, pivmin) > j;  // lam_j < x
    const unsigned b = __ballot_sync(gmask, above) & gmask;
    // the first lane whose point lies above lam_j bounds it from above
    const int first = b ? __ffs(b) - 1 - ((threadIdx.x & 31) & ~(kMsLanes - 1)) : kMsLanes;
    const double nlo = first == 0 ? lo : lo + first * step;
    const double nhi = first == kMsLanes ? hi : lo + (first + 1) * step;
    if (!(nlo >= lo && nhi <= hi && nlo < nhi)) break;  // no progress left in FP64
    lo = nlo;
    hi = nhi;
  }
  if (g < n && l == 0) lam[j] = 0.5 * (lo + hi);
}

// Eigenvalue j by multisection on the Sturm count in a group of L lanes (the
// L lanes of the warp at (lane & ~(L - 1))): the interval shrinks (L + 1)-fold
// per round.  Every lane of the group must call it with the same j; lane l of
// the group returns the result.
template <int L>
__device__ double multisect_eig(const double* __restrict__ d, const double* __restrict__ e2,
                                int n, const double* __restrict__ scal, int j) {
  const int lane = threadIdx.x & 31;
  const int l = lane & (L - 1);
  const unsigned gmask = ((1u << L) - 1u) << (lane & ~(L - 1));
  double lo = scal[0], hi = scal[1];
  const double pivmin = scal[2];
  for (int it = 0; it < 96; ++it) {
    if (hi - lo <= 2.0 * 2.2e-16 * fmax(fabs(lo), fabs(hi))) break;
    const double step = (hi - lo) / (L + 1);
    const double x = lo + (l + 1) * step;
    const bool above = sturm(d, e2, n, x, pivmin) > j;
    const unsigned b = __ballot_sync(gmask, above) & gmask;
    const int first = b ? __ffs(b) - 1 - (lane & ~(L - 1)) : L;
    const double nlo = first == 0 ? lo : lo + first * step;
    const double nhi = first == L ? hi : lo + (first + 1) * step;
    if (!(nlo >= lo && nhi <= hi && nlo < nhi)) break;
    lo = nlo;
    hi = nhi;
  }
  return 0.5 * (lo + hi);
}

// Eigenvalue j by plain bisection on the Sturm count: one count per halving,
// the fewest counts per bit.  The batched eigensolver takes this form: there
// one SM (or a few) holds all of a problem's eigenvalues, so the FP64 pipe,
// not the recurrence's latency, bounds the step.  Stops at the same relative
// width, when the midpoint no longer moves, or after 96 halvings.
__device__ double bisect_eig(const double* __restrict__ d, const double* __restrict__ e2, int n,
                             const double* __restrict__ scal, int j) {
  double lo = scal[0], hi = scal[1];
  const double pivmin = scal[2];
  for (int it = 0; it < 96; ++it) {
    if (hi - lo <= 2.0 * 2.2e-16 * fmax(fabs(lo), fabs(hi))) break;
    const double mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    if (sturm(d, e2, n, mid, pivmin) > j)
      hi = mid;
    else
      lo = mid;
  }
  return 0.5 * (lo + hi);
}

// Cluster bookkeeping: clus[j] = first index of j's cluster, clus[n + j] = its size.
__global__ void k_clusters(const double* lam, int n, const double* scal, int* clus) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double tol = 1e-9 * fmax(scal[3], 1e-300);
  int start = 0;
  for (int j = 1; j <= n; ++j) {
    if (j == n || lam[j] - lam[j - 1] > tol) {
      for (int t = start; t < j; ++t) {
        clus[t] = start;
        clus[n + t] = j - start;
      }
      start = j;
    }
  }
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double start_value(uint64_t seed, int i) {
  uint64_t z = mix64(seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ULL);
  return (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
}

// LU with partial pivoting of T - sigma I.  Factors at lu[(f * n + i) * stride + j]
// for f = 0 (u0), 1 (u1), 2 (u2), 3 (l); pivot flags in piv[i * stride + j].
struct TriLU {
  double* lu;
  int* piv;
  int n;
  int64_t stride;
  int j;
  __device__ double& at(int f, int i) const { return lu[((int64_t)f * n + i) * stride + j]; }
  __device__ int& pv(int i) const { return piv[(int64_t)i * stride + j]; }
};

__device__ void tri_factor(const TriLU& F, const double* d, const double* e, double sigma,
                           double pivmin) {
  const int n = F.n;
  double p0 = d[0] - sigma, p1 = n > 1 ? e[0] : 0.0, p2 = 0.0;
  for (int k = 0; k + 1 < n; ++k) {
    double ek = e[k];
    double a1 = d[k + 1] - sigma;
    double e1 = k + 2 < n ? e[k + 1] : 0.0;
    if (fabs(p0) >= fabs(ek)) {
      if (fabs(p0) < pivmin) p0 = p0 >= 0.0 ? pivmin : -pivmin;
      double l = ek / p0;
      F.at(0, k) = p0; F.at(1, k) = p1; F.at(2, k) = p2; F.at(3, k) = l; F.pv(k) = 0;
      double np0 = a1 - l * p1, np1 = e1 - l * p2;
      p0 = np0; p1 = np1; p2 = 0.0;
    } else {
      double l = p0 / ek;
      F.at(0, k) = ek; F.at(1, k) = a1; F.at(2, k) = e1; F.at(3, k) = l; F.pv(k) = 1;
      double np0 = p1 - l * a1, np1 = p2 - l * e1;
      p0 = np0; p1 = np1; p2 = 0.0;
    }
  }
  if (fabs(p0) < pivmin) p0 = p0 >= 0.0 ? pivmin : -pivmin;
  F.at(0, n - 1) = p0;
  F.at(1, n - 1) = 0.0;
  F.at(2, n - 1) = 0.0;
  F.at(3, n - 1) = 0.0;
  F.pv(n - 1) = 0;
}

// Solve (T - sigma) x = b in place in x (entry i at x[i sx]).
__device__ void tri_solve(const TriLU& F, double* x, int64_t sx = 1) {
  const int n = F.n;
  for (int k = 0; k + 1 < n; ++k) {
    if (F.pv(k)) {
      double t = x[k * sx];
      x[k * sx] = x[(k + 1) * sx];
      x[(k + 1) * sx] = t;
    }
    x[(k + 1) * sx] -= F.at(3, k) * x[k * sx];
  }
  for (int k = n - 1; k >= 0; --k) {
    double s = x[k * sx];
    if (k + 1 < n) s -= F.at(1, k) * x[(k + 1) * sx];
    if (k + 2 < n) s -= F.at(2, k) * x[(k + 2) * sx];
    x[k * sx] = s / F.at(0, k);
  }
}

__device__ void scale_maxabs(double* x, int n, int64_t sx = 1) {
  double m = 0.0;
  for (int i = 0; i < n; ++i) m = fmax(m, fabs(x[i * sx]));
  if (m > 0.0) {
    double inv = 1.0 / m;
    for (int i = 0; i < n; ++i) x[i * sx] *= inv;
  }
}

constexpr int kInvIters = 3;

// Thread per eigenvalue, singletons only: eigenvector j into the row-major
// scratch Xr (entry i of vector j at Xr[i n + j], so that the threads of a
// warp, which hold consecutive j, touch consecutive addresses); the caller
// transposes Xr into the column-major V.
__global__ void k_inviter_single(const double* __restrict__ d, const double* __restrict__ e,
                                 const double* __restrict__ lam, const double* __restrict__ scal,
                                 const int* __restrict__ clus, int n, double* lu, int* piv,
                                 double* Xr) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n || clus[n + j] != 1) return;
  TriLU F{lu, piv, n, n, j};
  const double pivmin = fmax(2.2e-16 * scal[3], 1e-300);
  tri_factor(F, d, e, lam[j], pivmin);
  double* x = Xr + j;
  const int64_t sx = n;
  for (int i = 0; i < n; ++i) x[i * sx] = start_value(0x5EEDull + j, i);
  for (int it = 0; it < kInvIters; ++it) {
    scale_maxabs(x, n, sx);
    tri_solve(F, x, sx);
  }
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += x[i * sx] * x[i * sx];
  double inv = 1.0 / sqrt(s);
  for (int i = 0; i < n; ++i) x[i * sx] *= inv;
}

// One CTA per cluster (launched for every j; only cluster starts of size > 1 work).
// Members are iterated in order; each iterate is orthogonalised against the
// earlier members (classical Gram-Schmidt, applied twice).
__global__ void k_inviter_cluster(const double* __restrict__ d, const double* __restrict__ e,
                                  const double* __restrict__ lam, const double* __restrict__ scal,
                                  const int* __restrict__ clus, int n, double* lu, int* piv,
                                  double* V) {
  __shared__ double sh[32];
  __shared__ double coef[1];
  const int j0 = blockIdx.x;
  if (clus[j0] != j0 || clus[n + j0] < 2) return;
  const int size = clus[n + j0];
  const double pivmin = fmax(2.2e-16 * scal[3], 1e-300);
  const double sep = 10.0 * 2.2e-16 * fmax(scal[3], 1e-300);
  double shift_prev = 0.0;
  for (int m = 0; m < size; ++m) {
    const int j = j0 + m;
    double sigma = lam[j];
    if (m > 0 && sigma - shift_prev < sep) sigma = shift_prev + sep;
    shift_prev = sigma;
    TriLU F{lu, piv, n, n, j};
    if (threadIdx.x == 0) tri_factor(F, d, e, sigma, pivmin);
    double* x = V + (int64_t)j * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = start_value(0x5EEDull + j, i);
    __syncthreads();
    for (int it = 0; it < kInvIters; ++it) {
      if (threadIdx.x == 0) {
        scale_maxabs(x, n);
        tri_solve(F, x);
      }
      __syncthreads();
      for (int pass = 0; pass < 2; ++pass) {
        for (int q = 0; q < m; ++q) {
          const double* y = V + (int64_t)(j0 + q) * n;
          double acc = 0.0;
          for (int i = threadIdx.x; i < n; i += blockDim.x) acc += y[i] * x[i];
          double c = block_sum_d(acc, sh);
          for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] -= c * y[i];
          __syncthreads();
        }
      }
      double acc = 0.0;
      for (int i = threadIdx.x; i < n; i += blockDim.x) acc += x[i] * x[i];
      double nrm = sqrt(block_sum_d(acc, sh));
      if (threadIdx.x == 0) coef[0] = nrm > 0.0 ? 1.0 / nrm : 0.0;
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] *= coef[0];
      __syncthreads();
    }
  }
}

// Apply all reflectors: V <- H_0 H_1 ... H_{n-3} V, warp per column of V.
constexpr int kBtWarps = 4;
__global__ void __launch_bounds__(kBtWarps * 32)
    k_backtransform(const double* __restrict__ Hv, double* __restrict__ V, int n) {
  extern __shared__ double cols[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + warp;
  if (c >= n) return;
  double* x = cols + (int64_t)warp * n;
  for (int i = lane; i < n; i += 32) x[i] = V[(int64_t)c * n + i];
  __syncwarp();
  for (int k = n - 3; k >= 0; --k) {
    const double* v = Hv + (int64_t)k * n;
    double s = 0.0;
    for (int i = k + 1 + lane; i < n; i += 32) s += v[i] * x[i];
    s = 2.0 * warp_sum_d(s);
    for (int i = k + 1 + lane; i < n; i += 32) x[i] -= s * v[i];
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) V[(int64_t)c * n + i] = x[i];
}

// Largest-magnitude entry of each column made positive (first index on ties);
// eigenvalue NaN/Inf check.
__global__ void k_fix_signs(double* Z, int n, const double* lam, int* status) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  double* z = Z + (int64_t)warp * n;
  double best = -1.0;
  int bi = 0;
  for (int i = lane; i < n; i += 32) {
    double a = fabs(z[i]);
    if (a > best) { best = a; bi = i; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double ob = __shfl_xor_sync(0xffffffffu, best, o);
    int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  bool neg = z[bi] < 0.0;
  if (neg)
    for (int i = lane; i < n; i += 32) z[i] = -z[i];
  if (lane == 0 && !isfinite(lam[warp])) atomicCAS(status, 0, ST_NUMERIC);
}

cudaError_t cholesky(double* A, int n, int* status, cudaStream_t st) {
  for (int j0 = 0; j0 < n; j0 += kNb) {
    int jb = min(kNb, n - j0);
    note_launch(), k_potrf_diag<<<1, kNb, 0, st>>>(A, n, j0, jb, status);
    int rem = n - j0 - jb;
    if (rem > 0) {
      note_launch(), k_potrf_panel<<<(rem + 127) / 128, 128, 0, st>>>(A, n, j0, jb, status);
      int nt = (rem + 31) / 32;
      note_launch(), k_potrf_update<<<dim3(nt, nt), 256, 0, st>>>(A, n, j0, jb, status);
    }
  }
  return cudaGetLastError();
}

// warps per block for the column-per-warp kernels: each warp keeps one n-vector
// in shared memory
int col_warps(int n) {
  int w = (int)((200 * 1024) / ((size_t)n * sizeof(double)));
  return w < 1 ? 1 : (w > 4 ? 4 : w);
}

template <bool FWD>
cudaError_t trsm(const double* Lt, const double* B, double* X, int n, const int* status,
                 cudaStream_t st) {
  int wpb = col_warps(n);
  size_t smem = (size_t)wpb * n * sizeof(double);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_trsm<FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  note_launch(), k_trsm<FWD><<<(n + wpb - 1) / wpb, wpb * 32, smem, st>>>(Lt, B, X, n, n, status);
  return cudaGetLastError();
}

int blocks_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 4096); }

}  // namespace

cudaError_t eig_alloc(EigWork& w, int nmax) {
  eig_free(w);
  w.nmax = nmax;
  size_t nn = (size_t)nmax * nmax;
  cudaError_t err = cudaSuccess;
  auto take = [&](auto** p, size_t bytes) {
    if (err == cudaSuccess) err = cudaMalloc((void**)p, bytes > 0 ? bytes : 8);
  };
  take(&w.L, nn * 8);
  take(&w.A, nn * 8);
  take(&w.W, nn * 8);
  take(&w.V, nn * 8);
  take(&w.d, (size_t)nmax * 8);
  take(&w.e, (size_t)nmax * 8 + 8);
  take(&w.tau, (size_t)nmax * 8 * 2 + 8);
  take(&w.lu, 4 * nn * 8);
  take(&w.scal, 64 * 8);
  take(&w.status, 64);
  take(&w.clus, (size_t)2 * nmax * 4 + 8);
  take(&w.piv, nn * 4);
  if (nmax >= kTcEigMin) {
    take(&w.X0, nn * 8);
    take(&w.X1, nn * 8);
  }
  if (err != cudaSuccess) eig_free(w);
  return err;
}

void eig_free(EigWork& w) {
  cudaFree(w.L); cudaFree(w.A); cudaFree(w.W); cudaFree(w.V); cudaFree(w.d); cudaFree(w.e);
  cudaFree(w.tau); cudaFree(w.lu); cudaFree(w.scal); cudaFree(w.status); cudaFree(w.clus);
  cudaFree(w.piv); cudaFree(w.X0); cudaFree(w.X1);
  w = EigWork{};
}

// ---------------------------------------------------------------------------
// Tensor-core mode (n >= kTcEigMin): the O(n^3) products of the reduction, the
// re-orthonormalisation and the back-substitution as FP64-accurate six-digit
// tensor-core GEMMs (tc_rotate: C = A B, A m x k with a leading dimension, B
// k x k contiguous), with the triangular factors inverted explicitly:
//   inv([[L11, 0], [L21, L22]]) = [[X11, 0], [-X22 L21 X11, X22]],
// X21 formed as -(U^T X22^T)^T with U = L21 X11, so that every product has a
// square right factor; blocks of <= 128 rows are inverted by substitution.
// ---------------------------------------------------------------------------
// B (n x m, ldb) = scale A^T (A m x n, lda), or B = scale A without transposing
__global__ void k_copy_scaled(const double* __restrict__ A, int64_t lda, int m, int n,
                              double* __restrict__ B, int64_t ldb, int transpose, double scale) {
  __shared__ double tile[32][33];
  const int bi = blockIdx.x * 32, bj = blockIdx.y * 32;  // A rows, columns
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = bi + threadIdx.x, j = bj + r;
    if (i < m && j < n) tile[r][threadIdx.x] = A[i + (int64_t)j * lda];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    if (transpose) {
      const int i = bj + threadIdx.x, j = bi + r;  // B row i = A column, B column j = A row
      if (i < n && j < m) B[i + (int64_t)j * ldb] = scale * tile[threadIdx.x][r];
    } else {
      const int i = bi + threadIdx.x, j = bj + r;
      if (i < m && j < n) B[i + (int64_t)j * ldb] = scale * tile[r][threadIdx.x];
    }
  }
}

// Leaf kernels of the tensor-core mode: one CTA of kLeafThreads works on an
// n x n block (n <= 128) held whole in shared memory.
constexpr int kLeafThreads = 512;
constexpr int kLeafMax = 128;
constexpr int kLeafCols = 16;  // columns of L staged per load

// X = L^-1 for a lower-triangular n x n block: forward substitution on the
// columns of I, right-looking (step k divides row k by L(k,k) and removes it
// from the rows below), so each entry sees the same operations in the same
// order as column-by-column substitution; the upper triangle is zeroed
__global__ void __launch_bounds__(kLeafThreads)
    k_trinv_leaf(const double* __restrict__ L, int64_t ldl, int n, double* X, int64_t ldx) {
  extern __shared__ double leaf_sm[];
  double* xs = leaf_sm;          // n x n, row-major
  double* lc = leaf_sm + n * n;  // kLeafCols staged columns of L
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < n * n; e += nt) xs[e] = (e / n == e % n) ? 1.0 : 0.0;
  for (int k0 = 0; k0 < n; k0 += kLeafCols) {
    const int kc = min(kLeafCols, n - k0);
    __syncthreads();
    for (int e = tid; e < kc * n; e += nt) {
      const int c = e / n, i = e - c * n;
      lc[e] = i >= k0 + c ? L[i + (int64_t)(k0 + c) * ldl] : 0.0;
    }
    __syncthreads();
    for (int kk = 0; kk < kc; ++kk) {
      const int k = k0 + kk;
      const double* lk = lc + kk * n;
      for (int c = tid; c <= k; c += nt) xs[k * n + c] /= lk[k];
      __syncthreads();
      const int rows = n - k - 1, cols = k + 1;
      for (int e = tid; e < rows * cols; e += nt) {
        const int i = k + 1 + e / cols, c = e % cols;
        xs[i * n + c] -= lk[i] * xs[k * n + c];
      }
      __syncthreads();
    }
  }
  for (int e = tid; e < n * n; e += nt) {
    const int c = e / n, i = e - c * n;
    X[i + (int64_t)c * ldx] = c <= i ? xs[i * n + c] : 0.0;
  }
}

// Cholesky of the n x n diagonal block at A (lda) in place (lower triangle),
// right-looking, in the operation order of k_potrf_diag; a non-positive or
// non-finite pivot records NOT_SPD (and continues with 1)
__global__ void __launch_bounds__(kLeafThreads)
    k_potrf_leaf(double* A, int64_t lda, int n, int* status) {
  extern __shared__ double leaf_sm[];
  __shared__ double piv;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < n * n; e += nt) {
    const int j = e / n, i = e - j * n;
    leaf_sm[e] = i >= j ? A[i + (int64_t)j * lda] : 0.0;
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      double d = leaf_sm[k + k * n];
      if (!(d > 0.0) || !isfinite(d)) {
        atomicCAS(status, 0, ST_NOT_SPD);
        d = 1.0;
      }
      piv = sqrt(d);
      leaf_sm[k + k * n] = piv;
    }
    __syncthreads();
    for (int i = k + 1 + tid; i < n; i += nt) leaf_sm[i + k * n] /= piv;
    __syncthreads();
    const int m = n - k - 1;
    for (int e = tid; e < m * m; e += nt) {
      const int i = k + 1 + e % m, j = k + 1 + e / m;
      if (j <= i) leaf_sm[i + j * n] -= leaf_sm[i + k * n] * leaf_sm[j + k * n];
    }
    __syncthreads();
  }
  for (int e = tid; e < n * n; e += nt) {
    const int j = e / n, i = e - j * n;
    if (i >= j) A[i + (int64_t)j * lda] = leaf_sm[e];
  }
}

cudaError_t trinv_leaf(const double* L, int64_t ldl, int n, double* X, int64_t ldx,
                       cudaStream_t st) {
  static unsigned long long bits = 0;
  const size_t smem = (size_t)(kLeafMax * kLeafMax + kLeafCols * kLeafMax) * sizeof(double);
  cudaError_t e = smem_limit_once(&bits, (const void*)k_trinv_leaf, (int)smem);
  if (e != cudaSuccess) return e;
  note_launch();
  k_trinv_leaf<<<1, kLeafThreads, (size_t)(n * n + kLeafCols * n) * sizeof(double), st>>>(
      L, ldl, n, X, ldx);
  return cudaGetLastError();
}

cudaError_t potrf_leaf(double* A, int64_t lda, int n, int* status, cudaStream_t st) {
  static unsigned long long bits = 0;
  const size_t smem = (size_t)kLeafMax * kLeafMax * sizeof(double);
  cudaError_t e = smem_limit_once(&bits, (const void*)k_potrf_leaf, (int)smem);
  if (e != cudaSuccess) return e;
  note_launch();
  k_potrf_leaf<<<1, kLeafThreads, (size_t)n * n * sizeof(double), st>>>(A, lda, n, status);
  return cudaGetLastError();
}

cudaError_t copy_scaled(const double* A, int64_t lda, int m, int n, double* B, int64_t ldb,
                        bool transpose, double scale, cudaStream_t st) {
  const dim3 g((unsigned)((m + 31) / 32), (unsigned)((n + 31) / 32));
  note_launch(), k_copy_scaled<<<g, dim3(32, 8), 0, st>>>(A, lda, m, n, B, ldb, transpose ? 1 : 0,
                                                          scale);
  return cudaGetLastError();
}

// C (m x k, ldc) = A (m x k, lda) B (k x k contiguous)
cudaError_t gemm_tc(const EigGemm& g, const double* A, int64_t lda, int m, int k, const double* B,
                    double* C, int64_t ldc, cudaStream_t st) {
  return tc_rotate(A, lda, m, k, B, C, ldc, g.SA, g.SZ, g.esc, g.status, st);
}

// X (ldx) = L^-1 for lower-triangular L (n x n, ldl); scratch: 2 n^2 doubles
cudaError_t trinv_lower(const EigGemm& g, const double* L, int64_t ldl, int n, double* X,
                        int64_t ldx, double* scratch, cudaStream_t st) {
  if (n <= kLeafMax) return trinv_leaf(L, ldl, n, X, ldx, st);
  const int n1 = (n / 2 + 63) / 64 * 64, n2 = n - n1;
  cudaError_t e;
  if ((e = trinv_lower(g, L, ldl, n1, X, ldx, scratch, st)) != cudaSuccess) return e;
  if ((e = trinv_lower(g, L + n1 + (int64_t)n1 * ldl, ldl, n2, X + n1 + (int64_t)n1 * ldx, ldx,
                       scratch, st)) != cudaSuccess)
    return e;
  double* S0 = scratch;                      // X11 contiguous (n1 x n1)
  double* U = S0 + (int64_t)n1 * n1;         // L21 X11 (n2 x n1)
  double* Ut = U + (int64_t)n2 * n1;         // U^T (n1 x n2)
  double* S3 = Ut + (int64_t)n1 * n2;        // X22^T contiguous (n2 x n2)
  double* W = S0;                            // U^T X22^T (n1 x n2), over S0 once U is made
  if ((e = copy_scaled(X, ldx, n1, n1, S0, n1, false, 1.0, st)) != cudaSuccess) return e;
  if ((e = gemm_tc(g, L + n1, ldl, n2, n1, S0, U, n2, st)) != cudaSuccess) return e;
  if ((e = copy_scaled(U, n2, n2, n1, Ut, n1, true, 1.0, st)) != cudaSuccess) return e;
  if ((e = copy_scaled(X + n1 + (int64_t)n1 * ldx, ldx, n2, n2, S3, n2, true, 1.0, st)) !=
      cudaSuccess)
    return e;
  if ((e = gemm_tc(g, Ut, n1, n1, n2, S3, W, n1, st)) != cudaSuccess) return e;
  // X21 = -W^T; X12 = 0
  if ((e = copy_scaled(W, n1, n1, n2, X + n1, ldx, true, -1.0, st)) != cudaSuccess) return e;
  return cudaMemset2DAsync(X + (int64_t)n1 * ldx, ldx * sizeof(double), 0, n1 * sizeof(double),
                           n2, st);
}

// Lw = strict lower triangle of S + I / 2 (b x b): the transpose of T^-1 for a
// block of unit reflectors H = I - 2 v v^T (S = Y^T Y)
__global__ void k_wy_tinv_t(const double* __restrict__ S, int b, double* __restrict__ Lw) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= b * b) return;
  const int i = t % b, j = t / b;
  Lw[t] = i > j ? S[t] : (i == j ? 0.5 : 0.0);
}

// X (m x n, ldx) -= P (m x n, ldp)
__global__ void k_sub_block(double* __restrict__ X, int64_t ldx, const double* __restrict__ P,
                            int64_t ldp, int m, int n) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)m * n) return;
  const int i = (int)(t % m), j = (int)(t / m);
  X[i + (int64_t)j * ldx] -= P[i + (int64_t)j * ldp];
}

// X <- H_0 H_1 ... H_{n-3} X for the reflectors stored as the columns of Hv
// (column k: v_k, entries k + 1 .. n - 1), in blocks of kWy reflectors from
// the last block to the first: a block is I - Y T Y^T with T upper triangular,
// T^-1 = strict upper triangle of Y^T Y + I / 2 (compact WY form), applied as
// X_r -= Y_r (T (Y_r^T X_r)) on the rows r >= j0 + 1 the block touches, all
// products tensor-core GEMMs.  scratch: 4 n^2 doubles.
constexpr int kWy = 128;
cudaError_t backtransform_wy(const EigGemm& g, const double* Hv, double* X, int n,
                             double* scratch, cudaStream_t st) {
  const int nref = n - 2;  // reflectors 0 .. n - 3
  if (nref <= 0) return cudaSuccess;
  double* Yt = scratch;                          // b x n_r
  double* S = Yt + (int64_t)kWy * n;             // b x b
  double* Lw = S + kWy * kWy;                    // b x b
  double* TT = Lw + kWy * kWy;                   // b x b (T^T)
  double* T = TT + kWy * kWy;                    // b x b
  double* W1 = T + kWy * kWy;                    // b x n
  double* W2 = W1 + (int64_t)kWy * n;            // b x n
  double* P = W2 + (int64_t)kWy * n;             // n_r x n
  cudaError_t e;
  for (int j0 = (nref - 1) / kWy * kWy; j0 >= 0; j0 -= kWy) {
    const int b = std::min(kWy, nref - j0);
    const int r0 = j0 + 1, nr = n - r0;
    const double* Yr = Hv + r0 + (int64_t)j0 * n;  // n_r x b, ld n
    if ((e = copy_scaled(Yr, n, nr, b, Yt, b, true, 1.0, st)) != cudaSuccess) return e;
    if ((e = tc_gemm_f64(Yt, b, b, nr, Yr, n, b, S, b, g.SA, g.SZ, g.esc, g.status, st)) !=
        cudaSuccess)
      return e;
    note_launch(), k_wy_tinv_t<<<(b * b + 255) / 256, 256, 0, st>>>(S, b, Lw);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = trinv_leaf(Lw, b, b, TT, b, st)) != cudaSuccess) return e;  // TT = T^T
    if ((e = copy_scaled(TT, b, b, b, T, b, true, 1.0, st)) != cudaSuccess) return e;
    if ((e = tc_gemm_f64(Yt, b, b, nr, X + r0, n, n, W1, b, g.SA, g.SZ, g.esc, g.status, st)) !=
        cudaSuccess)
      return e;
    if ((e = tc_gemm_f64(T, b, b, b, W1, b, n, W2, b, g.SA, g.SZ, g.esc, g.status, st)) !=
        cudaSuccess)
      return e;
    if ((e = tc_gemm_f64(Yr, n, nr, b, W2, b, n, P, nr, g.SA, g.SZ, g.esc, g.status, st)) !=
        cudaSuccess)
      return e;
    note_launch(), k_sub_block<<<(unsigned)(((int64_t)nr * n + 255) / 256), 256, 0, st>>>(
        X + r0, n, P, nr, nr, n);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Whether the tensor-core mode runs for n: the GEMM's digit buffers must hold
// six digits of an n x n operand (both factors) and its exponent tables.
// Blocked Cholesky A = L L^T (tensor-core mode), panels of kLeafMax columns:
// the diagonal block in shared memory (k_potrf_leaf); the panel below it
// L21 = A21 L11^-T with the leaf inverse and a tensor-core GEMM; the trailing
// matrix A22 -= L21 L21^T by a tensor-core GEMM and a subtraction.  The lower
// triangle of A holds L on return (the strict upper triangle is left as it
// was, except inside A22, where it is scratch).  big: (n - 128)^2 doubles;
// small: 2 * 128^2 + 256 n doubles.
cudaError_t cholesky_tc(const EigGemm& g, double* A, int n, int* status, double* big,
                        double* small, cudaStream_t st) {
  constexpr int nb = kLeafMax;
  cudaError_t e;
  for (int j0 = 0; j0 < n; j0 += nb) {
    const int jb = std::min(nb, n - j0), rem = n - j0 - jb;
    double* A11 = A + j0 + (int64_t)j0 * n;
    if ((e = potrf_leaf(A11, n, jb, status, st)) != cudaSuccess) return e;
    if (rem == 0) break;
    double* X11 = small;                       // L11^-1 (jb x jb)
    double* Xt = X11 + nb * nb;                // L11^-T
    double* P = Xt + nb * nb;                  // L21 (rem x jb)
    double* Pt = P + (int64_t)rem * jb;        // L21^T (jb x rem)
    double* A21 = A11 + jb;
    double* A22 = A21 + (int64_t)jb * n;
    if ((e = trinv_leaf(A11, n, jb, X11, jb, st)) != cudaSuccess) return e;
    if ((e = copy_scaled(X11, jb, jb, jb, Xt, jb, true, 1.0, st)) != cudaSuccess) return e;
    if ((e = gemm_tc(g, A21, n, rem, jb, Xt, P, rem, st)) != cudaSuccess) return e;
    if ((e = copy_scaled(P, rem, rem, jb, A21, n, false, 1.0, st)) != cudaSuccess) return e;
    if ((e = copy_scaled(P, rem, rem, jb, Pt, jb, true, 1.0, st)) != cudaSuccess) return e;
    if ((e = tc_gemm_f64(P, rem, rem, jb, Pt, jb, rem, big, rem, g.SA, g.SZ, g.esc, g.status,
                         st)) != cudaSuccess)
      return e;
    note_launch(), k_sub_block<<<(unsigned)(((int64_t)rem * rem + 255) / 256), 256, 0, st>>>(
        A22, n, big, rem, rem, rem);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

bool tc_eig_fits(const EigGemm* g, int n) {
  if (!g || !g->SA || !g->SZ || !g->esc || n < kTcEigMin) return false;
  const size_t ldk = (size_t)(n + 7) / 8 * 8;
  const size_t need = 6 * (size_t)((n + 127) / 128 * 128) * ldk;
  const size_t nq = (ldk + 255) / 256, MP = (n + 127) / 128 * 128;
  const size_t esc = 4 * ((n + 63) / 64 * 64) + nq * 2 * MP + 256;
  return g->sa_elems >= need && g->sz_elems >= 6 * ldk * n && g->esc_bytes >= esc;
}

// Checked enqueue: return the first failing runtime call's error at once.
#define EK(expr)                      \
  do {                                \
    const cudaError_t e_ = (expr);    \
    if (e_ != cudaSuccess) return e_; \
  } while (0)
// Kernel launch followed by the launch check.
#define EL(...)                   \
  do {                            \
    note_launch();                \
    __VA_ARGS__;                  \
    EK(cudaGetLastError());       \
  } while (0)

cudaError_t gen_eig(EigWork& w, const double* Hs, const double* Ms, int n, double* lam, double* Z,
                    cudaStream_t st, const EigGemm* g) {
  // Buffers (n x n unless noted): L (Cholesky factor of Ms, kept to the end),
  // A, W, V, lu (4 n x n), piv (n x n ints).  status[0]: NOT_SPD/NUMERIC of the
  // problem; status[1]: failure of the internal re-orthonormalisation.
  const int64_t nn = (int64_t)n * n;
  const int nb = blocks_for(nn);
  const dim3 tb(32, 8), tg((n + 31) / 32, (n + 31) / 32);
  int* st0 = w.status;
  int* st1 = w.status + 1;
  EK(cudaMemsetAsync(w.status, 0, 2 * sizeof(int), st));  // words 2, 3: GEMM / stencil waits
  const bool tcm = tc_eig_fits(g, n) && w.X0 && w.X1;
  // 1. Ms = L L^T
  EK(cudaMemcpyAsync(w.W, Ms, nn * 8, cudaMemcpyDeviceToDevice, st));
  if (tcm)
    EK(cholesky_tc(*g, w.W, n, st0, w.X0, w.lu, st));
  else
    EK(cholesky(w.W, n, st0, st));
  EL(k_tril_copy<<<nb, 256, 0, st>>>(w.W, w.L, n));
  EL(k_transpose<<<tg, tb, 0, st>>>(w.L, w.V, n));  // V = L row-major (forward solves)
  // 2. A = sym(L^-1 (L^-1 Hs)^T)
  if (tcm) {
    EK(trinv_lower(*g, w.L, n, n, w.X0, n, w.lu, st));           // X0 = L^-1
    EK(copy_scaled(w.X0, n, n, n, w.X1, n, true, 1.0, st));       // X1 = L^-T
    EK(gemm_tc(*g, Hs, n, n, n, w.X1, w.W, n, st));                // W = Hs L^-T
    EK(gemm_tc(*g, w.X0, n, n, n, w.W, w.V, n, st));               // V = L^-1 Hs L^-T
    EL(k_symmetrize<<<nb, 256, 0, st>>>(w.V, w.A, n));
  } else {
    EK(trsm<true>(w.V, Hs, w.W, n, st0, st));          // W = L^-1 Hs
    EL(k_transpose<<<tg, tb, 0, st>>>(w.W, w.A, n));  // A = W^T
    EK(trsm<true>(w.V, w.A, w.W, n, st0, st));         // W = L^-1 W^T
    EL(k_symmetrize<<<nb, 256, 0, st>>>(w.W, w.A, n));
  }
  // 3. Householder tridiagonalisation; reflectors in the rows of Hv = lu[0, nn)
  double* Hv = w.lu;
  double* p = w.tau;
  bool coop_done = false;
  if (n >= 64) {
    int dev = 0, per_sm = 0, coop = 0;
    EK(cudaGetDevice(&dev));
    EK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    const int sms = sm_count();
    // one CTA per SM (fewest arrivals per grid barrier): 256 threads while the
    // barriers dominate a step (measured: Ns = 1300 78 ms, 88 ms with 512 or
    // with two CTAs of 256 per SM), 512 once the rank-2 updates do (Ns = 4800:
    // 895 ms, 926 ms with two CTAs of 256, 1036 with one)
    const int hthreads = n < 2048 ? 256 : kHouseThreads;
    const size_t vbytes = (size_t)n * sizeof(double);
    if (vbytes > 48 * 1024)
      EK(cudaFuncSetAttribute(k_house_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)std::min<size_t>(vbytes, 200 * 1024)));
    if (vbytes <= 200 * 1024)
      EK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_house_persistent, hthreads,
                                                       vbytes));
    else
      per_sm = 0;  // the reflector would not fit in shared memory: per-step kernels
    if (coop && sms > 0 && per_sm > 0) {
      int blocks = sms * std::min(per_sm, 1);
      GridBar gb{reinterpret_cast<unsigned*>(w.status + 8), reinterpret_cast<unsigned*>(w.status + 9),
                 w.status + 4, wait_cycles()};
      EK(cudaMemsetAsync(w.status + 4, 0, sizeof(int), st));
      EK(cudaMemsetAsync(w.status + 8, 0, 2 * sizeof(int), st));
      double* Ap = w.A;
      double* dp = w.d;
      double* ep = w.e;
      int nn_ = n;
      void* args[] = {&Ap, &Hv, &dp, &ep, &p, &nn_, &gb};
      note_launch();
      // a refused cooperative launch (e.g. not enough co-resident blocks)
      // falls back to the per-step kernels below
      if (cudaLaunchCooperativeKernel((void*)k_house_persistent, dim3(blocks), dim3(hthreads), args,
                                      vbytes, st) == cudaSuccess)
        coop_done = true;
      else
        cudaGetLastError();
    }
  }
  for (int k = 0; !coop_done && k + 2 < n; ++k) {
    EL(k_house_vec<<<1, 256, 0, st>>>(w.A, Hv, w.d, w.e, n, k));
    int m = n - k - 1;
    EL(k_house_matvec<<<(m + 7) / 8, 256, 0, st>>>(w.A, Hv, p, n, k));
    int ub = (int)std::min<int64_t>(((int64_t)m * m + 255) / 256, 1024);
    EL(k_house_update<<<ub, 256, 0, st>>>(w.A, Hv, p, n, k));
  }
  EL(k_house_tail<<<1, 32, 0, st>>>(w.A, Hv, w.d, w.e, n));
  EK(cudaMemcpyAsync(w.A, Hv, nn * 8, cudaMemcpyDeviceToDevice, st));  // reflectors -> A
  // 4. eigenvalues of T (ascending)
  double* e2 = w.tau + n;
  EL(k_gersh<<<1, 1024, 0, st>>>(w.d, w.e, n, e2, w.scal));
  if (n < 2048)
    EL(k_bisect<8><<<(n * 8 + 127) / 128, 128, 0, st>>>(w.d, e2, n, w.scal, lam));
  else
    EL(k_bisect<4><<<(n * 4 + 127) / 128, 128, 0, st>>>(w.d, e2, n, w.scal, lam));
  // 5. eigenvectors of T into W (column-major); factors in lu (4 n x n)
  EL(k_clusters<<<1, 32, 0, st>>>(lam, n, w.scal, w.clus));
  double* VT = w.W;
  // (V is idle here: it holds the singletons' vectors row-major, then they
  // are transposed into VT before the clusters are iterated there)
  EL(k_inviter_single<<<(n + 31) / 32, 32, 0, st>>>(w.d, w.e, lam, w.scal, w.clus, n, w.lu,
                                                    w.piv, w.V));
  EL(k_transpose<<<tg, tb, 0, st>>>(w.V, VT, n));
  EL(k_inviter_cluster<<<n, 256, 0, st>>>(w.d, w.e, lam, w.scal, w.clus, n, w.lu, w.piv, VT));
  //    Cholesky-QR pass: G = VT^T VT = R R^T, Q = VT R^-T  (Q^T = R^-1 VT^T)
  if (tcm) {
    double* G = w.lu + nn;
    EK(copy_scaled(VT, n, n, n, w.V, n, true, 1.0, st));            // V = VT^T
    EK(gemm_tc(*g, w.V, n, n, n, VT, G, n, st));                     // G = VT^T VT
    EK(cholesky_tc(*g, G, n, st1, w.X0, w.lu + 2 * nn, st));
    EL(k_tril_copy<<<nb, 256, 0, st>>>(G, w.V, n));                  // V = R (lower)
    EK(trinv_lower(*g, w.V, n, n, w.X0, n, w.lu + 2 * nn, st));      // X0 = R^-1
    EK(copy_scaled(w.X0, n, n, n, G, n, true, 1.0, st));             // G = R^-T
    EK(gemm_tc(*g, VT, n, n, n, G, w.V, n, st));                     // V = VT R^-T = Q
    EK(cudaMemcpyAsync(VT, w.V, nn * 8, cudaMemcpyDeviceToDevice, st));
  } else {
    double* G1 = w.lu;           // unused copy (projection writes two outputs)
    double* G = w.lu + nn;
    double* work = w.lu + 2 * nn;  // 2 nn doubles for one split
    EK(project_simt<double>(VT, VT, n, n, n, G1, G, work, 1, st));
    EK(cholesky(G, n, st1, st));
    EL(k_tril_copy<<<nb, 256, 0, st>>>(G, w.V, n));            // V = R (column-major)
    EL(k_transpose<<<tg, tb, 0, st>>>(w.V, w.lu, n));          // lu0 = R row-major
    EL(k_transpose<<<tg, tb, 0, st>>>(VT, w.lu + 2 * nn, n));  // lu2 = VT^T column-major
    EK(trsm<true>(w.lu, w.lu + 2 * nn, w.lu + nn, n, st1, st));  // lu1 = Q^T
    EL(k_transpose<<<tg, tb, 0, st>>>(w.lu + nn, VT, n));      // VT = Q
  }
  // 6. V = Q_house VT (all reflectors, warp per column)
  if (tcm) {
    EK(backtransform_wy(*g, w.A, VT, n, w.lu, st));
  } else {
    int wpb = col_warps(n);
    size_t smem = (size_t)wpb * n * sizeof(double);
    if (smem > 48 * 1024)
      EK(cudaFuncSetAttribute(k_backtransform, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem));
    EL(k_backtransform<<<(n + wpb - 1) / wpb, wpb * 32, smem, st>>>(w.A, VT, n));
  }
  // 7. Z = L^-T V; sign convention; NaN check
  if (tcm)
    EK(gemm_tc(*g, w.X1, n, n, n, VT, Z, n, st));
  else
    EK(trsm<false>(w.L, VT, Z, n, st0, st));
  EL(k_fix_signs<<<(n * 32 + 255) / 256, 256, 0, st>>>(Z, n, lam, st0));
  return cudaSuccess;
}
#undef EL
#undef EK

// ---------------------------------------------------------------------------
// Batched eigensolver.  One thread-block cluster ("team") per problem runs the
// steps of gen_eig above, in the same order, with cluster barriers (release /
// acquire at cluster scope, so each step sees the global-memory writes of the
// previous one) in place of kernel boundaries and grid barriers.  On one SM or
// a few, the FP64 pipe bounds this kernel, so two steps take a form with fewer
// FP64 instructions than gen_eig's: the triangular solves go 32 unknowns at a
// time (a reciprocal of each pivot instead of a division per row, no
// reduction across the warp per row), and the eigenvalues of T come from plain
// bisection (one Sturm count per bit) instead of multisection.  Work inside a
// step is spread over the team's threads (element loops), warps (one
// right-hand side or matrix column per warp) or single threads (one
// eigenvalue each).  Buffers: A (Ms copy, then the reduced matrix, then the
// reflectors, reflector k in column k below the diagonal), L / V (Cholesky
// factor column- and row-major), W (L^-1 Hs, later the eigenvectors of T), lu
// (4 n^2: scratch, then the inverse-iteration factors, then the
// re-orthonormalisation's factor, Gram matrix and Q).  Every control decision
// (loop bounds, a non-positive pivot) depends only on values that every
// thread of the team reads after the same barrier, so all CTAs of a cluster
// pass the same barriers and leave together.
// ---------------------------------------------------------------------------
namespace {

constexpr int kEbThreads = 512;
constexpr int kEbWarps = kEbThreads / 32;

struct Team {
  int tid, nthr, warp, nwarps, lane;
  bool lead;  // thread 0 of the team's first CTA
};

__device__ __forceinline__ void team_sync() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Cholesky S = L L^T of the symmetric n x n S (column-major; the lower triangle
// is read and updated in place, right-looking, one column per step).  Writes
// the factor column-major into Lc and row-major into Lr (lower entries only).
// Returns false, on every thread alike, at a non-positive or non-finite pivot.
// The pivot's square root and reciprocal are formed once per CTA (thread 0)
// and shared through bc[0..1]: every warp computing them would cost the FP64
// pipe as much as distinct values.
__device__ bool team_cholesky(double* S, double* Lc, double* Lr, int n, const Team& t,
                              double* bc) {
  for (int k = 0; k < n; ++k) {
    const double akk = S[k + (int64_t)k * n];
    if (!(akk > 0.0) || !isfinite(akk)) return false;
    if (threadIdx.x == 0) {
      const double r = sqrt(akk);
      bc[0] = r;
      bc[1] = 1.0 / r;
    }
    __syncthreads();
    const double s = bc[0];
    const double linv = bc[1];
    for (int i = k + t.tid; i < n; i += t.nthr) {
      const double l = i == k ? s : S[i + (int64_t)k * n] * linv;
      Lc[i + (int64_t)k * n] = l;
      Lr[(int64_t)i * n + k] = l;
    }
    for (int j = k + 1 + t.warp; j < n; j += t.nwarps) {
      const double lj = S[j + (int64_t)k * n] * linv;
      for (int i = j + t.lane; i < n; i += 32)
        S[i + (int64_t)j * n] -= (S[i + (int64_t)k * n] * linv) * lj;
    }
    team_sync();
  }
  return true;
}

// One warp solves L x = b (FWD) or L^T x = b (!FWD) for lower-triangular L,
// with b and x in the warp's shared memory, 32 unknowns at a time: lane l
// owns unknown i = i0 + l.  The sum over the unknowns of earlier blocks is
// each lane's own dot product, read coalesced from F (FWD: L column-major,
// F[i + k n] = L(i, k); !FWD: L row-major, F[k n + i] = L(k, i)); inside the
// 32 x 32 diagonal block the unknowns follow one another, each broadcast by a
// shuffle and multiplied by the reciprocal of its pivot.
template <bool FWD>
__device__ void warp_trsv(const double* __restrict__ F, int n, const double* b, double* x,
                          int lane) {
  const int nblk = (n + 31) / 32;
  for (int bq = 0; bq < nblk; ++bq) {
    const int i0 = FWD ? bq * 32 : (nblk - 1 - bq) * 32;
    const int nb = min(32, n - i0);
    const int i = i0 + lane;
    const bool act = lane < nb;
    double s0 = 0.0, s1 = 0.0;
    if (act) {
      if (FWD) {
        int k = 0;
        for (; k + 1 < i0; k += 2) {
          s0 += F[i + (int64_t)k * n] * x[k];
          s1 += F[i + (int64_t)(k + 1) * n] * x[k + 1];
        }
        if (k < i0) s0 += F[i + (int64_t)k * n] * x[k];
      } else {
        int k = i0 + 32;
        for (; k + 1 < n; k += 2) {
          s0 += F[(int64_t)k * n + i] * x[k];
          s1 += F[(int64_t)(k + 1) * n + i] * x[k + 1];
        }
        if (k < n) s0 += F[(int64_t)k * n + i] * x[k];
      }
    }
    double r = act ? b[i] - (s0 + s1) : 0.0;
    const double dinv = act ? 1.0 / F[i + (int64_t)i * n] : 0.0;
    for (int q = 0; q < nb; ++q) {
      const int qq = FWD ? q : nb - 1 - q;
      const double xq = __shfl_sync(0xffffffffu, r * dinv, qq);
      if (lane == qq) x[i] = xq;
      if (act && (FWD ? lane > qq : lane < qq))
        r -= (FWD ? F[i + (int64_t)(i0 + qq) * n] : F[(int64_t)(i0 + qq) * n + i]) * xq;
    }
    __syncwarp();
  }
}

// Columns c = warp, warp + nwarps, ...: x = L^-1 b with b[i] = B[c bc + i bs],
// stored to X[c xc + i xs]; Lc: L column-major.
__device__ void team_forward(const double* Lc, const double* B, int64_t bc, int64_t bs, double* X,
                             int64_t xc, int64_t xs, int n, double* wb, double* wx,
                             const Team& t) {
  for (int c = t.warp; c < n; c += t.nwarps) {
    for (int i = t.lane; i < n; i += 32) wb[i] = B[c * bc + i * bs];
    __syncwarp();
    warp_trsv<true>(Lc, n, wb, wx, t.lane);
    for (int i = t.lane; i < n; i += 32) X[c * xc + i * xs] = wx[i];
    __syncwarp();
  }
}

// block-wide sum over the CTA's threads (every thread gets the result)
__device__ double cta_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum_d(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  // every warp sums the warps' partials by shuffles (the same order in each)
  const double w = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
  return warp_sum_d(w);
}

__global__ void __launch_bounds__(kEbThreads, 1)
    k_eig_batch(const EigBatchItem* __restrict__ items, int count) {
  extern __shared__ double ebsh[];
  __shared__ double red[32];
  unsigned rank, csize;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(csize));
  const int item = (int)(blockIdx.x / csize);
  if (item >= count) return;  // whole clusters only
  const EigBatchItem P = items[item];
  const int n = P.n;
  const int64_t nn = (int64_t)n * n;
  Team t;
  t.tid = (int)(rank * blockDim.x + threadIdx.x);
  t.nthr = (int)(csize * blockDim.x);
  t.lane = threadIdx.x & 31;
  t.warp = t.tid >> 5;
  t.nwarps = t.nthr >> 5;
  t.lead = t.tid == 0;
  double* vsh = ebsh;      // reflector (n)
  double* qsh = ebsh + n;  // 2 q of the rank-2 update (n)
  double* wb = ebsh + 2 * (int64_t)n + (int64_t)(threadIdx.x >> 5) * 2 * n;  // per warp
  double* wx = wb + n;
  double *A = P.A, *L = P.L, *V = P.V, *W = P.W, *lu = P.lu;

  // 1. Ms = L L^T (A <- Ms; factor into L column-major and V row-major)
  for (int64_t q = t.tid; q < nn; q += t.nthr) A[q] = P.Ms[q];
  team_sync();
  if (!team_cholesky(A, L, V, n, t, red + 16)) {
    if (t.lead) atomicCAS(P.status, 0, ST_NOT_SPD);
    return;
  }
  // 2. W = L^-1 Hs; lu = L^-1 W^T; A = sym(lu)
  team_forward(L, P.Hs, n, 1, W, n, 1, n, wb, wx, t);
  team_sync();
  team_forward(L, W, 1, n, lu, n, 1, n, wb, wx, t);
  team_sync();
  for (int j = t.warp; j < n; j += t.nwarps)
    for (int i = t.lane; i < n; i += 32)
      A[i + (int64_t)j * n] = 0.5 * (lu[i + (int64_t)j * n] + lu[j + (int64_t)i * n]);
  team_sync();
  // 3. Householder reduction (steps as in k_house_persistent); reflector k is
  //    kept in column k of A below the diagonal (no later step reads it)
  double* p = P.tau;
  for (int k = 0; k + 2 < n; ++k) {
    const double* col = A + (int64_t)k * n;
    double acc = 0.0;
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) acc += col[i] * col[i];
    const double xx = cta_sum(acc, red);  // (every warp holds the same sum)
    if (threadIdx.x == 0) red[16] = sqrt(xx);
    __syncthreads();
    const double xn = red[16];
    const double x0 = col[k + 1];
    const double alpha = x0 >= 0.0 ? -xn : xn;
    double vn2 = 0.0;
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) {
      const double v = col[i] - (i == k + 1 ? alpha : 0.0);
      vn2 += v * v;
    }
    const double vv = cta_sum(vn2, red);
    if (threadIdx.x == 0) red[17] = sqrt(vv);
    __syncthreads();
    const double vn = red[17];
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x)
      vsh[i] = (xn > 0.0 && vn > 0.0) ? (col[i] - (i == k + 1 ? alpha : 0.0)) / vn : 0.0;
    __syncthreads();
    if (t.lead) {
      P.d[k] = col[k];
      P.e[k] = xn > 0.0 ? alpha : 0.0;
    }
    // p = A v, warp per row, four rows at a time (their loads overlap)
    for (int i0 = k + 1 + 4 * t.warp; i0 < n; i0 += 4 * t.nwarps) {
      double s4[4] = {0.0, 0.0, 0.0, 0.0};
      for (int j = k + 1 + t.lane; j < n; j += 32) {
        const double vj = vsh[j];
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (i0 + r < n) s4[r] += A[(int64_t)(i0 + r) * n + j] * vj;
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const double v = warp_sum_d(s4[r]);
        if (t.lane == 0 && i0 + r < n) p[i0 + r] = v;
      }
    }
    team_sync();
    acc = 0.0;
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) acc += vsh[i] * p[i];
    const double K = cta_sum(acc, red);
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) qsh[i] = 2.0 * (p[i] - K * vsh[i]);
    __syncthreads();
    // element q = r + m c of the trailing block (row k+1+r, column k+1+c);
    // each thread steps q by the team size, carrying (r, c) without dividing
    const int m = n - k - 1;
    const int sq = t.nthr / m, sr = t.nthr % m;
    for (int r = t.tid % m, c = t.tid / m; c < m;) {
      const int i = k + 1 + r, j = k + 1 + c;
      A[i + (int64_t)j * n] -= vsh[i] * qsh[j] + qsh[i] * vsh[j];
      r += sr;
      c += sq;
      if (r >= m) {
        r -= m;
        ++c;
      }
    }
    if (rank == 0)
      for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[i + (int64_t)k * n] = vsh[i];
    team_sync();
  }
  if (t.lead) {
    for (int k = n >= 2 ? n - 2 : 0; k < n; ++k) P.d[k] = A[k + (int64_t)k * n];
    if (n >= 2) P.e[n - 2] = A[(n - 1) + (int64_t)(n - 2) * n];
  }
  team_sync();
  // 4. eigenvalues of T: Gershgorin interval (first CTA), then bisection
  double* e2 = P.tau + n;
  if (rank == 0) {
    double lo = 1e300, hi = -1e300, emax = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double r = (i > 0 ? fabs(P.e[i - 1]) : 0.0) + (i + 1 < n ? fabs(P.e[i]) : 0.0);
      lo = fmin(lo, P.d[i] - r);
      hi = fmax(hi, P.d[i] + r);
      if (i + 1 < n) {
        e2[i] = P.e[i] * P.e[i];
        emax = fmax(emax, e2[i]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    }
    __shared__ double gsh[3][32];
    if (t.lane == 0) {
      gsh[0][threadIdx.x >> 5] = lo;
      gsh[1][threadIdx.x >> 5] = hi;
      gsh[2][threadIdx.x >> 5] = emax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        lo = fmin(lo, gsh[0][w]);
        hi = fmax(hi, gsh[1][w]);
        emax = fmax(emax, gsh[2][w]);
      }
      const double tnorm = fmax(fabs(lo), fabs(hi));
      const double pad = 2.2e-16 * tnorm * n + 1e-300;
      P.scal[0] = lo - pad;
      P.scal[1] = hi + pad;
      P.scal[2] = fmax(2.2250738585072014e-308 * fmax(1.0, emax), 1e-300);
      P.scal[3] = tnorm;
    }
  }
  team_sync();
  {
    // eigenvalues dealt round-robin over the cluster's CTAs, L lanes each:
    // where a CTA holds few eigenvalues the Sturm recurrence's latency binds
    // and multisection's fewer rounds win, where it holds many the FP64 pipe
    // binds and bisection's fewer counts do
    const int per_cta = (n + (int)csize - 1) / (int)csize;
    const int L = per_cta > 96 ? 1 : per_cta > 48 ? 2 : 4;
    const int groups = (int)blockDim.x / L;
    for (int g0 = 0; g0 * (int)csize < n; g0 += groups) {
      const int j = (int)rank + (int)csize * (g0 + (int)threadIdx.x / L);
      if (j < n) {
        double v;
        if (L == 4)
          v = multisect_eig<4>(P.d, e2, n, P.scal, j);
        else if (L == 2)
          v = multisect_eig<2>(P.d, e2, n, P.scal, j);
        else
          v = bisect_eig(P.d, e2, n, P.scal, j);
        if ((threadIdx.x & (L - 1)) == 0) P.lam[j] = v;
      }
    }
  }
  team_sync();
  if (t.lead) {  // clusters of nearly equal eigenvalues (as k_clusters)
    const double tol = 1e-9 * fmax(P.scal[3], 1e-300);
    int start = 0;
    for (int j = 1; j <= n; ++j) {
      if (j == n || P.lam[j] - P.lam[j - 1] > tol) {
        for (int q = start; q < j; ++q) {
          P.clus[q] = start;
          P.clus[n + q] = j - start;
        }
        start = j;
      }
    }
  }
  team_sync();
  // 5. eigenvectors of T into W by inverse iteration: singletons thread per
  //    eigenvalue, clusters warp per cluster (members in order, Gram-Schmidt
  //    twice against the earlier ones), then Cholesky-QR
  {
    const double pivmin = fmax(2.2e-16 * P.scal[3], 1e-300);
    for (int j = (int)(rank + csize * threadIdx.x); j < n; j += t.nthr) {
      if (P.clus[n + j] != 1) continue;
      TriLU F{lu, P.piv, n, n, j};
      tri_factor(F, P.d, P.e, P.lam[j], pivmin);
      double* x = W + (int64_t)j * n;
      for (int i = 0; i < n; ++i) x[i] = start_value(0x5EEDull + j, i);
      for (int it = 0; it < kInvIters; ++it) {
        scale_maxabs(x, n);
        tri_solve(F, x);
      }
      double s = 0.0;
      for (int i = 0; i < n; ++i) s += x[i] * x[i];
      const double inv = 1.0 / sqrt(s);
      for (int i = 0; i < n; ++i) x[i] *= inv;
    }
    const double sep = 10.0 * 2.2e-16 * fmax(P.scal[3], 1e-300);
    for (int j0 = t.warp; j0 < n; j0 += t.nwarps) {
      if (P.clus[j0] != j0 || P.clus[n + j0] < 2) continue;
      const int size = P.clus[n + j0];
      double shift_prev = 0.0;
      for (int m = 0; m < size; ++m) {
        const int j = j0 + m;
        double sigma = P.lam[j];
        if (m > 0 && sigma - shift_prev < sep) sigma = shift_prev + sep;
        shift_prev = sigma;
        TriLU F{lu, P.piv, n, n, j};
        if (t.lane == 0) tri_factor(F, P.d, P.e, sigma, pivmin);
        double* x = W + (int64_t)j * n;
        for (int i = t.lane; i < n; i += 32) x[i] = start_value(0x5EEDull + j, i);
        __syncwarp();
        for (int it = 0; it < kInvIters; ++it) {
          if (t.lane == 0) {
            scale_maxabs(x, n);
            tri_solve(F, x);
          }
          __syncwarp();
          for (int pass = 0; pass < 2; ++pass) {
            for (int q = 0; q < m; ++q) {
              const double* y = W + (int64_t)(j0 + q) * n;
              double acc = 0.0;
              for (int i = t.lane; i < n; i += 32) acc += y[i] * x[i];
              const double c = warp_sum_d(acc);
              for (int i = t.lane; i < n; i += 32) x[i] -= c * y[i];
              __syncwarp();
            }
          }
          double acc = 0.0;
          for (int i = t.lane; i < n; i += 32) acc += x[i] * x[i];
          const double nrm = sqrt(warp_sum_d(acc));
          const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
          for (int i = t.lane; i < n; i += 32) x[i] *= inv;
          __syncwarp();
        }
      }
    }
  }
  team_sync();
  //    G = W^T W (lower triangle, into lu[n^2, 2n^2)), G = R R^T, Q = W R^-T
  double* G = lu + nn;
  for (int j = t.warp; j < n; j += t.nwarps) {
    const double* wj = W + (int64_t)j * n;
    for (int i = t.lane; i < n; i += 32) wb[i] = wj[i];
    __syncwarp();
    for (int i = j; i < n; ++i) {
      const double* wi = W + (int64_t)i * n;
      double acc = 0.0;
      for (int r = t.lane; r < n; r += 32) acc += wi[r] * wb[r];
      acc = warp_sum_d(acc);
      if (t.lane == 0) G[i + (int64_t)j * n] = acc;
    }
    __syncwarp();
  }
  team_sync();
  if (!team_cholesky(G, lu, lu + 2 * nn, n, t, red + 16)) {
    if (t.lead) atomicCAS(P.status + 1, 0, ST_NUMERIC);
    return;
  }
  //    row c of Q = R^-1 (row c of W), into lu[3 n^2, 4 n^2)
  double* Q = lu + 3 * nn;
  team_forward(lu, W, 1, n, Q, 1, n, n, wb, wx, t);
  team_sync();
  // 6.-7. per column c (warp): apply the reflectors to column c of Q, solve
  //    L^T z = (that column), make its largest-magnitude entry positive
  for (int c = t.warp; c < n; c += t.nwarps) {
    for (int i = t.lane; i < n; i += 32) wb[i] = Q[i + (int64_t)c * n];
    __syncwarp();
    for (int k = n - 3; k >= 0; --k) {
      const double* v = A + (int64_t)k * n;
      double s = 0.0;
      for (int i = k + 1 + t.lane; i < n; i += 32) s += v[i] * wb[i];
      s = 2.0 * warp_sum_d(s);
      for (int i = k + 1 + t.lane; i < n; i += 32) wb[i] -= s * v[i];
      __syncwarp();
    }
    warp_trsv<false>(V, n, wb, wx, t.lane);
    double best = -1.0;
    int bi = 0;
    bool finite = true;
    for (int i = t.lane; i < n; i += 32) {
      const double a = fabs(wx[i]);
      finite = finite && isfinite(wx[i]);
      if (a > best) {
        best = a;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    const double sg = wx[bi] < 0.0 ? -1.0 : 1.0;
    for (int i = t.lane; i < n; i += 32) P.Z[i + (int64_t)c * n] = sg * wx[i];
    if (!__all_sync(0xffffffffu, finite) && t.lane == 0) atomicCAS(P.status, 0, ST_NUMERIC);
    __syncwarp();
  }
  for (int j = t.tid; j < n; j += t.nthr)
    if (!isfinite(P.lam[j])) atomicCAS(P.status, 0, ST_NUMERIC);
}

size_t eig_batch_smem(int nmax) { return (size_t)(2 + 2 * kEbWarps) * nmax * sizeof(double); }

}  // namespace

EigBatchItem eig_batch_item(const EigWork& w, const double* Hs, const double* Ms, int n,
                            double* lam, double* Z) {
  EigBatchItem it{};
  it.Hs = Hs; it.Ms = Ms; it.lam = lam; it.Z = Z;
  it.L = w.L; it.A = w.A; it.W = w.W; it.V = w.V; it.lu = w.lu;
  it.d = w.d; it.e = w.e; it.tau = w.tau; it.scal = w.scal;
  it.status = w.status; it.clus = w.clus; it.piv = w.piv;
  it.n = n;
  return it;
}

int eig_batch_cluster(int n) {
  int c = n <= 128 ? 1 : n <= 176 ? 2 : n <= 240 ? 4 : 8;
  // largest cluster the device co-schedules with this kernel's shared memory
  static int max_ok[9] = {0};
  static bool probed = false;
  if (!probed) {
    probed = true;
    const size_t smem = eig_batch_smem(kEigBatchMax);
    cudaFuncSetAttribute(k_eig_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    for (int cs = 1; cs <= 8; cs *= 2) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = cs;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(cs);
      cfg.blockDim = dim3(kEbThreads);
      cfg.dynamicSmemBytes = smem;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int nc = 0;
      max_ok[cs] = cudaOccupancyMaxActiveClusters(&nc, k_eig_batch, &cfg) == cudaSuccess && nc > 0;
      cudaGetLastError();
    }
  }
  while (c > 1 && !max_ok[c]) c /= 2;
  return c;
}

cudaError_t eig_batch(const EigBatchItem* items, int count, int cluster, int nmax,
                      cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const size_t smem = eig_batch_smem(std::max(nmax, 1));
  cudaError_t e =
      cudaFuncSetAttribute(k_eig_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)(count * cluster));
  cfg.blockDim = dim3(kEbThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  note_launch();
  return cudaLaunchKernelEx(&cfg, k_eig_batch, items, count);
}

}  // namespace sparc
