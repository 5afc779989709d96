// CheFSI step at a Bloch wavevector k (complex FP64).  The paper computes at
// Gamma in real arithmetic; at any other wavevector of the Brillouin-zone
// sampling every operation of Algorithm 1 is complex (Sec. III, introduction:
// the TiO2 slabs of Sec. IV use Monkhorst-Pack grids).
//
//   H(k) x = -1/2 Lap_k x + Veff o x + sum_J chi^k_J Gamma_J h^3 chi^k_J^H x
//
// Bloch condition psi(r + L_d e_d) = exp(i k_d L_d) psi(r) on periodic axes
// (L_d = N_d h): a neighbour index j = i +- p of the radius-6 stencil is read
// at j mod N_d and multiplied by exp(i k_d L_d q), q = floor(j / N_d); on a
// Dirichlet axis an index outside the grid reads 0 and k_d is unused.  The
// projectors are Bloch sums; with a cut-off below half of every periodic cell
// one image T_i contributes at each support point i (the one nearest r_i), so
// chi^k(r_i) = chi(r_i - R_J - T_i) exp(i k.T_i): the tabulated values times a
// phase made once at create time.
//
// The Rayleigh-Ritz step is Algorithm 1's with ^T replaced by ^H: Hs = Xt^H Yt
// and Ms = Xt^H Xt (Hermitian), Cholesky Ms = L L^H, A = L^-1 Hs L^-H, the
// eigenpairs of the Hermitian A by cyclic Jacobi rotations (unitary by
// construction, so degenerate levels keep orthonormal vectors), Z = L^-H V.
//
// Layout: complex blocks are column-major Nd x Ns with interleaved (re, im)
// FP64 pairs, leading dimension in complex elements; ns x ns matrices are
// column-major complex.  Every reduction runs in a fixed order.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "internal.cuh"

namespace sparc {

namespace {

using cd = double2;  // (re, im)

__device__ __forceinline__ cd cadd(cd a, cd b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cd csub(cd a, cd b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ cd cmul(cd a, cd b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ cd cconj(cd a) { return make_double2(a.x, -a.y); }
// conj(a) * b
__device__ __forceinline__ cd cmulc(cd a, cd b) {
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ cd cscale(double s, cd a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ double cabs2(cd a) { return fma(a.x, a.x, a.y * a.y); }

constexpr int R = kRadius;
constexpr int kQ = 2 * R + 1;  // phases for cell crossings q in [-R, R]

struct KArgs {
  const cd* x;
  int64_t ldx;
  cd* y;
  int64_t ldy;
  const cd* prev;
  int64_t ldp;
  const double* veff;
  const int* pull_ptr;
  const int* pull_k;
  const cd* pull_chi;
  const cd* D;  // D[n * kp + k]
  int kp;
  int n[3], bc[3];
  cd phase[3][kQ];  // exp(i k_d L_d q), q = -R..R
  double diag_minus_shift, off[R + 1], s_h, s_p;
  int ns;
};

// neighbour value at coordinate c + s along axis d (periodic: wrapped with
// the Bloch phase of the crossings; Dirichlet: 0 outside)
__device__ __forceinline__ cd nb(const KArgs& a, const cd* xn, int64_t base, int64_t stride, int c,
                                 int s, int d) {
  const int nn = a.n[d];
  int j = c + s;
  if (j >= 0 && j < nn) return xn[base + (int64_t)(j - c) * stride];
  if (a.bc[d] == SPARC_DIRICHLET) return make_double2(0.0, 0.0);
  int q = j >= 0 ? j / nn : -((-j + nn - 1) / nn);
  const int jm = j - q * nn;
  return cmul(xn[base + (int64_t)(jm - c) * stride], a.phase[d][q + R]);
}

// y = s_h ((H(k) - shift) x) + s_p prev, one thread per (point, orbital)
__global__ void __launch_bounds__(256) k_hpsi_c(const KArgs a) {
  const int64_t nd = (int64_t)a.n[0] * a.n[1] * a.n[2];
  const int n = blockIdx.y;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nd) return;
  const int ix = (int)(i % a.n[0]), iy = (int)((i / a.n[0]) % a.n[1]),
            iz = (int)(i / ((int64_t)a.n[0] * a.n[1]));
  const cd* xn = a.x + (int64_t)n * a.ldx;
  const cd xc = xn[i];
  cd acc = cscale(a.diag_minus_shift + a.veff[i], xc);
  const int64_t sx = 1, sy = a.n[0], sz = (int64_t)a.n[0] * a.n[1];
#pragma unroll
  for (int p = 1; p <= R; ++p) {
    cd s = cadd(nb(a, xn, i, sx, ix, p, 0), nb(a, xn, i, sx, ix, -p, 0));
    s = cadd(s, cadd(nb(a, xn, i, sy, iy, p, 1), nb(a, xn, i, sy, iy, -p, 1)));
    s = cadd(s, cadd(nb(a, xn, i, sz, iz, p, 2), nb(a, xn, i, sz, iz, -p, 2)));
    acc = cadd(acc, cscale(a.off[p], s));
  }
  if (a.kp > 0) {
    const cd* Dn = a.D + (int64_t)n * a.kp;
    for (int e = a.pull_ptr[i]; e < a.pull_ptr[i + 1]; ++e)
      acc = cadd(acc, cmul(a.pull_chi[e], Dn[a.pull_k[e]]));
  }
  cd out = cscale(a.s_h, acc);
  if (a.prev) out = cadd(out, cscale(a.s_p, a.prev[(int64_t)n * a.ldp + i]));
  a.y[(int64_t)n * a.ldy + i] = out;
}

// block sum in a fixed order (thread 0 gets the result)
template <int NT>
__device__ cd block_sum_c(cd v, cd* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = NT / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] = cadd(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  const cd r = sh[0];
  __syncthreads();
  return r;
}

// D[n kp + k] = gamma_k h^3 sum_s conj(chi^k_k(s)) x_n(idx_s): one block per
// (atom, orbital), projectors in turn
__global__ void __launch_bounds__(256)
    k_nl_coef_c(const int64_t* supp_ptr, const int* supp_idx, const int* nproj,
                const int64_t* chi_ptr, const cd* chi, const int* proj_ptr, const double* gamma,
                double h3, const cd* x, int64_t ldx, int kp, cd* D) {
  __shared__ cd sh[256];
  const int J = blockIdx.x, n = blockIdx.y;
  const int64_t s0 = supp_ptr[J];
  const int ns_ = (int)(supp_ptr[J + 1] - s0);
  const cd* xn = x + (int64_t)n * ldx;
  for (int q = 0; q < nproj[J]; ++q) {
    const cd* c = chi + chi_ptr[J] + (int64_t)q * ns_;
    cd acc = make_double2(0.0, 0.0);
    for (int t = threadIdx.x; t < ns_; t += blockDim.x)
      acc = cadd(acc, cmulc(c[t], xn[supp_idx[s0 + t]]));
    acc = block_sum_c<256>(acc, sh);
    if (threadIdx.x == 0) {
      const int k = proj_ptr[J] + q;
      D[(int64_t)n * kp + k] = cscale(gamma[k] * h3, acc);
    }
  }
}

// Hs[p, q] = sum_i conj(X_p(i)) Y_q(i), Ms likewise with X, for p <= q; the
// lower triangle is the conjugate, the diagonal real.  One block per (p, q).
__global__ void __launch_bounds__(256)
    k_project_c(const cd* X, const cd* Y, int64_t ld, int64_t nd, int ns, cd* Hs, cd* Ms) {
  __shared__ cd sh[256];
  const int p = blockIdx.x, q = blockIdx.y;
  if (p > q) return;
  const cd* xp = X + (int64_t)p * ld;
  const cd* xq = X + (int64_t)q * ld;
  const cd* yq = Y + (int64_t)q * ld;
  cd h = make_double2(0.0, 0.0), m = make_double2(0.0, 0.0);
  for (int64_t i = threadIdx.x; i < nd; i += blockDim.x) {
    const cd a = xp[i];
    h = cadd(h, cmulc(a, yq[i]));
    m = cadd(m, cmulc(a, xq[i]));
  }
  h = block_sum_c<256>(h, sh);
  m = block_sum_c<256>(m, sh);
  if (threadIdx.x == 0) {
    if (p == q) {
      h.y = 0.0;
      m.y = 0.0;
    }
    Hs[p + (int64_t)q * ns] = h;
    Ms[p + (int64_t)q * ns] = m;
    Hs[q + (int64_t)p * ns] = cconj(h);
    Ms[q + (int64_t)p * ns] = cconj(m);
  }
}

// Xout_q(i) = sum_p Xt_p(i) Z[p, q], one thread per (point, output column)
__global__ void __launch_bounds__(256)
    k_rotate_c(const cd* Xt, int64_t ld, int64_t nd, int ns, const cd* Z, cd* Xo, int64_t ldo) {
  const int q = blockIdx.y;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nd) return;
  cd acc = make_double2(0.0, 0.0);
  for (int p = 0; p < ns; ++p) acc = cadd(acc, cmul(Xt[(int64_t)p * ld + i], Z[p + (int64_t)q * ns]));
  Xo[(int64_t)q * ldo + i] = acc;
}

// ---- Hermitian generalised eigensolver ----------------------------------
constexpr int kEigThreads = 1024;
constexpr int kMaxSweeps = 40;

// Cholesky M = L L^H (lower, column-major, one block): column j's diagonal,
// then the rows below it; status 4 (NOT_SPD) on a non-positive pivot.
__global__ void __launch_bounds__(kEigThreads) k_cholesky_c(const cd* M, cd* L, int n, int* status) {
  __shared__ double red[kEigThreads];
  __shared__ double djj;
  for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x) L[t] = make_double2(0.0, 0.0);
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int k = threadIdx.x; k < j; k += blockDim.x) s += cabs2(L[j + (int64_t)k * n]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = kEigThreads / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const double d = M[j + (int64_t)j * n].x - red[0];
      if (!(d > 0.0) || !isfinite(d)) {
        atomicCAS(status, 0, SPARC_ERR_NOT_SPD);
        djj = 1.0;
      } else {
        djj = sqrt(d);
      }
      L[j + (int64_t)j * n] = make_double2(djj, 0.0);
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
      cd a = M[i + (int64_t)j * n];
      for (int k = 0; k < j; ++k) a = csub(a, cmul(L[i + (int64_t)k * n], cconj(L[j + (int64_t)k * n])));
      L[i + (int64_t)j * n] = cscale(1.0 / djj, a);
    }
    __syncthreads();
  }
}

// W = L^-1 B (forward substitution), one thread per column of B
__global__ void k_solve_lower_c(const cd* L, const cd* B, cd* W, int n) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  for (int i = 0; i < n; ++i) {
    cd a = B[i + (int64_t)c * n];
    for (int k = 0; k < i; ++k) a = csub(a, cmul(L[i + (int64_t)k * n], W[k + (int64_t)c * n]));
    W[i + (int64_t)c * n] = cscale(1.0 / L[i + (int64_t)i * n].x, a);
  }
}

// W = L^-H B (back substitution on the upper-triangular L^H), one thread per column
__global__ void k_solve_upper_h_c(const cd* L, const cd* B, cd* W, int n) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  for (int i = n - 1; i >= 0; --i) {
    cd a = B[i + (int64_t)c * n];
    for (int k = i + 1; k < n; ++k)
      a = csub(a, cmul(cconj(L[k + (int64_t)i * n]), W[k + (int64_t)c * n]));
    W[i + (int64_t)c * n] = cscale(1.0 / L[i + (int64_t)i * n].x, a);
  }
}

// B = A^H
__global__ void k_conj_transpose_c(const cd* A, cd* B, int n) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  const int i = (int)(t % n), j = (int)(t / n);
  B[j + (int64_t)i * n] = cconj(A[t]);
}

// B = (A + A^H) / 2 (the diagonal real)
__global__ void k_hermitize_c(const cd* A, cd* B, int n) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  const int i = (int)(t % n), j = (int)(t / n);
  const cd a = A[t], b = cconj(A[j + (int64_t)i * n]);
  cd r = cscale(0.5, cadd(a, b));
  if (i == j) r.y = 0.0;
  B[t] = r;
}

// Eigenpairs of Hermitian A (n x n, column-major, overwritten) by cyclic
// Jacobi rotations in parallel rounds: the n (even-padded) indices are paired
// by the circle method, so each round's rotations act on disjoint index pairs
// and apply together (columns first, then rows).  A rotation of the pair (p, q)
// with A[p, q] = r exp(i phi) is J = diag(1, exp(-i phi)) R, R the real
// Jacobi rotation of [[a_pp, r], [r, a_qq]] (tau = (a_qq - a_pp) / 2r,
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1 / sqrt(1 + t^2), s = t c).
// Sweeps stop when the off-diagonal Frobenius norm is below 1e-15 of the
// whole, or after kMaxSweeps (status 5 then).  V (n x n) receives the
// eigenvectors, lam the eigenvalues, ascending; each column of V is scaled
// so that its largest-magnitude entry is real and positive.
__global__ void __launch_bounds__(kEigThreads)
    k_jacobi_c(cd* A, cd* V, cd* Vs, double* lam, int n, int* status) {
  __shared__ int pp[512], qq[512];
  __shared__ double cs[512], sn[512];
  __shared__ cd ph[512];  // exp(-i phi)
  __shared__ double red[kEigThreads];
  const int m = n + (n & 1);  // even number of players (index n is a dummy)
  for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x) {
    const int i = (int)(t % n), j = (int)(t / n);
    V[t] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  auto reduce = [&](double v) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int o = kEigThreads / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
  };
  bool converged = n < 2;
  for (int sweep = 0; sweep < kMaxSweeps && !converged; ++sweep) {
    double off = 0.0, all = 0.0;
    for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x) {
      const int i = (int)(t % n), j = (int)(t / n);
      const double v = cabs2(A[t]);
      all += v;
      if (i != j) off += v;
    }
    off = reduce(off);
    all = reduce(all);
    if (off <= 1e-30 * all) {
      converged = true;
      break;
    }
    for (int round = 0; round < m - 1; ++round) {
      // pairs of this round: (round, m - 1) and (round + i, round - i) mod (m - 1)
      for (int t = threadIdx.x; t < m / 2; t += blockDim.x) {
        int p, q;
        if (t == 0) {
          p = round;
          q = m - 1;
        } else {
          p = (round + t) % (m - 1);
          q = (round - t + (m - 1)) % (m - 1);
        }
        if (p > q) {
          const int tmp = p;
          p = q;
          q = tmp;
        }
        double c = 1.0, s = 0.0;
        cd e = make_double2(1.0, 0.0);
        if (q < n) {
          const cd b = A[p + (int64_t)q * n];
          const double r = sqrt(cabs2(b));
          if (r > 0.0) {
            const double app = A[p + (int64_t)p * n].x, aqq = A[q + (int64_t)q * n].x;
            const double tau = (aqq - app) / (2.0 * r);
            const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + tt * tt);
            s = tt * c;
            e = make_double2(b.x / r, -b.y / r);
          }
        }
        pp[t] = p;
        qq[t] = q;
        cs[t] = c;
        sn[t] = s;
        ph[t] = e;
      }
      __syncthreads();
      // columns: (x_p, x_q) <- (c x_p - s e x_q, s x_p + c e x_q), for A and V
      for (int64_t w = threadIdx.x; w < (int64_t)(m / 2) * n; w += blockDim.x) {
        const int t = (int)(w / n), i = (int)(w % n);
        const int p = pp[t], q = qq[t];
        if (q >= n || sn[t] == 0.0) continue;
        const double c = cs[t], s = sn[t];
        const cd e = ph[t];
        cd* Ap = A + (int64_t)p * n;
        cd* Aq = A + (int64_t)q * n;
        const cd xp = Ap[i], xqe = cmul(Aq[i], e);
        Ap[i] = csub(cscale(c, xp), cscale(s, xqe));
        Aq[i] = cadd(cscale(s, xp), cscale(c, xqe));
        cd* Vp = V + (int64_t)p * n;
        cd* Vq = V + (int64_t)q * n;
        const cd vp = Vp[i], vqe = cmul(Vq[i], e);
        Vp[i] = csub(cscale(c, vp), cscale(s, vqe));
        Vq[i] = cadd(cscale(s, vp), cscale(c, vqe));
      }
      __syncthreads();
      // rows: (y_p, y_q) <- (c y_p - s conj(e) y_q, s y_p + c conj(e) y_q)
      for (int64_t w = threadIdx.x; w < (int64_t)(m / 2) * n; w += blockDim.x) {
        const int t = (int)(w / n), j = (int)(w % n);
        const int p = pp[t], q = qq[t];
        if (q >= n || sn[t] == 0.0) continue;
        const double c = cs[t], s = sn[t];
        const cd ec = cconj(ph[t]);
        const cd yp = A[p + (int64_t)j * n], yqe = cmul(A[q + (int64_t)j * n], ec);
        A[p + (int64_t)j * n] = csub(cscale(c, yp), cscale(s, yqe));
        A[q + (int64_t)j * n] = cadd(cscale(s, yp), cscale(c, yqe));
      }
      __syncthreads();
    }
  }
  if (!converged && threadIdx.x == 0) atomicCAS(status, 0, SPARC_ERR_NUMERIC);
  // ascending order (ties by index), columns permuted into Vs and phased
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double li = A[i + (int64_t)i * n].x;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double lj = A[j + (int64_t)j * n].x;
      rank += (lj < li || (lj == li && j < i)) ? 1 : 0;
    }
    lam[rank] = li;
    if (!isfinite(li)) atomicCAS(status, 0, SPARC_ERR_NUMERIC);
    const cd* v = V + (int64_t)i * n;
    int imax = 0;
    double amax = -1.0;
    for (int r = 0; r < n; ++r) {
      const double a = cabs2(v[r]);
      if (a > amax) {
        amax = a;
        imax = r;
      }
    }
    const double am = sqrt(amax);
    const cd f = am > 0.0 ? make_double2(v[imax].x / am, -v[imax].y / am) : make_double2(1.0, 0.0);
    for (int r = 0; r < n; ++r) Vs[r + (int64_t)rank * n] = cmul(v[r], f);
  }
}

int blocks1(int64_t n, int t = 256) { return (int)std::min<int64_t>((n + t - 1) / t, 1 << 30); }

}  // namespace

// ---------------------------------------------------------------------------
// Handle-side state and entry points used by api.cu
// ---------------------------------------------------------------------------
struct KpointState {
  double kvec[3] = {0, 0, 0};
  cd phase[3][kQ];
  // nonlocal tables with phases
  cd* chi = nullptr;
  cd* pull_chi = nullptr;
  // workspaces
  cd* W1 = nullptr;
  cd* W2 = nullptr;
  cd* D = nullptr;
  cd* Hs = nullptr;
  cd* Ms = nullptr;
  cd* Z = nullptr;
  cd* L = nullptr;
  cd* A = nullptr;
  cd* T1 = nullptr;
  cd* T2 = nullptr;
  double* lam = nullptr;
  double* lz = nullptr;  // Lanczos: 3 complex vectors + coefficients + partials
  int64_t ld = 0;        // complex elements
};

namespace {

int kfail(sparc_context* c, cudaError_t e, const char* what) {
  c->err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? SPARC_ERR_OOM : SPARC_ERR_CUDA;
}
#define KC(expr)                                    \
  do {                                              \
    const cudaError_t e_ = (expr);                  \
    if (e_ != cudaSuccess) return kfail(c, e_, #expr); \
  } while (0)

KArgs base_args(const sparc_context* c, const KpointState& k) {
  KArgs a{};
  a.veff = c->veff64;
  a.pull_ptr = c->nl64.pull_ptr;
  a.pull_k = c->nl64.pull_k;
  a.pull_chi = k.pull_chi;
  a.D = k.D;
  a.kp = c->nl64.kp;
  a.n[0] = c->grid.nx; a.n[1] = c->grid.ny; a.n[2] = c->grid.nz;
  for (int d = 0; d < 3; ++d) {
    a.bc[d] = c->grid.bc[d];
    for (int q = 0; q < kQ; ++q) a.phase[d][q] = k.phase[d][q];
  }
  for (int p = 0; p <= R; ++p) a.off[p] = c->lap.off[p];
  return a;
}

// y = s_h (H(k) - shift) x + s_p prev (gathering D of x first)
int khstep(sparc_context* c, const cd* x, int64_t ldx, cd* y, int64_t ldy, const cd* prev,
           int64_t ldp, int ns, double shift, double s_h, double s_p, cudaStream_t st) {
  KpointState& k = *c->kpt;
  const Nonlocal<double>& nl = c->nl64;
  if (nl.natoms > 0 && nl.kp > 0) {
    note_launch();
    k_nl_coef_c<<<dim3(nl.natoms, ns), 256, 0, st>>>(nl.supp_ptr, nl.supp_idx, nl.nproj,
                                                      nl.chi_ptr, k.chi, nl.proj_ptr, nl.gamma,
                                                      c->h * c->h * c->h, x, ldx, nl.kp, k.D);
    KC(cudaGetLastError());
  }
  KArgs a = base_args(c, k);
  a.x = x; a.ldx = ldx; a.y = y; a.ldy = ldy; a.prev = prev; a.ldp = ldp;
  a.diag_minus_shift = c->lap.diag - shift;
  a.s_h = s_h; a.s_p = s_p; a.ns = ns;
  note_launch();
  k_hpsi_c<<<dim3(blocks1(c->nd), ns), 256, 0, st>>>(a);
  KC(cudaGetLastError());
  return SPARC_OK;
}

int kfilter(sparc_context* c, cd* X, int64_t ldx, int ns, int m, double a, double b, double a0,
            bool land_in_workspace, cd** result, int64_t* ldr, cudaStream_t st) {
  KpointState& k = *c->kpt;
  const double e = (b - a) / 2.0, cc = (b + a) / 2.0;
  double sigma = e / (a0 - cc);
  const double sigma1 = sigma, tau = 2.0 / sigma1;
  std::vector<cd*> buf(m + 1);
  std::vector<int64_t> lds(m + 1);
  buf[0] = X;
  lds[0] = ldx;
  for (int i = 1; i <= m; ++i) {
    cd* out;
    if (land_in_workspace) out = (m % 2 == 1) ? ((i % 2 == 1) ? k.W1 : X) : ((i % 2 == 1) ? k.W1 : k.W2);
    else out = (i % 2 == 1) ? k.W1 : X;
    buf[i] = out;
    lds[i] = out == X ? ldx : k.ld;
  }
  for (int i = 1; i <= m; ++i) {
    int rc;
    if (i == 1) {
      rc = khstep(c, buf[0], lds[0], buf[1], lds[1], nullptr, 0, ns, cc, sigma1 / e, 0.0, st);
    } else {
      const double sn = 1.0 / (tau - sigma);
      rc = khstep(c, buf[i - 1], lds[i - 1], buf[i], lds[i], buf[i - 2], lds[i - 2], ns, cc,
                  2.0 * sn / e, -sigma * sn, st);
      sigma = sn;
    }
    if (rc) return rc;
  }
  *result = buf[m];
  *ldr = lds[m];
  return SPARC_OK;
}

int kread_status(sparc_context* c, cudaStream_t st) {
  int hs[2] = {0, 0};
  KC(cudaMemcpyAsync(hs, c->eig.status, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  KC(cudaStreamSynchronize(st));
  if (hs[0] == SPARC_ERR_NOT_SPD) {
    c->err = "subspace overlap Ms is not positive definite";
    return SPARC_ERR_NOT_SPD;
  }
  if (hs[0]) {
    c->err = "non-finite value or no convergence in the subspace eigensolve";
    return SPARC_ERR_NUMERIC;
  }
  return SPARC_OK;
}

int keig(sparc_context* c, const cd* Hs, const cd* Ms, int n, double* lam, cd* Z, cudaStream_t st) {
  KpointState& k = *c->kpt;
  KC(cudaMemsetAsync(c->eig.status, 0, 2 * sizeof(int), st));
  const int64_t nn = (int64_t)n * n;
  note_launch();
  k_cholesky_c<<<1, kEigThreads, 0, st>>>(Ms, k.L, n, c->eig.status);
  KC(cudaGetLastError());
  const int cb = blocks1(n, 64);
  note_launch();
  k_solve_lower_c<<<cb, 64, 0, st>>>(k.L, Hs, k.T1, n);  // T1 = L^-1 Hs
  KC(cudaGetLastError());
  note_launch();
  k_conj_transpose_c<<<blocks1(nn), 256, 0, st>>>(k.T1, k.T2, n);  // T2 = T1^H
  KC(cudaGetLastError());
  note_launch();
  k_solve_lower_c<<<cb, 64, 0, st>>>(k.L, k.T2, k.T1, n);  // T1 = L^-1 Hs L^-H
  KC(cudaGetLastError());
  note_launch();
  k_hermitize_c<<<blocks1(nn), 256, 0, st>>>(k.T1, k.A, n);
  KC(cudaGetLastError());
  note_launch();
  k_jacobi_c<<<1, kEigThreads, 0, st>>>(k.A, k.T1, k.T2, lam, n, c->eig.status);
  KC(cudaGetLastError());
  note_launch();
  k_solve_upper_h_c<<<cb, 64, 0, st>>>(k.L, k.T2, Z, n);  // Z = L^-H V
  KC(cudaGetLastError());
  return SPARC_OK;
}

int kproject(sparc_context* c, const cd* X, const cd* Y, int64_t ld, int ns, cd* Hs, cd* Ms,
             cudaStream_t st) {
  note_launch();
  k_project_c<<<dim3(ns, ns), 256, 0, st>>>(X, Y, ld, c->nd, ns, Hs, Ms);
  KC(cudaGetLastError());
  return SPARC_OK;
}

int krotate(sparc_context* c, const cd* Xt, int64_t ld, int ns, const cd* Z, cd* Xo, int64_t ldo,
            cudaStream_t st) {
  note_launch();
  k_rotate_c<<<dim3(blocks1(c->nd), ns), 256, 0, st>>>(Xt, ld, c->nd, ns, Z, Xo, ldo);
  KC(cudaGetLastError());
  return SPARC_OK;
}

int klanczos(sparc_context* c, int iters, uint64_t seed, double* a0, double* b, cudaStream_t st) {
  KpointState& k = *c->kpt;
  const int64_t nd = c->nd, n2 = 2 * nd;  // the complex vectors as real arrays
  double* v = k.lz;
  double* w = v + n2;
  double* vp = w + n2;
  double* ab = vp + n2;
  double* partial = ab + 1024;
  double* out2 = partial + 320;
  KC(fill_uniform_re_c128(v, nd, seed, st));
  KC(cudaMemsetAsync(vp, 0, n2 * sizeof(double), st));
  // Re(u^H w) is the real dot product of the interleaved arrays, and alpha_j,
  // beta_j are real for Hermitian H: the real Lanczos kernels apply as they are
  KC(lanczos_normalize(v, w, vp, ab, -1, n2, partial, st));
  for (int j = 0; j < iters; ++j) {
    int rc = khstep(c, reinterpret_cast<const cd*>(v), nd, reinterpret_cast<cd*>(w), nd, nullptr,
                    0, 1, 0.0, 1.0, 0.0, st);
    if (rc) return rc;
    KC(lanczos_update(w, v, vp, ab, j, n2, st));
    KC(lanczos_normalize(v, w, vp, ab, j, n2, partial, st));
  }
  KC(lanczos_bounds(ab, iters, out2, st));
  double hb[2];
  KC(cudaMemcpyAsync(hb, out2, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  KC(cudaStreamSynchronize(st));
  if (!std::isfinite(hb[0]) || !std::isfinite(hb[1])) {
    c->err = "Lanczos produced a non-finite bound";
    return SPARC_ERR_NUMERIC;
  }
  *a0 = hb[0];
  *b = hb[1];
  return SPARC_OK;
}

}  // namespace

int kpoint_init(sparc_context* c, const double kvec[3], const double* positions,
                const sparc_nonlocal* nl) {
  KpointState* k = new KpointState();
  c->kpt = k;
  for (int d = 0; d < 3; ++d) k->kvec[d] = kvec[d];
  const int nn[3] = {c->grid.nx, c->grid.ny, c->grid.nz};
  for (int d = 0; d < 3; ++d) {
    const double th = kvec[d] * nn[d] * c->h;  // k_d L_d
    for (int q = -R; q <= R; ++q) {
      const double a = th * q;
      k->phase[d][q + R] = c->grid.bc[d] == SPARC_PERIODIC ? make_double2(cos(a), sin(a))
                                                            : make_double2(1.0, 0.0);
    }
  }
  const int64_t nd = c->nd;
  k->ld = (nd + 15) / 16 * 16;
  const int natoms = nl ? nl->natoms : 0;
  if (natoms > 0) {
    // projector values with the Bloch phase of their image, per atom (support
    // order) and per grid point (the pull table's order: atom, then projector)
    const int64_t nsupp = nl->supp_ptr[natoms];
    std::vector<double> ph_re(nsupp), ph_im(nsupp);
    for (int J = 0; J < natoms; ++J)
      for (int64_t t = nl->supp_ptr[J]; t < nl->supp_ptr[J + 1]; ++t) {
        const int64_t i = nl->supp_idx[t];
        const int64_t ic[3] = {i % nn[0], (i / nn[0]) % nn[1], i / ((int64_t)nn[0] * nn[1])};
        double kt = 0.0;
        for (int d = 0; d < 3; ++d) {
          if (c->grid.bc[d] != SPARC_PERIODIC) continue;
          const double L = nn[d] * c->h;
          const double T = L * std::nearbyint((ic[d] * c->h - positions[3 * J + d]) / L);
          kt += kvec[d] * T;
        }
        ph_re[t] = cos(kt);
        ph_im[t] = sin(kt);
      }
    const int64_t nchi = nl->chi_ptr[natoms];
    std::vector<cd> chi(std::max<int64_t>(nchi, 1));
    std::vector<int> pull_ptr(nd + 1, 0);
    for (int J = 0; J < natoms; ++J) {
      const int64_t s0 = nl->supp_ptr[J], ns_ = nl->supp_ptr[J + 1] - s0;
      for (int q = 0; q < nl->nproj[J]; ++q)
        for (int64_t t = 0; t < ns_; ++t) {
          const double v = nl->chi[nl->chi_ptr[J] + q * ns_ + t];
          chi[nl->chi_ptr[J] + q * ns_ + t] = make_double2(v * ph_re[s0 + t], v * ph_im[s0 + t]);
        }
      for (int64_t t = 0; t < ns_; ++t) pull_ptr[nl->supp_idx[s0 + t] + 1] += nl->nproj[J];
    }
    for (int64_t i = 0; i < nd; ++i) pull_ptr[i + 1] += pull_ptr[i];
    std::vector<cd> pull_chi(std::max(pull_ptr[nd], 1));
    std::vector<int> fill(pull_ptr.begin(), pull_ptr.end() - 1);
    for (int J = 0; J < natoms; ++J) {
      const int64_t s0 = nl->supp_ptr[J], ns_ = nl->supp_ptr[J + 1] - s0;
      for (int64_t t = 0; t < ns_; ++t) {
        const int i = nl->supp_idx[s0 + t];
        for (int q = 0; q < nl->nproj[J]; ++q)
          pull_chi[fill[i]++] = chi[nl->chi_ptr[J] + q * ns_ + t];
      }
    }
    KC(cudaMalloc(&k->chi, chi.size() * sizeof(cd)));
    KC(cudaMemcpy(k->chi, chi.data(), chi.size() * sizeof(cd), cudaMemcpyHostToDevice));
    KC(cudaMalloc(&k->pull_chi, pull_chi.size() * sizeof(cd)));
    KC(cudaMemcpy(k->pull_chi, pull_chi.data(), pull_chi.size() * sizeof(cd),
                  cudaMemcpyHostToDevice));
  }
  const size_t blk = (size_t)k->ld * c->ns_max * sizeof(cd);
  const size_t nn2 = (size_t)c->ns_max * c->ns_max * sizeof(cd);
  KC(cudaMalloc(&k->W1, blk));
  KC(cudaMalloc(&k->W2, blk));
  KC(cudaMemset(k->W1, 0, blk));
  KC(cudaMemset(k->W2, 0, blk));
  KC(cudaMalloc(&k->D, (size_t)std::max(c->nl64.kp, 1) * c->ns_max * sizeof(cd)));
  for (cd** p : {&k->Hs, &k->Ms, &k->Z, &k->L, &k->A, &k->T1, &k->T2}) KC(cudaMalloc(p, nn2));
  KC(cudaMalloc(&k->lam, (size_t)c->ns_max * sizeof(double)));
  KC(cudaMalloc(&k->lz, ((size_t)6 * nd + 1024 + 384) * sizeof(double)));
  return SPARC_OK;
}

void kpoint_free(sparc_context* c) {
  KpointState* k = c->kpt;
  if (!k) return;
  for (void* p : {(void*)k->chi, (void*)k->pull_chi, (void*)k->W1, (void*)k->W2, (void*)k->D,
                  (void*)k->Hs, (void*)k->Ms, (void*)k->Z, (void*)k->L, (void*)k->A,
                  (void*)k->T1, (void*)k->T2, (void*)k->lam, (void*)k->lz})
    cudaFree(p);
  delete k;
  c->kpt = nullptr;
}

int kpoint_hpsi(sparc_context* c, const void* X, void* Y, int ns, int64_t ld, cudaStream_t st) {
  return khstep(c, (const cd*)X, ld, (cd*)Y, ld, nullptr, 0, ns, 0.0, 1.0, 0.0, st);
}

int kpoint_bounds(sparc_context* c, int iters, uint64_t seed, double* a0, double* b,
                  cudaStream_t st) {
  return klanczos(c, iters, seed, a0, b, st);
}

int kpoint_filter(sparc_context* c, void* X, int ns, int64_t ld, int m, double a, double b,
                  double a0, cudaStream_t st) {
  cd* res;
  int64_t ldr;
  int rc = kfilter(c, (cd*)X, ld, ns, m, a, b, a0, false, &res, &ldr, st);
  if (rc) return rc;
  if (res != (cd*)X)
    KC(cudaMemcpy2DAsync(X, ld * sizeof(cd), res, ldr * sizeof(cd), c->nd * sizeof(cd), ns,
                         cudaMemcpyDeviceToDevice, st));
  return SPARC_OK;
}

int kpoint_project(sparc_context* c, const void* Xt, const void* Yt, int ns, int64_t ld, double* Hs,
                   double* Ms, cudaStream_t st) {
  return kproject(c, (const cd*)Xt, (const cd*)Yt, ld, ns, (cd*)Hs, (cd*)Ms, st);
}

int kpoint_eig(sparc_context* c, const double* Hs, const double* Ms, int ns, double* lam, double* Z,
               cudaStream_t st) {
  int rc = keig(c, (const cd*)Hs, (const cd*)Ms, ns, lam, (cd*)Z, st);
  return rc ? rc : kread_status(c, st);
}

int kpoint_rotate(sparc_context* c, const void* Xt, void* Xout, const double* Z, int ns, int64_t ld,
                  cudaStream_t st) {
  return krotate(c, (const cd*)Xt, ld, ns, (const cd*)Z, (cd*)Xout, ld, st);
}

int kpoint_step(sparc_context* c, void* Xv, int ns, int64_t ldx, int m, double a, double b,
                double a0, double* eig, int eig_on_host, cudaStream_t st) {
  KpointState& k = *c->kpt;
  cd* X = (cd*)Xv;
  KC(cudaEventRecord(c->ev[1], st));
  cd* Xt;
  int64_t ldt;
  int rc = kfilter(c, X, ldx, ns, m, a, b, a0, true, &Xt, &ldt, st);
  if (rc) return rc;
  KC(cudaEventRecord(c->ev[2], st));
  cd* Yt = Xt == k.W1 ? k.W2 : k.W1;
  if ((rc = khstep(c, Xt, ldt, Yt, k.ld, nullptr, 0, ns, 0.0, 1.0, 0.0, st))) return rc;
  KC(cudaEventRecord(c->ev[3], st));
  if (ldt != k.ld) {
    c->err = "internal: filter result outside the workspace";
    return SPARC_ERR_CUDA;
  }
  if ((rc = kproject(c, Xt, Yt, k.ld, ns, k.Hs, k.Ms, st))) return rc;
  KC(cudaEventRecord(c->ev[4], st));
  if ((rc = keig(c, k.Hs, k.Ms, ns, k.lam, k.Z, st))) return rc;
  KC(cudaEventRecord(c->ev[5], st));
  if ((rc = krotate(c, Xt, k.ld, ns, k.Z, X, ldx, st))) return rc;
  KC(cudaEventRecord(c->ev[6], st));
  c->timed = true;
  if ((rc = kread_status(c, st))) return rc;
  double lmax;
  KC(cudaMemcpy(&lmax, k.lam + ns - 1, sizeof(double), cudaMemcpyDeviceToHost));
  c->have_prev = true;
  c->prev_max = lmax;
  if (eig) {
    if (eig_on_host) KC(cudaMemcpy(eig, k.lam, ns * sizeof(double), cudaMemcpyDeviceToHost));
    else KC(cudaMemcpyAsync(eig, k.lam, ns * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  return SPARC_OK;
}

}  // namespace sparc
