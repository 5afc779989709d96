// Fermi-Dirac occupations of the Ritz values and the electron density of the
// occupied orbitals (the quantities a self-consistent cycle takes from one
// CheFSI step, Section 2.1):
//   f_n = 1 / (1 + exp((lambda_n - mu) / kT)),  mu such that 2 sum_n f_n = Ne,
//   rho_i = (2 / h^3) sum_n f_n X_{i n}^2.
// X is column-major and normalised by X^T X = I, so h^3 sum_i rho_i = Ne.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "internal.cuh"

namespace sparc {
namespace {

constexpr int kFermiThreads = 512;

__device__ __forceinline__ double fermi(double lam, double mu, double kT) {
  const double t = fmin(fmax((lam - mu) / kT, -700.0), 700.0);
  return 1.0 / (1.0 + exp(t));
}

// 2 sum_n f_n(mu) over the block, in a fixed reduction order.
__device__ double electron_count(const double* lam, int ns, double mu, double kT, double* red) {
  double s = 0.0;
  for (int n = threadIdx.x; n < ns; n += blockDim.x) s += fermi(lam[n], mu, kT);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();  // red[] of the previous call is consumed
  if ((threadIdx.x & 31) == 0) red[w] = s;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; ++i) t += red[i];
  return 2.0 * t;
}

// One block: bisection on mu over [min lambda - 1, max lambda + 1] until
// |2 sum f - Ne| < tol (at most 400 halvings), then f_n at that mu.
__global__ void __launch_bounds__(kFermiThreads) k_fermi(const double* __restrict__ lam, int ns,
                                                         double ne, double kT, double tol,
                                                         double* __restrict__ occ,
                                                         double* __restrict__ mu_out) {
  __shared__ double red[kFermiThreads / 32];
  __shared__ double ext[2][kFermiThreads / 32];
  double lo = INFINITY, hi = -INFINITY;
  for (int n = threadIdx.x; n < ns; n += blockDim.x) {
    lo = fmin(lo, lam[n]);
    hi = fmax(hi, lam[n]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    ext[0][threadIdx.x >> 5] = lo;
    ext[1][threadIdx.x >> 5] = hi;
  }
  __syncthreads();
  lo = INFINITY;
  hi = -INFINITY;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
    lo = fmin(lo, ext[0][i]);
    hi = fmax(hi, ext[1][i]);
  }
  lo -= 1.0;
  hi += 1.0;
  double mu = 0.5 * (lo + hi);
  for (int it = 0; it < 400; ++it) {
    mu = 0.5 * (lo + hi);
    const double c = electron_count(lam, ns, mu, kT, red);
    if (fabs(c - ne) < tol) break;
    if (c < ne) lo = mu;
    else hi = mu;
  }
  for (int n = threadIdx.x; n < ns; n += blockDim.x) occ[n] = fermi(lam[n], mu, kT);
  if (threadIdx.x == 0) *mu_out = mu;
}

// rho over a range of points: V consecutive points per thread (one vector
// load per orbital), orbitals [n0, n1) of this split, taken G at a time with
// all G loads issued before the arithmetic (the loads, not the FMAs, set the
// pace).  FP32 blocks sum f_n x^2 in FP32 within a group of G = 16 orbitals
// and add each group in FP64; FP64 blocks accumulate in FP64 throughout.
template <typename T, int V>
__global__ void __launch_bounds__(256) k_density(const T* __restrict__ X, int64_t ld, int64_t nd,
                                                 int ns, int nsplit,
                                                 const double* __restrict__ occ, double scale,
                                                 double* __restrict__ out) {
  using Vec = typename std::conditional<
      std::is_same<T, float>::value,
      typename std::conditional<V == 4, float4, float2>::type,
      typename std::conditional<V == 2, double2, double>::type>::type;
  constexpr int G = std::is_same<T, float>::value ? 16 : 8;
  const int split = blockIdx.y;
  const int per = (ns + nsplit - 1) / nsplit;
  const int n0 = split * per, n1 = min(ns, n0 + per);
  double acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = 0.0;
  const int64_t i0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * V;
  if (i0 >= nd) return;
  const bool full = i0 + V <= nd;
  for (int g0 = n0; g0 < n1; g0 += G) {
    const int cnt = min(G, n1 - g0);
    T x[G][V];
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const T* col = X + i0 + (int64_t)(g0 + u) * ld;
      if (u < cnt && full) {
        const Vec w = __ldg(reinterpret_cast<const Vec*>(col));
        const T* wp = reinterpret_cast<const T*>(&w);
#pragma unroll
        for (int v = 0; v < V; ++v) x[u][v] = wp[v];
      } else {
#pragma unroll
        for (int v = 0; v < V; ++v) x[u][v] = (u < cnt && i0 + v < nd) ? col[v] : T(0);
      }
    }
    T part[V];
#pragma unroll
    for (int v = 0; v < V; ++v) part[v] = T(0);
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const T f = u < cnt ? (T)__ldg(occ + g0 + u) : T(0);
#pragma unroll
      for (int v = 0; v < V; ++v) part[v] = fma(f * x[u][v], x[u][v], part[v]);
    }
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] += (double)part[v];
  }
  double* o = out + (int64_t)split * nd;
#pragma unroll
  for (int v = 0; v < V; ++v)
    if (i0 + v < nd) o[i0 + v] = nsplit == 1 ? acc[v] * scale : acc[v];
}

// rho_i = scale * sum over splits of the partial sums, in split order.
__global__ void k_density_reduce(const double* __restrict__ part, int64_t nd, int nsplit,
                                 double scale, double* __restrict__ rho) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nd;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < nsplit; ++k) s += part[(int64_t)k * nd + i];
    rho[i] = s * scale;
  }
}

template <typename T, int V>
cudaError_t launch_density(const T* X, int64_t ld, int64_t nd, int ns, const double* occ,
                           double scale, double* rho, double* work, int64_t work_elems,
                           cudaStream_t st) {
  const int64_t threads = (nd + V - 1) / V;
  const unsigned bx = (unsigned)((threads + 255) / 256);
  // enough orbital splits to give every SM about 1024 threads, bounded by the
  // orbitals (at least 8 per split) and by the scratch
  int nsplit = (int)std::max<int64_t>(1, (int64_t)sm_count() * 1024 / std::max<int64_t>(threads, 1));
  nsplit = std::min(nsplit, std::max(1, ns / 8));
  nsplit = (int)std::min<int64_t>(nsplit, std::max<int64_t>(1, work_elems / std::max<int64_t>(nd, 1)));
  nsplit = std::min(nsplit, 64);
  if (nsplit == 1) {
    note_launch();
    k_density<T, V><<<dim3(bx, 1), 256, 0, st>>>(X, ld, nd, ns, 1, occ, scale, rho);
    return cudaGetLastError();
  }
  note_launch();
  k_density<T, V><<<dim3(bx, nsplit), 256, 0, st>>>(X, ld, nd, ns, nsplit, occ, scale, work);
  note_launch();
  k_density_reduce<<<(unsigned)std::min<int64_t>((nd + 255) / 256, 4096), 256, 0, st>>>(
      work, nd, nsplit, scale, rho);
  return cudaGetLastError();
}

}  // namespace

cudaError_t fermi_occupations(const double* lam, int ns, double ne, double kT, double* occ,
                              double* mu, cudaStream_t st) {
  note_launch();
  k_fermi<<<1, kFermiThreads, 0, st>>>(lam, ns, ne, kT, 1e-12, occ, mu);
  return cudaGetLastError();
}

cudaError_t density(const void* X, int64_t ld, int64_t nd, int ns, bool fp32, const double* occ,
                    double h, double* rho, double* work, int64_t work_elems, cudaStream_t st) {
  const double scale = 2.0 / (h * h * h);
  if (ns == 0) return cudaMemsetAsync(rho, 0, (size_t)nd * sizeof(double), st);
  const uintptr_t p = (uintptr_t)X;
  if (fp32) {
    if (p % 16 == 0 && ld % 4 == 0)
      return launch_density<float, 4>((const float*)X, ld, nd, ns, occ, scale, rho, work,
                                      work_elems, st);
    return launch_density<float, 1>((const float*)X, ld, nd, ns, occ, scale, rho, work,
                                    work_elems, st);
  }
  if (p % 16 == 0 && ld % 2 == 0)
    return launch_density<double, 2>((const double*)X, ld, nd, ns, occ, scale, rho, work,
                                     work_elems, st);
  return launch_density<double, 1>((const double*)X, ld, nd, ns, occ, scale, rho, work,
                                   work_elems, st);
}

}  // namespace sparc
