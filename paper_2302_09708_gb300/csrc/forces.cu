// Nonlocal Hellmann-Feynman forces on the atoms (the force kernels that the
// paper moves to the GPU beside the filter, Sec. III: the gradient of the
// orbitals, then the nonlocal projectors applied to it).  For real orbitals
// X_n with occupations f_n (spin degeneracy 2):
//   c_{Jp n}  = h^3 sum_i chi_Jp(i) X_n(i)
//   g_{Jp n d} = h^3 sum_i chi_Jp(i) (D_d X_n)(i)
//   F_Jd = -4 sum_n f_n sum_p gamma_Jp c_{Jp n} g_{Jp n d},
// with D_d the radius-6 central first derivative along axis d, under the
// Laplacian's boundary rules (periodic wrap, Dirichlet zero ghosts).
//
// One block per (orbital, atom) walks the atom's support points, forms X and
// its three derivatives there, and reduces the 16 sums of each group of four
// projectors in a fixed order. The per-(atom, orbital) contributions are then
// summed over orbitals in order by a second kernel, so the result is
// deterministic and uses no atomics.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "internal.cuh"

namespace sparc {
namespace {

constexpr int kForceThreads = 128;
constexpr int kForceWarps = kForceThreads / 32;

// Central first-derivative weights of radius 6 (order 12): w_p for p = 1..6.
__constant__ double kD1[7] = {0.0,        6.0 / 7.0, -15.0 / 56.0, 5.0 / 63.0,
                              -1.0 / 56.0, 1.0 / 385.0, -1.0 / 5544.0};

// sum_p w_p (x[i + p] - x[i - p]) along one axis of length n and stride
// `stride`, for the point `lin` whose coordinate on that axis is i.
template <typename T>
__device__ __forceinline__ double axis_diff(const T* __restrict__ x, int64_t lin, int i, int n,
                                            int64_t stride, int periodic) {
  double s = 0.0;
#pragma unroll
  for (int p = 1; p <= kRadius; ++p) {
    int jp = i + p, jm = i - p;
    double vp = 0.0, vm = 0.0;
    if (periodic) {
      jp = ((jp % n) + n) % n;
      jm = ((jm % n) + n) % n;
      vp = (double)x[lin + (int64_t)(jp - i) * stride];
      vm = (double)x[lin + (int64_t)(jm - i) * stride];
    } else {
      if (jp < n) vp = (double)x[lin + (int64_t)p * stride];
      if (jm >= 0) vm = (double)x[lin - (int64_t)p * stride];
    }
    s += kD1[p] * (vp - vm);
  }
  return s;
}

template <typename T>
__global__ void __launch_bounds__(kForceThreads)
k_nl_force(Grid g, double inv_h, double h3, Nonlocal<double> nl, int atom0,
           const T* __restrict__ X, int64_t ld, int ns, const double* __restrict__ occ,
           double* __restrict__ part) {
  const int n = blockIdx.x;
  const int J = atom0 + blockIdx.y;
  const int64_t s0 = nl.supp_ptr[J];
  const int64_t nsupp = nl.supp_ptr[J + 1] - s0;
  const int np = nl.nproj[J];
  const double* chi = nl.chi + nl.chi_ptr[J];  // column-major nsupp x np
  const double* gam = nl.gamma + nl.proj_ptr[J];
  const T* x = X + (int64_t)n * ld;
  const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
  __shared__ double red[kForceWarps][16];
  double fd[3] = {0.0, 0.0, 0.0};  // meaningful in thread 0
  for (int p0 = 0; p0 < np; p0 += 4) {
    double acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = 0.0;
    for (int64_t t = threadIdx.x; t < nsupp; t += kForceThreads) {
      const int64_t lin = nl.supp_idx[s0 + t];
      const int ix = (int)(lin % g.nx);
      const int64_t r = lin / g.nx;
      const int iy = (int)(r % g.ny);
      const int iz = (int)(r / g.ny);
      const double x0 = (double)x[lin];
      const double gx = axis_diff(x, lin, ix, g.nx, 1, g.bc[0] == 0);
      const double gy = axis_diff(x, lin, iy, g.ny, sy, g.bc[1] == 0);
      const double gz = axis_diff(x, lin, iz, g.nz, sz, g.bc[2] == 0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (p0 + q < np) {
          const double cq = chi[(int64_t)(p0 + q) * nsupp + t];
          acc[q] += cq * x0;
          acc[4 + 3 * q + 0] += cq * gx;
          acc[4 + 3 * q + 1] += cq * gy;
          acc[4 + 3 * q + 2] += cq * gz;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      double v = acc[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        double v = 0.0;
        for (int w = 0; w < kForceWarps; ++w) v += red[w][k];
        tot[k] = v;
      }
      for (int q = 0; q < 4 && p0 + q < np; ++q) {
        const double c = h3 * tot[q] * gam[p0 + q];
        fd[0] += c * h3 * inv_h * tot[4 + 3 * q + 0];
        fd[1] += c * h3 * inv_h * tot[4 + 3 * q + 1];
        fd[2] += c * h3 * inv_h * tot[4 + 3 * q + 2];
      }
    }
    __syncthreads();  // red[] is rewritten by the next projector group
  }
  if (threadIdx.x == 0) {
    const double f = -4.0 * occ[n];
    double* o = part + ((int64_t)J * ns + n) * 3;
    o[0] = f * fd[0];
    o[1] = f * fd[1];
    o[2] = f * fd[2];
  }
}

// F[J][d] = sum over orbitals n (in order) of part[J][n][d].
__global__ void k_nl_force_reduce(const double* __restrict__ part, int natoms, int ns,
                                  double* __restrict__ F) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)natoms * 3) return;
  const int64_t J = t / 3, d = t % 3;
  double s = 0.0;
  for (int n = 0; n < ns; ++n) s += part[(J * ns + n) * 3 + d];
  F[t] = s;
}

}  // namespace

template <typename T>
cudaError_t nonlocal_forces(const Grid& g, double h, const Nonlocal<double>& nl, const T* X,
                            int64_t ld, int ns, const double* occ, double* F, double* part,
                            cudaStream_t st) {
  if (nl.natoms == 0) return cudaSuccess;
  if (ns == 0) return cudaMemsetAsync(F, 0, sizeof(double) * 3 * nl.natoms, st);
  const double h3 = h * h * h;
  constexpr int kAtomsPerLaunch = 65535;
  for (int a0 = 0; a0 < nl.natoms; a0 += kAtomsPerLaunch) {
    const int na = std::min(kAtomsPerLaunch, nl.natoms - a0);
    note_launch();
    k_nl_force<T><<<dim3((unsigned)ns, (unsigned)na), kForceThreads, 0, st>>>(
        g, 1.0 / h, h3, nl, a0, X, ld, ns, occ, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int64_t outs = (int64_t)nl.natoms * 3;
  note_launch();
  k_nl_force_reduce<<<(unsigned)((outs + 127) / 128), 128, 0, st>>>(part, nl.natoms, ns, F);
  return cudaGetLastError();
}

template cudaError_t nonlocal_forces<double>(const Grid&, double, const Nonlocal<double>&,
                                             const double*, int64_t, int, const double*,
                                             double*, double*, cudaStream_t);
template cudaError_t nonlocal_forces<float>(const Grid&, double, const Nonlocal<double>&,
                                            const float*, int64_t, int, const double*, double*,
                                            double*, cudaStream_t);

}  // namespace sparc
