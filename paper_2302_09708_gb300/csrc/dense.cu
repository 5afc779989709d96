// Dense FP64 SIMT kernels for the Rayleigh-Ritz step (Algorithm 1):
//   projection  Hs = Xt^T Yt, Ms = Xt^T Xt  (paper Sec. II B),
//   rotation    X  = Xt Z                     (paper Sec. II D).
// Projection computes only the upper-triangular 64 x 64 tiles of both outputs
// (both are symmetric in exact arithmetic), splits the long K = Nd dimension
// across CTAs and sums the split partials in a fixed order (deterministic).
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "internal.cuh"

namespace sparc {

namespace {

constexpr int kT = 64;   // output tile
constexpr int kK = 16;   // K step
constexpr int kThreads = 256;

__device__ __forceinline__ void upper_tile(int t, int nb, int& bi, int& bj) {
  // enumerate (bi <= bj) row by row
  int r = 0;
  while (t >= nb - r) {
    t -= nb - r;
    ++r;
  }
  bi = r;
  bj = r + t;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_project_partial(const T* __restrict__ X, const T* __restrict__ Y, int64_t ld, int64_t nd,
                      int ns, int64_t kchunk, double* __restrict__ work) {
  __shared__ double As[kK][kT + 1];
  __shared__ double Bs[kK][kT + 1];
  __shared__ double Cs[kK][kT + 1];
  const int nb = (ns + kT - 1) / kT;
  int bi, bj;
  upper_tile(blockIdx.x, nb, bi, bj);
  const int i0 = bi * kT, j0 = bj * kT;
  const int64_t k0 = blockIdx.y * kchunk;
  const int64_t k1 = min(k0 + kchunk, nd);
  const int tid = threadIdx.x;
  const int tr = tid / 16, tc = tid % 16;
  double ah[4][4] = {}, am[4][4] = {};
  const int lk = tid % kK, lc = tid / kK;  // load coordinates (16 x 16)
  for (int64_t kb = k0; kb < k1; kb += kK) {
    const int64_t kk = kb + lk;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int c = lc + 16 * r;
      int gi = i0 + c, gj = j0 + c;
      bool okk = kk < k1;
      As[lk][c] = (okk && gi < ns) ? (double)X[kk + gi * ld] : 0.0;
      Bs[lk][c] = (okk && gj < ns) ? (double)Y[kk + gj * ld] : 0.0;
      Cs[lk][c] = (okk && gj < ns) ? (double)X[kk + gj * ld] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kK; ++k) {
      double a[4], b[4], c[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        a[r] = As[k][tr * 4 + r];
        b[r] = Bs[k][tc * 4 + r];
        c[r] = Cs[k][tc * 4 + r];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          ah[r][s] = fma(a[r], b[s], ah[r][s]);
          am[r][s] = fma(a[r], c[s], am[r][s]);
        }
    }
    __syncthreads();
  }
  double* wh = work + (int64_t)blockIdx.y * 2 * ns * ns;
  double* wm = wh + (int64_t)ns * ns;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      int gi = i0 + tr * 4 + r, gj = j0 + tc * 4 + s;
      if (gi < ns && gj < ns) {
        wh[gi + (int64_t)gj * ns] = ah[r][s];
        wm[gi + (int64_t)gj * ns] = am[r][s];
      }
    }
}

// Sum the split partials of each upper element (i <= j) in split order and
// write both (i, j) and (j, i).
__global__ void k_project_reduce(const double* __restrict__ work, int nsplit, int ns,
                                 double* __restrict__ Hs, double* __restrict__ Ms) {
  const int64_t nn = (int64_t)ns * ns;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nn;
       t += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(t % ns), j = (int)(t / ns);
    if (i > j) continue;
    double h = 0.0, m = 0.0;
    for (int s = 0; s < nsplit; ++s) {
      h += work[(int64_t)s * 2 * nn + t];
      m += work[(int64_t)s * 2 * nn + nn + t];
    }
    Hs[t] = h;
    Ms[t] = m;
    Hs[j + (int64_t)i * ns] = h;
    Ms[j + (int64_t)i * ns] = m;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_rotate(const T* __restrict__ X, int64_t ld, int64_t nd, int ns, const double* __restrict__ Z,
             T* __restrict__ Out, int64_t ldo) {
  __shared__ double As[kK][kT + 1];
  __shared__ double Zs[kK][kT + 1];
  const int64_t t0 = (int64_t)blockIdx.x * kT;
  const int j0 = blockIdx.y * kT;
  const int tid = threadIdx.x;
  const int tr = tid % 16, tc = tid / 16;
  double acc[4][4] = {};
  for (int kb = 0; kb < ns; kb += kK) {
    // A tile: 64 rows (t) x 16 k; consecutive threads walk t
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int e = tid + r * kThreads;  // 0..1023
      int tt = e % kT, kk = e / kT;
      int64_t gt = t0 + tt;
      int gk = kb + kk;
      As[kk][tt] = (gt < nd && gk < ns) ? (double)X[gt + (int64_t)gk * ld] : 0.0;
      int kz = e % kK, jz = e / kK;
      int gj = j0 + jz, gkz = kb + kz;
      Zs[kz][jz] = (gj < ns && gkz < ns) ? Z[gkz + (int64_t)gj * ns] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kK; ++k) {
      double a[4], z[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        a[r] = As[k][tr * 4 + r];
        z[r] = Zs[k][tc * 4 + r];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s) acc[r][s] = fma(a[r], z[s], acc[r][s]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    int gj = j0 + tc * 4 + s;
    if (gj >= ns) continue;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int64_t gt = t0 + tr * 4 + r;
      if (gt < nd) Out[gt + (int64_t)gj * ldo] = (T)acc[r][s];
    }
  }
}

}  // namespace

int project_nsplit(int64_t nd, int ns) {
  // ~8 waves of the 3-CTA-per-SM residency so the last wave's tail is small
  int nb = (ns + kT - 1) / kT;
  int64_t tiles = (int64_t)nb * (nb + 1) / 2;
  int64_t want = (8 * 3 * sm_count() + tiles - 1) / tiles;
  int64_t maxk = (nd + 1023) / 1024;  // at least ~1024 K per split
  int64_t s = want < maxk ? want : maxk;
  if (s < 1) s = 1;
  if (s > 64) s = 64;
  return (int)s;
}

template <typename T>
cudaError_t project_simt(const T* Xt, const T* Yt, int64_t ld, int64_t nd, int ns, double* Hs,
                         double* Ms, double* work, int nsplit, cudaStream_t st) {
  int nb = (ns + kT - 1) / kT;
  int tiles = nb * (nb + 1) / 2;
  int64_t kchunk = (nd + nsplit - 1) / nsplit;
  kchunk = (kchunk + kK - 1) / kK * kK;
  note_launch(), k_project_partial<T><<<dim3(tiles, nsplit), kThreads, 0, st>>>(Xt, Yt, ld, nd, ns, kchunk, work);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return project_reduce(work, nsplit, ns, Hs, Ms, st);
}

cudaError_t project_reduce(const double* work, int nsplit, int ns, double* Hs, double* Ms,
                           cudaStream_t st) {
  int64_t nn = (int64_t)ns * ns;
  int blocks = (int)std::min<int64_t>((nn + 255) / 256, 4096);
  note_launch(), k_project_reduce<<<blocks, 256, 0, st>>>(work, nsplit, ns, Hs, Ms);
  return cudaGetLastError();
}

template <typename T>
cudaError_t rotate_simt(const T* Xt, int64_t ld, int64_t nd, int ns, const double* Z, T* Xout,
                        int64_t ldo, cudaStream_t st) {
  dim3 grid((unsigned)((nd + kT - 1) / kT), (ns + kT - 1) / kT);
  note_launch(), k_rotate<T><<<grid, kThreads, 0, st>>>(Xt, ld, nd, ns, Z, Xout, ldo);
  return cudaGetLastError();
}

template cudaError_t project_simt<double>(const double*, const double*, int64_t, int64_t, int,
                                          double*, double*, double*, int, cudaStream_t);
template cudaError_t project_simt<float>(const float*, const float*, int64_t, int64_t, int,
                                         double*, double*, double*, int, cudaStream_t);
template cudaError_t rotate_simt<double>(const double*, int64_t, int64_t, int, const double*,
                                         double*, int64_t, cudaStream_t);
template cudaError_t rotate_simt<float>(const float*, int64_t, int64_t, int, const double*, float*,
                                        int64_t, cudaStream_t);

}  // namespace sparc

// ---------------------------------------------------------------------------
// Projection without any device allocation (sparc_project_noalloc).
//
// The split-K partial sums of the projection live in one file-scope device
// array instead of a handle's cudaMalloc'd workspace, so the call needs no
// handle and allocates nothing.  The array is created when the library is
// loaded onto a device and stays resident until the process exits.  Host code
// must not hand the symbol g_noalloc_scratch to a kernel (on the host it is only
// a stand-in); its device address is looked up once per device with
// cudaGetSymbolAddress and passed to the kernels.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoallocScratchDoubles = size_t(1) << 22;  // 32 MiB per device
static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
cudaError_t noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

// True for memory the current device can address without peer access: device
// memory of the current device, or managed memory.  A failed attribute query
// clears only the error it raised itself, never one the caller left pending.
bool device_pointer(const void* p) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  const cudaError_t pending = cudaPeekAtLastError();
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    if (pending == cudaSuccess) cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" int sparc_project_noalloc(const double* Xt, const double* Yt, int ns, int64_t nd,
                                     int64_t ld, double* Hs, double* Ms, void* stream) {
  using sparc::set_global_error;
  if (!Xt || !Yt || !Hs || !Ms) {
    set_global_error("invalid argument: null pointer");
    return SPARC_ERR_INVALID_ARG;
  }
  if (ns < 1 || nd < 1 || ld < nd) {
    set_global_error("invalid argument: need ns >= 1, nd >= 1, ld >= nd");
    return SPARC_ERR_INVALID_ARG;
  }
  // one split needs the two ns x ns partial outputs
  if ((size_t)2 * ns * ns > kNoallocScratchDoubles) {
    set_global_error("invalid argument: ns exceeds 1448, the largest size the static scratch "
                     "of sparc_project_noalloc (2 ns^2 doubles of 4194304) can hold");
    return SPARC_ERR_INVALID_ARG;
  }
  if (!device_pointer(Xt) || !device_pointer(Yt) || !device_pointer(Hs) ||
      !device_pointer(Ms)) {
    set_global_error("invalid argument: sparc_project_noalloc takes device pointers of the "
                     "current device");
    return SPARC_ERR_INVALID_ARG;
  }
  double* work = nullptr;
  cudaError_t e = noalloc_scratch(&work);
  if (e != cudaSuccess) {
    set_global_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    return SPARC_ERR_CUDA;
  }
  int nsplit = sparc::project_nsplit(nd, ns);
  int fit = (int)(kNoallocScratchDoubles / ((size_t)2 * ns * ns));
  if (nsplit > fit) nsplit = fit;
  // every partial the reduction reads is written by the same call, so the
  // scratch needs no clearing between calls
  e = sparc::project_simt<double>(Xt, Yt, ld, nd, ns, Hs, Ms, work, nsplit,
                                  static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    set_global_error(std::string("projection launch: ") + cudaGetErrorString(e));
    return SPARC_ERR_CUDA;
  }
  return SPARC_OK;
}
