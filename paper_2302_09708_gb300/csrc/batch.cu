// Batched CheFSI step over many independent systems (the paper treats the
// eigenproblems of different k-points, spins or configurations as independent,
// Sec. II): every Chebyshev degree of every system in the batch is one launch
// of the nonlocal-coefficient kernel and one launch of the stencil kernel,
// whose CTAs look up their system in a device descriptor table.  The
// Rayleigh-Ritz pieces (projection, eigensolve, rotation) of each system run on
// a pool of forked streams.  The whole step is captured once as a CUDA graph
// and replayed on later calls with the same buffers; only the per-degree
// scalars (which depend on the bounds) are uploaded before each replay.
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace sparc {

namespace {

constexpr int kR = kRadius;
constexpr int kBX = 32, kBY = 8;  // stencil tile (one thread per point)

// Per-system, per-degree work description.
struct BatchItem {
  const void* x;
  void* y;
  const void* prev;
  int64_t ldx, ldy, ldp;
  double shift, s_h, s_p;
  int active;
  int pad;
};

// Per-system constant description.
struct BatchSys {
  int nx, ny, nz, bcx, bcy, bcz;
  int ns, tiles_x, tiles_y, nzc, bz;
  int natoms, kp;
  int64_t cta_begin;      // first stencil CTA of this system
  int64_t nl_cta_begin;   // first nonlocal CTA of this system
  double diag, off[kR + 1], h3;
  const void* veff;
  const int* pull_ptr;
  const int* pull_k;
  const void* pull_chi;
  const int64_t* supp_ptr;
  const int* supp_idx;
  const int* nproj;
  const int64_t* chi_ptr;
  const void* chi;
  const int* proj_ptr;
  const double* gamma;
  void* D;
};

__device__ __forceinline__ int find_sys(const BatchSys* sys, int nsys, int64_t cta, bool nl) {
  int lo = 0, hi = nsys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int64_t b = nl ? sys[mid].nl_cta_begin : sys[mid].cta_begin;
    if (b <= cta) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ bool wrap(int& c, int n, int bc) {
  if (c >= 0 && c < n) return true;
  if (bc == SPARC_DIRICHLET) return false;
  c %= n;
  if (c < 0) c += n;
  return true;
}

constexpr int kNlOrb = 4;

template <typename T>
__global__ void __launch_bounds__(256)
    k_nl_coef_batched(const BatchSys* __restrict__ sys, const BatchItem* __restrict__ items,
                      int nsys) {
  __shared__ T red[4][8];
  const int si = find_sys(sys, nsys, blockIdx.x, true);
  const BatchSys& S = sys[si];
  const BatchItem& it = items[si];
  if (!it.active || S.kp == 0) return;
  const int64_t local = blockIdx.x - S.nl_cta_begin;
  const int ngroups = (S.ns + kNlOrb - 1) / kNlOrb;
  const int J = (int)(local / ngroups), grp = (int)(local % ngroups);
  if (J >= S.natoms) return;
  const T* __restrict__ x = (const T*)it.x;
  const int64_t s0 = S.supp_ptr[J];
  const int nsup = (int)(S.supp_ptr[J + 1] - s0);
  const int np = S.nproj[J];
  const T* __restrict__ chi = (const T*)S.chi + S.chi_ptr[J];
  const int k0 = S.proj_ptr[J];
  const int* __restrict__ idx = S.supp_idx + s0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T* D = (T*)S.D;
  for (int n = grp * kNlOrb; n < min(grp * kNlOrb + kNlOrb, S.ns); ++n) {
    const T* __restrict__ xn = x + (int64_t)n * it.ldx;
    for (int qb = 0; qb < np; qb += 4) {
      T acc[4] = {T(0), T(0), T(0), T(0)};
      for (int t = threadIdx.x; t < nsup; t += blockDim.x) {
        const T xv = xn[idx[t]];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (qb + q < np) acc[q] += chi[(int64_t)(qb + q) * nsup + t] * xv;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        T v = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[q][wid] = v;
      }
      __syncthreads();
      if (threadIdx.x < 4 && qb + (int)threadIdx.x < np) {
        T v = T(0);
        for (int w = 0; w < 8; ++w) v += red[threadIdx.x][w];
        const int k = k0 + qb + threadIdx.x;
        D[(int64_t)n * S.kp + k] = T(v * (S.gamma[k] * S.h3));
      }
      __syncthreads();
    }
  }
}

// One thread per output point of a kBX x kBY xy-tile, marching z through a
// plane-sized shared tile with a 13-deep register queue.
template <typename T>
__global__ void __launch_bounds__(kBX* kBY)
    k_apply_h_batched(const BatchSys* __restrict__ sys, const BatchItem* __restrict__ items,
                      int nsys) {
  __shared__ T s[kBY + 2 * kR][kBX + 2 * kR];
  const int si = find_sys(sys, nsys, blockIdx.x, false);
  const BatchSys& S = sys[si];
  const BatchItem& it = items[si];
  if (!it.active) return;
  int64_t local = blockIdx.x - S.cta_begin;
  const int zc = (int)(local % S.nzc);
  local /= S.nzc;
  const int tile = (int)(local % (S.tiles_x * S.tiles_y));
  const int n = (int)(local / (S.tiles_x * S.tiles_y));
  const int x0 = (tile % S.tiles_x) * kBX, y0 = (tile / S.tiles_x) * kBY;
  const int z0 = zc * S.bz, z1 = min(z0 + S.bz, S.nz);
  const int tx = threadIdx.x % kBX, ty = threadIdx.x / kBX;
  const int px = x0 + tx, py = y0 + ty;
  const bool valid = px < S.nx && py < S.ny;
  const int64_t nxy = (int64_t)S.nx * S.ny;
  const T* __restrict__ xn = (const T*)it.x + (int64_t)n * it.ldx;
  T q[2 * kR + 1];
#pragma unroll
  for (int j = 0; j < 2 * kR + 1; ++j) {
    int zz = z0 - kR + j;
    q[j] = (valid && wrap(zz, S.nz, S.bcz)) ? xn[zz * nxy + (int64_t)py * S.nx + px] : T(0);
  }
  const T dms = T(S.diag - it.shift);
  const T sh = T(it.s_h), sp = T(it.s_p);
  for (int z = z0; z < z1; ++z) {
    __syncthreads();
    for (int e = threadIdx.x; e < (kBY + 2 * kR) * (kBX + 2 * kR); e += blockDim.x) {
      const int r = e / (kBX + 2 * kR), c = e % (kBX + 2 * kR);
      int gx = x0 + c - kR, gy = y0 + r - kR;
      const bool ok = wrap(gx, S.nx, S.bcx) && wrap(gy, S.ny, S.bcy);
      s[r][c] = ok ? xn[z * nxy + (int64_t)gy * S.nx + gx] : T(0);
    }
    __syncthreads();
    if (valid) {
      T acc = dms * q[kR];
#pragma unroll
      for (int p = 1; p <= kR; ++p)
        acc += T(S.off[p]) * ((s[ty + kR][tx + kR + p] + s[ty + kR][tx + kR - p]) +
                              (s[ty + kR + p][tx + kR] + s[ty + kR - p][tx + kR]) +
                              (q[kR + p] + q[kR - p]));
      const int64_t g = z * nxy + (int64_t)py * S.nx + px;
      acc += ((const T*)S.veff)[g] * q[kR];
      if (S.kp > 0) {
        const T* Dn = (const T*)S.D + (int64_t)n * S.kp;
        const T* pc = (const T*)S.pull_chi;
        T nlv = T(0);
        for (int e = S.pull_ptr[g]; e < S.pull_ptr[g + 1]; ++e) nlv += pc[e] * Dn[S.pull_k[e]];
        acc += nlv;
      }
      T out = sh * acc;
      if (it.prev) out += sp * ((const T*)it.prev)[(int64_t)n * it.ldp + g];
      ((T*)it.y)[(int64_t)n * it.ldy + g] = out;
    }
#pragma unroll
    for (int j = 0; j < 2 * kR; ++j) q[j] = q[j + 1];
    int zz = z + kR + 1;
    q[2 * kR] = (valid && wrap(zz, S.nz, S.bcz)) ? xn[zz * nxy + (int64_t)py * S.nx + px] : T(0);
  }
}

}  // namespace

// Host-side layout helper: fills the per-system constants (CTA offsets, tiling)
// and returns the total CTA counts of the two batched kernels.
template <typename T>
void batch_layout(std::vector<BatchSysHost>& hs, int64_t* cta_total, int64_t* nl_total) {
  int64_t c = 0, nlc = 0;
  for (auto& b : hs) {
    b.tiles_x = (b.nx + kBX - 1) / kBX;
    b.tiles_y = (b.ny + kBY - 1) / kBY;
    b.nzc = std::max(1, std::min(b.nz / 8, 4));
    b.bz = (b.nz + b.nzc - 1) / b.nzc;
    b.nzc = (b.nz + b.bz - 1) / b.bz;
    b.cta_begin = c;
    c += (int64_t)b.tiles_x * b.tiles_y * b.ns * b.nzc;
    b.nl_cta_begin = nlc;
    nlc += (int64_t)std::max(b.natoms, 1) * ((b.ns + kNlOrb - 1) / kNlOrb);
  }
  *cta_total = c;
  *nl_total = nlc;
}

size_t batch_sys_bytes() { return sizeof(BatchSys); }
size_t batch_item_bytes() { return sizeof(BatchItem); }

void batch_pack_sys(const BatchSysHost& h, void* out) {
  BatchSys s{};
  s.nx = h.nx; s.ny = h.ny; s.nz = h.nz; s.bcx = h.bc[0]; s.bcy = h.bc[1]; s.bcz = h.bc[2];
  s.ns = h.ns; s.tiles_x = h.tiles_x; s.tiles_y = h.tiles_y; s.nzc = h.nzc; s.bz = h.bz;
  s.natoms = h.natoms; s.kp = h.kp; s.cta_begin = h.cta_begin; s.nl_cta_begin = h.nl_cta_begin;
  s.diag = h.diag;
  for (int p = 0; p <= kR; ++p) s.off[p] = h.off[p];
  s.h3 = h.h3;
  s.veff = h.veff; s.pull_ptr = h.pull_ptr; s.pull_k = h.pull_k; s.pull_chi = h.pull_chi;
  s.supp_ptr = h.supp_ptr; s.supp_idx = h.supp_idx; s.nproj = h.nproj; s.chi_ptr = h.chi_ptr;
  s.chi = h.chi; s.proj_ptr = h.proj_ptr; s.gamma = h.gamma; s.D = h.D;
  *reinterpret_cast<BatchSys*>(out) = s;
}

void batch_pack_item(const BatchItemHost& h, void* out) {
  BatchItem it{};
  it.x = h.x; it.y = h.y; it.prev = h.prev; it.ldx = h.ldx; it.ldy = h.ldy; it.ldp = h.ldp;
  it.shift = h.shift; it.s_h = h.s_h; it.s_p = h.s_p; it.active = h.active;
  *reinterpret_cast<BatchItem*>(out) = it;
}

template <typename T>
cudaError_t batch_degree(const void* sys, const void* items, int nsys, int64_t cta_total,
                         int64_t nl_total, cudaStream_t st) {
  const BatchSys* s = (const BatchSys*)sys;
  const BatchItem* it = (const BatchItem*)items;
  if (nl_total > 0) note_launch(), k_nl_coef_batched<T><<<(unsigned)nl_total, 256, 0, st>>>(s, it, nsys);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  note_launch(), k_apply_h_batched<T><<<(unsigned)cta_total, kBX * kBY, 0, st>>>(s, it, nsys);
  return cudaGetLastError();
}

template void batch_layout<float>(std::vector<BatchSysHost>&, int64_t*, int64_t*);
template void batch_layout<double>(std::vector<BatchSysHost>&, int64_t*, int64_t*);
template cudaError_t batch_degree<float>(const void*, const void*, int, int64_t, int64_t,
                                         cudaStream_t);
template cudaError_t batch_degree<double>(const void*, const void*, int, int64_t, int64_t,
                                          cudaStream_t);

}  // namespace sparc
