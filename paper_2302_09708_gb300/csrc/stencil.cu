// Matrix-free Hamiltonian application on the GPU (paper Sec. II A):
//   K1  finite-difference Laplacian + Veff + nonlocal pull-add, fused with the
//       Chebyshev recurrence axpy (y = s_h (H - shift) x + s_p prev);
//   K2  nonlocal projector coefficients D = Gamma h^3 chi^T x per atom;
//   small FP64 vector kernels for the Lanczos bound estimate.
//
// K1 layout: one CTA owns a BX x BY tile of an xy-plane for one orbital and
// marches along z.  The current plane (with a 6-point halo in x and y) sits in
// shared memory; the 13 values along z at each of the thread's VX points sit in
// a register queue.  Each thread computes VX consecutive x points, so its x
// neighbours and the y neighbour rows are read with vector loads.
#include <stdint.h>

#include <algorithm>

#include "internal.cuh"

namespace sparc {

namespace {

template <typename T, int V>
struct VecT;
template <>
struct VecT<float, 4> { using type = float4; };
template <>
struct VecT<float, 2> { using type = float2; };
template <>
struct VecT<double, 2> { using type = double2; };

template <typename T, int V, bool VEC>
__device__ __forceinline__ void load_v(T (&dst)[V], const T* __restrict__ p) {
  if constexpr (VEC) {
    using VT = typename VecT<T, V>::type;
    VT t = __ldg(reinterpret_cast<const VT*>(p));
    const T* tt = reinterpret_cast<const T*>(&t);
#pragma unroll
    for (int i = 0; i < V; ++i) dst[i] = tt[i];
  } else {
#pragma unroll
    for (int i = 0; i < V; ++i) dst[i] = __ldg(p + i);
  }
}

// Vector load from shared memory (16-byte aligned address).
template <typename T, int V>
__device__ __forceinline__ void lds_v(T (&dst)[V], const T* p) {
  using VT = typename VecT<T, V>::type;
  VT t = *reinterpret_cast<const VT*>(p);
  const T* tt = reinterpret_cast<const T*>(&t);
#pragma unroll
  for (int i = 0; i < V; ++i) dst[i] = tt[i];
}

// Global load of V consecutive values of which the first nv are in range.
template <typename T, int V, bool VEC>
__device__ __forceinline__ void load_part(T (&dst)[V], const T* __restrict__ p, int nv) {
  if constexpr (VEC) {
    load_v<T, V, true>(dst, p);
  } else {
#pragma unroll
    for (int i = 0; i < V; ++i) dst[i] = i < nv ? __ldg(p + i) : T(0);
  }
}

template <typename T, int V, bool VEC>
__device__ __forceinline__ void store_v(T* p, const T (&src)[V]) {
  if constexpr (VEC) {
    using VT = typename VecT<T, V>::type;
    VT t;
    T* tt = reinterpret_cast<T*>(&t);
#pragma unroll
    for (int i = 0; i < V; ++i) tt[i] = src[i];
    *reinterpret_cast<VT*>(p) = t;
  } else {
#pragma unroll
    for (int i = 0; i < V; ++i) p[i] = src[i];
  }
}

// Map a grid coordinate into [0, n) (periodic) or report it outside (Dirichlet).
__device__ __forceinline__ bool map_coord(int& c, int n, int bc) {
  if (c >= 0 && c < n) return true;
  if (bc == SPARC_DIRICHLET) return false;
  c %= n;
  if (c < 0) c += n;
  return true;
}

template <typename T>
struct HArgs {
  const T* x;
  int64_t ldx;
  T* y;
  int64_t ldy;
  const T* prev;
  int64_t ldp;
  const T* veff;
  const int* pull_ptr;
  const int* pull_k;
  const T* pull_chi;
  const T* D;
  int kp;
  int nx, ny, nz, bcx, bcy, bcz;
  T diag_minus_shift;  // -1/2 * 3 w0/h^2 - shift
  T off[kRadius + 1];  // -1/2 w_p/h^2
  T s_h, s_p;
  int bz, tiles_x;
};

constexpr int kPad = 8;  // x halo padding in shared memory (>= kRadius, keeps vector alignment)

template <typename T, int VX, int BX, int BY, bool VEC>
__global__ void __launch_bounds__((BX / VX) * BY)
    k_apply_h(const HArgs<T> a) {
  constexpr int R = kRadius;
  constexpr int TX = BX / VX;
  constexpr int NT = TX * BY;
  constexpr int SW = BX + 2 * kPad;  // shared row width
  constexpr int SH = BY + 2 * R;
  constexpr int FW = BX + 2 * R;     // columns actually filled: [kPad - R, kPad + BX + R)
  constexpr int FN = FW * SH;
  constexpr int PER = (FN + NT - 1) / NT;
  __shared__ __align__(16) T s[SH][SW];

  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int tile_x = blockIdx.x % a.tiles_x, tile_y = blockIdx.x / a.tiles_x;
  const int x0 = tile_x * BX, y0 = tile_y * BY;
  const int n = blockIdx.y;
  const int z0 = blockIdx.z * a.bz;
  const int z1 = min(z0 + a.bz, a.nz);
  const int64_t nxy = (int64_t)a.nx * a.ny;
  const T* __restrict__ xn = a.x + (int64_t)n * a.ldx;

  // In-plane source offsets of this thread's shared-memory fill elements
  // (-1: zero ghost, -2: nothing to do).
  int src[PER];
#pragma unroll
  for (int e = 0; e < PER; ++e) {
    int idx = threadIdx.x + e * NT;
    int o = -2;
    if (idx < FN) {
      int r = idx / FW, c = idx % FW;
      int gx = x0 + c - R, gy = y0 + r - R;
      bool ok = map_coord(gx, a.nx, a.bcx) && map_coord(gy, a.ny, a.bcy);
      o = ok ? gx + a.nx * gy : -1;
    }
    src[e] = o;
  }

  const int px = x0 + tx * VX, py = y0 + ty;
  const bool valid = px < a.nx && py < a.ny;
  const int nv = valid ? min(VX, a.nx - px) : 0;  // in-range points of this thread
  const int64_t pofs = valid ? (int64_t)px + (int64_t)a.nx * py : 0;

  // z register queue: q[j] holds plane z - R + j at the thread's points
  T q[2 * R + 1][VX];
  auto load_plane = [&](int zz, T(&dst)[VX]) {
    bool ok = valid && map_coord(zz, a.nz, a.bcz);
    if (ok) {
      load_part<T, VX, VEC>(dst, xn + zz * nxy + pofs, nv);
    } else {
#pragma unroll
      for (int v = 0; v < VX; ++v) dst[v] = T(0);
    }
  };
#pragma unroll
  for (int j = 0; j < 2 * R + 1; ++j) load_plane(z0 - R + j, q[j]);

  const int sx = tx * VX + kPad, sy = ty + R;
  for (int z = z0; z < z1; ++z) {
    __syncthreads();
    const T* __restrict__ plane = xn + z * nxy;
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      int idx = threadIdx.x + e * NT;
      if (src[e] != -2) {
        int r = idx / FW, c = idx % FW;
        s[r][c + kPad - R] = src[e] >= 0 ? __ldg(plane + src[e]) : T(0);
      }
    }
    __syncthreads();
    if (valid) {
      // x window: columns sx - R .. sx + VX - 1 + R, loaded from an aligned start
      constexpr int XW = VX + 2 * kPad;
      T xw[XW];
#pragma unroll
      for (int i = 0; i < XW; i += VX) {
        T t[VX];
        lds_v<T, VX>(t, &s[sy][tx * VX + i]);
#pragma unroll
        for (int v = 0; v < VX; ++v) xw[i + v] = t[v];
      }
      T acc[VX];
#pragma unroll
      for (int v = 0; v < VX; ++v) acc[v] = a.diag_minus_shift * q[R][v];
#pragma unroll
      for (int p = 1; p <= R; ++p) {
        T up[VX], dn[VX];
        lds_v<T, VX>(up, &s[sy + p][sx]);
        lds_v<T, VX>(dn, &s[sy - p][sx]);
#pragma unroll
        for (int v = 0; v < VX; ++v) {
          T sum = (xw[kPad + v + p] + xw[kPad + v - p]) + (up[v] + dn[v]) +
                  (q[R + p][v] + q[R - p][v]);
          acc[v] += a.off[p] * sum;
        }
      }
      const int64_t g = z * nxy + pofs;
      T vf[VX];
      load_part<T, VX, VEC>(vf, a.veff + g, nv);
#pragma unroll
      for (int v = 0; v < VX; ++v) acc[v] += vf[v] * q[R][v];
      if (a.kp > 0) {
        const T* __restrict__ Dn = a.D + (int64_t)n * a.kp;
#pragma unroll
        for (int v = 0; v < VX; ++v) {
          if (v >= nv) break;
          int e0 = __ldg(a.pull_ptr + g + v), e1 = __ldg(a.pull_ptr + g + v + 1);
          T nlv = T(0);
          for (int e = e0; e < e1; ++e) nlv += __ldg(a.pull_chi + e) * __ldg(Dn + __ldg(a.pull_k + e));
          acc[v] += nlv;
        }
      }
      T out[VX];
      if (a.prev) {
        T pv[VX];
        load_part<T, VX, VEC>(pv, a.prev + (int64_t)n * a.ldp + g, nv);
#pragma unroll
        for (int v = 0; v < VX; ++v) out[v] = a.s_h * acc[v] + a.s_p * pv[v];
      } else {
#pragma unroll
        for (int v = 0; v < VX; ++v) out[v] = a.s_h * acc[v];
      }
      T* yo = a.y + (int64_t)n * a.ldy + g;
      if (VEC) {
        store_v<T, VX, true>(yo, out);
      } else {
        for (int v = 0; v < nv; ++v) yo[v] = out[v];
      }
    }
    // advance the z queue
#pragma unroll
    for (int j = 0; j < 2 * R; ++j)
#pragma unroll
      for (int v = 0; v < VX; ++v) q[j][v] = q[j + 1][v];
    load_plane(z + R + 1, q[2 * R]);
  }
}

template <typename T>
struct TileCfg;
template <>
struct TileCfg<float> { static constexpr int VX = 4, BX = 32, BY = 16; };
template <>
struct TileCfg<double> { static constexpr int VX = 2, BX = 32, BY = 16; };

}  // namespace

template <typename T>
cudaError_t apply_h(const Grid& g, const LapCoef& lc, const T* veff, const Nonlocal<T>& nl,
                    const T* D, const T* x, int64_t ldx, T* y, int64_t ldy, const T* prev,
                    int64_t ldp, int ns, double shift, double s_h, double s_p, cudaStream_t st) {
  using C = TileCfg<T>;
  HArgs<T> a;
  a.x = x; a.ldx = ldx; a.y = y; a.ldy = ldy; a.prev = prev; a.ldp = ldp; a.veff = veff;
  a.pull_ptr = nl.pull_ptr; a.pull_k = nl.pull_k; a.pull_chi = nl.pull_chi; a.D = D;
  a.kp = nl.kp;
  a.nx = g.nx; a.ny = g.ny; a.nz = g.nz;
  a.bcx = g.bc[0]; a.bcy = g.bc[1]; a.bcz = g.bc[2];
  a.diag_minus_shift = T(lc.diag - shift);
  for (int p = 0; p <= kRadius; ++p) a.off[p] = T(lc.off[p]);
  a.s_h = T(s_h);
  a.s_p = T(s_p);
  a.tiles_x = (g.nx + C::BX - 1) / C::BX;
  int tiles_y = (g.ny + C::BY - 1) / C::BY;
  int64_t xy_ctas = (int64_t)a.tiles_x * tiles_y * ns;
  // split z so that the grid covers the SMs several times over
  int nzc = (int)((4 * sm_count() + xy_ctas - 1) / xy_ctas);
  nzc = max(1, min(nzc, max(1, g.nz / 8)));
  a.bz = (g.nz + nzc - 1) / nzc;
  nzc = (g.nz + a.bz - 1) / a.bz;
  dim3 grid(a.tiles_x * tiles_y, ns, nzc);
  dim3 block((C::BX / C::VX) * C::BY);
  const bool vec = (g.nx % C::VX == 0) && (ldx % C::VX == 0) && (ldy % C::VX == 0) &&
                   (!prev || ldp % C::VX == 0) &&
                   ((uintptr_t)x % (C::VX * sizeof(T)) == 0) &&
                   ((uintptr_t)y % (C::VX * sizeof(T)) == 0) &&
                   (!prev || (uintptr_t)prev % (C::VX * sizeof(T)) == 0) &&
                   ((uintptr_t)veff % (C::VX * sizeof(T)) == 0);
  if (vec)
    note_launch(), k_apply_h<T, C::VX, C::BX, C::BY, true><<<grid, block, 0, st>>>(a);
  else
    note_launch(), k_apply_h<T, C::VX, C::BX, C::BY, false><<<grid, block, 0, st>>>(a);
  return cudaGetLastError();
}

template cudaError_t apply_h<double>(const Grid&, const LapCoef&, const double*,
                                     const Nonlocal<double>&, const double*, const double*,
                                     int64_t, double*, int64_t, const double*, int64_t, int,
                                     double, double, double, cudaStream_t);
template cudaError_t apply_h<float>(const Grid&, const LapCoef&, const float*,
                                    const Nonlocal<float>&, const float*, const float*, int64_t,
                                    float*, int64_t, const float*, int64_t, int, double, double,
                                    double, cudaStream_t);

// ---------------------------------------------------------------------------
// Generic local stencil by y-slabs of whole rows (any nx >= kRadius):
// y = s_h ((-1/2 Lap + Veff - shift) x) + s_p prev, the nonlocal term added
// afterwards by the tiled pass.  One CTA owns rows y0 .. y0 + by - 1 of one
// orbital for a z range and marches along z; each thread owns PPT points of
// the slab (consecutive threads, consecutive points, so every global access
// is coalesced) and keeps their 13 values along z in a register queue.  Per
// plane the CTA writes its own centre values into shared memory, loads the 2R
// halo rows above and below, and repeats the first and last R columns of
// every row beside it (periodic x; zero columns for Dirichlet x), so that the
// x and y neighbours are read from shared memory without index wrapping.
// Global reads per plane: the own points once, plus 2R / by halo rows.
// Arithmetic in the same order as k_apply_h's local part.
// ---------------------------------------------------------------------------
namespace {

constexpr int kSlabThreads = 256;

template <typename T>
struct SlabArgs {
  const T* x;
  int64_t ldx;
  T* y;
  int64_t ldy;
  const T* prev;
  int64_t ldp;
  const T* veff;
  int nx, ny, nz, bcx, bcy, bcz;
  int by, bz;
  T dms;               // -1/2 * 3 w0/h^2 - shift
  T off[kRadius + 1];  // -1/2 w_p/h^2
  T s_h, s_p;
};

template <typename T, int PPT>
__global__ void __launch_bounds__(kSlabThreads, sizeof(T) == 4 ? 4 : 2)
    k_apply_h_slab(const SlabArgs<T> a) {
  constexpr int R = kRadius;
  extern __shared__ __align__(16) unsigned char slab_raw[];
  T* const s = reinterpret_cast<T*>(slab_raw);
  const int W = a.nx + 2 * R;  // shared row: R ghost columns, nx, R ghost columns
  const int n = blockIdx.y;
  const int y0 = blockIdx.x * a.by;
  const int byl = min(a.by, a.ny - y0);
  const int npts = byl * a.nx;
  const int z0 = blockIdx.z * a.bz, z1 = min(z0 + a.bz, a.nz);
  const int64_t nxy = (int64_t)a.nx * a.ny;
  const T* __restrict__ xn = a.x + (int64_t)n * a.ldx;
  const bool perx = a.bcx == SPARC_PERIODIC;
  for (int e = threadIdx.x; e < (a.by + 2 * R) * W; e += blockDim.x) s[e] = T(0);

  int pofs[PPT], sidx[PPT];
  unsigned own = 0, dup_r = 0, dup_l = 0;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int p = threadIdx.x + k * blockDim.x;
    pofs[k] = 0;
    sidx[k] = R * W + R;
    if (p < npts) {
      const int ry = p / a.nx, rx = p - ry * a.nx;
      pofs[k] = (y0 + ry) * a.nx + rx;
      sidx[k] = (ry + R) * W + rx + R;
      own |= 1u << k;
      if (perx && rx < R) dup_r |= 1u << k;           // also right of the row
      if (perx && rx >= a.nx - R) dup_l |= 1u << k;   // also left of the row
    }
  }
  T q[2 * R + 1][PPT];
  auto load_q = [&](int zz, T(&d)[PPT]) {
    const bool ok = map_coord(zz, a.nz, a.bcz);
    const T* __restrict__ pl = xn + (int64_t)zz * nxy;
#pragma unroll
    for (int k = 0; k < PPT; ++k) d[k] = (ok && ((own >> k) & 1u)) ? __ldg(pl + pofs[k]) : T(0);
  };
#pragma unroll
  for (int j = 0; j < 2 * R + 1; ++j) load_q(z0 - R + j, q[j]);

  for (int z = z0; z < z1; ++z) {
    // this plane's Veff and previous iterate, and the queue's next plane, are
    // requested first, so that their latency overlaps the barrier below
    const int64_t gz = (int64_t)z * nxy;
    T vf[PPT], pv[PPT], nq[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const bool o = (own >> k) & 1u;
      vf[k] = o ? __ldg(a.veff + gz + pofs[k]) : T(0);
      pv[k] = (o && a.prev) ? a.prev[(int64_t)n * a.ldp + gz + pofs[k]] : T(0);
    }
    load_q(z + R + 1, nq);
    // own centre values of plane z, with their ghost copies
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      if ((own >> k) & 1u) {
        s[sidx[k]] = q[R][k];
        if ((dup_r >> k) & 1u) s[sidx[k] + a.nx] = q[R][k];
        if ((dup_l >> k) & 1u) s[sidx[k] - a.nx] = q[R][k];
      }
    }
    // R halo rows above and below the slab (wrapped, or zero outside)
    const T* __restrict__ pl = xn + (int64_t)z * nxy;
    for (int e = threadIdx.x; e < 2 * R * a.nx; e += blockDim.x) {
      const int hr = e / a.nx, hx = e - hr * a.nx;
      const int srow = hr < R ? hr : byl + hr;
      int gy = hr < R ? y0 - R + hr : y0 + byl + hr - R;
      const bool ok = map_coord(gy, a.ny, a.bcy);
      const T v = ok ? __ldg(pl + (int64_t)gy * a.nx + hx) : T(0);
      const int si = srow * W + hx + R;
      s[si] = v;
      if (perx && hx < R) s[si + a.nx] = v;
      if (perx && hx >= a.nx - R) s[si - a.nx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      if ((own >> k) & 1u) {
        const T* c = s + sidx[k];
        T acc = a.dms * q[R][k];
#pragma unroll
        for (int p = 1; p <= R; ++p) {
          const T sum = (c[p] + c[-p]) + (c[p * W] + c[-p * W]) + (q[R + p][k] + q[R - p][k]);
          acc += a.off[p] * sum;
        }
        acc += vf[k] * q[R][k];
        const T out = a.prev ? a.s_h * acc + a.s_p * pv[k] : a.s_h * acc;
        a.y[(int64_t)n * a.ldy + gz + pofs[k]] = out;
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 2 * R; ++j)
#pragma unroll
      for (int k = 0; k < PPT; ++k) q[j][k] = q[j + 1][k];
#pragma unroll
    for (int k = 0; k < PPT; ++k) q[2 * R][k] = nq[k];
  }
}

template <typename T>
struct SlabPpt;
template <>
struct SlabPpt<float> { static constexpr int v = 2; };
template <>
struct SlabPpt<double> { static constexpr int v = 2; };

}  // namespace

template <typename T>
cudaError_t apply_h_local(const Grid& g, const LapCoef& lc, const T* veff, const T* x,
                          int64_t ldx, T* y, int64_t ldy, const T* prev, int64_t ldp, int ns,
                          double shift, double s_h, double s_p, cudaStream_t st, bool* used) {
  constexpr int PPT = SlabPpt<T>::v;
  constexpr int R = kRadius;
  *used = false;
  const int maxpts = PPT * kSlabThreads;
  if (g.nx < R || g.nx > maxpts || ns < 1 || ns > 65535) return cudaSuccess;
  int by = std::min(g.ny, maxpts / g.nx);
  const int nslab = (g.ny + by - 1) / by;
  by = (g.ny + nslab - 1) / nslab;
  const int threads = ((by * g.nx + PPT - 1) / PPT + 31) / 32 * 32;
  const size_t smem = (size_t)(by + 2 * R) * (g.nx + 2 * R) * sizeof(T);
  if (smem > 48 * 1024) return cudaSuccess;
  // z chunks: enough CTAs to cover the SMs several times, each chunk at least
  // 2R planes deep (its queue reads 2R planes beyond it)
  const int64_t xy_ctas = (int64_t)nslab * ns;
  int nzc = (int)std::min<int64_t>((8 * sm_count() + xy_ctas - 1) / xy_ctas, 1 << 20);
  nzc = std::max(1, std::min(nzc, std::max(1, g.nz / (2 * R))));
  const int bz = (g.nz + nzc - 1) / nzc;
  nzc = (g.nz + bz - 1) / bz;
  SlabArgs<T> a;
  a.x = x; a.ldx = ldx; a.y = y; a.ldy = ldy; a.prev = prev; a.ldp = ldp; a.veff = veff;
  a.nx = g.nx; a.ny = g.ny; a.nz = g.nz; a.bcx = g.bc[0]; a.bcy = g.bc[1]; a.bcz = g.bc[2];
  a.by = by;
  a.bz = bz;
  a.dms = T(lc.diag - shift);
  for (int p = 0; p <= R; ++p) a.off[p] = T(lc.off[p]);
  a.s_h = T(s_h);
  a.s_p = T(s_p);
  note_launch();
  k_apply_h_slab<T, PPT><<<dim3(nslab, ns, nzc), threads, smem, st>>>(a);
  *used = true;
  return cudaGetLastError();
}

template cudaError_t apply_h_local<float>(const Grid&, const LapCoef&, const float*, const float*,
                                          int64_t, float*, int64_t, const float*, int64_t, int,
                                          double, double, double, cudaStream_t, bool*);
template cudaError_t apply_h_local<double>(const Grid&, const LapCoef&, const double*,
                                           const double*, int64_t, double*, int64_t,
                                           const double*, int64_t, int, double, double, double,
                                           cudaStream_t, bool*);

// ---------------------------------------------------------------------------
// K2: nonlocal coefficients D[n][k] = gamma_k h^3 sum_t chi_k(t) x_n(t).  One
// CTA per (atom, group of kNlOrb orbitals): threads stride over the atom's
// support points, load the point's projector values once and apply them to
// every orbital of the group; warp partial sums go through shared memory and
// are added in a fixed order (deterministic).
// ---------------------------------------------------------------------------
namespace {

constexpr int kNlThreads = 256;
constexpr int kNlOrb = 8;
constexpr int kNlProj = 4;  // projectors per pass

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void __launch_bounds__(kNlThreads)
    k_nl_coef(const Nonlocal<T> nl, double h3, const T* __restrict__ x, int64_t ldx, int ns,
              T* __restrict__ D, bool kmajor) {
  __shared__ T red[kNlThreads / 32][kNlOrb][kNlProj];
  const int J = blockIdx.x;
  const int64_t s0 = nl.supp_ptr[J];
  const int nsup = (int)(nl.supp_ptr[J + 1] - s0);
  const int np = nl.nproj[J];
  const T* __restrict__ chi = nl.chi + nl.chi_ptr[J];
  const int k0 = nl.proj_ptr[J];
  const int* __restrict__ idx = nl.supp_idx + s0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nb = blockIdx.y * kNlOrb;
  const int norb = min(kNlOrb, ns - nb);
  const T* __restrict__ xb = x + (int64_t)nb * ldx;
  for (int qb = 0; qb < np; qb += kNlProj) {
    T acc[kNlOrb][kNlProj];
#pragma unroll
    for (int n = 0; n < kNlOrb; ++n)
#pragma unroll
      for (int q = 0; q < kNlProj; ++q) acc[n][q] = T(0);
    for (int t = threadIdx.x; t < nsup; t += kNlThreads) {
      const int64_t i = __ldg(idx + t);
      T c[kNlProj];
#pragma unroll
      for (int q = 0; q < kNlProj; ++q)
        c[q] = qb + q < np ? __ldg(chi + (int64_t)(qb + q) * nsup + t) : T(0);
      T xv[kNlOrb];
#pragma unroll
      for (int n = 0; n < kNlOrb; ++n) xv[n] = n < norb ? __ldg(xb + (int64_t)n * ldx + i) : T(0);
#pragma unroll
      for (int n = 0; n < kNlOrb; ++n)
#pragma unroll
        for (int q = 0; q < kNlProj; ++q) acc[n][q] += c[q] * xv[n];
    }
#pragma unroll
    for (int n = 0; n < kNlOrb; ++n)
#pragma unroll
      for (int q = 0; q < kNlProj; ++q) {
        const T v = warp_sum(acc[n][q]);
        if (lane == 0) red[wid][n][q] = v;
      }
    __syncthreads();
    if (threadIdx.x < kNlOrb * kNlProj) {
      const int n = threadIdx.x / kNlProj, q = threadIdx.x % kNlProj;
      if (n < norb && qb + q < np) {
        T v = T(0);
        for (int w = 0; w < kNlThreads / 32; ++w) v += red[w][n][q];
        const int k = k0 + qb + q;
        D[kmajor ? (int64_t)k * ns + nb + n : (int64_t)(nb + n) * nl.kp + k] =
            T(v * (nl.gamma[k] * h3));
      }
    }
    __syncthreads();
  }
}

}  // namespace

template <typename T>
cudaError_t nl_coefficients(const Nonlocal<T>& nl, double h3, const T* x, int64_t ldx, int ns,
                            T* D, cudaStream_t st, bool kmajor) {
  if (nl.natoms == 0 || nl.kp == 0) return cudaSuccess;
  dim3 grid(nl.natoms, (ns + kNlOrb - 1) / kNlOrb);
  note_launch(), k_nl_coef<T><<<grid, kNlThreads, 0, st>>>(nl, h3, x, ldx, ns, D, kmajor);
  return cudaGetLastError();
}

template cudaError_t nl_coefficients<double>(const Nonlocal<double>&, double, const double*,
                                             int64_t, int, double*, cudaStream_t, bool);
template cudaError_t nl_coefficients<float>(const Nonlocal<float>&, double, const float*,
                                            int64_t, int, float*, cudaStream_t, bool);

// ---------------------------------------------------------------------------
// Block copy between leading dimensions.
// ---------------------------------------------------------------------------
namespace {
template <typename T, typename U>
__global__ void k_copy_block(const T* __restrict__ src, int64_t lds, U* __restrict__ dst,
                             int64_t ldd, int64_t nd) {
  const int n = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nd;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[n * ldd + i] = (U)src[n * lds + i];
}
}  // namespace

template <typename T, typename U>
cudaError_t copy_block(const T* src, int64_t lds, U* dst, int64_t ldd, int64_t nd, int ns,
                       cudaStream_t st) {
  int bx = (int)std::min<int64_t>((nd + 255) / 256, 1024);
  note_launch(), k_copy_block<T, U><<<dim3(bx, ns), 256, 0, st>>>(src, lds, dst, ldd, nd);
  return cudaGetLastError();
}
template cudaError_t copy_block<double, double>(const double*, int64_t, double*, int64_t, int64_t,
                                                int, cudaStream_t);
template cudaError_t copy_block<float, float>(const float*, int64_t, float*, int64_t, int64_t,
                                              int, cudaStream_t);
template cudaError_t copy_block<float, double>(const float*, int64_t, double*, int64_t, int64_t,
                                               int, cudaStream_t);

// ---------------------------------------------------------------------------
// FP64 vector kernels for Lanczos.  Reductions: kRedBlocks fixed partial sums
// (grid-stride, fixed order) then one block sums the partials in order.
// ---------------------------------------------------------------------------
namespace {

constexpr int kRedBlocks = 256;
constexpr int kRedThreads = 256;

__device__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  __syncthreads();
  return t;  // valid in thread 0
}

__global__ void k_dot_partial(const double* __restrict__ u, const double* __restrict__ v,
                              int64_t n, double* __restrict__ partial) {
  __shared__ double sh[kRedThreads / 32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc += u[i] * v[i];
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void k_sum_partials(const double* __restrict__ partial, int np, double* out,
                               int mode) {
  __shared__ double sh[kRedThreads / 32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += partial[i];
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) *out = mode == 1 ? sqrt(t) : t;
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__global__ void k_fill_uniform(double* v, int64_t n, uint64_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = mix64(seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ULL);
    v[i] = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
  }
}

// complex (interleaved) vector with real part u(seed, i) - 1/2, imaginary part 0
__global__ void k_fill_uniform_re(double* v, int64_t n, uint64_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = mix64(seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ULL);
    v[2 * i] = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    v[2 * i + 1] = 0.0;
  }
}

// ab layout: ab[2j] = alpha_j, ab[2j+1] = beta_j; ab[-1] slot handled by j == 0.
__global__ void k_lz_sub_prev(double* __restrict__ w, const double* __restrict__ vp,
                              const double* __restrict__ ab, int j, int64_t n) {
  double bprev = j > 0 ? ab[2 * (j - 1) + 1] : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    w[i] -= bprev * vp[i];
}

__global__ void k_lz_sub_alpha(double* __restrict__ w, const double* __restrict__ v,
                               const double* __restrict__ ab, int j, int64_t n) {
  double al = ab[2 * j];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    w[i] -= al * v[i];
}

__global__ void k_lz_shift(double* __restrict__ v, const double* __restrict__ w,
                           double* __restrict__ vp, const double* __restrict__ ab, int j,
                           int64_t n) {
  double bt = ab[2 * j + 1];
  double inv = bt > 0.0 ? 1.0 / bt : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    vp[i] = v[i];
    v[i] = w[i] * inv;
  }
}

__global__ void k_scale_inv(double* v, const double* nrm, int64_t n) {
  double inv = 1.0 / *nrm;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] *= inv;
}

// Number of eigenvalues of the k x k tridiagonal (alpha, beta) below x (Sturm count).
__device__ int sturm_count(const double* ab, int k, double x) {
  int cnt = 0;
  double q = 1.0;
  for (int i = 0; i < k; ++i) {
    double b2 = i > 0 ? ab[2 * (i - 1) + 1] * ab[2 * (i - 1) + 1] : 0.0;
    q = (ab[2 * i] - x) - (i > 0 ? b2 / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// Extreme eigenvalues of the Lanczos tridiagonal by bisection; out2 = {a0, b}.
__global__ void k_lz_bounds(const double* ab, int k, double* out2) {
  if (threadIdx.x >= 2) return;
  double lo = ab[0], hi = ab[0];
  for (int i = 0; i < k; ++i) {
    double r = (i > 0 ? fabs(ab[2 * (i - 1) + 1]) : 0.0) + (i + 1 < k ? fabs(ab[2 * i + 1]) : 0.0);
    lo = fmin(lo, ab[2 * i] - r);
    hi = fmax(hi, ab[2 * i] + r);
  }
  const int target = threadIdx.x == 0 ? 0 : k - 1;  // index of the wanted eigenvalue
  double a = lo, b = hi;
  for (int it = 0; it < 200 && b - a > 2.2e-16 * fmax(fabs(a), fabs(b)); ++it) {
    double m = 0.5 * (a + b);
    if (m <= a || m >= b) break;
    if (sturm_count(ab, k, m) > target) b = m; else a = m;
  }
  double theta = 0.5 * (a + b);
  if (threadIdx.x == 0) out2[0] = theta;
  else out2[1] = theta + fabs(ab[2 * (k - 1) + 1]);
}

int grid_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 2048); }

}  // namespace

cudaError_t dot_f64(const double* u, const double* v, int64_t n, double* partial, double* out,
                    cudaStream_t st) {
  note_launch(), k_dot_partial<<<kRedBlocks, kRedThreads, 0, st>>>(u, v, n, partial);
  note_launch(), k_sum_partials<<<1, kRedThreads, 0, st>>>(partial, kRedBlocks, out, 0);
  return cudaGetLastError();
}

cudaError_t fill_uniform_f64(double* v, int64_t n, uint64_t seed, cudaStream_t st) {
  note_launch(), k_fill_uniform<<<grid_for(n), 256, 0, st>>>(v, n, seed);
  return cudaGetLastError();
}

cudaError_t fill_uniform_re_c128(double* v, int64_t n, uint64_t seed, cudaStream_t st) {
  note_launch(), k_fill_uniform_re<<<grid_for(n), 256, 0, st>>>(v, n, seed);
  return cudaGetLastError();
}

// w -= beta_{j-1} vp; alpha_j = w.v; w -= alpha_j v
cudaError_t lanczos_update(double* w, const double* v, double* vp, const double* ab, int j,
                           int64_t n, cudaStream_t st) {
  note_launch(), k_lz_sub_prev<<<grid_for(n), 256, 0, st>>>(w, vp, ab, j, n);
  return cudaGetLastError();
}

// alpha_j = w.v; w -= alpha_j v; beta_j = |w|; vp = v; v = w / beta_j.
// For j < 0: normalise v in place (start vector).
cudaError_t lanczos_normalize(double* v, double* w, double* vp, double* ab, int j, int64_t n,
                              double* partial, cudaStream_t st) {
  if (j < 0) {
    note_launch(), k_dot_partial<<<kRedBlocks, kRedThreads, 0, st>>>(v, v, n, partial);
    note_launch(), k_sum_partials<<<1, kRedThreads, 0, st>>>(partial, kRedBlocks, partial + kRedBlocks, 1);
    note_launch(), k_scale_inv<<<grid_for(n), 256, 0, st>>>(v, partial + kRedBlocks, n);
    return cudaGetLastError();
  }
  note_launch(), k_dot_partial<<<kRedBlocks, kRedThreads, 0, st>>>(w, v, n, partial);
  note_launch(), k_sum_partials<<<1, kRedThreads, 0, st>>>(partial, kRedBlocks, ab + 2 * j, 0);
  note_launch(), k_lz_sub_alpha<<<grid_for(n), 256, 0, st>>>(w, v, ab, j, n);
  note_launch(), k_dot_partial<<<kRedBlocks, kRedThreads, 0, st>>>(w, w, n, partial);
  note_launch(), k_sum_partials<<<1, kRedThreads, 0, st>>>(partial, kRedBlocks, ab + 2 * j + 1, 1);
  note_launch(), k_lz_shift<<<grid_for(n), 256, 0, st>>>(v, w, vp, ab, j, n);
  return cudaGetLastError();
}

cudaError_t lanczos_bounds(const double* ab, int k, double* out2, cudaStream_t st) {
  note_launch(), k_lz_bounds<<<1, 32, 0, st>>>(ab, k, out2);
  return cudaGetLastError();
}

}  // namespace sparc
