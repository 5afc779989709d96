// Hamiltonian application (paper Sec. II A) with a TMA plane ring — the fast
// form of K1 used when the grid rows are TMA-friendly.
//
// One CTA owns one orbital and one y-slab of BY rows spanning the full x
// extent, and marches along z.  For every z-plane a single thread issues TMA
// loads of the slab plus its 6-row y halos (wrapped for periodic y, zero-filled
// outside the grid for Dirichlet y; zero-filled planes for Dirichlet z) into a
// ring of S shared-memory slots, up to S - 7 planes ahead of use, with one
// full/empty mbarrier pair per slot.  Each thread computes VY = 2 rows x VX
// consecutive x points: x and y neighbours come from the slot of the current
// plane (vector shared-memory loads), z neighbours from a 13-deep register
// queue fed from the ring.  Veff, the nonlocal pull-add and the Chebyshev
// recurrence axpy are fused as in the generic kernel.  Every mbarrier wait is
// bounded; on expiry the CTA records SPARC_ERR_TIMEOUT and leaves its loop.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "internal.cuh"

namespace sparc {

namespace {

constexpr int R = kRadius;
constexpr int VY = 2;
constexpr long long kWait = 4000000000LL;

__device__ __forceinline__ uint32_t su32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ bool bar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait.  Gives up when its own budget runs out (recording the timeout)
// or as soon as any CTA of the launch has recorded one in the status word.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, int* status) {
  if (bar_test(bar, parity)) return true;
  const long long t0 = clock64();
  while (!bar_test(bar, parity)) {
    if (*(volatile int*)status != 0) return false;
    if (clock64() - t0 > kWait) {
      atomicCAS(status, 0, SPARC_ERR_TIMEOUT);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void tma4(uint32_t dst, const CUtensorMap* m, int x, int y, int z,
                                     int n, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(m), "r"(x), "r"(y), "r"(z), "r"(n), "r"(bar)
      : "memory");
}

template <typename T, int V>
struct Vec;
template <>
struct Vec<float, 4> { using t = float4; };
template <>
struct Vec<double, 2> { using t = double2; };

template <typename T, int V>
__device__ __forceinline__ void lds(T (&d)[V], const T* p) {
  typename Vec<T, V>::t v = *reinterpret_cast<const typename Vec<T, V>::t*>(p);
  const T* s = reinterpret_cast<const T*>(&v);
#pragma unroll
  for (int i = 0; i < V; ++i) d[i] = s[i];
}
template <typename T, int V>
__device__ __forceinline__ void ldg(T (&d)[V], const T* p) {
  typename Vec<T, V>::t v = __ldg(reinterpret_cast<const typename Vec<T, V>::t*>(p));
  const T* s = reinterpret_cast<const T*>(&v);
#pragma unroll
  for (int i = 0; i < V; ++i) d[i] = s[i];
}
template <int V>
__device__ __forceinline__ void ldg_idx(int (&d)[V], const int* p) {
  if constexpr (V == 4) {
    const int4 v = __ldg(reinterpret_cast<const int4*>(p));
    d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
  } else {
    const int2 v = __ldg(reinterpret_cast<const int2*>(p));
    d[0] = v.x; d[1] = v.y;
  }
}
template <typename T, int V>
__device__ __forceinline__ void stg(T* p, const T (&d)[V]) {
  typename Vec<T, V>::t v;
  T* s = reinterpret_cast<T*>(&v);
#pragma unroll
  for (int i = 0; i < V; ++i) s[i] = d[i];
  *reinterpret_cast<typename Vec<T, V>::t*>(p) = v;
}

template <typename T>
struct RingArgs {
  T* y;
  int64_t ldy;
  const T* prev;
  int64_t ldp;
  const T* veff;
  const int* grp_ptr;  // grouped nonlocal slots, VX points per group
  const int* grp_k;
  const T* grp_chi;
  const T* D;
  int kp;
  uint32_t d_off;  // byte offset of the orbital's D column in dynamic shared memory
  int nx, ny, nz, bcx, bcy, bcz;
  int by;        // slab rows
  int nslab;     // ny / by (rounded up)
  int bz;        // z planes per CTA
  int slots;     // ring depth S
  uint32_t slot_bytes;
  T diag_minus_shift;
  T off[R + 1];
  T s_h, s_p;
  int* status;
};

template <typename T, int VX>
__global__ void __launch_bounds__(384, 1)
    k_apply_h_ring(const __grid_constant__ CUtensorMap mid, const __grid_constant__ CUtensorMap halo,
                   const RingArgs<T> a) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full[16], empty[16];
  __shared__ int abort_sh;
  __shared__ int issued_hi;  // one past the last issued plane

  const int nwarps = (blockDim.x + 31) >> 5;
  const int qpr = a.nx / VX;  // x quads per row
  const int tid = threadIdx.x;
  const int ry = tid / qpr, qx = tid % qpr;
  const int x = qx * VX;
  const int yy = ry * VY;  // first of the thread's two rows within the slab
  const int n = blockIdx.x / a.nslab;
  const int slab = blockIdx.x % a.nslab;
  const int y0 = slab * a.by;
  const int z0 = blockIdx.y * a.bz;
  const int z1 = min(z0 + a.bz, a.nz);
  const int pbase = z0 - R;
  const int S = a.slots;
  const int rowe = a.nx;  // elements per shared row
  const uint32_t base = (su32(smem_raw) + 127u) & ~127u;
  T* const ring = reinterpret_cast<T*>(smem_raw + (base - su32(smem_raw)));
  const int64_t nxy = (int64_t)a.nx * a.ny;
  const int slab_rows = a.by + 2 * R;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&full[s])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&empty[s])), "r"(nwarps));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_sh = 0;
    issued_hi = z0 - R;
  }
  // this CTA's orbital column of the nonlocal coefficients D, kept on chip
  T* const dsh = reinterpret_cast<T*>(smem_raw + (base - su32(smem_raw)) + a.d_off);
  for (int k = tid; k < a.kp; k += blockDim.x) dsh[k] = __ldg(a.D + (int64_t)n * a.kp + k);
  __syncthreads();
  volatile int* abort = &abort_sh;
  const unsigned full_mask = 0xffffffffu;

  // issue plane p into its slot (thread 0 only)
  auto issue = [&](int p) {
    const int k = p - pbase;
    const int s = k % S;
    const uint32_t fb = su32(&full[s]);
    const uint32_t dst = base + (uint32_t)s * a.slot_bytes;
    int zc = p;
    if (a.bcz == SPARC_PERIODIC) {
      zc %= a.nz;
      if (zc < 0) zc += a.nz;
    }
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                 "r"((uint32_t)(slab_rows * rowe * sizeof(T)))
                 : "memory");
    int yt = y0 - R, yb = y0 + a.by;
    if (a.bcy == SPARC_PERIODIC) {
      if (yt < 0) yt += a.ny;
      if (yb >= a.ny) yb -= a.ny;
    }
    const uint32_t rb = (uint32_t)(rowe * sizeof(T));
    tma4(dst, &halo, 0, yt, zc, n, fb);
    tma4(dst + R * rb, &mid, 0, y0, zc, n, fb);
    tma4(dst + (R + a.by) * rb, &halo, 0, yb, zc, n, fb);
    issued_hi = p + 1;
  };
  // bounded wait; any timeout aborts the whole CTA
  auto wait = [&](uint32_t bar, uint32_t parity) {
    if (*abort) return false;
    if (!bar_wait(bar, parity, a.status)) {
      *abort = 1;
      return false;
    }
    return true;
  };
  // slot, phase of plane p
  auto slot_of = [&](int p) { return (p - pbase) % S; };
  auto round_of = [&](int p) { return (uint32_t)((p - pbase) / S); };

  const int plast = z1 + R;  // planes [pbase, plast) are needed
  if (tid == 0)
    for (int p = pbase; p < min(plast, pbase + S); ++p) issue(p);

  T q[2 * R + 1][VY][VX];
  // initial queue: planes z0-R .. z0+R-1.  The first R of them (before z0) serve
  // only the queue, so each is released as soon as it is read and its slot is
  // refilled at once: the ring then needs only 2R - R + 1 = R + 1 < S slots of
  // look-ahead here instead of all 2R planes at the same time.
#pragma unroll
  for (int j = 0; j < 2 * R; ++j) {
    const int p = pbase + j;
    const int s = slot_of(p);
    wait(su32(&full[s]), round_of(p) & 1);
    const T* row = ring + (size_t)s * (a.slot_bytes / sizeof(T));
#pragma unroll
    for (int r = 0; r < VY; ++r) lds<T, VX>(q[j][r], row + (R + yy + r) * rowe + x);
    if (j < R) {
      __syncwarp();
      if ((tid & 31) == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&empty[s]))
                     : "memory");
      if (tid == 0 && p + S < plast)
        if (wait(su32(&empty[s]), round_of(p) & 1)) issue(p + S);
      __syncwarp();
    }
  }

  T* __restrict__ yn = a.y + (int64_t)n * a.ldy;
  const T* __restrict__ pn = a.prev ? a.prev + (int64_t)n * a.ldp : nullptr;
  const int gy0 = y0 + yy;

  for (int z = z0; z < z1; ++z) {
    if (__shfl_sync(full_mask, *abort, 0)) break;
    // Veff, prev and the nonlocal slot range of this plane (used after the
    // stencil sums, which cover their latency)
    const int64_t g0 = z * nxy + (int64_t)gy0 * a.nx + x;
    T vf[VY][VX], pv[VY][VX];
    int gs[VY], ge[VY];
#pragma unroll
    for (int r = 0; r < VY; ++r) {
      gs[r] = ge[r] = 0;
      if (gy0 + r < a.ny) {
        ldg<T, VX>(vf[r], a.veff + g0 + r * a.nx);
        if (pn) ldg<T, VX>(pv[r], pn + g0 + r * a.nx);
        if (a.kp > 0) {
          const int64_t q = (g0 + r * a.nx) / VX;
          gs[r] = __ldg(a.grp_ptr + q);
          ge[r] = __ldg(a.grp_ptr + q + 1);
        }
      }
    }
    // push plane z + R into the queue
    {
      const int p = z + R;
      const int s = slot_of(p);
      const bool got = wait(su32(&full[s]), round_of(p) & 1);
      if (!__all_sync(full_mask, got)) break;
      const T* row = ring + (size_t)s * (a.slot_bytes / sizeof(T));
#pragma unroll
      for (int r = 0; r < VY; ++r) lds<T, VX>(q[2 * R][r], row + (R + yy + r) * rowe + x);
    }
    const int sz = slot_of(z);
    const T* pl = ring + (size_t)sz * (a.slot_bytes / sizeof(T));
    T acc[VY][VX];
#pragma unroll
    for (int r = 0; r < VY; ++r)
#pragma unroll
      for (int v = 0; v < VX; ++v) acc[r][v] = a.diag_minus_shift * q[R][r][v];
    // y and z neighbours
#pragma unroll
    for (int p = 1; p <= R; ++p) {
      T up[VY][VX], dn[VY][VX];
#pragma unroll
      for (int r = 0; r < VY; ++r) {
        lds<T, VX>(up[r], pl + (R + yy + r + p) * rowe + x);
        lds<T, VX>(dn[r], pl + (R + yy + r - p) * rowe + x);
      }
#pragma unroll
      for (int r = 0; r < VY; ++r)
#pragma unroll
        for (int v = 0; v < VX; ++v)
          acc[r][v] += a.off[p] * ((up[r][v] + dn[r][v]) + (q[R + p][r][v] + q[R - p][r][v]));
    }
    // x neighbours
#pragma unroll
    for (int r = 0; r < VY; ++r) {
      const T* rowp = pl + (R + yy + r) * rowe;
      // window x - R .. x + VX - 1 + R; interior threads read it with aligned
      // vector loads starting at x - WL (bank-conflict free), edge threads wrap
      T w[VX + 2 * R];
      constexpr int WL = (R + VX - 1) / VX * VX;  // >= R, multiple of VX
      constexpr int NV = (2 * WL + VX) / VX;
      if (x >= WL && x + VX + WL <= a.nx) {
        T buf[NV * VX];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          T t4[VX];
          lds<T, VX>(t4, rowp + x - WL + k * VX);
#pragma unroll
          for (int v = 0; v < VX; ++v) buf[k * VX + v] = t4[v];
        }
#pragma unroll
        for (int i = 0; i < VX + 2 * R; ++i) w[i] = buf[i + WL - R];
      } else {
#pragma unroll
        for (int i = 0; i < VX + 2 * R; ++i) {
          int xx = x - R + i;
          bool inside = true;
          if (xx < 0 || xx >= a.nx) {
            if (a.bcx == SPARC_DIRICHLET) inside = false;
            else xx = xx < 0 ? xx + a.nx : xx - a.nx;
          }
          w[i] = inside ? rowp[xx] : T(0);
        }
      }
#pragma unroll
      for (int p = 1; p <= R; ++p)
#pragma unroll
        for (int v = 0; v < VX; ++v) acc[r][v] += a.off[p] * (w[R + v + p] + w[R + v - p]);
    }
    // release the slot of plane z (all warps), refill it with plane z + S
    __syncwarp();
    if ((tid & 31) == 0)
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&empty[sz])) : "memory");
    if (tid == 0 && z + S < plast) {
      if (wait(su32(&empty[sz]), round_of(z) & 1)) issue(z + S);
    }
    __syncwarp();
    // Veff, nonlocal pull-add (one slot = VX (k, chi) pairs), recurrence, store
#pragma unroll
    for (int r = 0; r < VY; ++r) {
      if (gy0 + r >= a.ny) continue;
      const int64_t g = g0 + r * a.nx;
      T h[VX];
#pragma unroll
      for (int v = 0; v < VX; ++v) h[v] = acc[r][v] + vf[r][v] * q[R][r][v];
      // up to four slots' loads in flight before their FMAs (the loads are L2
      // round trips; one at a time they would serialise)
      for (int sl = gs[r]; sl < ge[r]; sl += 4) {
        int kk[4][VX];
        T ch[4][VX];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (sl + u < ge[r]) {
            ldg_idx<VX>(kk[u], a.grp_k + (int64_t)(sl + u) * VX);
            ldg<T, VX>(ch[u], a.grp_chi + (int64_t)(sl + u) * VX);
          } else {
#pragma unroll
            for (int v = 0; v < VX; ++v) {
              kk[u][v] = 0;
              ch[u][v] = T(0);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < VX; ++v) h[v] += ch[u][v] * dsh[kk[u][v]];
      }
      T out[VX];
#pragma unroll
      for (int v = 0; v < VX; ++v) out[v] = pn ? a.s_h * h[v] + a.s_p * pv[r][v] : a.s_h * h[v];
      stg<T, VX>(yn + g, out);
    }

#pragma unroll
    for (int j = 0; j < 2 * R; ++j)
#pragma unroll
      for (int r = 0; r < VY; ++r)
#pragma unroll
        for (int v = 0; v < VX; ++v) q[j][r][v] = q[j + 1][r][v];
  }
  // drain: every issued load must have landed before the CTA exits
  if (tid == 0) {
    const int hi = issued_hi;
    for (int p = max(pbase, hi - S); p < hi; ++p) {
      const long long t0 = clock64();
      while (!bar_test(su32(&full[slot_of(p)]), round_of(p) & 1) && clock64() - t0 < kWait) {
      }
    }
  }
  __syncthreads();
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

template <typename T>
bool block_map(CUtensorMap* m, const T* x, int64_t ldx, const Grid& g, int ns, int rows) {
  auto enc = encoder();
  if (!enc) return false;
  const size_t es = sizeof(T);
  cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)ns};
  cuuint64_t strides[3] = {(cuuint64_t)g.nx * es, (cuuint64_t)g.nx * g.ny * es,
                           (cuuint64_t)ldx * es};
  cuuint32_t box[4] = {(cuuint32_t)g.nx, (cuuint32_t)rows, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(m, sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                   4, const_cast<T*>(x), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

// Ring-kernel plan for a grid/dtype, or false if the generic kernel must be used.
template <typename T>
bool ring_plan(const Grid& g, int kp, int& by, int& slots, uint32_t& slot_bytes, int& threads) {
  constexpr int VX = sizeof(T) == 4 ? 4 : 2;
  const int es = sizeof(T);
  if (g.nx % (sizeof(T) == 4 ? 16 : 8) != 0 || g.nx > 256) return false;
  const int cands[3] = {sizeof(T) == 4 ? 32 : 16, 16, 8};
  by = 0;
  for (int c : cands) {
    if (g.ny % c == 0 || (g.bc[1] == SPARC_DIRICHLET && c <= g.ny)) {
      if ((c / VY) * (g.nx / VX) <= 384) {
        by = c;
        break;
      }
    }
  }
  if (by == 0) return false;
  if (g.bc[1] == SPARC_PERIODIC && g.ny < by + 2 * R && g.ny != by) return false;
  if (g.bc[1] == SPARC_PERIODIC && g.ny < 2 * R) return false;
  slot_bytes = (uint32_t)((by + 2 * R) * g.nx * es);
  slot_bytes = (slot_bytes + 127u) & ~127u;
  const int64_t dbytes = (int64_t)kp * es;
  if (dbytes > 64 * 1024) return false;
  const uint32_t budget = (uint32_t)(200 * 1024 - dbytes);
  slots = std::min<int>(13, (int)(budget / slot_bytes));
  if (slots < 8) return false;  // the march needs plane z + R resident S - 7 planes ahead
  threads = (by / VY) * (g.nx / VX);
  return threads >= 32 && threads % 32 == 0;
}

template <typename T>
cudaError_t apply_h_ring(const Grid& g, const LapCoef& lc, const T* veff, const Nonlocal<T>& nl,
                         const T* D, const T* x, int64_t ldx, T* y, int64_t ldy, const T* prev,
                         int64_t ldp, int ns, double shift, double s_h, double s_p, int* status,
                         cudaStream_t st, bool* used) {
  *used = false;
  constexpr int VX = sizeof(T) == 4 ? 4 : 2;
  int by, slots, threads;
  uint32_t slot_bytes;
  if (!ring_plan<T>(g, nl.kp, by, slots, slot_bytes, threads)) return cudaSuccess;
  if (nl.kp > 0 && (!nl.grp_ptr || nl.grp != VX)) return cudaSuccess;
  const int va = 16 / sizeof(T);
  if (ldx % va || ldy % va || (prev && ldp % va) || ((uintptr_t)x % 16) || ((uintptr_t)y % 16) ||
      (prev && ((uintptr_t)prev % 16)) || ((uintptr_t)veff % 16))
    return cudaSuccess;
  CUtensorMap mmid, mhalo;
  if (!block_map<T>(&mmid, x, ldx, g, ns, by) || !block_map<T>(&mhalo, x, ldx, g, ns, R))
    return cudaSuccess;
  RingArgs<T> a;
  a.y = y; a.ldy = ldy; a.prev = prev; a.ldp = ldp; a.veff = veff;
  a.grp_ptr = nl.grp_ptr; a.grp_k = nl.grp_k; a.grp_chi = nl.grp_chi; a.D = D; a.kp = nl.kp;
  a.nx = g.nx; a.ny = g.ny; a.nz = g.nz; a.bcx = g.bc[0]; a.bcy = g.bc[1]; a.bcz = g.bc[2];
  a.by = by;
  a.nslab = (g.ny + by - 1) / by;
  a.slots = slots;
  a.slot_bytes = slot_bytes;
  a.diag_minus_shift = T(lc.diag - shift);
  for (int p = 0; p <= R; ++p) a.off[p] = T(lc.off[p]);
  a.s_h = T(s_h);
  a.s_p = T(s_p);
  a.status = status;
  // z split: enough CTAs to cover the SMs a few times
  const int64_t xy = (int64_t)a.nslab * ns;
  int nzc = (int)std::max<int64_t>(1, (2 * sm_count() + xy - 1) / xy);
  nzc = std::min(nzc, std::max(1, g.nz / 16));
  a.bz = (g.nz + nzc - 1) / nzc;
  nzc = (g.nz + a.bz - 1) / a.bz;
  a.d_off = (uint32_t)slots * slot_bytes;
  const size_t smem = (size_t)slots * slot_bytes + (size_t)nl.kp * sizeof(T) + 128;
  static unsigned long long attr_bits = 0;
  cudaError_t ae = smem_limit_once(&attr_bits, (const void*)k_apply_h_ring<T, VX>, 210 * 1024);
  if (ae != cudaSuccess) return ae;
  dim3 grid((unsigned)(a.nslab * ns), (unsigned)nzc);
  note_launch(), k_apply_h_ring<T, VX><<<grid, threads, smem, st>>>(mmid, mhalo, a);
  *used = true;
  return cudaGetLastError();
}

template bool ring_plan<float>(const Grid&, int, int&, int&, uint32_t&, int&);
template bool ring_plan<double>(const Grid&, int, int&, int&, uint32_t&, int&);
template cudaError_t apply_h_ring<float>(const Grid&, const LapCoef&, const float*,
                                         const Nonlocal<float>&, const float*, const float*,
                                         int64_t, float*, int64_t, const float*, int64_t, int,
                                         double, double, double, int*, cudaStream_t, bool*);
template cudaError_t apply_h_ring<double>(const Grid&, const LapCoef&, const double*,
                                          const Nonlocal<double>&, const double*, const double*,
                                          int64_t, double*, int64_t, const double*, int64_t, int,
                                          double, double, double, int*, cudaStream_t, bool*);

}  // namespace sparc
