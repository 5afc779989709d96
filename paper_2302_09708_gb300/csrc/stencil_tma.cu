// Hamiltonian application (paper Sec. II A) with a TMA plane ring: the local
// part of H (the radius-6 finite-difference Laplacian and Veff) fused with the
// Chebyshev recurrence axpy, for grids whose rows are TMA-friendly.  The
// nonlocal projector term is applied afterwards by nl_apply (nonlocal.cu).
//
// One CTA owns one orbital and one y-slab of BY rows spanning the full x
// extent, and marches along z.  For every z-plane a single thread issues TMA
// loads of the slab plus its 6-row y halos (wrapped for periodic y, zero-filled
// outside the grid for Dirichlet y; zero-filled planes for Dirichlet z) into a
// ring of S shared-memory slots, up to S - 7 planes ahead of use, with one
// full/empty mbarrier pair per slot.  Every mbarrier wait is bounded; on expiry
// the CTA records SPARC_ERR_TIMEOUT and leaves its loop.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "internal.cuh"

namespace sparc {

namespace {

constexpr int R = kRadius;

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
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, int* status,
                                         long long budget) {
  if (bar_test(bar, parity)) return true;
  const long long t0 = clock64();
  while (!bar_test(bar, parity)) {
    if (*(volatile int*)status != 0) return false;
    if (clock64() - t0 > budget) {
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
template <typename T, int V>
__device__ __forceinline__ void stg(T* p, const T (&d)[V]) {
  typename Vec<T, V>::t v;
  T* s = reinterpret_cast<T*>(&v);
#pragma unroll
  for (int i = 0; i < V; ++i) s[i] = d[i];
  *reinterpret_cast<typename Vec<T, V>::t*>(p) = v;
}

// Two-lane arithmetic on pairs of neighbouring x points: FP32 pairs run as
// packed f32x2 instructions (one instruction per two points), FP64 pairs as
// two scalar operations.
template <typename T>
struct Two;
template <>
struct Two<float> {
  using t = float2;
  static __device__ __forceinline__ t add(t a, t b) { return __fadd2_rn(a, b); }
  static __device__ __forceinline__ t mul(t a, t b) { return __fmul2_rn(a, b); }
  static __device__ __forceinline__ t fma(t a, t b, t c) { return __ffma2_rn(a, b, c); }
  static __device__ __forceinline__ t make(float a, float b) { return make_float2(a, b); }
  static __device__ __forceinline__ t zero() { return make_float2(0.f, 0.f); }
};
template <>
struct Two<double> {
  using t = double2;
  static __device__ __forceinline__ t add(t a, t b) {
    return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y));
  }
  static __device__ __forceinline__ t mul(t a, t b) {
    return make_double2(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y));
  }
  static __device__ __forceinline__ t fma(t a, t b, t c) {
    return make_double2(__fma_rn(a.x, b.x, c.x), __fma_rn(a.y, b.y, c.y));
  }
  static __device__ __forceinline__ t make(double a, double b) { return make_double2(a, b); }
  static __device__ __forceinline__ t zero() { return make_double2(0.0, 0.0); }
};

template <typename T>
struct RingArgs {
  T* y;
  int64_t ldy;
  const T* prev;
  int64_t ldp;
  const T* veff;
  int nx, ny, nz, bcx, bcy, bcz;
  int by;        // slab rows
  int nslab;     // ny / by (rounded up)
  int bz;        // z planes per CTA
  int slots;     // ring depth S
  uint32_t slot_bytes;
  // coefficients duplicated into both lanes of a pair (kernel-argument
  // operands of the pair instructions, so they take no registers)
  typename Two<T>::t dms2;      // (-1/2 Laplacian diagonal) - shift
  typename Two<T>::t off2[R + 1];  // -1/2 w_p / h^2
  typename Two<T>::t sh2, sp2;
  long long wait_cycles;  // bound of every mbarrier wait (SM clock cycles)
  int* status;
  int stall;  // test hook: first wait on a barrier that nothing completes
};

// Local part of y = s_h (H - shift) x + s_p prev: the radius-6 Laplacian, Veff
// and the Chebyshev recurrence axpy.  The nonlocal term is added afterwards by
// nl_apply (nonlocal.cu), which reads the support points of a block of
// orbitals at once.  One CTA owns one orbital and one y-slab (BY rows x full x)
// and marches along z; TMA loads every plane of the slab with its y halos into
// a ring of S shared-memory slots.  Each thread computes VY rows x VX points per
// plane and U planes per step: y neighbours and the x window come from the
// plane's slot, z neighbours from a register queue of 2R + U planes that moves
// by U planes per step.  The x window is NC aligned vector loads at offsets
// wrapped once per thread (zero chunks for Dirichlet x), so no thread takes a
// per-element path.  Even x distances are summed as pairs, odd ones (whose
// pairs straddle two vector registers) as two scalar adds.
template <typename T, int VX, int VY, int U, int MAXT, bool XDIR>
__global__ void __launch_bounds__(MAXT, 1)
    k_apply_h_ring(const __grid_constant__ CUtensorMap mid, const __grid_constant__ CUtensorMap halo,
                   const RingArgs<T> a) {
  using TW = Two<T>;
  using P = typename TW::t;
  constexpr int NP = VX / 2;                   // point pairs per row
  constexpr int WL = (R + VX - 1) / VX * VX;   // window start x - WL (multiple of VX, >= R)
  constexpr int NC = (2 * WL + VX) / VX;       // window chunks of VX elements
  constexpr int Q = 2 * R + U;                 // queue depth (planes)
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full[16], empty[16];
  __shared__ uint64_t never;    // test hook: a barrier no thread arrives on
  __shared__ int released[16];  // warps that have released each slot this round
  __shared__ int abort_sh;
  __shared__ int issued_hi;  // one past the last issued plane

  const int nwarps = (blockDim.x + 31) >> 5;
  const int nq = a.nx / VX;  // x chunks per row
  const int tid = threadIdx.x;
  const int ry = tid / nq, qx = tid % nq;
  const int x = qx * VX;
  const int yy = ry * VY;  // first of the thread's rows within the slab
  const int n = blockIdx.x / a.nslab;
  const int slab = blockIdx.x % a.nslab;
  const int y0 = slab * a.by;
  const int z0 = blockIdx.y * a.bz;
  const int z1 = min(z0 + a.bz, a.nz);
  const int pbase = z0 - R;
  const int S = a.slots;
  const int rowe = a.nx;  // elements per shared row
  const int slot_elems = (int)(a.slot_bytes / sizeof(T));
  const uint32_t base = (su32(smem_raw) + 127u) & ~127u;
  T* const ring = reinterpret_cast<T*>(smem_raw + (base - su32(smem_raw)));
  const int64_t nxy = (int64_t)a.nx * a.ny;
  const int slab_rows = a.by + 2 * R;
  const long long wmax = a.wait_cycles;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&full[s])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&empty[s])), "r"(nwarps));
      released[s] = 0;
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&never)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_sh = 0;
    issued_hi = z0 - R;
  }
  __syncthreads();
  volatile int* abort = &abort_sh;
  const unsigned full_mask = 0xffffffffu;

  // plane p (in slot s) to the ring
  auto issue = [&](int p, int s) {
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
    atomicMax(&issued_hi, p + 1);
  };
  // bounded wait; any timeout aborts the whole CTA
  auto wait = [&](uint32_t bar, uint32_t parity) {
    if (*abort) return false;
    if (!bar_wait(bar, parity, a.status, wmax)) {
      *abort = 1;
      return false;
    }
    return true;
  };
  // slot and round of a plane, advanced one plane at a time (no division)
  struct Pos {
    int s, r;
  };
  auto advance = [&](Pos& q) {
    if (++q.s == S) {
      q.s = 0;
      ++q.r;
    }
  };

  const int plast = z1 + R;  // planes [pbase, plast) are needed
  if (tid == 0)
    for (int p = pbase; p < min(plast, pbase + S); ++p) issue(p, p - pbase);
  // test hook: this wait can only run out (after wait_cycles); the CTA then
  // stops like on any other timeout, its loads in flight drained below
  if (a.stall) wait(su32(&never), 0);
  // Release plane p's slot (lane 0 of every warp, after the warp's reads).  The
  // last warp to release it refills it with plane p + S, once the slot's empty
  // barrier has completed (bounded wait; it completes with that last arrival),
  // so no warp waits for the others and the ring stays S - 7 planes ahead.
  auto release = [&](int p, Pos ps) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&empty[ps.s])) : "memory");
    if (atomicAdd(&released[ps.s], 1) == nwarps - 1) {
      released[ps.s] = 0;
      if (p + S < plast && wait(su32(&empty[ps.s]), ps.r & 1)) issue(p + S, ps.s);
    }
  };

  // x window: chunk c covers x - WL + c VX .. + VX - 1; its row offset wrapped
  // once here (periodic x), or marked for zero fill (Dirichlet x)
  int coff[NC];
  unsigned cvalid = 0;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    int qi = qx - WL / VX + c;
    bool ok = true;
    if (qi < 0 || qi >= nq) {
      ok = !XDIR;
      qi = ((qi % nq) + nq) % nq;
    }
    coff[c] = qi * VX;
    if (ok) cvalid |= 1u << c;
  }

  auto load_pairs = [&](P (&d)[NP], const T* p) {
    T t[VX];
    lds<T, VX>(t, p);
#pragma unroll
    for (int u = 0; u < NP; ++u) d[u] = TW::make(t[2 * u], t[2 * u + 1]);
  };

  P q[Q][VY][NP];
  // initial queue: planes z0-R .. z0+R-1.  The first R of them (before z0) serve
  // only the queue, so each is released as soon as it is read and its slot is
  // refilled at once.
  {
    Pos ps{0, 0};
#pragma unroll
    for (int j = 0; j < 2 * R; ++j) {
      const int p = pbase + j;
      wait(su32(&full[ps.s]), ps.r & 1);
      const T* row = ring + (size_t)ps.s * slot_elems;
#pragma unroll
      for (int r = 0; r < VY; ++r) load_pairs(q[j][r], row + (R + yy + r) * rowe + x);
      if (j < R) {
        __syncwarp();
        if ((tid & 31) == 0) release(p, ps);
        __syncwarp();
      }
      advance(ps);
    }
  }

  T* __restrict__ yn = a.y + (int64_t)n * a.ldy;
  const T* __restrict__ pn = a.prev ? a.prev + (int64_t)n * a.ldp : nullptr;
  const int gy0 = y0 + yy;
  bool rowok[VY];
#pragma unroll
  for (int r = 0; r < VY; ++r) rowok[r] = gy0 + r < a.ny;

  // slot/round of the next plane to push (z + R) and of the next plane to compute (z)
  Pos push{(2 * R) % S, (2 * R) / S};
  Pos cur{R % S, R / S};
  for (int z = z0; z < z1; z += U) {
    if (__shfl_sync(full_mask, *abort, 0)) break;
    const int nu = min(U, z1 - z);
    // push planes z + R .. z + R + nu - 1 into the queue
    bool got = true;
#pragma unroll
    for (int t = 0; t < U; ++t) {
      if (t < nu) {
        got = got && wait(su32(&full[push.s]), push.r & 1);
        const T* row = ring + (size_t)push.s * slot_elems;
#pragma unroll
        for (int r = 0; r < VY; ++r) load_pairs(q[2 * R + t][r], row + (R + yy + r) * rowe + x);
        advance(push);
      }
    }
    if (!__all_sync(full_mask, got)) break;
#pragma unroll
    for (int t = 0; t < U; ++t) {
      if (t >= nu) break;
      const int zz = z + t;
      // Veff and prev of this plane, used after the neighbour sums
      const int64_t g0 = zz * nxy + (int64_t)gy0 * a.nx + x;
      P vc[VY][NP], pc[VY][NP];
#pragma unroll
      for (int r = 0; r < VY; ++r) {
        T tv[VX], tp[VX];
#pragma unroll
        for (int v = 0; v < VX; ++v) tv[v] = tp[v] = T(0);
        if (rowok[r]) {
          ldg<T, VX>(tv, a.veff + g0 + r * a.nx);
          if (pn) ldg<T, VX>(tp, pn + g0 + r * a.nx);
        }
#pragma unroll
        for (int w = 0; w < NP; ++w) {
          vc[r][w] = TW::make(tv[2 * w], tv[2 * w + 1]);
          pc[r][w] = TW::make(tp[2 * w], tp[2 * w + 1]);
        }
      }
      const T* pl = ring + (size_t)cur.s * slot_elems;
      // even and odd neighbour distances accumulate separately (two independent
      // dependency chains)
      P acc[VY][NP], acc1[VY][NP];
#pragma unroll
      for (int r = 0; r < VY; ++r) {
        const T* rowp = pl + (R + yy + r) * rowe;
        T b[NC * VX];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          T tt[VX];
          lds<T, VX>(tt, rowp + coff[c]);
          if (XDIR && !((cvalid >> c) & 1u)) {
#pragma unroll
            for (int v = 0; v < VX; ++v) tt[v] = T(0);
          }
#pragma unroll
          for (int v = 0; v < VX; ++v) b[c * VX + v] = tt[v];
        }
#pragma unroll
        for (int u = 0; u < NP; ++u) {
          acc[r][u] = TW::mul(a.dms2, q[R + t][r][u]);
          acc1[r][u] = TW::zero();
        }
#pragma unroll
        for (int p = 1; p <= R; ++p) {
          P up[NP], dn[NP];
          load_pairs(up, pl + (R + yy + r + p) * rowe + x);
          load_pairs(dn, pl + (R + yy + r - p) * rowe + x);
#pragma unroll
          for (int u = 0; u < NP; ++u) {
            const int o = WL + 2 * u;
            P xs;
            if (p & 1)  // b[o + p] starts a pair only for even p
              xs = TW::make(b[o + p] + b[o - p], b[o + 1 + p] + b[o + 1 - p]);
            else
              xs = TW::add(TW::make(b[o + p], b[o + 1 + p]), TW::make(b[o - p], b[o + 1 - p]));
            const P ys = TW::add(up[u], dn[u]);
            const P zs = TW::add(q[R + t + p][r][u], q[R + t - p][r][u]);
            const P sum = TW::add(TW::add(ys, zs), xs);
            if (p & 1)
              acc1[r][u] = TW::fma(a.off2[p], sum, acc1[r][u]);
            else
              acc[r][u] = TW::fma(a.off2[p], sum, acc[r][u]);
          }
        }
      }
      // release the slot of plane zz (the last warp refills it)
      __syncwarp();
      if ((tid & 31) == 0) release(zz, cur);
      __syncwarp();
      advance(cur);
      // Veff, recurrence and store
#pragma unroll
      for (int r = 0; r < VY; ++r) {
        if (!rowok[r]) continue;
        T out[VX];
#pragma unroll
        for (int u = 0; u < NP; ++u) {
          const P h = TW::fma(vc[r][u], q[R + t][r][u], TW::add(acc[r][u], acc1[r][u]));
          const P o2 = pn ? TW::fma(a.sh2, h, TW::mul(a.sp2, pc[r][u])) : TW::mul(a.sh2, h);
          out[2 * u] = o2.x;
          out[2 * u + 1] = o2.y;
        }
        stg<T, VX>(yn + g0 + r * a.nx, out);
      }
    }
#pragma unroll
    for (int j = 0; j < 2 * R; ++j)
#pragma unroll
      for (int r = 0; r < VY; ++r)
#pragma unroll
        for (int u = 0; u < NP; ++u) q[j][r][u] = q[j + U][r][u];
  }
  // drain: every issued load must have landed before the CTA exits
  __syncthreads();
  if (tid == 0) {
    const int hi = issued_hi;
    for (int p = max(pbase, hi - S); p < hi; ++p) {
      const int k = p - pbase;
      const long long t0 = clock64();
      while (!bar_test(su32(&full[k % S]), (k / S) & 1) &&
             clock64() - t0 < max(wmax, kDrainCycles)) {
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

// Plan of the double-FP32 ring kernel (stencil_df.cu: two rows per thread, the
// nonlocal coefficients D staged in shared memory), or false if the generic
// kernel must be used.
template <typename T>
bool ring_plan(const Grid& g, int kp, int& by, int& slots, uint32_t& slot_bytes, int& threads) {
  constexpr int VX = sizeof(T) == 4 ? 4 : 2;
  const int es = sizeof(T);
  if (g.nx % (sizeof(T) == 4 ? 16 : 8) != 0 || g.nx > 256) return false;
  const int cands[3] = {sizeof(T) == 4 ? 32 : 16, 16, 8};
  by = 0;
  for (int c : cands) {
    if (g.ny % c == 0 || (g.bc[1] == SPARC_DIRICHLET && c <= g.ny)) {
      if ((c / 2) * (g.nx / VX) <= 384) {
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
  threads = (by / 2) * (g.nx / VX);
  return threads >= 32 && threads % 32 == 0;
}

// Plan of the local ring kernel for a grid, element type and thread shape
// (vy rows per thread, at most maxt threads): slab rows, ring slots, slot bytes
// and threads, or false when the grid does not fit the ring form.
template <typename T>
bool local_ring_plan(const Grid& g, int vy, int maxt, int& by, int& slots,
                     uint32_t& slot_bytes, int& threads) {
  constexpr int VX = sizeof(T) == 4 ? 4 : 2;
  const int es = sizeof(T);
  if (g.nx % (sizeof(T) == 4 ? 16 : 8) != 0 || g.nx > 256) return false;
  const int cands[7] = {64, 48, 32, 24, 16, 12, 8};
  by = 0;
  for (int c : cands) {
    if (c % vy) continue;
    if (g.ny % c == 0 || (g.bc[1] == SPARC_DIRICHLET && c <= g.ny)) {
      const int th = (c / vy) * (g.nx / VX);
      const uint32_t sb = ((uint32_t)((c + 2 * R) * g.nx * es) + 127u) & ~127u;
      if (th <= maxt && th % 32 == 0 && (200 * 1024) / sb >= 8) {
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
  slots = std::min<int>(16, (int)((200 * 1024) / slot_bytes));
  if (slots < 8) return false;  // the march needs plane z + R resident S - 7 planes ahead
  threads = (by / vy) * (g.nx / VX);
  return threads >= 32 && threads % 32 == 0;
}

// Thread shapes of the local ring kernel: rows per thread, planes per step and
// the CTA's thread limit (which bounds the registers per thread).  Every shape
// computes each point with the same operations in the same order, so the
// results do not depend on the shape; the fastest one is picked by timing
// (ring_tune).
struct RingShapeDef {
  int vy, u, maxt;
};
constexpr RingShapeDef kShapesF32[] = {{1, 4, 384}, {1, 1, 576}, {1, 2, 512}};
constexpr RingShapeDef kShapesF64[] = {{1, 2, 384}, {1, 1, 576}};
template <typename T>
constexpr int num_shapes() {
  return sizeof(T) == 4 ? (int)(sizeof(kShapesF32) / sizeof(RingShapeDef))
                        : (int)(sizeof(kShapesF64) / sizeof(RingShapeDef));
}
template <typename T>
constexpr RingShapeDef shape_def(int i) {
  return sizeof(T) == 4 ? kShapesF32[i] : kShapesF64[i];
}

template <typename T, int VX, int VY, int U, int MAXT>
cudaError_t launch_ring(bool xdir, dim3 grid, int threads, size_t smem, cudaStream_t st,
                        const CUtensorMap& mmid, const CUtensorMap& mhalo, const RingArgs<T>& a) {
  static unsigned long long bits[2] = {0, 0};
  const void* fn = xdir ? (const void*)k_apply_h_ring<T, VX, VY, U, MAXT, true>
                        : (const void*)k_apply_h_ring<T, VX, VY, U, MAXT, false>;
  cudaError_t ae = smem_limit_once(&bits[xdir ? 1 : 0], fn, 210 * 1024);
  if (ae != cudaSuccess) return ae;
  note_launch();
  if (xdir)
    k_apply_h_ring<T, VX, VY, U, MAXT, true><<<grid, threads, smem, st>>>(mmid, mhalo, a);
  else
    k_apply_h_ring<T, VX, VY, U, MAXT, false><<<grid, threads, smem, st>>>(mmid, mhalo, a);
  return cudaGetLastError();
}

template <typename T>
int ring_num_shapes() {
  return num_shapes<T>();
}

template <typename T>
bool ring_shape_info(const Grid& g, int shape, int* vy, int* u, int* by, int* threads) {
  if (shape < 0 || shape >= num_shapes<T>()) return false;
  const RingShapeDef d = shape_def<T>(shape);
  int slots;
  uint32_t sb;
  if (!local_ring_plan<T>(g, d.vy, d.maxt, *by, slots, sb, *threads)) return false;
  *vy = d.vy;
  *u = d.u;
  return true;
}

template <typename T>
bool ring_applicable(const Grid& g, const T* x, int64_t ldx, const T* y, int64_t ldy,
                     const T* prev, int64_t ldp, const T* veff) {
  bool any = false;
  for (int s = 0; s < num_shapes<T>() && !any; ++s) {
    const RingShapeDef d = shape_def<T>(s);
    int by, slots, th;
    uint32_t sb;
    any = local_ring_plan<T>(g, d.vy, d.maxt, by, slots, sb, th);
  }
  const int va = 16 / sizeof(T);
  if (!any || !encoder() || ldx % va || ldy % va || (prev && ldp % va) || ((uintptr_t)x % 16) ||
      ((uintptr_t)y % 16) || (prev && ((uintptr_t)prev % 16)) || ((uintptr_t)veff % 16))
    return false;
  return true;
}

template <typename T>
cudaError_t apply_h_ring(const Grid& g, const LapCoef& lc, const T* veff, const T* x, int64_t ldx,
                         T* y, int64_t ldy, const T* prev, int64_t ldp, int ns, double shift,
                         double s_h, double s_p, long long wait_cycles, int* status,
                         cudaStream_t st, int shape, bool stall, bool* used) {
  *used = false;
  constexpr int VX = sizeof(T) == 4 ? 4 : 2;
  if (shape < 0 || shape >= num_shapes<T>()) shape = 0;
  const RingShapeDef d = shape_def<T>(shape);
  int by, slots, threads;
  uint32_t slot_bytes;
  if (!local_ring_plan<T>(g, d.vy, d.maxt, by, slots, slot_bytes, threads)) return cudaSuccess;
  const int va = 16 / sizeof(T);
  if (ldx % va || ldy % va || (prev && ldp % va) || ((uintptr_t)x % 16) || ((uintptr_t)y % 16) ||
      (prev && ((uintptr_t)prev % 16)) || ((uintptr_t)veff % 16))
    return cudaSuccess;
  CUtensorMap mmid, mhalo;
  if (!block_map<T>(&mmid, x, ldx, g, ns, by) || !block_map<T>(&mhalo, x, ldx, g, ns, R))
    return cudaSuccess;
  RingArgs<T> a;
  a.y = y; a.ldy = ldy; a.prev = prev; a.ldp = ldp; a.veff = veff;
  a.nx = g.nx; a.ny = g.ny; a.nz = g.nz; a.bcx = g.bc[0]; a.bcy = g.bc[1]; a.bcz = g.bc[2];
  a.by = by;
  a.nslab = (g.ny + by - 1) / by;
  a.slots = slots;
  a.slot_bytes = slot_bytes;
  const T dms = T(lc.diag - shift);
  a.dms2 = {dms, dms};
  for (int p = 0; p <= R; ++p) a.off2[p] = {T(lc.off[p]), T(lc.off[p])};
  a.sh2 = {T(s_h), T(s_h)};
  a.sp2 = {T(s_p), T(s_p)};
  a.wait_cycles = wait_cycles;
  a.status = status;
  a.stall = stall ? 1 : 0;
  // z split: enough CTAs to cover the SMs a few times
  const int64_t xy = (int64_t)a.nslab * ns;
  int nzc = (int)std::max<int64_t>(1, (2 * sm_count() + xy - 1) / xy);
  nzc = std::min(nzc, std::max(1, g.nz / 16));
  a.bz = (g.nz + nzc - 1) / nzc;
  nzc = (g.nz + a.bz - 1) / a.bz;
  const size_t smem = (size_t)slots * slot_bytes + 128;
  const dim3 grid((unsigned)(a.nslab * ns), (unsigned)nzc);
  const bool xd = g.bc[0] == SPARC_DIRICHLET;
  cudaError_t e = cudaSuccess;
  if constexpr (sizeof(T) == 4) {
    switch (shape) {
      case 0: e = launch_ring<T, VX, 1, 4, 384>(xd, grid, threads, smem, st, mmid, mhalo, a); break;
      case 1: e = launch_ring<T, VX, 1, 1, 576>(xd, grid, threads, smem, st, mmid, mhalo, a); break;
      default: e = launch_ring<T, VX, 1, 2, 512>(xd, grid, threads, smem, st, mmid, mhalo, a); break;
    }
  } else {
    switch (shape) {
      case 0: e = launch_ring<T, VX, 1, 2, 384>(xd, grid, threads, smem, st, mmid, mhalo, a); break;
      default: e = launch_ring<T, VX, 1, 1, 576>(xd, grid, threads, smem, st, mmid, mhalo, a); break;
    }
  }
  if (e == cudaSuccess) *used = true;
  return e;
}

template bool ring_plan<float>(const Grid&, int, int&, int&, uint32_t&, int&);
template bool ring_plan<double>(const Grid&, int, int&, int&, uint32_t&, int&);
template cudaError_t apply_h_ring<float>(const Grid&, const LapCoef&, const float*, const float*,
                                         int64_t, float*, int64_t, const float*, int64_t, int,
                                         double, double, double, long long, int*, cudaStream_t,
                                         int, bool, bool*);
template cudaError_t apply_h_ring<double>(const Grid&, const LapCoef&, const double*,
                                          const double*, int64_t, double*, int64_t, const double*,
                                          int64_t, int, double, double, double, long long, int*,
                                          cudaStream_t, int, bool, bool*);
template bool ring_applicable<float>(const Grid&, const float*, int64_t, const float*, int64_t,
                                     const float*, int64_t, const float*);
template bool ring_applicable<double>(const Grid&, const double*, int64_t, const double*, int64_t,
                                      const double*, int64_t, const double*);
template int ring_num_shapes<float>();
template int ring_num_shapes<double>();
template bool ring_shape_info<float>(const Grid&, int, int*, int*, int*, int*);
template bool ring_shape_info<double>(const Grid&, int, int*, int*, int*, int*);

}  // namespace sparc
