// FP64 Hamiltonian application (paper Sec. II A) in double-FP32 arithmetic:
// the TMA plane-ring kernel of stencil_tma.cu for FP64 orbital blocks, with
// every sum and product carried as an unevaluated pair hi + lo of FP32 numbers
// (48-bit significand) on the FP32 pipe.  GB300 runs FP64 at 1/64 of the FP32
// rate, so the FP64 stencil (≈ 42 FP64 instructions per point) is bound by its
// FP64 pipe; in pair arithmetic the same point costs ≈ 400 FP32 instructions.  Errors: each pair operation is accurate to ≈ 2^-48
// of its operands, so H x agrees with FP64 arithmetic to ≈ 1e-13 relative
// (FP64's own rounding, amplified by the stencil's cancellation, is ≈ 3e-14).
//
// FP64 inputs become pairs with integer operations only (no FP64 pipe): each
// ring slot is converted in place once, when its plane is first used, and
// the previous recurrence term per point as it is loaded.  The result is
// written as FP64 (one FP64 add per point).  Veff and the grouped projector
// values come as pair tables made at handle creation; the CTA's nonlocal
// coefficients D are converted when they are staged in shared memory.
//
// The pair operations are the published error-free transformations: the sum
// of two numbers as TwoSum (Knuth, TAOCP vol. 2, Sec. 4.2.2) or FastTwoSum
// when the order of magnitudes is known (Dekker 1971), the product as an exact
// TwoProduct by one FMA for the rounding error, followed by the usual
// renormalisation of hi + lo.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "internal.cuh"

namespace sparc {

namespace {

constexpr int R = kRadius;
constexpr int VX = 2;  // points per thread along x (one 16-byte load of two pairs)
constexpr int VY = 2;  // rows per thread

struct df {
  float h, l;
};

// error-free transformations (no contraction: explicit round-to-nearest ops)
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df add(df a, df b) {
  const df s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ df mul(df a, df b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ df fma(df a, df b, df c) { return add(mul(a, b), c); }

// Unnormalised accumulator: the high parts are summed error-free (TwoSum), the
// low parts and the rounding errors in a plain FP32 word, which is 2^-24 below
// and needs no more than FP32 accuracy.  Equivalent in accuracy to a chain of
// pair additions at about 2/3 of the cost.
struct acc_t {
  float h, l;
};
__device__ __forceinline__ void acc_add(acc_t& a, df v) {
  const df s = two_sum(a.h, v.h);
  a.h = s.h;
  a.l = __fadd_rn(a.l, __fadd_rn(s.l, v.l));
}
// a += w * v (w, v pairs): the product's high part exactly (FMA), its cross
// terms into the low word
__device__ __forceinline__ void acc_fma(acc_t& a, df w, acc_t v) {
  const float p = __fmul_rn(w.h, v.h);
  float e = __fmaf_rn(w.h, v.h, -p);
  e = __fmaf_rn(w.h, v.l, e);
  e = __fmaf_rn(w.l, v.h, e);
  const df s = two_sum(a.h, p);
  a.h = s.h;
  a.l = __fadd_rn(a.l, __fadd_rn(s.l, e));
}
__device__ __forceinline__ df normalise(acc_t a) { return fast_two_sum(a.h, a.l); }

// 2^n as a float for -126 <= n <= 127
__device__ __forceinline__ float pow2f(int n) { return __int_as_float((n + 127) << 23); }

// FP64 -> pair with integer operations: h = x rounded to nearest FP32, l the
// rounded remainder (|x - h - l| <= 2^-48 |x|).  Magnitudes outside
// [2^-100, 2^100] (and zero, inf, nan) take the FP64 conversions instead.
__device__ __forceinline__ df d2df(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7FF);
  if (e < 1023 - 100 || e > 1023 + 100) {
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
  }
  const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);  // 53-bit significand
  unsigned int hm = (unsigned int)(m >> 29);                              // leading 24 bits
  const unsigned int r = (unsigned int)(m & 0x1FFFFFFFull);               // trailing 29 bits
  if (r > 0x10000000u || (r == 0x10000000u && (hm & 1u))) ++hm;           // round to nearest even
  const int rem = (int)((long long)m - ((long long)hm << 29));            // |rem| <= 2^28
  int eh = e;
  if (hm == (1u << 24)) {  // rounding carried into a new binade
    hm >>= 1;
    ++eh;
  }
  const unsigned int sign = (unsigned int)(u >> 32) & 0x80000000u;
  const float h = __uint_as_float(sign | ((unsigned int)(eh - 1023 + 127) << 23) | (hm & 0x7FFFFFu));
  // float(rem) without an int-to-float instruction (an FP64-pipe operation on
  // GB300): rem = hi 2^14 + lo, each half exact through the 1.5 * 2^23 offset,
  // recombined with one rounding
  const int rh = rem >> 14, rl = rem & 0x3FFF;
  const float fh = __fsub_rn(__int_as_float(0x4B400000 + rh), 12582912.0f);
  const float fl = __fsub_rn(__int_as_float(0x4B400000 + rl), 12582912.0f);
  const float frem = __fmaf_rn(fh, 16384.0f, fl);
  float l = __fmul_rn(__fmul_rn(frem, 0x1p-29f), pow2f(e - 1046));
  if (sign) l = -l;
  return {h, l};
}

// exact FP32 -> FP64 by moving the IEEE-754 fields (no FP64 conversion)
__device__ __forceinline__ double widen(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFFu;
  if (e == 0u || e == 0xFFu) return (double)f;
  const uint64_t d = ((uint64_t)(u & 0x80000000u) << 32) | ((uint64_t)(e + 896u) << 52) |
                     ((uint64_t)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)d);
}

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
// Bounded wait: false on its own timeout (recorded) or once any CTA of the
// launch has recorded a status.
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

// two consecutive pairs from shared memory (one 16-byte load)
__device__ __forceinline__ void lds2(df (&d)[VX], const df* p) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  d[0] = {v.x, v.y};
  d[1] = {v.z, v.w};
}

struct RingArgsDF {
  double* y;
  int64_t ldy;
  const double* prev;
  int64_t ldp;
  const float2* veff;      // Veff as pairs
  const int* grp_ptr;      // grouped nonlocal slots, two points per group
  const int* grp_k;
  const float2* grp_chi;   // chi as pairs
  const double* D;
  int kp;
  uint32_t d_off;          // byte offset of the orbital's D pairs in dynamic shared memory
  int nx, ny, nz, bcx, bcy, bcz;
  int by, nslab, bz, slots;
  uint32_t slot_bytes;
  df diag_minus_shift;
  df off[R + 1];
  df s_h, s_p;
  int* status;
  long long wait;  // bound of every mbarrier wait (SM clock cycles)
};

__global__ void __launch_bounds__(384, 1)
    k_apply_h_ring_df(const __grid_constant__ CUtensorMap mid,
                      const __grid_constant__ CUtensorMap halo, const RingArgsDF a) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full[16], empty[16];
  __shared__ int issued_hi;  // one past the last issued plane

  const int nwarps = (blockDim.x + 31) >> 5;
  const int qpr = a.nx / VX;
  const int tid = threadIdx.x;
  const int ry = tid / qpr, qx = tid % qpr;
  const int x = qx * VX;
  const int yy = ry * VY;
  const int n = blockIdx.x / a.nslab;
  const int slab = blockIdx.x % a.nslab;
  const int y0 = slab * a.by;
  const int z0 = blockIdx.y * a.bz;
  const int z1 = min(z0 + a.bz, a.nz);
  const int pbase = z0 - R;
  const int S = a.slots;
  const int rowe = a.nx;  // pairs (8 bytes) per shared row
  const uint32_t base = (su32(smem_raw) + 127u) & ~127u;
  uint8_t* const ring_b = smem_raw + (base - su32(smem_raw));
  const int64_t nxy = (int64_t)a.nx * a.ny;
  const int slab_rows = a.by + 2 * R;
  const int slot_elems = slab_rows * rowe;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&full[s])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&empty[s])), "r"(nwarps));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    issued_hi = z0 - R;
  }
  // this CTA's orbital column of the nonlocal coefficients, as pairs
  df* const dsh = reinterpret_cast<df*>(ring_b + a.d_off);
  for (int k = tid; k < a.kp; k += blockDim.x) dsh[k] = d2df(__ldg(a.D + (int64_t)n * a.kp + k));
  __syncthreads();

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
                 "r"((uint32_t)(slot_elems * 8))
                 : "memory");
    int yt = y0 - R, yb = y0 + a.by;
    if (a.bcy == SPARC_PERIODIC) {
      if (yt < 0) yt += a.ny;
      if (yb >= a.ny) yb -= a.ny;
    }
    const uint32_t rb = (uint32_t)(rowe * 8);
    tma4(dst, &halo, 0, yt, zc, n, fb);
    tma4(dst + R * rb, &mid, 0, y0, zc, n, fb);
    tma4(dst + (R + a.by) * rb, &halo, 0, yb, zc, n, fb);
    issued_hi = p + 1;
  };
  auto slot_of = [&](int p) { return (p - pbase) % S; };
  auto round_of = [&](int p) { return (uint32_t)((p - pbase) / S); };
  auto slot_ptr = [&](int s) { return reinterpret_cast<df*>(ring_b + (size_t)s * a.slot_bytes); };
  // Wait for plane p (every thread), convert its slot to pairs in place and
  // make that visible to the CTA.  Returns false, uniformly, if any thread's
  // wait gave up.
  auto arrive_convert = [&](int p) {
    const int s = slot_of(p);
    const bool got = bar_wait(su32(&full[s]), round_of(p) & 1, a.status, a.wait);
    if (got) {
      df* sl = slot_ptr(s);
      const double* sd = reinterpret_cast<const double*>(sl);
      for (int i = tid; i < slot_elems; i += blockDim.x) {
        const df v = d2df(sd[i]);
        sl[i] = v;
      }
      // the slot goes back to the TMA (async proxy) after these generic writes
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    return __syncthreads_or(!got) == 0;
  };
  auto release = [&](int p) {  // every warp is done with plane p's slot
    const int s = slot_of(p);
    __syncwarp();
    if ((tid & 31) == 0)
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&empty[s])) : "memory");
    if (tid == 0 && p + S < z1 + R)
      if (bar_wait(su32(&empty[s]), round_of(p) & 1, a.status, a.wait)) issue(p + S);
    __syncwarp();
  };

  const int plast = z1 + R;
  if (tid == 0)
    for (int p = pbase; p < min(plast, pbase + S); ++p) issue(p);

  df q[2 * R + 1][VY][VX];
  bool ok = true;
  // initial queue: planes z0-R .. z0+R-1; those before z0 serve only the queue
#pragma unroll
  for (int j = 0; j < 2 * R; ++j) {
    const int p = pbase + j;
    if (ok) ok = arrive_convert(p);
    if (ok) {
      const df* row = slot_ptr(slot_of(p));
#pragma unroll
      for (int r = 0; r < VY; ++r) lds2(q[j][r], row + (R + yy + r) * rowe + x);
      if (j < R) release(p);
    }
  }

  double* __restrict__ yn = a.y + (int64_t)n * a.ldy;
  const double* __restrict__ pn = a.prev ? a.prev + (int64_t)n * a.ldp : nullptr;
  const int gy0 = y0 + yy;

  for (int z = z0; ok && z < z1; ++z) {
    const int64_t g0 = z * nxy + (int64_t)gy0 * a.nx + x;
    // plane z + R: wait, convert, push into the queue
    if (!arrive_convert(z + R)) break;
    {
      const df* row = slot_ptr(slot_of(z + R));
#pragma unroll
      for (int r = 0; r < VY; ++r) lds2(q[2 * R][r], row + (R + yy + r) * rowe + x);
    }
    const df* pl = slot_ptr(slot_of(z));
    acc_t acc[VY][VX];
#pragma unroll
    for (int r = 0; r < VY; ++r)
#pragma unroll
      for (int v = 0; v < VX; ++v) {
        const df c = mul(a.diag_minus_shift, q[R][r][v]);
        acc[r][v] = {c.h, c.l};
      }
    // per row and distance: y and z neighbours from the slot and the queue,
    // x neighbours read singly (periodic wrap or zero ghosts)
#pragma unroll
    for (int r = 0; r < VY; ++r) {
      const df* rowp = pl + (R + yy + r) * rowe;
#pragma unroll
      for (int p = 1; p <= R; ++p) {
        df up[VX], dn[VX];
        lds2(up, pl + (R + yy + r + p) * rowe + x);
        lds2(dn, pl + (R + yy + r - p) * rowe + x);
#pragma unroll
        for (int v = 0; v < VX; ++v) {
          int xl = x + v - p, xr = x + v + p;
          bool il = true, ir = true;
          if (xl < 0) {
            if (a.bcx == SPARC_DIRICHLET) il = false;
            else xl += a.nx;
          }
          if (xr >= a.nx) {
            if (a.bcx == SPARC_DIRICHLET) ir = false;
            else xr -= a.nx;
          }
          acc_t sm = {up[v].h, up[v].l};
          acc_add(sm, dn[v]);
          acc_add(sm, q[R + p][r][v]);
          acc_add(sm, q[R - p][r][v]);
          acc_add(sm, il ? rowp[xl] : df{0.f, 0.f});
          acc_add(sm, ir ? rowp[xr] : df{0.f, 0.f});
          acc_fma(acc[r][v], a.off[p], sm);
        }
      }
    }
    release(z);
    // Veff, prev and the nonlocal slot range of this plane (loaded after the
    // stencil sums: the registers go to the queue and the neighbour sums)
    float4 vf4[VY];
    double2 pv2[VY];
    int gs[VY], ge[VY];
#pragma unroll
    for (int r = 0; r < VY; ++r) {
      gs[r] = ge[r] = 0;
      if (gy0 + r < a.ny) {
        vf4[r] = __ldg(reinterpret_cast<const float4*>(a.veff + g0 + r * a.nx));
        if (pn) pv2[r] = __ldg(reinterpret_cast<const double2*>(pn + g0 + r * a.nx));
        if (a.kp > 0) {
          const int64_t qg = (g0 + r * a.nx) / VX;
          gs[r] = __ldg(a.grp_ptr + qg);
          ge[r] = __ldg(a.grp_ptr + qg + 1);
        }
      }
    }
    // Veff, nonlocal pull-add, recurrence, store as FP64
#pragma unroll
    for (int r = 0; r < VY; ++r) {
      if (gy0 + r >= a.ny) continue;
      df h[VX];
      const df vf[VX] = {{vf4[r].x, vf4[r].y}, {vf4[r].z, vf4[r].w}};
#pragma unroll
      for (int v = 0; v < VX; ++v) h[v] = fma(vf[v], q[R][r][v], normalise(acc[r][v]));
      // up to four slots' loads in flight before their products
      for (int sl = gs[r]; sl < ge[r]; sl += 4) {
        int2 kk[4];
        float4 c4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (sl + u < ge[r]) {
            kk[u] = __ldg(reinterpret_cast<const int2*>(a.grp_k + (int64_t)(sl + u) * VX));
            c4[u] = __ldg(reinterpret_cast<const float4*>(a.grp_chi + (int64_t)(sl + u) * VX));
          } else {
            kk[u] = make_int2(0, 0);
            c4[u] = make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          h[0] = fma(df{c4[u].x, c4[u].y}, dsh[kk[u].x], h[0]);
          h[1] = fma(df{c4[u].z, c4[u].w}, dsh[kk[u].y], h[1]);
        }
      }
      double out[VX];
#pragma unroll
      for (int v = 0; v < VX; ++v) {
        df o = mul(a.s_h, h[v]);
        if (pn) o = fma(a.s_p, d2df(v == 0 ? pv2[r].x : pv2[r].y), o);
        out[v] = __dadd_rn(widen(o.h), widen(o.l));
      }
      *reinterpret_cast<double2*>(yn + g0 + r * a.nx) = make_double2(out[0], out[1]);
    }
#pragma unroll
    for (int j = 0; j < 2 * R; ++j)
#pragma unroll
      for (int r = 0; r < VY; ++r)
#pragma unroll
        for (int v = 0; v < VX; ++v) q[j][r][v] = q[j + 1][r][v];
  }
  // drain: every issued load must have landed before the CTA exits
  __syncthreads();
  if (tid == 0) {
    const int hi = issued_hi;
    for (int p = max(pbase, hi - S); p < hi; ++p) {
      const long long t0 = clock64();
      while (!bar_test(su32(&full[slot_of(p)]), round_of(p) & 1) &&
             clock64() - t0 < max(a.wait, kDrainCycles)) {
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

bool block_map(CUtensorMap* m, const double* x, int64_t ldx, const Grid& g, int ns, int rows) {
  auto enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)ns};
  cuuint64_t strides[3] = {(cuuint64_t)g.nx * 8, (cuuint64_t)g.nx * g.ny * 8,
                           (cuuint64_t)ldx * 8};
  cuuint32_t box[4] = {(cuuint32_t)g.nx, (cuuint32_t)rows, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, const_cast<double*>(x), dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

df host_df(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}

}  // namespace

cudaError_t apply_h_ring_df(const Grid& g, const LapCoef& lc, const float2* veff_df,
                            const Nonlocal<double>& nl, const double* D, const double* x,
                            int64_t ldx, double* y, int64_t ldy, const double* prev, int64_t ldp,
                            int ns, double shift, double s_h, double s_p, int* status,
                            cudaStream_t st, bool* used) {
  *used = false;
  int by, slots, threads;
  uint32_t slot_bytes;
  if (!ring_plan<double>(g, nl.kp, by, slots, slot_bytes, threads)) return cudaSuccess;
  if (nl.kp > 0 && (!nl.grp_ptr || nl.grp != VX || !nl.grp_chi_df)) return cudaSuccess;
  if (!veff_df) return cudaSuccess;
  if (ldx % 2 || ldy % 2 || (prev && ldp % 2) || ((uintptr_t)x % 16) || ((uintptr_t)y % 16) ||
      (prev && ((uintptr_t)prev % 16)) || ((uintptr_t)veff_df % 16))
    return cudaSuccess;
  CUtensorMap mmid, mhalo;
  if (!block_map(&mmid, x, ldx, g, ns, by) || !block_map(&mhalo, x, ldx, g, ns, R))
    return cudaSuccess;
  RingArgsDF a;
  a.y = y; a.ldy = ldy; a.prev = prev; a.ldp = ldp; a.veff = veff_df;
  a.grp_ptr = nl.grp_ptr; a.grp_k = nl.grp_k; a.grp_chi = nl.grp_chi_df; a.D = D; a.kp = nl.kp;
  a.nx = g.nx; a.ny = g.ny; a.nz = g.nz; a.bcx = g.bc[0]; a.bcy = g.bc[1]; a.bcz = g.bc[2];
  a.by = by;
  a.nslab = (g.ny + by - 1) / by;
  a.slots = slots;
  a.slot_bytes = slot_bytes;
  a.diag_minus_shift = host_df(lc.diag - shift);
  for (int p = 0; p <= R; ++p) a.off[p] = host_df(lc.off[p]);
  a.s_h = host_df(s_h);
  a.s_p = host_df(s_p);
  a.status = status;
  a.wait = wait_cycles();
  const int64_t xy = (int64_t)a.nslab * ns;
  int nzc = (int)std::max<int64_t>(1, (2 * sm_count() + xy - 1) / xy);
  nzc = std::min(nzc, std::max(1, g.nz / 16));
  a.bz = (g.nz + nzc - 1) / nzc;
  nzc = (g.nz + a.bz - 1) / a.bz;
  a.d_off = (uint32_t)slots * slot_bytes;
  const size_t smem = (size_t)slots * slot_bytes + (size_t)nl.kp * 8 + 128;
  static unsigned long long attr_bits = 0;
  cudaError_t ae = smem_limit_once(&attr_bits, (const void*)k_apply_h_ring_df, 210 * 1024);
  if (ae != cudaSuccess) return ae;
  dim3 grid((unsigned)(a.nslab * ns), (unsigned)nzc);
  note_launch(), k_apply_h_ring_df<<<grid, threads, smem, st>>>(mmid, mhalo, a);
  *used = true;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Generic local stencil in double-FP32 arithmetic, by y-slabs of whole rows,
// for FP64 blocks on grids the ring does not fit (any nx >= R): the slab
// structure of stencil.cu's k_apply_h_slab (register z queue, own rows and the
// halo rows in shared memory with repeated ghost columns) with the per-point
// operation order of k_apply_h_ring_df (neighbour sums in the error-free
// accumulator, coefficient products by acc_fma, Veff, then the recurrence);
// the nonlocal term follows with the tiled pass.
// ---------------------------------------------------------------------------
namespace {

constexpr int kSlabDfThreads = 256;
constexpr int kSlabDfPpt = 2;  // points per thread

struct SlabArgsDF {
  const double* x;
  int64_t ldx;
  double* y;
  int64_t ldy;
  const double* prev;
  int64_t ldp;
  const float2* veff;  // Veff as pairs
  int nx, ny, nz, bcx, bcy, bcz;
  int by, bz;
  df dms;  // diagonal - shift
  df off[R + 1];
  df s_h, s_p;
};

__global__ void __launch_bounds__(kSlabDfThreads, 2) k_apply_h_slab_df(const SlabArgsDF a) {
  constexpr int PPT = kSlabDfPpt;
  extern __shared__ __align__(16) uint8_t slabdf_raw[];
  df* const s = reinterpret_cast<df*>(slabdf_raw);
  const int W = a.nx + 2 * R;
  const int n = blockIdx.y;
  const int y0 = blockIdx.x * a.by;
  const int byl = min(a.by, a.ny - y0);
  const int npts = byl * a.nx;
  const int z0 = blockIdx.z * a.bz, z1 = min(z0 + a.bz, a.nz);
  const int64_t nxy = (int64_t)a.nx * a.ny;
  const double* __restrict__ xn = a.x + (int64_t)n * a.ldx;
  const bool perx = a.bcx == SPARC_PERIODIC;
  for (int e = threadIdx.x; e < (a.by + 2 * R) * W; e += blockDim.x) s[e] = df{0.f, 0.f};

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
      if (perx && rx < R) dup_r |= 1u << k;
      if (perx && rx >= a.nx - R) dup_l |= 1u << k;
    }
  }
  auto wrap = [](int& c, int nn, int bc) {
    if (c >= 0 && c < nn) return true;
    if (bc == SPARC_DIRICHLET) return false;
    c %= nn;
    if (c < 0) c += nn;
    return true;
  };
  df q[2 * R + 1][PPT];
  auto load_q = [&](int zz, df(&d)[PPT]) {
    const bool ok = wrap(zz, a.nz, a.bcz);
    const double* __restrict__ pl = xn + (int64_t)zz * nxy;
#pragma unroll
    for (int k = 0; k < PPT; ++k)
      d[k] = (ok && ((own >> k) & 1u)) ? d2df(__ldg(pl + pofs[k])) : df{0.f, 0.f};
  };
#pragma unroll
  for (int j = 0; j < 2 * R + 1; ++j) load_q(z0 - R + j, q[j]);

  for (int z = z0; z < z1; ++z) {
    const int64_t gz = (int64_t)z * nxy;
    float2 vf[PPT];
    double pv[PPT];
    df nq[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const bool o = (own >> k) & 1u;
      vf[k] = o ? __ldg(a.veff + gz + pofs[k]) : make_float2(0.f, 0.f);
      pv[k] = (o && a.prev) ? a.prev[(int64_t)n * a.ldp + gz + pofs[k]] : 0.0;
    }
    load_q(z + R + 1, nq);
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      if ((own >> k) & 1u) {
        s[sidx[k]] = q[R][k];
        if ((dup_r >> k) & 1u) s[sidx[k] + a.nx] = q[R][k];
        if ((dup_l >> k) & 1u) s[sidx[k] - a.nx] = q[R][k];
      }
    }
    const double* __restrict__ pl = xn + gz;
    for (int e = threadIdx.x; e < 2 * R * a.nx; e += blockDim.x) {
      const int hr = e / a.nx, hx = e - hr * a.nx;
      const int srow = hr < R ? hr : byl + hr;
      int gy = hr < R ? y0 - R + hr : y0 + byl + hr - R;
      const bool ok = wrap(gy, a.ny, a.bcy);
      const df v = ok ? d2df(__ldg(pl + (int64_t)gy * a.nx + hx)) : df{0.f, 0.f};
      const int si = srow * W + hx + R;
      s[si] = v;
      if (perx && hx < R) s[si + a.nx] = v;
      if (perx && hx >= a.nx - R) s[si - a.nx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      if ((own >> k) & 1u) {
        const df* c = s + sidx[k];
        const df c0 = mul(a.dms, q[R][k]);
        acc_t acc = {c0.h, c0.l};
#pragma unroll
        for (int p = 1; p <= R; ++p) {
          acc_t sm = {c[p * W].h, c[p * W].l};
          acc_add(sm, c[-p * W]);
          acc_add(sm, q[R + p][k]);
          acc_add(sm, q[R - p][k]);
          acc_add(sm, c[-p]);
          acc_add(sm, c[p]);
          acc_fma(acc, a.off[p], sm);
        }
        const df h = fma(df{vf[k].x, vf[k].y}, q[R][k], normalise(acc));
        df o = mul(a.s_h, h);
        if (a.prev) o = fma(a.s_p, d2df(pv[k]), o);
        a.y[(int64_t)n * a.ldy + gz + pofs[k]] = __dadd_rn(widen(o.h), widen(o.l));
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

}  // namespace

cudaError_t apply_h_local_df(const Grid& g, const LapCoef& lc, const float2* veff_df,
                             const double* x, int64_t ldx, double* y, int64_t ldy,
                             const double* prev, int64_t ldp, int ns, double shift, double s_h,
                             double s_p, cudaStream_t st, bool* used) {
  *used = false;
  const int maxpts = kSlabDfPpt * kSlabDfThreads;
  if (!veff_df || g.nx < R || g.nx > maxpts || ns < 1 || ns > 65535) return cudaSuccess;
  int by = std::min(g.ny, maxpts / g.nx);
  const int nslab = (g.ny + by - 1) / by;
  by = (g.ny + nslab - 1) / nslab;
  const int threads = ((by * g.nx + kSlabDfPpt - 1) / kSlabDfPpt + 31) / 32 * 32;
  const size_t smem = (size_t)(by + 2 * R) * (g.nx + 2 * R) * sizeof(df);
  if (smem > 48 * 1024) return cudaSuccess;
  const int64_t xy_ctas = (int64_t)nslab * ns;
  int nzc = (int)std::min<int64_t>((8 * sm_count() + xy_ctas - 1) / xy_ctas, 1 << 20);
  nzc = std::max(1, std::min(nzc, std::max(1, g.nz / (2 * R))));
  const int bz = (g.nz + nzc - 1) / nzc;
  nzc = (g.nz + bz - 1) / bz;
  SlabArgsDF a;
  a.x = x; a.ldx = ldx; a.y = y; a.ldy = ldy; a.prev = prev; a.ldp = ldp; a.veff = veff_df;
  a.nx = g.nx; a.ny = g.ny; a.nz = g.nz; a.bcx = g.bc[0]; a.bcy = g.bc[1]; a.bcz = g.bc[2];
  a.by = by;
  a.bz = bz;
  a.dms = host_df(lc.diag - shift);
  for (int p = 0; p <= R; ++p) a.off[p] = host_df(lc.off[p]);
  a.s_h = host_df(s_h);
  a.s_p = host_df(s_p);
  note_launch();
  k_apply_h_slab_df<<<dim3(nslab, ns, nzc), threads, smem, st>>>(a);
  *used = true;
  return cudaGetLastError();
}

}  // namespace sparc
