// Split-precision tensor-core GEMMs (tcgen05 + TMA + TMEM) for the projection
// and rotation of Algorithm 1 (paper Sec. II B, II D), in two accuracies:
//   FP32 operands (mixed precision): 4 digits, levels 0..3 (10 products);
//   FP64 operands (plain form):      6 digits, levels 0..5 (21 products).
//
// Block fixed-point split (Ozaki-style): for every operand row r (a row of the
// GEMM's M or N dimension) and every chunk q of 256 K values, the entries are
// scaled by 2^-e_rq, e_rq the binary exponent of the chunk's largest entry, and
// every entry u = x 2^-e_rq in (-1, 1) is written as D signed 8-bit integer
// digits, u = 2^-7 (d0 + 2^-8 d1 + 2^-16 d2 + ...) + O(2^-(8D-1)), each exactly
// representable in BF16.  A product is formed from the digit products of
// level l = i + j < NL,
//   L_l = sum_{i+j=l} a_i b_j,   a b ~ 2^(e_a + e_b - 14) sum_l 2^-8l L_l,
// each level accumulating in its own tensor-memory accumulator.  Digit products
// are integers of magnitude <= 2^14, so over a chunk of 256 K values the sums of
// levels 0..3 stay integers of magnitude <= 2^24 and the tensor core adds them
// exactly; levels >= 4 (FP64 form only) may round, at 2^-56 of the leading level.
// At the end of every chunk the level sums are scaled by 2^(e_a + e_b - 14) of
// that chunk and folded into a double-FP32 (hi, lo) running sum held in
// registers: the leading levels by error-free TwoSum, the remaining ones first
// combined in FP32 (Horner in 2^-8).  Per-chunk exponents keep the digits
// relative to local magnitudes, so the first dropped level (whose diagonal terms
// never cancel) stays ~2^-8NL of the local values instead of biasing long sums.
// Relative to sum_k |a_k b_k| the result is accurate to ~2^-32 (FP32 form) and
// ~2^-45 (FP64 form).  The running sums are FP32 pairs, so results below about
// 1e-30 in magnitude lose relative accuracy (FP64 orbital entries that small
// carry no weight in a normalised block).
//
// Kernel structure: persistent, one CTA of 320 threads per SM walks the work
// items (128 x 64 output tile, K split, output) with a grid stride; the
// pipeline counters run on across items, so one tile's TMA loads overlap the
// previous tile's epilogue:
//   warp 0     TMA producer: one 3-D TMA load per operand per K-step brings the
//              D BF16 digit tiles (swizzled) into a shared-memory ring
//              (full/empty mbarriers);
//   warp 1     allocates 512 TMEM columns and issues tcgen05.mma (one thread):
//              NL level accumulators of 64 columns, double-buffered when they fit;
//   warps 2-9  epilogue: two warps per TMEM lane quarter, 32 columns each; fold
//              a finished accumulator set into (hi, lo), finally write hi + lo.
// Every mbarrier wait is bounded; on expiry the CTA records SPARC_ERR_TIMEOUT
// in the status word, stops issuing work, drains what it issued (bounded) and
// frees its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "internal.cuh"

namespace sparc {

namespace {

constexpr int kBM = 128, kBN = 64;
constexpr int kQ = 256;  // K values per exponent chunk
constexpr uint32_t kTmemCols = 512;
constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;

// Compile-time plan of one accuracy form: D digits, levels 0..NL-1.
template <int D, int NL>
struct Plan {
  static_assert(NL <= D, "levels beyond the digits");
  static constexpr int kD = D, kNL = NL;
  static constexpr int kBK = D <= 4 ? 64 : 32;           // K per stage (one swizzle row)
  static constexpr int kSwizzle = kBK * 2;                // bytes: 128 or 64
  static constexpr int kSteps = kQ / kBK;                 // stages per exponent chunk
  static constexpr int kProducts = NL * (NL + 1) / 2;     // digit pairs with i + j < NL
  static constexpr int kBufs = (int)kTmemCols / (NL * kBN);  // accumulator sets in TMEM
  static constexpr int kExact = D <= 4 ? 1 : 3;           // levels folded by TwoSum
  static constexpr uint32_t kTileA = kBM * kBK * 2;       // one A digit tile
  static constexpr uint32_t kTileB = kBN * kBK * 2;       // one B digit tile
  static constexpr uint32_t kOpA = D * kTileA;
  static constexpr uint32_t kStageBytes = D * (kTileA + kTileB);
  static constexpr int kStages = (int)((220u * 1024u) / kStageBytes) > 4
                                     ? 4
                                     : (int)((220u * 1024u) / kStageBytes);
  // 1 KB for the alignment of the ring, and a margin behind it
  static constexpr uint32_t kSmemBytes = kStages * kStageBytes + 1024 + 4096;
  static_assert(kBufs >= 1 && kStages >= 2, "plan does not fit");
  static_assert(kSmemBytes <= 227 * 1024, "shared memory");
};
using PlanF32 = Plan<4, 4>;
using PlanF64 = Plan<6, 6>;

// Digit pair of product p, ordered by level l = i + j, then by i.
__host__ __device__ constexpr int prod_level(int p) {
  int l = 0;
  while ((l + 1) * (l + 2) / 2 <= p) ++l;
  return l;
}
__host__ __device__ constexpr int prod_a(int p) {
  return p - prod_level(p) * (prod_level(p) + 1) / 2;
}
__host__ __device__ constexpr int prod_b(int p) { return prod_level(p) - prod_a(p); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait; false on timeout (and then *abort is set).  Also gives up when
// another CTA of the launch has already recorded a status.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort,
                                          const int* status, long long budget) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_test(bar, parity)) return true;
    if (*abort) return false;
    if (*(volatile const int*)status != 0 || clock64() - t0 > budget) {
      *abort = 1;
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor (tcgen05 version 1) of a K-major operand whose
// rows are one swizzle span long (SW = 128 or 64 bytes): 8-row groups are
// 8 * SW bytes apart; layout code 2 = 128-byte swizzle, 4 = 64-byte swizzle.
template <int SW>
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  static_assert(SW == 128 || SW == 64, "swizzle");
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)((8 * SW) >> 4) << 32;   // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                 // descriptor version
  d |= (uint64_t)(SW == 128 ? 2 : 4) << 61;
  return d;
}

// Instruction descriptor: BF16 x BF16 -> FP32, A and B K-major, M = 128, N = 64.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 2^n as a float, built from the IEEE-754 exponent field for normal results.
__device__ __forceinline__ float pow2i(int n) {
  return n >= -126 ? __int_as_float((min(n, 127) + 127) << 23) : ldexpf(1.0f, n);
}

// Exact float -> double by moving the IEEE-754 fields with integer operations
// (GB300's FP64 pipe, which would otherwise do the conversion, is 1/64 of FP32).
__device__ __forceinline__ double widen(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFFu;
  if (e == 0u || e == 0xFFu) return (double)f;  // zero, subnormal, inf, nan
  const uint64_t d = ((uint64_t)(u & 0x80000000u) << 32) | ((uint64_t)(e + 896u) << 52) |
                     ((uint64_t)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)d);
}

// 2^-8l (0 <= l <= 15), from the IEEE-754 exponent field
__device__ __forceinline__ float exp2_neg8(int l) { return __int_as_float((127 - 8 * l) << 23); }

struct TcArgs {
  int M, N;
  int64_t K;
  int64_t kchunk;   // K per split (multiple of kQ)
  int upper;        // 1: enumerate only tiles with bi <= bj (symmetric outputs)
  int tiles_m, tiles_n;
  int nout;         // outputs per tile (2 for the projection: Hs and Ms)
  int ntiles_upper; // upper-triangle tiles (symmetric outputs)
  double* work;     // mode 0: work[(split * 2 + out) * M * N + m + n * M]
  float* out32;     // mode 1: out32[m + n * ldo]
  double* out64;    // mode 2: out64[m + n * ldo]
  int64_t ldo;
  int mode;
  const int8_t* escA;   // exponent of A row r in chunk q at [q * MP + r]
  const int8_t* escB0;  // exponent of B row c (output 0) in chunk q at [q * NP + c]
  const int8_t* escB1;  // same for output 1
  int MP, NP;           // row strides of the exponent arrays (multiples of 128)
  int* status;
  long long wait_cycles;  // bound of every wait (SM clock cycles)
};

template <int D, int NL>
// 10 warps are allotted registers as 12 (whole warp quads): at most 168 each
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB0,
              const __grid_constant__ CUtensorMap tB1, const TcArgs a) {
  using P = Plan<D, NL>;
  constexpr int kStages = P::kStages, kBufs = P::kBufs, kBK = P::kBK;
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t bars[2 * kStages + 2 * kBufs + 1];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t full0 = smem_u32(&bars[0]);
  const uint32_t empty0 = smem_u32(&bars[kStages]);
  const uint32_t accf0 = smem_u32(&bars[2 * kStages]);          // kBufs barriers
  const uint32_t acce0 = smem_u32(&bars[2 * kStages + kBufs]);  // kBufs barriers
  const uint32_t drain = smem_u32(&bars[2 * kStages + 2 * kBufs]);

  // Work items (persistent CTAs walk them with a grid stride): item w is
  // (tile, split, output) with the tile fastest, so the CTAs running together
  // share a split's K range (projection) or a row block's A digits (rotation)
  // in L2.  Every role decodes the same sequence; stage and accumulator
  // counters run on across items.
  // symmetric outputs list only the tiles that reach the upper triangle
  // (bi * 128 <= bj * 64 + 63): column bj holds bj / 2 + 1 of them
  const int ntiles = a.upper ? a.ntiles_upper : a.tiles_m * a.tiles_n;
  const int nsplit = (int)((a.K + a.kchunk - 1) / a.kchunk);
  const int nitems = ntiles * nsplit * a.nout;
  struct Item {
    int bi, bj, out;
    int64_t k0;
    int nk;
    bool skip;
  };
  auto decode = [&](int w) {
    Item it;
    const int tile = w % ntiles, rest = w / ntiles;
    it.out = rest % a.nout;
    const int split = rest / a.nout;
    if (a.upper) {
      int t = tile, bj = 0;
      while (bj + 1 < a.tiles_n && t >= min(a.tiles_m, (bj * kBN + kBN - 1) / kBM + 1)) {
        t -= min(a.tiles_m, (bj * kBN + kBN - 1) / kBM + 1);
        ++bj;
      }
      it.bi = t;
      it.bj = bj;
    } else {
      it.bj = tile % a.tiles_n;
      it.bi = tile / a.tiles_n;
    }
    it.skip = false;
    it.k0 = (int64_t)split * a.kchunk;
    const int64_t k1 = min(a.K, it.k0 + a.kchunk);
    it.nk = k1 > it.k0 ? (int)((k1 - it.k0 + kBK - 1) / kBK) : 0;
    return it;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < kBufs; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, kEpiWarps);
    }
    mbar_init(drain, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  volatile int* abort = &abort_sh;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int g = 0;  // stages issued so far (all items)
      bool ok = true;
      for (int w = blockIdx.x; ok && w < nitems; w += gridDim.x) {
        const Item itm = decode(w);
        const CUtensorMap* tB = itm.out == 0 ? &tB0 : &tB1;
        for (int it = 0; it < itm.nk; ++it, ++g) {
          const int s = g % kStages;
          const uint32_t round = (uint32_t)(g / kStages);
          if (!mbar_wait(empty0 + 8 * s, (round & 1) ^ 1, abort, a.status, a.wait_cycles)) {
            ok = false;
            break;
          }
          const uint32_t sa = base + s * P::kStageBytes;
          mbar_expect_tx(full0 + 8 * s, P::kStageBytes);
          const int kx = (int)(itm.k0 + (int64_t)it * kBK);
          tma_load_3d(sa, &tA, kx, itm.bi * kBM, 0, full0 + 8 * s);
          tma_load_3d(sa + P::kOpA, tB, kx, itm.bj * kBN, 0, full0 + 8 * s);
        }
      }
      if (*abort) {
        // drain: the loads already issued must land before the CTA exits
        for (int it = max(0, g - kStages); it < g; ++it) {
          const long long t0 = clock64();
          while (!mbar_test(full0 + 8 * (it % kStages), (uint32_t)(it / kStages) & 1) &&
                 clock64() - t0 < max(a.wait_cycles, kDrainCycles)) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int g = 0;   // stages consumed so far
      int gc = 0;  // accumulator chunks started so far
      bool ok = true;
      for (int w = blockIdx.x; ok && w < nitems; w += gridDim.x) {
        const Item itm = decode(w);
        for (int it = 0; it < itm.nk; ++it, ++g) {
          const int s = g % kStages;
          const uint32_t round = (uint32_t)(g / kStages);
          const int in_chunk = it % P::kSteps;
          const int buf = gc % kBufs;
          const uint32_t use = (uint32_t)(gc / kBufs);
          if (in_chunk == 0) {
            if (!mbar_wait(acce0 + 8 * buf, (use & 1) ^ 1, abort, a.status, a.wait_cycles)) {
              ok = false;
              break;
            }
            tc_fence_after();
          }
          if (!mbar_wait(full0 + 8 * s, round & 1, abort, a.status, a.wait_cycles)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = base + s * P::kStageBytes, sb = sa + P::kOpA;
          // descriptors of this stage's first A and B tiles; every other operand
          // is a compile-time offset (the address field holds addr >> 4 and the
          // ring ends below 256 KB, so the additions never carry out of it)
          const uint64_t da0 = smem_desc<P::kSwizzle>(sa), db0 = smem_desc<P::kSwizzle>(sb);
          const uint32_t d0 = tmem + (uint32_t)(buf * NL * kBN);
#pragma unroll
          for (int p = 0; p < P::kProducts; ++p) {
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk) {
              const uint64_t da = da0 + (uint64_t)((prod_a(p) * P::kTileA + kk * 32) >> 4);
              const uint64_t db = db0 + (uint64_t)((prod_b(p) * P::kTileB + kk * 32) >> 4);
              tc_mma(d0 + (uint32_t)(prod_level(p) * kBN), da, db,
                     !(in_chunk == 0 && kk == 0 && prod_a(p) == 0));
            }
          }
          tc_commit(empty0 + 8 * s);
          if (in_chunk == P::kSteps - 1 || it == itm.nk - 1) {
            tc_commit(accf0 + 8 * buf);
            ++gc;
          }
        }
      }
      // all issued MMAs complete before tensor memory is released
      tc_commit(drain);
      const long long t0 = clock64();
      while (!mbar_test(drain, 0) && clock64() - t0 < max(a.wait_cycles, kDrainCycles)) {
      }
    }
  } else {
    // ---------------- epilogue (warps 2..9) ----------------
    const int q = warp & 3;             // TMEM lane quarter of this warp
    const int half = (warp - 2) >> 2;   // which 32 of the tile's 64 columns
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    bool ok = true;
    int gc = 0;  // accumulator chunks consumed so far (all items)
    for (int w = blockIdx.x; ok && w < nitems; w += gridDim.x) {
    const Item itm = decode(w);
    if (itm.skip) continue;
    const int bi = itm.bi, bj = itm.bj, out = itm.out;
    const int nchunks = (itm.nk + P::kSteps - 1) / P::kSteps;
    float hi[32], lo[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      hi[i] = 0.f;
      lo[i] = 0.f;
    }
    for (int c = 0; c < nchunks && ok; ++c, ++gc) {
      const int buf = gc % kBufs;
      const uint32_t use = (uint32_t)(gc / kBufs);
      if (!mbar_wait(accf0 + 8 * buf, use & 1, abort, a.status, a.wait_cycles)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t t_acc =
          tmem + lane_off + (uint32_t)(buf * NL * kBN) + (uint32_t)(half * 32);
      // exponents of this chunk: the thread's A row and the warp's 32 B rows
      const int qg = (int)(itm.k0 / kQ) + c;
      const int rowc = min(bi * kBM + q * 32 + lane, a.MP - 1);
      const int ea = (int)a.escA[(int64_t)qg * a.MP + rowc] - 14;
      const uint4* eb_src = reinterpret_cast<const uint4*>(
          (out == 0 ? a.escB0 : a.escB1) + (int64_t)qg * a.NP + bj * kBN + half * 32);
      // columns in slices of 8: all NL level loads of a slice are issued
      // before one wait (TMEM load latency is paid once per slice)
      constexpr int W = 8;
#pragma unroll
      for (int cq = 0; cq < 32 / W; ++cq) {
        const uint32_t tq = t_acc + cq * W;
        const uint2 ew = __ldg(reinterpret_cast<const uint2*>(eb_src) + cq);
        uint32_t L[NL][W];
#pragma unroll
        for (int l = 0; l < NL; ++l) tmem_ld8(tq + l * kBN, L[l]);
        tmem_wait_ld();
        if (cq == 32 / W - 1) {
          // every level of this buffer is in registers: hand it back to the MMA warp
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(acce0 + 8 * buf);
        }
#pragma unroll
        for (int i = 0; i < W; ++i) {
          // tail t = L_kExact + 2^-8 L_(kExact+1) + ... (Horner from the last level)
          float t = __uint_as_float(L[NL - 1][i]);
#pragma unroll
          for (int l = NL - 2; l >= P::kExact; --l)
            t = __fmaf_rn(t, 0.00390625f, __uint_as_float(L[l][i]));
          // chunk value (ch, cl) = L0 + 2^-8 L1 + ... + 2^-8kExact t, the exact
          // integer levels added error-free
          float ch = __uint_as_float(L[0][i]), cl = 0.f;
#pragma unroll
          for (int l = 1; l <= P::kExact; ++l) {
            const float x = (l < P::kExact ? __uint_as_float(L[l][i]) : t) * exp2_neg8(l);
            if (l < P::kExact || P::kExact == 1) {
              const float sm = __fadd_rn(ch, x);
              const float bp = __fsub_rn(sm, ch);
              cl = __fadd_rn(cl, __fadd_rn(__fsub_rn(ch, __fsub_rn(sm, bp)), __fsub_rn(x, bp)));
              ch = sm;
            } else {
              cl = __fadd_rn(cl, x);  // six-level tail: 2^-24 of L0 and below, low word
            }
          }
          // scale by 2^(e_a + e_b - 14) and add to the running (hi, lo)
          const int eb = (int)(int8_t)((i < 4 ? ew.x : ew.y) >> (8 * (i & 3)));
          const float sc = pow2i(ea + eb);
          const int j = cq * W + i;
          const float x = ch * sc;
          const float sm = __fadd_rn(hi[j], x);
          const float bp = __fsub_rn(sm, hi[j]);
          const float err = __fadd_rn(__fsub_rn(hi[j], __fsub_rn(sm, bp)), __fsub_rn(x, bp));
          const float l2 = __fadd_rn(lo[j], __fadd_rn(err, cl * sc));
          // renormalise so that |lo| stays within half an ulp of hi
          hi[j] = __fadd_rn(sm, l2);
          lo[j] = __fsub_rn(l2, __fsub_rn(hi[j], sm));
        }
      }
    }
    if (ok && nchunks > 0) {
      const int row = bi * kBM + q * 32 + lane;
      const int split = (int)(itm.k0 / a.kchunk);
      if (row < a.M) {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int col = bj * kBN + half * 32 + i;
          if (col < a.N) {
            if (a.mode == 0) {
              a.work[((int64_t)split * 2 + out) * a.M * a.N + row + (int64_t)col * a.M] =
                  __dadd_rn(widen(hi[i]), widen(lo[i]));
            } else if (a.mode == 1) {
              a.out32[row + (int64_t)col * a.ldo] = __fadd_rn(hi[i], lo[i]);
            } else {
              a.out64[row + (int64_t)col * a.ldo] = __dadd_rn(widen(hi[i]), widen(lo[i]));
            }
          }
        }
      }
    }
    }  // items
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
  if (threadIdx.x == 0 && abort_sh) atomicCAS(a.status, 0, SPARC_ERR_TIMEOUT);
}

// ---------------------------------------------------------------------------
// Fixed-point digit slicing
// ---------------------------------------------------------------------------
// Binary exponent E with |v| < 2^E for the largest |v| (0 for an all-zero row).
__device__ __forceinline__ int row_exponent(double vmax) {
  if (!(vmax > 0.0)) return 0;
  int e;
  frexp(vmax, &e);  // vmax = m 2^e, m in [0.5, 1)
  return e;
}

// Chunk exponent stored as int8. Raising E keeps |x 2^-E| < 1, so the clamp
// only costs digits of chunks whose largest entry is below 2^-120.
__device__ __forceinline__ int8_t chunk_exponent(double vmax) {
  return (int8_t)max(-120, min(127, row_exponent(vmax)));
}

// D signed 8-bit digits of u = x 2^-E (|u| < 1):
// u = 2^-7 (d0 + d1/2^8 + d2/2^16 + ...), each |d| <= 128.  Every step is exact
// in the input's own precision (FP32 input: its 24-bit mantissa spans at most
// four digits).
// BF16 of an integer digit |d| <= 128 without a conversion instruction (on
// GB300 those run on the FP64 pipe): d + 1.5 * 2^23 is exact as a float whose
// low mantissa bits hold d, and a float with at most 8 significant bits is
// its BF16 bit pattern in the upper half word.
__device__ __forceinline__ __nv_bfloat16 digit_bf16(int d) {
  const float f = __fsub_rn(__int_as_float(0x4B400000 + d), 12582912.0f);
  return __ushort_as_bfloat16((unsigned short)(__float_as_uint(f) >> 16));
}

// FP64 input: integer arithmetic on the IEEE-754 fields (GB300's FP64 pipe is
// 1/64 of its FP32 rate): F = x 2^(7 + 8(D-1) - E) rounded to an integer
// (|F| < 2^(7 + 8(D-1))), then d_k = round(F / 2^s), F -= d_k 2^s for
// s = 8(D-1-k); the remainders stay within half a digit, so |d_k| <= 128.
template <int D>
__device__ __forceinline__ void digits(double x, int E, __nv_bfloat16 (&d)[D]) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7FF);
  long long F = 0;
  if (e != 0 && e != 0x7FF) {  // zero and subnormals give zero digits
    const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = e - 1075 + 7 + 8 * (D - 1) - E;  // F = m 2^sh
    unsigned long long f = 0;
    if (sh >= 0) f = sh < 11 ? (m << sh) : 0ull;  // |x| < 2^E keeps sh < 0 in practice
    else if (sh > -64) f = (m >> (-sh)) + ((m >> (-sh - 1)) & 1ull);  // round half up
    F = (u >> 63) ? -(long long)f : (long long)f;
  }
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const int s = 8 * (D - 1 - k);
    long long dk;
    if (s > 0) {
      dk = (F + (1ll << (s - 1))) >> s;
      F -= dk << s;
    } else {
      dk = F;
    }
    d[k] = digit_bf16((int)dk);
  }
}
template <int D>
__device__ __forceinline__ void digits(float x, int E, __nv_bfloat16 (&d)[D]) {
  float u = ldexpf(x, 7 - E);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const float r = rintf(u);
    d[k] = __ushort_as_bfloat16((unsigned short)(__float_as_uint(r) >> 16));  // exact: |r| <= 128
    u = (u - r) * 256.0f;
  }
}

// |x| 2^-f as an order-preserving integer key (the IEEE-754 bits of the
// magnitude, exponent lowered by f; 0 for zero and values that would leave the
// normal range downwards).  key_exponent gives frexp's exponent of the value.
__device__ __forceinline__ long long mag_key(double x, int f = 0) {
  const long long b = __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFll;
  const long long e = b >> 52;
  if (e == 0) return 0;
  const long long e2 = e - f;
  if (e2 <= 0) return 0;
  if (e2 >= 0x7FF) return 0x7FEFFFFFFFFFFFFFll;
  return b - ((long long)f << 52);
}
__device__ __forceinline__ int key_exponent(long long k) {
  return k == 0 ? 0 : (int)(k >> 52) - 1022;  // m 2^e, m in [0.5, 1)
}
__device__ __forceinline__ int8_t chunk_exponent_key(long long k) {
  return (int8_t)max(-120, min(127, key_exponent(k)));
}
__device__ __forceinline__ long long warp_max(long long m) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  return m;
}

__device__ __forceinline__ float absmax(float m, float x) { return fmaxf(m, fabsf(x)); }
__device__ __forceinline__ float warp_max(float m) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  return m;
}

// Chunk exponents of the columns of X: esc[q * NP + col] = E(max over t in chunk
// q of |X[t + col ldx]|), one warp per (column, chunk).
template <typename T>
__global__ void k_chunk_exp_cols(const T* __restrict__ X, int64_t ldx, int64_t nd, int ncol,
                                 int nq, int NP, int8_t* __restrict__ esc) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (int64_t)ncol * nq) return;
  const int col = (int)(w % ncol), q = (int)(w / ncol);
  const T* x = X + (int64_t)col * ldx;
  const int64_t t1 = min((int64_t)(q + 1) * kQ, nd);
  if constexpr (std::is_same<T, double>::value) {
    long long m = 0;
    for (int64_t t = (int64_t)q * kQ + lane; t < t1; t += 32) m = max(m, mag_key(x[t]));
    m = warp_max(m);
    if (lane == 0) esc[(int64_t)q * NP + col] = chunk_exponent_key(m);
  } else {
    T m = 0;
    for (int64_t t = (int64_t)q * kQ + lane; t < t1; t += 32) m = absmax(m, x[t]);
    m = warp_max(m);
    if (lane == 0) esc[(int64_t)q * NP + col] = chunk_exponent((double)m);
  }
}

// Column exponents f_k of X (one block per column), used to balance columns.
template <typename T>
__global__ void k_col_exponent(const T* __restrict__ X, int64_t ldx, int64_t nd,
                               int* __restrict__ esc) {
  // magnitudes compared as integer keys (order-preserving for both types)
  __shared__ long long sm[32];
  const T* x = X + (int64_t)blockIdx.x * ldx;
  long long m = 0;
  for (int64_t t = threadIdx.x; t < nd; t += blockDim.x) {
    if constexpr (std::is_same<T, double>::value) m = max(m, mag_key(x[t]));
    else m = max(m, (long long)(__float_as_uint(x[t]) & 0x7FFFFFFFu));
  }
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long r = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = max(r, sm[w]);
    if constexpr (std::is_same<T, double>::value) esc[blockIdx.x] = key_exponent(r);
    else esc[blockIdx.x] = row_exponent((double)__uint_as_float((unsigned)r));
  }
}

// Chunk exponents of the rows of the column-balanced X (rotation A operand):
// esc[q * MP + t] = E(max over k in chunk q of |X[t + k ldx]| 2^-f_k).
template <typename T>
__global__ void k_chunk_exp_rows(const T* __restrict__ X, int64_t ldx, int64_t nd, int ns,
                                 const int* __restrict__ fcol, int MP, int8_t* __restrict__ esc) {
  const int q = blockIdx.y;
  const int k1 = min((q + 1) * kQ, ns);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nd;
       t += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (std::is_same<T, double>::value) {
      long long m = 0;
      for (int k = q * kQ; k < k1; ++k) m = max(m, mag_key(X[t + (int64_t)k * ldx], fcol[k]));
      esc[(int64_t)q * MP + t] = chunk_exponent_key(m);
    } else {
      float m = 0.f;
      for (int k = q * kQ; k < k1; ++k)
        m = fmaxf(m, ldexpf(fabsf(X[t + (int64_t)k * ldx]), -fcol[k]));
      esc[(int64_t)q * MP + t] = chunk_exponent((double)m);
    }
  }
}

// Chunk exponents of the rows of the row-scaled Z (rotation B operand, row j =
// output column j): esc[q * NP + j] = E(max over k in chunk q of |Z[k + j n]| 2^f_k).
// Z: K x N, column-major with leading dimension ldz
__global__ void k_chunk_exp_z(const double* __restrict__ Z, int K, int N, int64_t ldz,
                              const int* __restrict__ fcol, int nq, int NP,
                              int8_t* __restrict__ esc) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (int64_t)N * nq) return;
  const int j = (int)(w % N), q = (int)(w / N);
  long long m = 0;
  const int k1 = min((q + 1) * kQ, K);
  for (int k = q * kQ + lane; k < k1; k += 32)
    m = max(m, mag_key(Z[k + (int64_t)j * ldz], -fcol[k]));
  m = warp_max(m);
  if (lane == 0) esc[(int64_t)q * NP + j] = chunk_exponent_key(m);
}

// S[s][col][t] = digit s of X[t + col ldx] at its chunk's exponent (ld = lds)
template <typename T, int D>
__global__ void k_slice_cols(const T* __restrict__ X, int64_t ldx, int64_t nd, int ncol,
                             const int8_t* __restrict__ esc, int NP,
                             __nv_bfloat16* __restrict__ S, int64_t lds) {
  const int col = blockIdx.y;
  const int64_t plane = lds * ncol;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < lds;
       t += (int64_t)gridDim.x * blockDim.x) {
    __nv_bfloat16 d[D];
    const int E = esc[(t / kQ) * NP + col];
    digits<D>(t < nd ? X[t + col * ldx] : T(0), E, d);
    const int64_t o = t + col * lds;
#pragma unroll
    for (int k = 0; k < D; ++k) S[k * plane + o] = d[k];
  }
}

// Transposed digits of the column-balanced X: S[s][t][k] = digit s of
// X[t + k ldx] 2^-f_k at row t's exponent (ld = ldk)
template <typename T, int D>
__global__ void k_slice_transpose(const T* __restrict__ X, int64_t ldx, int64_t nd, int ns,
                                  const int* __restrict__ fcol, const int8_t* __restrict__ esc,
                                  int MP, __nv_bfloat16* __restrict__ S, int64_t ldk) {
  // digits of x 2^-f at exponent E are the digits of x at exponent E + f
  __shared__ T tile[32][33];
  const int64_t t0 = (int64_t)blockIdx.x * 32;
  const int k0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r;
    const int64_t t = t0 + threadIdx.x;
    tile[r][threadIdx.x] = (k < ns && t < nd) ? X[t + (int64_t)k * ldx] : T(0);
  }
  __syncthreads();
  const int64_t plane = ldk * nd;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t t = t0 + r;
    const int k = k0 + threadIdx.x;
    if (t < nd && k < ldk) {
      __nv_bfloat16 d[D];
      const int f = k < ns ? fcol[k] : 0;
      digits<D>(tile[threadIdx.x][r], (int)esc[(int64_t)(k / kQ) * MP + t] + f, d);
      const int64_t o = t * ldk + k;
#pragma unroll
      for (int q = 0; q < D; ++q) S[q * plane + o] = d[q];
    }
  }
}

// Z digits of the row-scaled Z: S[s][j][k] = digit s of Z[k + j n] 2^f_k at
// column j's exponent, ld = ldk  (X Z = (X 2^-f) (2^f Z): the scalings cancel)
template <int D>
__global__ void k_slice_z(const double* __restrict__ Z, int K, int N, int64_t ldz,
                          const int* __restrict__ fcol, const int8_t* __restrict__ esc, int NP,
                          __nv_bfloat16* __restrict__ S, int64_t ldk) {
  const int64_t plane = ldk * N;
  const int64_t tot = (int64_t)N * ldk;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / ldk), k = (int)(e % ldk);
    __nv_bfloat16 d[D];
    // digits of z 2^f at exponent E are the digits of z at exponent E - f
    digits<D>(k < K ? Z[k + (int64_t)j * ldz] : 0.0,
              (int)esc[(int64_t)(k / kQ) * NP + j] - (k < K ? fcol[k] : 0), d);
#pragma unroll
    for (int q = 0; q < D; ++q) S[q * plane + e] = d[q];
  }
}

// cuTensorMapEncodeTiled, resolved through the runtime so that the library does
// not link the driver library directly (it then also loads on hosts without one).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

// 3-D BF16 tensor map of D digit planes: dims (inner, rows, D), box
// (kBK, box_rows, D), swizzle of one kBK-element row (128 or 64 bytes).
template <class P>
bool make_map(CUtensorMap* m, const void* base, uint64_t inner, uint64_t rows, uint64_t ld,
              uint32_t box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[3] = {inner, rows, (cuuint64_t)P::kD};
  cuuint64_t strides[2] = {ld * 2, ld * rows * 2};
  cuuint32_t box[3] = {(cuuint32_t)P::kBK, box_rows, (cuuint32_t)P::kD};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   P::kSwizzle == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int D, int NL>
cudaError_t launch_tc(const CUtensorMap& tA, const CUtensorMap& tB0, const CUtensorMap& tB1,
                      const TcArgs& a, dim3 grid, cudaStream_t st) {
  using P = Plan<D, NL>;
  // the shared-memory opt-in is per device: set it once on each
  static std::mutex mu;
  static bool done[128] = {};
  static int sms[128] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int nsm;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    if (!done[dev]) {
      e = cudaFuncSetAttribute(k_tc_gemm<D, NL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               P::kSmemBytes);
      if (e != cudaSuccess) return e;
      e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return e;
      done[dev] = true;
    }
    nsm = sms[dev];
  }
  // persistent CTAs: one per SM (shared memory allows no second), at most one
  // per work item
  const long long items = (long long)(a.upper ? a.ntiles_upper : a.tiles_m * a.tiles_n) *
                          ((a.K + a.kchunk - 1) / a.kchunk) * a.nout;
  const unsigned ctas = (unsigned)std::max(1LL, std::min<long long>(items, nsm));
  (void)grid;
  note_launch(), k_tc_gemm<D, NL><<<ctas, kThreads, P::kSmemBytes, st>>>(tA, tB0, tB1, a);
  return cudaGetLastError();
}

template <typename T>
struct PlanOf;
template <>
struct PlanOf<float> {
  using type = PlanF32;
};
template <>
struct PlanOf<double> {
  using type = PlanF64;
};

template <class P, typename TX, typename TY>
cudaError_t tc_project_t(const TX* Xt, int64_t ldx, const TY* Yt, int64_t ldy, int64_t nd, int ns,
                         double* Hs, double* Ms, double* work, int nsplit, __nv_bfloat16* SX,
                         __nv_bfloat16* SY, int* esc, int* status, cudaStream_t st) {
  constexpr int D = P::kD;
  // digits of both operands, K-major (t contiguous per orbital column), each
  // (orbital column, chunk) at its own exponent
  const int64_t lds = (nd + 63) / 64 * 64;
  const int nq = (int)((lds + kQ - 1) / kQ);
  const int NP = (ns + 127) / 128 * 128;
  int8_t* escX = reinterpret_cast<int8_t*>(esc);
  int8_t* escY = escX + (size_t)nq * NP;
  const unsigned eg = (unsigned)(((int64_t)ns * nq * 32 + 255) / 256);
  note_launch(), k_chunk_exp_cols<TX><<<eg, 256, 0, st>>>(Xt, ldx, nd, ns, nq, NP, escX);
  note_launch(), k_chunk_exp_cols<TY><<<eg, 256, 0, st>>>(Yt, ldy, nd, ns, nq, NP, escY);
  dim3 sg((unsigned)std::min<int64_t>((lds + 255) / 256, 64), ns);
  note_launch(), k_slice_cols<TX, D><<<sg, 256, 0, st>>>(Xt, ldx, nd, ns, escX, NP, SX, lds);
  note_launch(), k_slice_cols<TY, D><<<sg, 256, 0, st>>>(Yt, ldy, nd, ns, escY, NP, SY, lds);
  CUtensorMap mXa, mXb, mYb;
  if (!make_map<P>(&mXa, SX, (uint64_t)lds, (uint64_t)ns, (uint64_t)lds, kBM) ||
      !make_map<P>(&mXb, SX, (uint64_t)lds, (uint64_t)ns, (uint64_t)lds, kBN) ||
      !make_map<P>(&mYb, SY, (uint64_t)lds, (uint64_t)ns, (uint64_t)lds, kBN))
    return cudaErrorInvalidValue;
  TcArgs a{};
  a.M = ns;
  a.N = ns;
  a.K = lds;
  int64_t kc = (lds + nsplit - 1) / nsplit;
  a.kchunk = (kc + kQ - 1) / kQ * kQ;  // splits start on exponent chunks
  a.upper = 1;
  a.tiles_m = (ns + kBM - 1) / kBM;
  a.tiles_n = (ns + kBN - 1) / kBN;
  a.work = work;
  a.mode = 0;
  a.escA = escX;
  a.escB0 = escY;
  a.escB1 = escX;
  a.MP = NP;
  a.NP = NP;
  a.nout = 2;
  a.ntiles_upper = 0;
  for (int bj = 0; bj < a.tiles_n; ++bj)
    a.ntiles_upper += std::min(a.tiles_m, (bj * kBN + kBN - 1) / kBM + 1);
  a.status = status;
  a.wait_cycles = wait_cycles();
  const int nsp = (int)((lds + a.kchunk - 1) / a.kchunk);
  // out 0: Hs = X^T Y (B = Y slices), out 1: Ms = X^T X (B = X slices); tiles
  // entirely below the diagonal exit at once
  cudaError_t e = launch_tc<P::kD, P::kNL>(mXa, mYb, mXb, a, dim3(a.tiles_m * a.tiles_n, nsp, 2),
                                           st);
  if (e != cudaSuccess) return e;
  // the SIMT path's deterministic split reduction (upper elements, mirrored)
  return project_reduce(work, nsp, ns, Hs, Ms, st);
}

// Xout (nd x N, ldo) = Xt (nd x ns, ld) Z (ns x N, column-major, ldz)
template <typename T>
cudaError_t tc_rotate_t(const T* Xt, int64_t ld, int64_t nd, int ns, const double* Z, int64_t ldz,
                        int N, T* Xout, int64_t ldo, __nv_bfloat16* SA, __nv_bfloat16* SZ,
                        int* esc, int* status, cudaStream_t st) {
  using P = typename PlanOf<T>::type;
  constexpr int D = P::kD;
  // digits of Xt per grid point t (over its ns entries) and of Z per column j
  const int64_t ldk = (ns + 7) / 8 * 8;
  const int nq = (int)((ldk + kQ - 1) / kQ);
  const int MP = (int)((nd + 127) / 128 * 128), NP = (N + 127) / 128 * 128;
  int* fcol = esc;  // ns entries: column exponents of Xt
  int8_t* escT = reinterpret_cast<int8_t*>(esc + ((ns + 63) / 64 * 64));
  int8_t* escZ = escT + (size_t)nq * MP;
  note_launch(), k_col_exponent<T><<<ns, 256, 0, st>>>(Xt, ld, nd, fcol);
  note_launch(), k_chunk_exp_rows<T><<<dim3((unsigned)std::min<int64_t>((nd + 255) / 256, 4096),
                                            nq),
                                       256, 0, st>>>(Xt, ld, nd, ns, fcol, MP, escT);
  note_launch(), k_chunk_exp_z<<<(unsigned)(((int64_t)N * nq * 32 + 255) / 256), 256, 0, st>>>(
      Z, ns, N, ldz, fcol, nq, NP, escZ);
  dim3 tg((unsigned)((nd + 31) / 32), (unsigned)((ldk + 31) / 32));
  note_launch(), k_slice_transpose<T, D><<<tg, dim3(32, 8), 0, st>>>(Xt, ld, nd, ns, fcol, escT,
                                                                     MP, SA, ldk);
  note_launch(), k_slice_z<D><<<(unsigned)std::min<int64_t>(((int64_t)N * ldk + 255) / 256,
                                                            4096),
                                256, 0, st>>>(Z, ns, N, ldz, fcol, escZ, NP, SZ, ldk);
  CUtensorMap mA, mZ;
  if (!make_map<P>(&mA, SA, (uint64_t)ldk, (uint64_t)nd, (uint64_t)ldk, kBM) ||
      !make_map<P>(&mZ, SZ, (uint64_t)ldk, (uint64_t)N, (uint64_t)ldk, kBN))
    return cudaErrorInvalidValue;
  TcArgs a{};
  a.M = (int)nd;
  a.N = N;
  a.K = ldk;
  a.kchunk = (ldk + kQ - 1) / kQ * kQ;
  a.upper = 0;
  a.tiles_m = (int)((nd + kBM - 1) / kBM);
  a.tiles_n = (N + kBN - 1) / kBN;
  if (std::is_same<T, float>::value) {
    a.out32 = reinterpret_cast<float*>(Xout);
    a.mode = 1;
  } else {
    a.out64 = reinterpret_cast<double*>(Xout);
    a.mode = 2;
  }
  a.ldo = ldo;
  a.escA = escT;
  a.escB0 = escZ;
  a.escB1 = escZ;
  a.MP = MP;
  a.NP = NP;
  a.nout = 1;
  a.status = status;
  a.wait_cycles = wait_cycles();
  return launch_tc<P::kD, P::kNL>(mA, mZ, mZ, a, dim3(a.tiles_m * a.tiles_n, 1, 1), st);
}

}  // namespace

size_t tc_esc_bytes(int64_t ld, int64_t nd, int ns_max) {
  const int64_t lds = (nd + 63) / 64 * 64;
  const int64_t nqp = (lds + kQ - 1) / kQ, NP = (ns_max + 127) / 128 * 128;
  const int64_t ldk = (ns_max + 7) / 8 * 8, nqr = (ldk + kQ - 1) / kQ;
  const int64_t MP = (nd + 127) / 128 * 128;
  const int64_t proj = 2 * nqp * NP;
  const int64_t rot = 4 * ((ns_max + 63) / 64 * 64) + nqr * (MP + NP);
  (void)ld;
  return (size_t)std::max(proj, rot) + 256;
}

int tc_digits(bool fp64) { return fp64 ? PlanF64::kD : PlanF32::kD; }

size_t tc_slice_elems(int64_t ld, int64_t nd, int ns_max, bool fp64) {
  const int64_t ldk = (ns_max + 7) / 8 * 8;
  const int64_t lds = (nd + 63) / 64 * 64;
  return (size_t)tc_digits(fp64) *
         std::max<int64_t>(std::max(ld, lds) * ns_max, nd * ldk);
}

int tc_project_nsplit(int ns) {
  const int tm = (ns + kBM - 1) / kBM, tn = (ns + kBN - 1) / kBN;
  int tiles = 0;
  for (int bj = 0; bj < tn; ++bj)
    for (int bi = 0; bi < tm; ++bi)
      if (bi * kBM <= bj * kBN + kBN - 1) ++tiles;
  tiles *= 2;  // Hs and Ms
  // enough (tile, split) items for the persistent CTAs to balance: ~4 per SM
  int s = (4 * sm_count() + tiles - 1) / tiles;
  return std::max(1, std::min(s, 64));
}

cudaError_t tc_project(const float* Xt, const float* Yt, int64_t ld, int64_t nd, int ns,
                       double* Hs, double* Ms, double* work, int nsplit, __nv_bfloat16* SX,
                       __nv_bfloat16* SY, int* esc, int* status, cudaStream_t st) {
  return tc_project_t<PlanF32>(Xt, ld, Yt, ld, nd, ns, Hs, Ms, work, nsplit, SX, SY, esc, status,
                               st);
}
cudaError_t tc_project(const float* Xt, int64_t ldx, const double* Yt, int64_t ldy, int64_t nd,
                       int ns, double* Hs, double* Ms, double* work, int nsplit,
                       __nv_bfloat16* SX, __nv_bfloat16* SY, int* esc, int* status,
                       cudaStream_t st) {
  return tc_project_t<PlanF32>(Xt, ldx, Yt, ldy, nd, ns, Hs, Ms, work, nsplit, SX, SY, esc,
                               status, st);
}
cudaError_t tc_project(const double* Xt, const double* Yt, int64_t ld, int64_t nd, int ns,
                       double* Hs, double* Ms, double* work, int nsplit, __nv_bfloat16* SX,
                       __nv_bfloat16* SY, int* esc, int* status, cudaStream_t st) {
  return tc_project_t<PlanF64>(Xt, ld, Yt, ld, nd, ns, Hs, Ms, work, nsplit, SX, SY, esc, status,
                               st);
}
cudaError_t tc_rotate(const float* Xt, int64_t ld, int64_t nd, int ns, const double* Z, float* Xout,
                      int64_t ldo, __nv_bfloat16* SA, __nv_bfloat16* SZ, int* esc, int* status,
                      cudaStream_t st) {
  return tc_rotate_t<float>(Xt, ld, nd, ns, Z, ns, ns, Xout, ldo, SA, SZ, esc, status, st);
}
cudaError_t tc_rotate(const double* Xt, int64_t ld, int64_t nd, int ns, const double* Z,
                      double* Xout, int64_t ldo, __nv_bfloat16* SA, __nv_bfloat16* SZ, int* esc,
                      int* status, cudaStream_t st) {
  return tc_rotate_t<double>(Xt, ld, nd, ns, Z, ns, ns, Xout, ldo, SA, SZ, esc, status, st);
}
cudaError_t tc_gemm_f64(const double* A, int64_t lda, int64_t m, int k, const double* B,
                        int64_t ldb, int n, double* C, int64_t ldc, __nv_bfloat16* SA,
                        __nv_bfloat16* SZ, int* esc, int* status, cudaStream_t st) {
  return tc_rotate_t<double>(A, lda, m, k, B, ldb, n, C, ldc, SA, SZ, esc, status, st);
}

}  // namespace sparc
