// C ABI of libsparc.so (declared in include/sparc.h): handle set-up, argument
// validation and the orchestration of Algorithm 1 (filtering, projection,
// diagonalisation, rotation) over the kernels of stencil.cu, dense.cu,
// eig.cu and tc_gemm.cu.  All compute runs in those kernels; this file only
// validates, allocates, builds index tables and enqueues work.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <type_traits>
#include <string>
#include <vector>

#include "internal.cuh"

using namespace sparc;

namespace {
std::atomic<long long> g_launches{0};
}  // namespace


void sparc::note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long sparc::launch_count() { return g_launches.load(std::memory_order_relaxed); }

namespace {

thread_local std::string g_create_err;
}  // namespace

void sparc::set_global_error(const std::string& msg) { g_create_err = msg; }

namespace {
constexpr int kMaxDev = 64;
std::atomic<int> g_sms[kMaxDev];
}  // namespace

int sparc::sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 1;
  int v = g_sms[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
    cudaGetLastError();
    return 1;
  }
  g_sms[dev].store(v, std::memory_order_relaxed);
  return v;
}

namespace {
thread_local long long g_wait_cycles = 4000000000LL;
}  // namespace
long long sparc::wait_cycles() { return g_wait_cycles; }
void sparc::set_wait_cycles(long long cycles) { g_wait_cycles = cycles; }

int sparc::smem_optin() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return 48 * 1024;
  }
  return v;
}

cudaError_t sparc::smem_limit_once(unsigned long long* bits, const void* func, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDev)
    return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  const unsigned long long bit = 1ull << dev;
  auto* word = reinterpret_cast<std::atomic<unsigned long long>*>(bits);
  if (word->load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) word->fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

namespace {

// 12th-order central second-derivative weights (Fornberg 1988, radius 6):
// w0 = -5369/1800, w1..w6 = 12/7, -15/56, 10/189, -1/112, 2/1925, -1/16632.
const double kW[kRadius + 1] = {-5369.0 / 1800.0, 12.0 / 7.0,   -15.0 / 56.0,  10.0 / 189.0,
                                -1.0 / 112.0,     2.0 / 1925.0, -1.0 / 16632.0};

// (hi, lo) FP32 pair of a double: hi = nearest float, lo = nearest float to the rest
float2 df_pair(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

struct Fail {
  int code;
};

int cuda_status(cudaError_t e) {
  return e == cudaErrorMemoryAllocation ? SPARC_ERR_OOM : SPARC_ERR_CUDA;
}

#define CK(ctx, expr)                                                               \
  do {                                                                              \
    cudaError_t e_ = (expr);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      (ctx)->err = std::string(#expr) + ": " + cudaGetErrorString(e_);              \
      return cuda_status(e_);                                                       \
    }                                                                               \
  } while (0)

#define ARG(ctx, cond, msg)                         \
  do {                                              \
    if (!(cond)) {                                  \
      (ctx)->err = std::string("invalid argument: ") + (msg); \
      return SPARC_ERR_INVALID_ARG;                 \
    }                                               \
  } while (0)

size_t elem_size(int dtype) { return dtype == SPARC_F32 ? 4 : 8; }

// Device or managed memory.  A failed attribute query (an unregistered host
// pointer) clears only the error it raised, never one left pending before it.
bool is_device_ptr(const void* p) {
  const cudaError_t pending = cudaPeekAtLastError();
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    if (pending == cudaSuccess) cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename T>
int upload(sparc_context* c, const T* host, size_t count, T** dev) {
  *dev = nullptr;
  if (count == 0) count = 1;
  if (c->nl_nmem >= (int)(sizeof(c->nl_mem) / sizeof(c->nl_mem[0]))) {
    c->err = "internal: too many operator tables";
    return SPARC_ERR_CUDA;
  }
  CK(c, cudaMalloc((void**)dev, count * sizeof(T)));
  c->nl_mem[c->nl_nmem++] = *dev;
  if (host) CK(c, cudaMemcpy(*dev, host, count * sizeof(T), cudaMemcpyHostToDevice));
  return SPARC_OK;
}

int check_block(sparc_context* c, const void* X, int ns, int64_t ld, int dtype) {
  ARG(c, X != nullptr, "null orbital block");
  ARG(c, ns >= 1 && ns <= c->ns_max, "ns must be in [1, ns_max]");
  ARG(c, ld >= c->nd, "ld must be >= Nd");
  if (c->kpt) {
    ARG(c, dtype == SPARC_C128, "k-point handles take SPARC_C128 blocks");
    ARG(c, is_device_ptr(X), "k-point handles take device blocks");
    return SPARC_OK;
  }
  int want = c->precision == SPARC_PREC_MIXED ? SPARC_F32 : SPARC_F64;
  ARG(c, dtype == want, "dtype must be SPARC_F64 on FP64 handles and SPARC_F32 on mixed handles");
  return SPARC_OK;
}

template <typename T>
const NlTiles<T>& tiles_of(const sparc_context* c);
template <>
const NlTiles<double>& tiles_of<double>(const sparc_context* c) { return c->tiles64; }
template <>
const NlTiles<float>& tiles_of<float>(const sparc_context* c) { return c->tiles32; }
// The support-point tables exist for the handle's working precision only (FP64
// handles: double, mixed handles: float).
template <typename T>
bool tiles_usable(const sparc_context* c) {
  const bool mixed = c->precision == SPARC_PREC_MIXED;
  return std::is_same<T, float>::value ? (mixed && c->tiles32_ok) : c->tiles64_ok;
}

// Thread shape of the ring stencil for ns orbitals of type T: the fixed one,
// one tuned before for this ns, or the fastest of the shapes that fit the grid
// timed now: one warm-up and two timed launches each, reading the call's own
// input block x (ldx) both as the operand and as the recurrence's previous
// block (as every filter degree after the first reads one) and writing a
// transient buffer, so no live data is touched.  The shapes give bit-identical
// results.  Tuning waits for the stream; during a stream capture the first
// shape is used untimed.
template <typename T>
int ring_shape(sparc_context* c, const T* x, int64_t ldx, int ns, cudaStream_t st, int* shape) {
  *shape = 0;
  const int nsh = ring_num_shapes<T>();
  if (c->shape_fixed >= 0) {
    *shape = std::min(c->shape_fixed, nsh - 1);
    return SPARC_OK;
  }
  for (const auto& e : c->shape_by_ns)
    if (e.first == ns) {
      *shape = e.second;
      return SPARC_OK;
    }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CK(c, cudaStreamIsCapturing(st, &cap));
  if (cap != cudaStreamCaptureStatusNone) return SPARC_OK;
  const T* veff = std::is_same<T, double>::value ? (const T*)c->veff64 : (const T*)c->veff32;
  T* y = nullptr;
  CK(c, cudaMalloc((void**)&y, (size_t)c->ld * ns * sizeof(T)));
  struct Free {
    void* p;
    ~Free() { cudaFree(p); }
  } free_y{y};
  sparc_tuning tu{};
  tu.candidates = std::min(nsh, 8);
  tu.ns = ns;
  float best = 0.f;
  int best_s = -1;
  for (int s_ = 0; s_ < tu.candidates; ++s_) {
    int vy, u, by, th;
    if (!ring_shape_info<T>(c->grid, s_, &vy, &u, &by, &th)) continue;
    float t = 0.f;
    for (int rep = 0; rep < 3; ++rep) {
      bool used = false;
      CK(c, cudaEventRecord(c->ev_tune[0], st));
      CK(c, apply_h_ring<T>(c->grid, c->lap, veff, x, ldx, y, c->ld, x, ldx, ns, 0.0, 1.0,
                            0.0, c->wait_cycles, c->eig.status + 3, st, s_, false, &used));
      CK(c, cudaEventRecord(c->ev_tune[1], st));
      CK(c, cudaEventSynchronize(c->ev_tune[1]));
      if (!used) break;
      float ms = 0.f;
      CK(c, cudaEventElapsedTime(&ms, c->ev_tune[0], c->ev_tune[1]));
      if (rep == 1 || (rep == 2 && ms < t)) t = ms;  // rep 0 warms up
    }
    tu.candidate_ms[s_] = t;
    if (t > 0.f && (best_s < 0 || t < best)) {
      best = t;
      best_s = s_;
    }
  }
  *shape = best_s < 0 ? 0 : best_s;
  c->shape_by_ns.emplace_back(ns, *shape);
  int vy = 0, u = 0, by = 0, th = 0;
  ring_shape_info<T>(c->grid, *shape, &vy, &u, &by, &th);
  tu.shape = *shape;
  tu.rows_per_thread = vy;
  tu.planes_per_step = u;
  tu.slab_rows = by;
  tu.threads = th;
  c->tuning = tu;
  return SPARC_OK;
}

// y = s_h (H - shift) x + s_p prev.  The nonlocal coefficients D of x are in
// c->D when `d_ready`, else they are gathered first (k_nl_coef).  In the split
// form (every handle with support-point tiles of its working precision) the
// local stencil runs first, the TMA ring where the grid and the blocks allow
// it and the generic tiled stencil elsewhere, and the nonlocal term follows by
// support-point tiles; with `want_next` that pass also leaves the
// coefficients of y in c->D (the next recurrence step's D) and sets
// *next_done.  Without tiles (the double-FP32 stencils, the mixed form's FP64
// Yt) the generic stencil adds the nonlocal term point by point.
// Projector entries per grid point above which the FP64 H application in
// double-FP32 arithmetic leaves the nonlocal term to the tiled pass instead of
// adding it point by point (bulk of the benchmark: 1.7; the 10-deep slab: 9.7)
constexpr double kDenseNonlocal = 4.0;

template <typename T>
int hstep(sparc_context* c, const T* x, int64_t ldx, T* y, int64_t ldy, const T* prev,
          int64_t ldp, int ns, double shift, double s_h, double s_p, cudaStream_t st,
          bool d_ready = false, bool want_next = false, bool* next_done = nullptr) {
  const Nonlocal<T>& nl = std::is_same<T, double>::value
                              ? reinterpret_cast<const Nonlocal<T>&>(c->nl64)
                              : reinterpret_cast<const Nonlocal<T>&>(c->nl32);
  const T* veff = std::is_same<T, double>::value ? (const T*)c->veff64 : (const T*)c->veff32;
  T* D = (T*)c->D;
  const double h3 = c->h * c->h * c->h;
  if (next_done) *next_done = false;
  // the split form keeps D projector-major (its nonlocal pass stages rows of
  // orbitals per projector); the fused stencils read it orbital-major
  const bool has_nl = nl.natoms > 0 && nl.kp > 0;
  const bool df = std::is_same<T, double>::value && c->ring_enabled && c->df_stencil;
  const bool split = !has_nl || tiles_usable<T>(c);
  const bool ring = split && !df && c->ring_enabled &&
                    ring_applicable<T>(c->grid, x, ldx, y, ldy, prev, ldp, veff);
  if (df && split && has_nl && c->nl_density > kDenseNonlocal) {
    // overlapping projectors (many entries per point): the double-FP32 ring
    // without its pull-add, then the tiled FP64 nonlocal pass
    if (!d_ready) CK(c, nl_coefficients<T>(nl, h3, x, ldx, ns, D, st, true));
    Nonlocal<double> local = c->nl64;
    local.kp = 0;
    bool used = false;
    CK(c, apply_h_ring_df(c->grid, c->lap, c->veff_df, local, nullptr, (const double*)x, ldx,
                          (double*)y, ldy, (const double*)prev, ldp, ns, shift, s_h, s_p,
                          c->eig.status + 3, st, &used));
    if (used) {
      const NlTiles<T>& t = tiles_of<T>(c);
      T* part = want_next ? (T*)c->part : nullptr;
      CK(c, nl_apply<T>(t, D, nl.kp, y, ldy, ns, s_h, part, st));
      if (want_next) {
        CK(c, nl_reduce<T>(t, part, ns, nl.kp, nl.gamma, h3, D, st));
        if (next_done) *next_done = true;
      }
      return SPARC_OK;
    }
    // the ring does not fit: the split generic form below, D already
    // projector-major
  } else if (df) {
    // the double-FP32 ring reads D orbital-major; where it does not fit the
    // grid, the split form follows (projector-major D) or, without tiles, the
    // fused generic stencil
    CK(c, nl_coefficients<T>(nl, h3, x, ldx, ns, D, st, false));
    bool used = false;
    CK(c, apply_h_ring_df(c->grid, c->lap, c->veff_df, c->nl64, (const double*)D,
                          (const double*)x, ldx, (double*)y, ldy, (const double*)prev, ldp, ns,
                          shift, s_h, s_p, c->eig.status + 3, st, &used));
    if (used) return SPARC_OK;
    if (split && has_nl) CK(c, nl_coefficients<T>(nl, h3, x, ldx, ns, D, st, true));
  } else if (!d_ready || !split) {
    // a D left by the previous degree's tiled pass is projector-major: any
    // other path gathers its own
    CK(c, nl_coefficients<T>(nl, h3, x, ldx, ns, D, st, split));
  }
  if (ring) {
    bool used = false;
    int shape = 0;
    int rc = ring_shape<T>(c, x, ldx, ns, st, &shape);
    if (rc) return rc;
    // kernel timing events of this degree (grown on first use)
    cudaEvent_t* kev = nullptr;
    if (c->kev_on) {
      while ((int)c->kev.size() < c->kev_n + 3) {
        cudaEvent_t e;
        CK(c, cudaEventCreate(&e));
        c->kev.push_back(e);
      }
      kev = c->kev.data() + c->kev_n;
      CK(c, cudaEventRecord(kev[0], st));
    }
    CK(c, apply_h_ring<T>(c->grid, c->lap, veff, x, ldx, y, ldy, prev, ldp, ns, shift, s_h, s_p,
                          c->wait_cycles, c->eig.status + 3, st, shape, c->stall_test, &used));
    if (kev) CK(c, cudaEventRecord(kev[1], st));
    if (used && c->shape_fixed >= 0 && c->tuning.shape != shape) {
      int vy = 0, u = 0, by = 0, th = 0;
      ring_shape_info<T>(c->grid, shape, &vy, &u, &by, &th);
      c->tuning = sparc_tuning{shape, vy, u, by, th, ns, ring_num_shapes<T>(), {}};
    }
    if (used) {
      if (nl.natoms > 0 && nl.kp > 0) {
        const NlTiles<T>& t = tiles_of<T>(c);
        T* part = want_next ? (T*)c->part : nullptr;
        CK(c, nl_apply<T>(t, D, nl.kp, y, ldy, ns, s_h, part, st));
        if (want_next) {
          CK(c, nl_reduce<T>(t, part, ns, nl.kp, nl.gamma, h3, D, st));
          if (next_done) *next_done = true;
        }
      }
      if (kev) {
        CK(c, cudaEventRecord(kev[2], st));
        c->kev_n += 3;
      }
      return SPARC_OK;
    }
    // the ring kernel declined after all: the generic local stencil follows
  }
  if (split) {
    // local part only (slab stencil, in double-FP32 arithmetic where the
    // handle asks for it, or the tiled one on grids it does not fit); the
    // tiled pass adds the nonlocal term
    bool used = false;
    if (df)
      CK(c, apply_h_local_df(c->grid, c->lap, c->veff_df, (const double*)x, ldx, (double*)y, ldy,
                             (const double*)prev, ldp, ns, shift, s_h, s_p, st, &used));
    if (!used)
      CK(c, apply_h_local<T>(c->grid, c->lap, veff, x, ldx, y, ldy, prev, ldp, ns, shift, s_h,
                             s_p, st, &used));
    if (!used) {
      Nonlocal<T> local = nl;
      local.kp = 0;
      CK(c, apply_h<T>(c->grid, c->lap, veff, local, D, x, ldx, y, ldy, prev, ldp, ns, shift, s_h,
                       s_p, st));
    }
    if (has_nl) {
      const NlTiles<T>& t = tiles_of<T>(c);
      T* part = want_next ? (T*)c->part : nullptr;
      CK(c, nl_apply<T>(t, D, nl.kp, y, ldy, ns, s_h, part, st));
      if (want_next) {
        CK(c, nl_reduce<T>(t, part, ns, nl.kp, nl.gamma, h3, D, st));
        if (next_done) *next_done = true;
      }
    }
    return SPARC_OK;
  }
  CK(c, apply_h<T>(c->grid, c->lap, veff, nl, D, x, ldx, y, ldy, prev, ldp, ns, shift, s_h, s_p,
                   st));
  return SPARC_OK;
}

// Chebyshev filter (Algorithm 1, scaled three-term recurrence).  Y_0 = X (ldx);
// Y_i goes to outs[i] (X, W1 or W2).  Returns the buffer holding Y_m; with
// `result_d`, *result_d tells whether c->D holds the nonlocal coefficients of
// Y_m on return (the ring path computes them from the last degree's values).
template <typename T>
int run_filter(sparc_context* c, T* X, int64_t ldx, int ns, int m, double a, double b, double a0,
               bool land_in_workspace, T** result, int64_t* ldr, cudaStream_t st,
               bool* result_d = nullptr) {
  const double e = (b - a) / 2.0, cc = (b + a) / 2.0;
  double sigma = e / (a0 - cc);
  const double sigma1 = sigma, tau = 2.0 / sigma1;
  T* W1 = (T*)c->W1;
  T* W2 = (T*)c->W2;
  // buffer plan: never write the buffer holding Y_{i-1}; writing over Y_{i-2}
  // is allowed (pointwise update).
  std::vector<T*> buf(m + 1);
  std::vector<int64_t> lds(m + 1);
  buf[0] = X;
  lds[0] = ldx;
  for (int i = 1; i <= m; ++i) {
    T* out;
    if (land_in_workspace) {
      if (m % 2 == 1) out = (i % 2 == 1) ? W1 : X;
      else out = (i % 2 == 1) ? W1 : W2;
    } else {
      out = (i % 2 == 1) ? W1 : X;
    }
    buf[i] = out;
    lds[i] = out == X ? ldx : c->ld;
  }
  bool d_ready = false;
  for (int i = 1; i <= m; ++i) {
    int rc;
    const bool want_next = i < m || result_d != nullptr;
    bool next = false;
    if (i == 1) {
      rc = hstep<T>(c, buf[0], lds[0], buf[1], lds[1], nullptr, 0, ns, cc, sigma1 / e, 0.0, st,
                    d_ready, want_next, &next);
    } else {
      double sigma_new = 1.0 / (tau - sigma);
      rc = hstep<T>(c, buf[i - 1], lds[i - 1], buf[i], lds[i], buf[i - 2], lds[i - 2], ns, cc,
                    2.0 * sigma_new / e, -sigma * sigma_new, st, d_ready, want_next, &next);
      sigma = sigma_new;
    }
    if (rc) return rc;
    d_ready = next;
  }
  *result = buf[m];
  *ldr = lds[m];
  if (result_d) *result_d = d_ready;
  return SPARC_OK;
}

int lanczos(sparc_context* c, int iters, uint64_t seed, double* a0, double* b, cudaStream_t st) {
  const int64_t nd = c->nd;
  double* v = c->lz;
  double* w = v + nd;
  double* vp = w + nd;
  double* ab = vp + nd;
  double* partial = ab + 1024;
  double* out2 = partial + 320;
  CK(c, fill_uniform_f64(v, nd, seed, st));
  CK(c, cudaMemsetAsync(vp, 0, nd * sizeof(double), st));
  CK(c, lanczos_normalize(v, w, vp, ab, -1, nd, partial, st));
  for (int j = 0; j < iters; ++j) {
    const Nonlocal<double>& nl = c->nl64;
    CK(c, nl_coefficients<double>(nl, c->h * c->h * c->h, v, nd, 1, c->lz + 3 * nd + 1024 + 384,
                                  st));
    CK(c, apply_h<double>(c->grid, c->lap, c->veff64, nl, c->lz + 3 * nd + 1024 + 384, v, nd, w,
                          nd, nullptr, 0, 1, 0.0, 1.0, 0.0, st));
    CK(c, lanczos_update(w, v, vp, ab, j, nd, st));
    CK(c, lanczos_normalize(v, w, vp, ab, j, nd, partial, st));
  }
  CK(c, lanczos_bounds(ab, iters, out2, st));
  double hb[2];
  CK(c, cudaMemcpyAsync(hb, out2, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(c, cudaStreamSynchronize(st));
  if (!std::isfinite(hb[0]) || !std::isfinite(hb[1])) {
    c->err = "Lanczos produced a non-finite bound";
    return SPARC_ERR_NUMERIC;
  }
  *a0 = hb[0];
  *b = hb[1];
  return SPARC_OK;
}

int read_status(sparc_context* c, cudaStream_t st) {
  int hs[5] = {0, 0, 0, 0, 0};
  CK(c, cudaMemcpyAsync(hs, c->eig.status, 5 * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(c, cudaStreamSynchronize(st));
  if (hs[2] == SPARC_ERR_TIMEOUT || hs[3] == SPARC_ERR_TIMEOUT || hs[4] == SPARC_ERR_TIMEOUT) {
    c->err = hs[2] ? "a bounded wait in a tensor-core GEMM ran out"
                   : hs[3] ? "a bounded wait in the TMA stencil ran out"
                           : "a bounded grid barrier in the eigensolver ran out";
    CK(c, cudaMemsetAsync(c->eig.status + 2, 0, 3 * sizeof(int), st));
    return SPARC_ERR_TIMEOUT;
  }
  if (hs[0] == SPARC_ERR_NOT_SPD) {
    c->err = "subspace overlap Ms is not positive definite";
    return SPARC_ERR_NOT_SPD;
  }
  if (hs[0] || hs[1]) {
    c->err = "non-finite value in the subspace eigensolve";
    return SPARC_ERR_NUMERIC;
  }
  return SPARC_OK;
}

template <typename T>
int do_project(sparc_context* c, const T* Xt, int64_t ldx, const T* Yt, int64_t ldy, int ns,
               double* Hs, double* Ms, cudaStream_t st) {
  // both operands share a leading dimension in the SIMT kernel
  if (ldx != ldy) {
    c->err = "projection operands must share a leading dimension";
    return SPARC_ERR_INVALID_ARG;
  }
  if (c->tc_gemm) {
    int nsplit = tc_project_nsplit(ns);
    CK(c, tc_project(Xt, Yt, ldx, c->nd, ns, Hs, Ms, c->proj_work, nsplit, c->S1, c->S2, c->esc,
                     c->eig.status + 2, st));
    return SPARC_OK;
  }
  int nsplit = project_nsplit(c->nd, ns);
  CK(c, project_simt<T>(Xt, Yt, ldx, c->nd, ns, Hs, Ms, c->proj_work, nsplit, st));
  return SPARC_OK;
}

template <typename T>
int do_rotate(sparc_context* c, const T* Xt, int64_t ldt, int ns, const double* Z, T* Xo,
              int64_t ldo, cudaStream_t st) {
  if (c->tc_gemm) {
    CK(c, tc_rotate(Xt, ldt, c->nd, ns, Z, Xo, ldo, c->S1, c->SZ, c->esc, c->eig.status + 2, st));
    return SPARC_OK;
  }
  CK(c, rotate_simt<T>(Xt, ldt, c->nd, ns, Z, Xo, ldo, st));
  return SPARC_OK;
}

// Mixed precision, Rayleigh-Ritz input: Yt = H Xt evaluated in FP64 from the
// FP32 filtered block, then the projection of (Xt, Yt).  In FP32 the stencil's
// largest terms (~|w0| 3/h^2 |x|) cancel to ~1/10 of themselves in H x, so the
// FP32 operator's rounding alone leaves ~1e-6 Ha in the Ritz values; with Yt in
// FP64 the remaining error is that of the FP32 filtered span (~1e-8 Ha).
// `mid` (optional) is recorded between the two.
int mixed_yt_project(sparc_context* c, const float* Xt, int64_t ldt, int ns, cudaEvent_t mid,
                     cudaStream_t st) {
  // the FP64 copy of Xt lives in the Yt-digit buffer until those digits are made
  double* X64 = reinterpret_cast<double*>(c->S2);
  CK(c, (copy_block<float, double>(Xt, ldt, X64, c->ld, c->nd, ns, st)));
  int rc = hstep<double>(c, X64, c->ld, c->Y64, c->ld, nullptr, 0, ns, 0.0, 1.0, 0.0, st);
  if (rc) return rc;
  if (mid) CK(c, cudaEventRecord(mid, st));
  const int nsplit = tc_project_nsplit(ns);
  CK(c, tc_project(Xt, ldt, c->Y64, c->ld, c->nd, ns, c->Hs, c->Ms, c->proj_work, nsplit, c->S1,
                   c->S2, c->esc, c->eig.status + 2, st));
  return SPARC_OK;
}

// The handle's tensor-core GEMM buffers, lent to the subspace eigensolver (idle
// between the projection and the rotation); null when the handle has none.
EigGemm eig_gemm_of(const sparc_context* c) {
  EigGemm g;
  if (!c->tc_gemm || !c->S1 || !c->SZ || !c->esc) return g;
  const bool f64 = c->precision != SPARC_PREC_MIXED;
  g.SA = c->S1;
  g.SZ = c->SZ;
  g.esc = c->esc;
  g.sa_elems = tc_slice_elems(c->ld, c->nd, c->ns_max, f64);
  g.sz_elems = (size_t)tc_digits(true) * ((c->ns_max + 7) / 8 * 8) * c->ns_max;
  g.esc_bytes = tc_esc_bytes(c->ld, c->nd, c->ns_max);
  g.status = c->eig.status + 2;
  return g;
}

template <typename T>
int do_step(sparc_context* c, T* X, int64_t ldx, int ns, int m, double a, double b, double a0,
            double* eig, int eig_on_host, cudaStream_t st) {
  CK(c, cudaEventRecord(c->ev[1], st));
  T* Xt;
  int64_t ldt;
  // FP64: the last filter degree also leaves the nonlocal coefficients of Xt
  // for Yt = H Xt; mixed precision evaluates Yt in FP64 from its own gather
  const bool f64 = std::is_same<T, double>::value;
  bool xt_d = false;
  c->kev_n = 0;
  c->kev_on = true;
  int rc = run_filter<T>(c, X, ldx, ns, m, a, b, a0, true, &Xt, &ldt, st, f64 ? &xt_d : nullptr);
  c->kev_on = false;
  if (rc) return rc;
  CK(c, cudaEventRecord(c->ev[2], st));
  if (!f64) {
    rc = mixed_yt_project(c, (const float*)Xt, ldt, ns, c->ev[3], st);
  } else {
    T* Yt = Xt == (T*)c->W1 ? (T*)c->W2 : (T*)c->W1;
    rc = hstep<T>(c, Xt, ldt, Yt, c->ld, nullptr, 0, ns, 0.0, 1.0, 0.0, st, xt_d);
    if (rc) return rc;
    CK(c, cudaEventRecord(c->ev[3], st));
    rc = do_project<T>(c, Xt, ldt, Yt, c->ld, ns, c->Hs, c->Ms, st);
  }
  if (rc) return rc;
  CK(c, cudaEventRecord(c->ev[4], st));
  {
    const EigGemm eg = eig_gemm_of(c);
    CK(c, gen_eig(c->eig, c->Hs, c->Ms, ns, c->lam, c->Z, st, &eg));
  }
  CK(c, cudaEventRecord(c->ev[5], st));
  rc = do_rotate<T>(c, Xt, ldt, ns, c->Z, X, ldx, st);
  if (rc) return rc;
  CK(c, cudaEventRecord(c->ev[6], st));
  c->timed = true;
  rc = read_status(c, st);  // synchronises the stream
  if (rc) return rc;
  double lmax;
  CK(c, cudaMemcpy(&lmax, c->lam + ns - 1, sizeof(double), cudaMemcpyDeviceToHost));
  c->have_prev = true;
  c->prev_max = lmax;
  if (eig) {
    if (eig_on_host)
      CK(c, cudaMemcpy(eig, c->lam, ns * sizeof(double), cudaMemcpyDeviceToHost));
    else
      CK(c, cudaMemcpyAsync(eig, c->lam, ns * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  return SPARC_OK;
}

// Stage a host block into the library's staging buffer (dtype elements).
int stage_in(sparc_context* c, const void* X, int ns, int64_t ld, int dtype, void** dev,
             int64_t* ldd, cudaStream_t st) {
  size_t es = elem_size(dtype);
  if (!c->Wstage) CK(c, cudaMalloc(&c->Wstage, (size_t)c->ld * c->ns_max * es));
  CK(c, cudaEventRecord(c->ev_stage[0], st));
  CK(c, cudaMemcpy2DAsync(c->Wstage, c->ld * es, X, ld * es, c->nd * es, ns,
                          cudaMemcpyHostToDevice, st));
  CK(c, cudaEventRecord(c->ev_stage[1], st));
  *dev = c->Wstage;
  *ldd = c->ld;
  return SPARC_OK;
}

int stage_out(sparc_context* c, void* X, int ns, int64_t ld, int dtype, cudaStream_t st) {
  size_t es = elem_size(dtype);
  CK(c, cudaEventRecord(c->ev_stage[2], st));
  CK(c, cudaMemcpy2DAsync(X, ld * es, c->Wstage, c->ld * es, c->nd * es, ns,
                          cudaMemcpyDeviceToHost, st));
  CK(c, cudaEventRecord(c->ev_stage[3], st));
  CK(c, cudaStreamSynchronize(st));
  return SPARC_OK;
}

void destroy_ctx(sparc_context* c) {
  if (!c) return;
  kpoint_free(c);
  for (int i = 0; i < c->nl_nmem; ++i) cudaFree(c->nl_mem[i]);
  cudaFree(c->veff64); cudaFree(c->veff32); cudaFree(c->veff_df);
  cudaFree(c->W1); cudaFree(c->W2); cudaFree(c->Wstage); cudaFree(c->D);
  cudaFree(c->S1); cudaFree(c->S2); cudaFree(c->SZ); cudaFree(c->esc); cudaFree(c->Y64);
  cudaFree(c->part);
  cudaFree(c->Hs); cudaFree(c->Ms); cudaFree(c->Z); cudaFree(c->lam); cudaFree(c->proj_work);
  cudaFree(c->lz);
  eig_free(c->eig);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : c->ev_stage)
    if (e) cudaEventDestroy(e);
  for (auto& e : c->ev_tune)
    if (e) cudaEventDestroy(e);
  for (auto& e : c->kev) cudaEventDestroy(e);
  delete c;
}

int create_impl(const sparc_grid* g, const double* veff, const sparc_nonlocal* nl,
                const sparc_options* opt, sparc_context* c, bool kpoint = false) {
  ARG(c, g != nullptr && veff != nullptr, "grid and veff are required");
  ARG(c, g->nx >= 1 && g->ny >= 1 && g->nz >= 1, "grid sizes must be >= 1");
  ARG(c, g->h > 0.0 && std::isfinite(g->h), "h must be positive");
  for (int d = 0; d < 3; ++d)
    ARG(c, g->bc[d] == SPARC_PERIODIC || g->bc[d] == SPARC_DIRICHLET, "bad boundary condition");
  const int64_t nd = (int64_t)g->nx * g->ny * g->nz;
  ARG(c, nd < (int64_t)1 << 31, "grid too large (Nd must fit in int32)");
  sparc_options o = opt ? *opt : sparc_options{SPARC_PREC_FP64, 1, 0, 0, 0, 0, 0};
  ARG(c, o.precision == SPARC_PREC_FP64 || o.precision == SPARC_PREC_MIXED, "bad precision");
  ARG(c, o.ns_max >= 1 && o.ns_max <= 65535, "ns_max must be in [1, 65535]");
  ARG(c, (o.flags & ~15) == 0 && o.reserved == 0, "unknown option flags or nonzero reserved");
  c->stall_test = (o.flags & 8) != 0;
  ARG(c, o.timeout_cycles >= 0, "timeout_cycles must be >= 0");
  {
    const int nsh = o.precision == SPARC_PREC_MIXED ? ring_num_shapes<float>()
                                                    : ring_num_shapes<double>();
    ARG(c, o.stencil_shape >= 0 && o.stencil_shape <= nsh, "stencil_shape out of range");
  }
  c->shape_fixed = o.stencil_shape - 1;
  if (o.timeout_cycles > 0) c->wait_cycles = o.timeout_cycles;
  c->tuning.shape = -1;
  CK(c, cudaSetDevice(o.device));
  c->device = o.device;
  c->grid.nx = g->nx; c->grid.ny = g->ny; c->grid.nz = g->nz;
  for (int d = 0; d < 3; ++d) c->grid.bc[d] = g->bc[d];
  c->h = g->h;
  c->nd = nd;
  c->ld = (nd + 31) / 32 * 32;
  c->precision = o.precision;
  c->ns_max = o.ns_max;
  const double h2 = g->h * g->h;
  c->lap.diag = -0.5 * 3.0 * kW[0] / h2;
  c->lap.off[0] = 0.0;
  for (int p = 1; p <= kRadius; ++p) c->lap.off[p] = -0.5 * kW[p] / h2;
  for (int64_t i = 0; i < nd; ++i) ARG(c, std::isfinite(veff[i]), "veff must be finite");

  // --- nonlocal tables -----------------------------------------------------
  int natoms = nl ? nl->natoms : 0;
  ARG(c, natoms >= 0, "natoms must be >= 0");
  std::vector<int> proj_ptr32(natoms + 1, 0);
  int64_t nsupp_tot = 0, nchi_tot = 0;
  int kp = 0;
  if (natoms > 0) {
    ARG(c, nl->supp_ptr && nl->supp_idx && nl->nproj && nl->chi_ptr && nl->chi && nl->proj_ptr &&
               nl->gamma, "null nonlocal table");
    ARG(c, nl->supp_ptr[0] == 0 && nl->chi_ptr[0] == 0 && nl->proj_ptr[0] == 0,
        "nonlocal offsets must start at 0");
    for (int J = 0; J < natoms; ++J) {
      int64_t ns_ = nl->supp_ptr[J + 1] - nl->supp_ptr[J];
      ARG(c, ns_ >= 0 && nl->nproj[J] >= 0 && nl->nproj[J] <= 64, "bad support/projector count");
      ARG(c, nl->chi_ptr[J + 1] - nl->chi_ptr[J] == ns_ * nl->nproj[J], "chi_ptr inconsistent");
      ARG(c, nl->proj_ptr[J + 1] - nl->proj_ptr[J] == nl->nproj[J], "proj_ptr inconsistent");
      proj_ptr32[J + 1] = (int)nl->proj_ptr[J + 1];
    }
    nsupp_tot = nl->supp_ptr[natoms];
    nchi_tot = nl->chi_ptr[natoms];
    kp = (int)nl->proj_ptr[natoms];
    for (int64_t t = 0; t < nsupp_tot; ++t)
      ARG(c, nl->supp_idx[t] >= 0 && nl->supp_idx[t] < nd, "support index out of range");
    for (int64_t t = 0; t < nchi_tot; ++t) ARG(c, std::isfinite(nl->chi[t]), "chi must be finite");
    for (int k = 0; k < kp; ++k) ARG(c, std::isfinite(nl->gamma[k]), "gamma must be finite");
  }
  // pull form: per grid point, (projector, chi) entries ordered by atom then projector
  std::vector<int> pull_ptr(nd + 1, 0);
  int64_t nent = 0;
  for (int J = 0; J < natoms; ++J) {
    for (int64_t t = nl->supp_ptr[J]; t < nl->supp_ptr[J + 1]; ++t)
      pull_ptr[nl->supp_idx[t] + 1] += nl->nproj[J];
    nent += (nl->supp_ptr[J + 1] - nl->supp_ptr[J]) * nl->nproj[J];
  }
  ARG(c, nent < (int64_t)1 << 31, "too many projector entries");
  c->nl_density = (double)nent / (double)std::max<int64_t>(nd, 1);
  for (int64_t i = 0; i < nd; ++i) pull_ptr[i + 1] += pull_ptr[i];
  std::vector<int> pull_k(nent > 0 ? nent : 1);
  std::vector<double> pull_chi(nent > 0 ? nent : 1);
  {
    std::vector<int> fill(pull_ptr.begin(), pull_ptr.end() - 1);
    for (int J = 0; J < natoms; ++J) {
      int64_t s0 = nl->supp_ptr[J], nsup = nl->supp_ptr[J + 1] - s0;
      for (int64_t t = 0; t < nsup; ++t) {
        int i = nl->supp_idx[s0 + t];
        for (int q = 0; q < nl->nproj[J]; ++q) {
          int slot = fill[i]++;
          pull_k[slot] = proj_ptr32[J] + q;
          pull_chi[slot] = nl->chi[nl->chi_ptr[J] + q * nsup + t];
        }
      }
    }
  }

  // grouped form of the pull table: G consecutive points per group, one slot
  // per entry of the group's fullest point (missing entries are (0, 0))
  auto build_groups = [&](int G, std::vector<int>& gptr, std::vector<int>& gk,
                          std::vector<double>& gchi) {
    const int64_t ng = (nd + G - 1) / G;
    gptr.assign(ng + 1, 0);
    for (int64_t q = 0; q < ng; ++q) {
      int mx = 0;
      for (int v = 0; v < G; ++v) {
        const int64_t i = q * G + v;
        if (i < nd) mx = std::max(mx, pull_ptr[i + 1] - pull_ptr[i]);
      }
      gptr[q + 1] = gptr[q] + mx;
    }
    const int64_t nslot = gptr[ng];
    gk.assign((size_t)std::max<int64_t>(nslot, 1) * G, 0);
    gchi.assign((size_t)std::max<int64_t>(nslot, 1) * G, 0.0);
    for (int64_t q = 0; q < ng; ++q)
      for (int v = 0; v < G; ++v) {
        const int64_t i = q * G + v;
        if (i >= nd) continue;
        for (int e = pull_ptr[i]; e < pull_ptr[i + 1]; ++e) {
          const int64_t slot = gptr[q] + (e - pull_ptr[i]);
          gk[slot * G + v] = pull_k[e];
          gchi[slot * G + v] = pull_chi[e];
        }
      }
  };

  // --- device copies --------------------------------------------------------
  CK(c, cudaMalloc(&c->veff64, nd * sizeof(double)));
  CK(c, cudaMemcpy(c->veff64, veff, nd * sizeof(double), cudaMemcpyHostToDevice));
  {
    std::vector<float2> vdf(nd);
    for (int64_t i = 0; i < nd; ++i) vdf[i] = df_pair(veff[i]);
    CK(c, cudaMalloc(&c->veff_df, nd * sizeof(float2)));
    CK(c, cudaMemcpy(c->veff_df, vdf.data(), nd * sizeof(float2), cudaMemcpyHostToDevice));
  }
  std::vector<float> f32(std::max<int64_t>(std::max<int64_t>(nd, nent), nchi_tot) + 1);
  if (c->precision == SPARC_PREC_MIXED) {
    for (int64_t i = 0; i < nd; ++i) f32[i] = (float)veff[i];
    CK(c, cudaMalloc(&c->veff32, nd * sizeof(float)));
    CK(c, cudaMemcpy(c->veff32, f32.data(), nd * sizeof(float), cudaMemcpyHostToDevice));
  }
  Nonlocal<double>& n64 = c->nl64;
  n64.natoms = natoms;
  n64.kp = kp;
  if (natoms > 0) {
    int64_t *sp, *cp;
    int *si, *npj, *pp;
    double *chi, *gam;
    int rc;
    if ((rc = upload<int64_t>(c, nl->supp_ptr, natoms + 1, &sp))) return rc;
    if ((rc = upload<int>(c, nl->supp_idx, nsupp_tot, &si))) return rc;
    if ((rc = upload<int>(c, nl->nproj, natoms, &npj))) return rc;
    if ((rc = upload<int64_t>(c, nl->chi_ptr, natoms + 1, &cp))) return rc;
    if ((rc = upload<double>(c, nl->chi, nchi_tot, &chi))) return rc;
    if ((rc = upload<int>(c, proj_ptr32.data(), natoms + 1, &pp))) return rc;
    if ((rc = upload<double>(c, nl->gamma, kp, &gam))) return rc;
    int *pptr, *pk;
    double* pchi;
    if ((rc = upload<int>(c, pull_ptr.data(), nd + 1, &pptr))) return rc;
    if ((rc = upload<int>(c, pull_k.data(), nent, &pk))) return rc;
    if ((rc = upload<double>(c, pull_chi.data(), nent, &pchi))) return rc;
    n64.supp_ptr = sp; n64.supp_idx = si; n64.nproj = npj; n64.chi_ptr = cp; n64.chi = chi;
    n64.proj_ptr = pp; n64.gamma = gam; n64.pull_ptr = pptr; n64.pull_k = pk;
    n64.pull_chi = pchi;
    {
      std::vector<PullEntry<double>> pk64(nent > 0 ? nent : 1);
      for (int64_t t = 0; t < nent; ++t) pk64[t] = PullEntry<double>{pull_k[t], pull_chi[t]};
      PullEntry<double>* d64;
      if ((rc = upload<PullEntry<double>>(c, pk64.data(), pk64.size(), &d64))) return rc;
      n64.pull_pk = d64;
      std::vector<int> gptr, gk;
      std::vector<double> gchi;
      build_groups(2, gptr, gk, gchi);
      int *dgp, *dgk;
      double* dgc;
      if ((rc = upload<int>(c, gptr.data(), gptr.size(), &dgp))) return rc;
      if ((rc = upload<int>(c, gk.data(), gk.size(), &dgk))) return rc;
      if ((rc = upload<double>(c, gchi.data(), gchi.size(), &dgc))) return rc;
      n64.grp = 2;
      n64.grp_ptr = dgp;
      n64.grp_k = dgk;
      n64.grp_chi = dgc;
      std::vector<float2> gdf(gchi.size());
      for (size_t t = 0; t < gchi.size(); ++t) gdf[t] = df_pair(gchi[t]);
      float2* dgdf;
      if ((rc = upload<float2>(c, gdf.data(), gdf.size(), &dgdf))) return rc;
      n64.grp_chi_df = dgdf;
    }
    Nonlocal<float>& n32 = c->nl32;
    n32.natoms = natoms; n32.kp = kp; n32.supp_ptr = sp; n32.supp_idx = si; n32.nproj = npj;
    n32.chi_ptr = cp; n32.proj_ptr = pp; n32.gamma = gam; n32.pull_ptr = pptr; n32.pull_k = pk;
    if (c->precision == SPARC_PREC_MIXED) {
      float *chi32, *pchi32;
      for (int64_t t = 0; t < nchi_tot; ++t) f32[t] = (float)nl->chi[t];
      if ((rc = upload<float>(c, f32.data(), nchi_tot, &chi32))) return rc;
      for (int64_t t = 0; t < nent; ++t) f32[t] = (float)pull_chi[t];
      if ((rc = upload<float>(c, f32.data(), nent, &pchi32))) return rc;
      n32.chi = chi32;
      n32.pull_chi = pchi32;
      std::vector<PullEntry<float>> pk32(nent > 0 ? nent : 1);
      for (int64_t t = 0; t < nent; ++t) pk32[t] = PullEntry<float>{pull_k[t], (float)pull_chi[t]};
      PullEntry<float>* d32;
      if ((rc = upload<PullEntry<float>>(c, pk32.data(), pk32.size(), &d32))) return rc;
      n32.pull_pk = d32;
      std::vector<int> gptr, gk;
      std::vector<double> gchi;
      build_groups(4, gptr, gk, gchi);
      std::vector<float> gchi32(gchi.begin(), gchi.end());
      int *dgp, *dgk;
      float* dgc;
      if ((rc = upload<int>(c, gptr.data(), gptr.size(), &dgp))) return rc;
      if ((rc = upload<int>(c, gk.data(), gk.size(), &dgk))) return rc;
      if ((rc = upload<float>(c, gchi32.data(), gchi32.size(), &dgc))) return rc;
      n32.grp = 4;
      n32.grp_ptr = dgp;
      n32.grp_k = dgk;
      n32.grp_chi = dgc;
    }
    // support-point tiles of the working precision (nonlocal pass of the split
    // form); mixed handles also get FP64 tiles, for their FP64 Yt = H Xt
    NlTilesHost th;
    nl_tiles_build(nd, pull_ptr.data(), pull_k.data(), pull_chi.data(), kp, th);
    const bool mixed = c->precision == SPARC_PREC_MIXED;
    auto put_tiles = [&](auto& t, auto tag) -> int {
      using TT = decltype(tag);
      int r;
      int *tp_, *pt_, *ep_, *ksp, *ksk, *kep, *kpp, *kpr;
      uint16_t *ekl, *kpt;
      TT *ech, *kch;
      std::vector<TT> ec(th.ent_chi.begin(), th.ent_chi.end());
      std::vector<TT> kc(th.kent_chi.begin(), th.kent_chi.end());
      if ((r = upload<int>(c, th.tile_ptr.data(), th.tile_ptr.size(), &tp_))) return r;
      if ((r = upload<int>(c, th.pts.data(), th.pts.size(), &pt_))) return r;
      if ((r = upload<int>(c, th.ent_ptr.data(), th.ent_ptr.size(), &ep_))) return r;
      if ((r = upload<uint16_t>(c, th.ent_kl.data(), th.ent_kl.size(), &ekl))) return r;
      if ((r = upload<TT>(c, ec.data(), ec.size(), &ech))) return r;
      if ((r = upload<int>(c, th.kset_ptr.data(), th.kset_ptr.size(), &ksp))) return r;
      if ((r = upload<int>(c, th.kset_k.data(), th.kset_k.size(), &ksk))) return r;
      if ((r = upload<int>(c, th.kent_ptr.data(), th.kent_ptr.size(), &kep))) return r;
      if ((r = upload<uint16_t>(c, th.kent_pt.data(), th.kent_pt.size(), &kpt))) return r;
      if ((r = upload<TT>(c, kc.data(), kc.size(), &kch))) return r;
      if ((r = upload<int>(c, th.kpair_ptr.data(), th.kpair_ptr.size(), &kpp))) return r;
      if ((r = upload<int>(c, th.kpair.data(), th.kpair.size(), &kpr))) return r;
      t.ntiles = (int)th.tile_ptr.size() - 1;
      t.npairs = (int)th.kset_k.size();
      t.kt_max = th.kt_max;
      t.et_max = th.et_max;
      t.tile_ptr = tp_; t.pts = pt_; t.ent_ptr = ep_; t.ent_kl = ekl; t.ent_chi = ech;
      t.kset_ptr = ksp; t.kset_k = ksk; t.kent_ptr = kep; t.kent_pt = kpt; t.kent_chi = kch;
      t.kpair_ptr = kpp; t.kpair = kpr;
      int optin = 0;
      CK(c, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
      const bool ok = nl_apply_smem(t) <= (size_t)optin;
      (sizeof(TT) == 4 ? c->tiles32_ok : c->tiles64_ok) = ok;
      // one partial-sum buffer serves both precisions (sized for the larger)
      const size_t pb = (size_t)std::max(t.npairs, 1) * c->ns_max * sizeof(TT);
      if (ok && pb > c->part_bytes) {
        cudaFree(c->part);
        c->part = nullptr;
        c->part_bytes = 0;
        CK(c, cudaMalloc(&c->part, pb));
        c->part_bytes = pb;
      }
      return SPARC_OK;
    };
    // (k-point handles keep complex tables of their own, kpoint.cu)
    if (!kpoint && mixed && (rc = put_tiles(c->tiles32, 0.0f))) return rc;
    if (!kpoint && (rc = put_tiles(c->tiles64, 0.0))) return rc;
  }

  // --- workspace ----------------------------------------------------------
  c->ring_enabled = !(opt && (opt->flags & 1));
  // double-FP32 stencil: always for the mixed form's FP64 Yt, opt-in (bit 2)
  // for FP64 handles, whose subspace target needs the full 53 bits
  c->df_stencil = c->precision == SPARC_PREC_MIXED || (opt && (opt->flags & 4));
  // mixed handles always take the tensor-core GEMMs; FP64 handles unless bit 1
  c->tc_gemm = c->precision == SPARC_PREC_MIXED || !(opt && (opt->flags & 2));
  if (kpoint) {  // the complex workspaces are kpoint.cu's; the status words are here
    CK(c, eig_alloc(c->eig, c->ns_max));
    CK(c, cudaMemset(c->eig.status, 0, 16 * sizeof(int)));
    for (auto& e : c->ev) CK(c, cudaEventCreate(&e));
    for (auto& e : c->ev_stage) CK(c, cudaEventCreate(&e));
    for (auto& e : c->ev_tune) CK(c, cudaEventCreate(&e));
    return SPARC_OK;
  }
  const size_t es = c->precision == SPARC_PREC_MIXED ? 4 : 8;
  const size_t blk = (size_t)c->ld * c->ns_max * es;
  CK(c, cudaMalloc(&c->W1, blk));
  CK(c, cudaMalloc(&c->W2, blk));
  CK(c, cudaMemset(c->W1, 0, blk));
  CK(c, cudaMemset(c->W2, 0, blk));
  CK(c, cudaMalloc(&c->D, (size_t)std::max(kp, 1) * c->ns_max * 8));
  const size_t nn = (size_t)c->ns_max * c->ns_max;
  CK(c, cudaMalloc(&c->Hs, nn * 8));
  CK(c, cudaMalloc(&c->Ms, nn * 8));
  CK(c, cudaMalloc(&c->Z, nn * 8));
  CK(c, cudaMalloc(&c->lam, (size_t)c->ns_max * 8));
  int64_t pw = 0;
  for (int n = 1; n <= c->ns_max; ++n) {
    pw = std::max<int64_t>(pw, (int64_t)project_nsplit(nd, n) * 2 * n * n);
    if (c->tc_gemm) pw = std::max<int64_t>(pw, (int64_t)tc_project_nsplit(n) * 2 * n * n);
  }
  if (c->tc_gemm) {
    const bool f64 = c->precision != SPARC_PREC_MIXED;
    const size_t se = tc_slice_elems(c->ld, nd, c->ns_max, f64);
    CK(c, cudaMalloc(&c->S1, se * sizeof(__nv_bfloat16)));
    CK(c, cudaMalloc(&c->S2, se * sizeof(__nv_bfloat16)));
    const size_t zk = (size_t)(c->ns_max + 7) / 8 * 8;
    // six digits whatever the precision: the subspace eigensolver's FP64-accurate
    // products borrow this buffer
    CK(c, cudaMalloc(&c->SZ, (size_t)tc_digits(true) * zk * c->ns_max * sizeof(__nv_bfloat16)));
    CK(c, cudaMalloc(&c->esc, tc_esc_bytes(c->ld, nd, c->ns_max)));
    if (!f64) CK(c, cudaMalloc(&c->Y64, (size_t)c->ld * c->ns_max * sizeof(double)));
  }
  c->proj_work_elems = pw;
  CK(c, cudaMalloc(&c->proj_work, pw * 8));
  CK(c, cudaMalloc(&c->lz, ((size_t)3 * nd + 1024 + 384 + std::max(kp, 1)) * 8));
  CK(c, eig_alloc(c->eig, c->ns_max));
  CK(c, cudaMemset(c->eig.status, 0, 16 * sizeof(int)));
  for (auto& e : c->ev) CK(c, cudaEventCreate(&e));
  for (auto& e : c->ev_stage) CK(c, cudaEventCreate(&e));
  for (auto& e : c->ev_tune) CK(c, cudaEventCreate(&e));
  return SPARC_OK;
}

}  // namespace

extern "C" {

int sparc_create(const sparc_grid* g, const double* veff, const sparc_nonlocal* nl,
                 const sparc_options* opt, sparc_handle* out) {
  if (!out) {
    g_create_err = "invalid argument: out is NULL";
    return SPARC_ERR_INVALID_ARG;
  }
  *out = nullptr;
  sparc_context* c = new sparc_context();
  int rc = create_impl(g, veff, nl, opt, c);
  if (rc) {
    g_create_err = c->err;
    destroy_ctx(c);
    return rc;
  }
  *out = c;
  return SPARC_OK;
}

int sparc_create_kpoint(const sparc_grid* g, const double* veff, const sparc_nonlocal* nl,
                        const double* positions, const sparc_options* opt, const double* kvec,
                        sparc_handle* out) {
  if (!out) {
    g_create_err = "invalid argument: out is NULL";
    return SPARC_ERR_INVALID_ARG;
  }
  *out = nullptr;
  sparc_context* c = new sparc_context();
  int rc = SPARC_OK;
  if (!kvec || !std::isfinite(kvec[0]) || !std::isfinite(kvec[1]) || !std::isfinite(kvec[2])) {
    c->err = "invalid argument: kvec must be three finite numbers";
    rc = SPARC_ERR_INVALID_ARG;
  } else if (opt && (opt->precision != SPARC_PREC_FP64 || opt->ns_max > 1022)) {
    c->err = "invalid argument: k-point handles are FP64 with ns_max <= 1022";
    rc = SPARC_ERR_INVALID_ARG;
  } else if (nl && nl->natoms > 0 && !positions) {
    c->err = "invalid argument: k-point handles with atoms need their positions";
    rc = SPARC_ERR_INVALID_ARG;
  }
  if (!rc) rc = create_impl(g, veff, nl, opt, c, true);
  if (!rc) rc = kpoint_init(c, kvec, positions, nl);
  if (rc) {
    g_create_err = c->err;
    destroy_ctx(c);
    return rc;
  }
  *out = c;
  return SPARC_OK;
}

int sparc_destroy(sparc_handle h) {
  if (!h) return SPARC_OK;
  cudaSetDevice(h->device);
  destroy_ctx(h);
  return SPARC_OK;
}

const char* sparc_last_error(sparc_handle h) {
  return h ? h->err.c_str() : g_create_err.c_str();
}

int sparc_hpsi(sparc_handle c, const void* X, void* Y, int ns, int64_t ld, int dtype,
               void* stream) {
  if (!c) return SPARC_ERR_INVALID_ARG;
  int rc = check_block(c, X, ns, ld, dtype);
  if (rc) return rc;
  ARG(c, Y != nullptr && X != Y, "Y must be non-null and distinct from X");
  ARG(c, is_device_ptr(X) && is_device_ptr(Y), "hpsi takes device blocks");
  CK(c, cudaSetDevice(c->device));
  set_wait_cycles(c->wait_cycles);
  cudaStream_t st = (cudaStream_t)stream;
  if (c->kpt) return kpoint_hpsi(c, X, Y, ns, ld, st);
  // a stencil wait that runs out is reported by the next call that reads status
  CK(c, cudaMemsetAsync(c->eig.status + 3, 0, sizeof(int), st));
  if (dtype == SPARC_F64)
    return hstep<double>(c, (const double*)X, ld, (double*)Y, ld, nullptr, 0, ns, 0.0, 1.0, 0.0, st);
  return hstep<float>(c, (const float*)X, ld, (float*)Y, ld, nullptr, 0, ns, 0.0, 1.0, 0.0, st);
}

int sparc_spectrum_bounds(sparc_handle c, int iters, uint64_t seed, double* a0, double* b,
                          void* stream) {
  if (!c) return SPARC_ERR_INVALID_ARG;
  ARG(c, iters >= 2 && iters <= 512, "iters must be in [2, 512]");
  ARG(c, a0 && b, "null output");
  CK(c, cudaSetDevice(c->device));
  set_wait_cycles(c->wait_cycles);
  if (c->kpt) return kpoint_bounds(c, iters, seed, a0, b, (cudaStream_t)stream);
  return lanczos(c, iters, seed, a0, b, (cudaStream_t)stream);
}

int sparc_cheb_filter(sparc_handle c, void* X, int ns, int64_t ld, int dtype, int degree, double a,
                      double b, double a0, void* stream) {
  if (!c) return SPARC_ERR_INVALID_ARG;
  int rc = check_block(c, X, ns, ld, dtype);
  if (rc) return rc;
  ARG(c, degree >= 1 && degree <= 1000, "degree must be in [1, 1000]");
  ARG(c, std::isfinite(a) && std::isfinite(b) && std::isfinite(a0) && a0 < a && a < b,
      "bounds must satisfy a0 < a < b");
  CK(c, cudaSetDevice(c->device));
  set_wait_cycles(c->wait_cycles);
  cudaStream_t st = (cudaStream_t)stream;
  if (c->kpt) return kpoint_filter(c, X, ns, ld, degree, a, b, a0, st);
  const bool host = !is_device_ptr(X);
  void* Xd = X;
  int64_t ldd = ld;
  CK(c, cudaMemsetAsync(c->eig.status + 3, 0, sizeof(int), st));
  if (host && (rc = stage_in(c, X, ns, ld, dtype, &Xd, &ldd, st))) return rc;
  void* res;
  int64_t ldr;
  if (dtype == SPARC_F64)
    rc = run_filter<double>(c, (double*)Xd, ldd, ns, degree, a, b, a0, false, (double**)&res, &ldr,
                            st);
  else
    rc = run_filter<float>(c, (float*)Xd, ldd, ns, degree, a, b, a0, false, (float**)&res, &ldr,
                           st);
  if (rc) return rc;
  if (res != Xd) {
    if (dtype == SPARC_F64)
      CK(c, copy_block<double>((const double*)res, ldr, (double*)Xd, ldd, c->nd, ns, st));
    else
      CK(c, copy_block<float>((const float*)res, ldr, (float*)Xd, ldd, c->nd, ns, st));
  }
  if (host) return stage_out(c, X, ns, ld, dtype, st);
  return SPARC_OK;
}

int sparc_project(sparc_handle c, const void* Xt, const void* Yt, int ns, int64_t ld, int dtype,
                  double* Hs, double* Ms, void* stream) {
  if (!c) return SPARC_ERR_INVALID_ARG;
  int rc = check_block(c, Xt, ns, ld, dtype);
  if (rc) return rc;
  ARG(c, Yt && Hs && Ms, "null argument");
  CK(c, cudaSetDevice(c->device));
  set_wait_cycles(c->wait_cycles);
  cudaStream_t st = (cudaStream_t)stream;
  if (c->kpt) return kpoint_project(c, Xt, Yt, ns, ld, Hs, Ms, st);
  // the tensor-core form's bounded waits report through the status word, which
  // this call then reads (synchronously); the FP64 SIMT form has no waits
  if (c->tc_gemm) CK(c, cudaMemsetAsync(c->eig.status, 0, 3 * sizeof(int), st));
  if (dtype == SPARC_F64)
    rc = do_project<double>(c, (const double*)Xt, ld, (const double*)Yt, ld, ns, Hs, Ms, st);
  else
    rc = do_project<float>(c, (const float*)Xt, ld, (const float*)Yt, ld, ns, Hs, Ms, st);
  if (rc) return rc;
  return c->tc_gemm ? read_status(c, st) : SPARC_OK;
}

int sparc_subspace_eig(sparc_handle c, const double* Hs, const double* Ms, int ns, double* lam,
                       double* Z, void* stream) {
  if (!c) return SPARC_ERR_INVALID_ARG;
  ARG(c, Hs && Ms && lam && Z, "null argument");
  ARG(c, ns >= 1 && ns <= c->ns_max, "ns must be in [1, ns_max]");
  CK(c, cudaSetDevice(c->device));
  set_wait_cycles(c->wait_cycles);
  cudaStream_t st = (cudaStream_t)stream;
  if (c->kpt) return kpoint_eig(c, Hs, Ms, ns, lam, Z, st);
  CK(c, cudaMemsetAsync(c->eig.status + 2, 0, sizeof(int), st));
  const EigGemm eg = eig_gemm_of(c);
  CK(c, gen_eig(c->eig, Hs, Ms, ns, lam, Z, st, &eg));
  return read_status(c, st);
}

int sparc_rotate(sparc_handle c, const void* Xt, void* Xout, const double* Z, int ns, int64_t ld,
                 int dtype, void* stream) {
  if (!c) return SPARC_ERR_INVALID_ARG;
  int rc = check_block(c, Xt, ns, ld, dtype);
  if (rc) return rc;
  ARG(c, Xout && Z && Xout != Xt, "Xout must be non-null and distinct from Xt");
  CK(c, cudaSetDevice(c->device));
  set_wait_cycles(c->wait_cycles);
  cudaStream_t st = (cudaStream_t)stream;
  if (c->kpt) return kpoint_rotate(c, Xt, Xout, Z, ns, ld, st);
  if (c->tc_gemm) CK(c, cudaMemsetAsync(c->eig.status, 0, 3 * sizeof(int), st));
  if (dtype == SPARC_F64)
    rc = do_rotate<double>(c, (const double*)Xt, ld, ns, Z, (double*)Xout, ld, st);
  else
    rc = do_rotate<float>(c, (const float*)Xt, ld, ns, Z, (float*)Xout, ld, st);
  if (rc) return rc;
  return c->tc_gemm ? read_status(c, st) : SPARC_OK;
}

int sparc_chefsi_step(sparc_handle c, void* X, int ns, int64_t ld, int dtype, int degree,
                      const double* bounds, double* eig, int eig_on_host, void* stream) {
  if (!c) return SPARC_ERR_INVALID_ARG;
  int rc = check_block(c, X, ns, ld, dtype);
  if (rc) return rc;
  ARG(c, degree >= 1 && degree <= 1000, "degree must be in [1, 1000]");
  CK(c, cudaSetDevice(c->device));
  set_wait_cycles(c->wait_cycles);
  cudaStream_t st = (cudaStream_t)stream;
  const auto wall0 = std::chrono::steady_clock::now();
  c->staged = false;
  const long long launches0 = launch_count();
  CK(c, cudaEventRecord(c->ev[0], st));
  CK(c, cudaMemsetAsync(c->eig.status + 2, 0, 2 * sizeof(int), st));
  double a, b, a0;
  if (bounds) {
    a = bounds[0];
    b = bounds[1];
    a0 = bounds[2];
  } else {
    if (!c->have_bounds) {
      rc = c->kpt ? kpoint_bounds(c, 32, 0, &c->a0, &c->b, st) : lanczos(c, 32, 0, &c->a0, &c->b, st);
      if (rc) return rc;
      c->have_bounds = true;
    }
    b = c->b;
    a0 = c->a0;
    a = c->have_prev ? c->prev_max : a0 + 0.1 * (b - a0);
    double lo = a0 + 1e-3 * (b - a0), hi = b - 1e-3 * (b - a0);
    a = std::min(std::max(a, lo), hi);
  }
  ARG(c, std::isfinite(a) && std::isfinite(b) && std::isfinite(a0) && a0 < a && a < b,
      "bounds must satisfy a0 < a < b");
  if (c->kpt) {
    c->kev_n = 0;
    if ((rc = kpoint_step(c, X, ns, ld, degree, a, b, a0, eig, eig_on_host, st))) return rc;
    c->step_launches = launch_count() - launches0;
    c->host_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
    return SPARC_OK;
  }
  const bool host = !is_device_ptr(X);
  void* Xd = X;
  int64_t ldd = ld;
  if (host && (rc = stage_in(c, X, ns, ld, dtype, &Xd, &ldd, st))) return rc;
  if (dtype == SPARC_F64)
    rc = do_step<double>(c, (double*)Xd, ldd, ns, degree, a, b, a0, eig, eig_on_host, st);
  else
    rc = do_step<float>(c, (float*)Xd, ldd, ns, degree, a, b, a0, eig, eig_on_host, st);
  if (rc) return rc;
  c->step_launches = launch_count() - launches0;
  if (host && (rc = stage_out(c, X, ns, ld, dtype, st))) return rc;
  c->staged = host;
  c->host_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0)
                   .count();
  return SPARC_OK;
}

int sparc_get_tuning(sparc_handle c, sparc_tuning* t) {
  if (!c) return SPARC_ERR_INVALID_ARG;
  ARG(c, t != nullptr, "null output");
  *t = c->tuning;
  return SPARC_OK;
}

int sparc_occupations(sparc_handle c, const double* lam, int ns, double ne, double kT,
                      double* occ, double* mu, void* stream) {
  if (!c) return SPARC_ERR_INVALID_ARG;
  ARG(c, ns >= 1, "ns must be >= 1");
  ARG(c, std::isfinite(kT) && kT > 0.0, "kT must be > 0");
  ARG(c, std::isfinite(ne) && ne > 0.0 && ne < 2.0 * ns, "ne must be in (0, 2 ns)");
  ARG(c, lam && occ && mu, "null pointer");
  ARG(c, is_device_ptr(lam) && is_device_ptr(occ) && is_device_ptr(mu),
      "occupations take device arrays");
  CK(c, cudaSetDevice(c->device));
  set_wait_cycles(c->wait_cycles);
  CK(c, fermi_occupations(lam, ns, ne, kT, occ, mu, (cudaStream_t)stream));
  return SPARC_OK;
}

int sparc_density(sparc_handle c, const void* X, int ns, int64_t ld, int dtype, const double* occ,
                  double* rho, void* stream) {
  if (!c) return SPARC_ERR_INVALID_ARG;
  ARG(c, !c->kpt, "sparc_density takes real (Gamma-point) handles");
  ARG(c, ns >= 0 && ns <= c->ns_max, "ns must be in [0, ns_max]");
  ARG(c, ld >= c->nd, "ld must be >= Nd");
  const int want = c->precision == SPARC_PREC_MIXED ? SPARC_F32 : SPARC_F64;
  ARG(c, dtype == want, "dtype must match the handle's precision");
  ARG(c, rho != nullptr && is_device_ptr(rho), "rho must be a device array");
  ARG(c, ns == 0 || (X && occ && is_device_ptr(X) && is_device_ptr(occ)),
      "X and occ must be device arrays");
  CK(c, cudaSetDevice(c->device));
  set_wait_cycles(c->wait_cycles);
  // scratch: the W1 filter buffer (ld x ns_max elements of the handle's type)
  const int64_t work_elems = c->ld * (int64_t)c->ns_max * (int64_t)elem_size(want) / 8;
  CK(c, density(X, ld, c->nd, ns, dtype == SPARC_F32, occ, c->h, rho, (double*)c->W1, work_elems,
                (cudaStream_t)stream));
  return SPARC_OK;
}

int sparc_nonlocal_forces(sparc_handle c, const void* X, int ns, int64_t ld, int dtype,
                          const double* occ, double* F, void* stream) {
  if (!c) return SPARC_ERR_INVALID_ARG;
  ARG(c, !c->kpt, "sparc_nonlocal_forces takes real (Gamma-point) handles");
  ARG(c, ns >= 0 && ns <= c->ns_max, "ns must be in [0, ns_max]");
  ARG(c, ld >= c->nd, "ld must be >= Nd");
  const int want = c->precision == SPARC_PREC_MIXED ? SPARC_F32 : SPARC_F64;
  ARG(c, dtype == want, "dtype must match the handle's precision");
  const int natoms = c->nl64.natoms;
  if (natoms == 0) return SPARC_OK;
  ARG(c, F != nullptr && is_device_ptr(F), "F must be a device array");
  ARG(c, ns == 0 || (X && occ && is_device_ptr(X) && is_device_ptr(occ)),
      "X and occ must be device arrays");
  // scratch: the W1 filter buffer holds natoms x ns x 3 doubles
  const int64_t work_doubles = c->ld * (int64_t)c->ns_max * (int64_t)elem_size(want) / 8;
  ARG(c, (int64_t)natoms * 3 * ns <= work_doubles, "too many atoms for the handle's workspace");
  CK(c, cudaSetDevice(c->device));
  set_wait_cycles(c->wait_cycles);
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == SPARC_F64)
    CK(c, nonlocal_forces<double>(c->grid, c->h, c->nl64, (const double*)X, ld, ns, occ, F,
                                  (double*)c->W1, st));
  else
    CK(c, nonlocal_forces<float>(c->grid, c->h, c->nl64, (const float*)X, ld, ns, occ, F,
                                 (double*)c->W1, st));
  return SPARC_OK;
}

int sparc_get_timings(sparc_handle c, sparc_timings* t) {
  if (!c || !t) return SPARC_ERR_INVALID_ARG;
  ARG(c, c->timed, "no step has run on this handle");
  CK(c, cudaEventSynchronize(c->ev[6]));
  float ms[6];
  for (int i = 0; i < 6; ++i) CK(c, cudaEventElapsedTime(&ms[i], c->ev[i], c->ev[i + 1]));
  t->bounds_ms = ms[0];
  t->filter_ms = ms[1];
  t->hx_ms = ms[2];
  t->project_ms = ms[3];
  t->eig_ms = ms[4];
  t->rotate_ms = ms[5];
  CK(c, cudaEventElapsedTime(&t->total_ms, c->ev[0], c->ev[6]));
  t->launches = c->step_launches;
  t->stage_in_ms = t->stage_out_ms = 0.0f;
  if (c->staged) {
    CK(c, cudaEventElapsedTime(&t->stage_in_ms, c->ev_stage[0], c->ev_stage[1]));
    CK(c, cudaEventElapsedTime(&t->stage_out_ms, c->ev_stage[2], c->ev_stage[3]));
  }
  t->host_ms = (float)c->host_ms;
  t->stencil_ms = t->nonlocal_ms = 0.0f;
  t->stencil_launches = c->kev_n / 3;
  for (int i = 0; i + 2 < c->kev_n; i += 3) {
    float a = 0.f, b = 0.f;
    CK(c, cudaEventElapsedTime(&a, c->kev[i], c->kev[i + 1]));
    CK(c, cudaEventElapsedTime(&b, c->kev[i + 1], c->kev[i + 2]));
    t->stencil_ms += a;
    t->nonlocal_ms += b;
  }
  return SPARC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched CheFSI step over many independent systems (the paper treats the
// eigenproblems of different k-points, spins or configurations as independent,
// Sec. II).  One CUDA graph holds the whole step of every member: each
// member's filter, Yt = H Xt and projection run as one chain of launches (the
// same kernels as sparc_chefsi_step: the TMA ring stencil where the grid
// allows it, the generic tiled stencil elsewhere, the tiled nonlocal pass) on
// one of a pool of forked streams, so that members proceed concurrently and
// fill the GPU together; then one batched eigensolve for all members (a
// thread-block cluster per member); then the rotations, again on the pool.
// The filter's scalars are launch arguments, so the graph is captured again
// (and the executable graph updated in place) when the blocks, sizes, degrees
// or bounds change.
// ---------------------------------------------------------------------------
struct sparc_batch_context {
  std::vector<sparc_context*> hs;
  int precision = SPARC_PREC_FP64;
  int device = 0;
  cudaStream_t cs = nullptr;
  std::vector<cudaStream_t> workers;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr, start = nullptr, stop = nullptr, done = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<int64_t> key;
  long long graph_launches = 0;
  long long last_launches = 0;
  // batched subspace eigensolve of the step: members with ns_max <=
  // kEigBatchMax, grouped by cluster size (one launch per group); the others
  // run gen_eig one by one
  struct EigGroup {
    int cluster, first, count, nmax;
  };
  std::vector<EigGroup> eig_groups;
  std::vector<int> eig_large;
  void* d_eig_items = nullptr;  // the step's table (fixed per batch)
  void* d_eig_call = nullptr;   // table of sparc_batch_subspace_eig calls
  std::string err;
};

namespace {

constexpr int kBatchWorkers = 16;

void batch_free(sparc_batch_context* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  cudaFree(b->d_eig_items);
  cudaFree(b->d_eig_call);
  for (auto s : b->workers) cudaStreamDestroy(s);
  for (auto e : b->joins) cudaEventDestroy(e);
  if (b->cs) cudaStreamDestroy(b->cs);
  for (auto e : {b->fork, b->start, b->stop, b->done})
    if (e) cudaEventDestroy(e);
  delete b;
}

// Groups of the batched eigensolve for problem sizes n[i]: members with
// n <= kEigBatchMax sorted by (cluster size, n) descending into `order`, one
// group per cluster size; the others listed in `large`.
void eig_plan(const std::vector<int>& n, std::vector<int>* order,
              std::vector<sparc_batch_context::EigGroup>* groups, std::vector<int>* large) {
  std::vector<std::pair<int, int>> key;  // (cluster, member)
  for (int i = 0; i < (int)n.size(); ++i) {
    if (n[i] > kEigBatchMax)
      large->push_back(i);
    else
      key.push_back({eig_batch_cluster(n[i]), i});
  }
  std::stable_sort(key.begin(), key.end(), [&](const std::pair<int, int>& a,
                                               const std::pair<int, int>& c) {
    return a.first != c.first ? a.first > c.first : n[a.second] > n[c.second];
  });
  for (size_t q = 0; q < key.size(); ++q) {
    order->push_back(key[q].second);
    if (groups->empty() || groups->back().cluster != key[q].first)
      groups->push_back({key[q].first, (int)q, 0, 0});
    groups->back().count++;
    groups->back().nmax = std::max(groups->back().nmax, n[key[q].second]);
  }
}

template <typename T>
int batch_step_impl(sparc_batch_context* b, void* const* X, const int* ns, const int64_t* ld,
                    const int* degree, const double* bounds, double* const* eig,
                    cudaStream_t caller) {
  const int n = (int)b->hs.size();
  constexpr bool f64 = std::is_same<T, double>::value;
  // per-member bounds, as sparc_chefsi_step takes them
  std::vector<double> A(n), Bv(n), A0(n);
  for (int i = 0; i < n; ++i) {
    sparc_context* c = b->hs[i];
    if (bounds) {
      A[i] = bounds[3 * i];
      Bv[i] = bounds[3 * i + 1];
      A0[i] = bounds[3 * i + 2];
    } else {
      if (!c->have_bounds) {
        int rc = lanczos(c, 32, 0, &c->a0, &c->b, b->cs);
        if (rc) {
          b->err = c->err;
          return rc;
        }
        c->have_bounds = true;
      }
      Bv[i] = c->b;
      A0[i] = c->a0;
      double a = c->have_prev ? c->prev_max : A0[i] + 0.1 * (Bv[i] - A0[i]);
      A[i] = std::min(std::max(a, A0[i] + 1e-3 * (Bv[i] - A0[i])), Bv[i] - 1e-3 * (Bv[i] - A0[i]));
    }
    if (!(A0[i] < A[i] && A[i] < Bv[i])) {
      b->err = "invalid argument: bounds must satisfy a0 < a < b";
      return SPARC_ERR_INVALID_ARG;
    }
  }
  auto bits = [](double v) {
    int64_t r;
    memcpy(&r, &v, sizeof(r));
    return r;
  };
  std::vector<int64_t> key;
  for (int i = 0; i < n; ++i) {
    key.push_back((int64_t)(uintptr_t)X[i]);
    key.push_back(ns[i]);
    key.push_back(ld[i]);
    key.push_back(degree[i]);
    key.push_back(bits(A[i]));
    key.push_back(bits(Bv[i]));
    key.push_back(bits(A0[i]));
  }
  CK(b, cudaEventRecord(b->start, caller));
  CK(b, cudaStreamWaitEvent(b->cs, b->start, 0));
  for (int i = 0; i < n; ++i)
    CK(b, cudaMemsetAsync(b->hs[i]->eig.status, 0, 4 * sizeof(int), b->cs));
  if (!b->exec || key != b->key) {
    // members to streams: largest filter work first, each to the stream with
    // the least work so far
    const int nw = (int)b->workers.size();
    std::vector<int> order(n), lane(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    auto work = [&](int i) { return (double)b->hs[i]->nd * ns[i] * degree[i]; };
    std::stable_sort(order.begin(), order.end(), [&](int p, int q) { return work(p) > work(q); });
    std::vector<double> load(nw, 0.0);
    for (int i : order) {
      const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      lane[i] = w;
      load[w] += work(i);
    }
    auto fork = [&]() {
      cudaEventRecord(b->fork, b->cs);
      for (auto w : b->workers) cudaStreamWaitEvent(w, b->fork, 0);
    };
    auto join = [&]() {
      for (size_t k = 0; k < b->workers.size(); ++k) {
        cudaEventRecord(b->joins[k], b->workers[k]);
        cudaStreamWaitEvent(b->cs, b->joins[k], 0);
      }
    };
    const long long l0 = launch_count();
    CK(b, cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal));
    int rc = SPARC_OK;
    std::vector<T*> xt(n);
    std::vector<int64_t> ldt(n);
    // filter, Yt = H Xt and projection, member by member on its stream
    fork();
    for (int i : order) {
      if (rc) break;
      sparc_context* c = b->hs[i];
      cudaStream_t w = b->workers[lane[i]];
      bool xt_d = false;
      rc = run_filter<T>(c, (T*)X[i], ld[i], ns[i], degree[i], A[i], Bv[i], A0[i], true, &xt[i],
                         &ldt[i], w, f64 ? &xt_d : nullptr);
      if (!rc) {
        if (!f64) {
          rc = mixed_yt_project(c, (const float*)xt[i], ldt[i], ns[i], nullptr, w);
        } else {
          T* Yt = xt[i] == (T*)c->W1 ? (T*)c->W2 : (T*)c->W1;
          rc = hstep<T>(c, xt[i], ldt[i], Yt, c->ld, nullptr, 0, ns[i], 0.0, 1.0, 0.0, w, xt_d);
          if (!rc) rc = do_project<T>(c, xt[i], ldt[i], Yt, c->ld, ns[i], c->Hs, c->Ms, w);
        }
      }
      if (rc) b->err = "system " + std::to_string(i) + ": " + c->err;
    }
    join();
    // batched eigensolve (one launch per cluster size, concurrent)
    fork();
    size_t wk = 0;
    for (const auto& g : b->eig_groups) {
      cudaStream_t w = b->workers[wk++ % b->workers.size()];
      const EigBatchItem* tab = static_cast<const EigBatchItem*>(b->d_eig_items) + g.first;
      if (!rc && eig_batch(tab, g.count, g.cluster, g.nmax, w) != cudaSuccess) {
        rc = SPARC_ERR_CUDA;
        b->err = "batched eigensolve launch failed";
      }
    }
    for (int i : b->eig_large) {
      sparc_context* c = b->hs[i];
      cudaStream_t w = b->workers[wk++ % b->workers.size()];
      const EigGemm eg = eig_gemm_of(c);
      if (!rc && gen_eig(c->eig, c->Hs, c->Ms, ns[i], c->lam, c->Z, w, &eg) != cudaSuccess) {
        rc = SPARC_ERR_CUDA;
        b->err = "eigensolve launch failed";
      }
    }
    join();
    // rotations
    fork();
    for (int i : order) {
      if (rc) break;
      sparc_context* c = b->hs[i];
      rc = do_rotate<T>(c, xt[i], ldt[i], ns[i], c->Z, (T*)X[i], ld[i], b->workers[lane[i]]);
      if (rc) b->err = "system " + std::to_string(i) + ": " + c->err;
    }
    join();
    cudaGraph_t graph;
    cudaError_t ec = cudaStreamEndCapture(b->cs, &graph);
    if (rc) {
      if (ec == cudaSuccess) cudaGraphDestroy(graph);
      return rc;
    }
    CK(b, ec);
    bool updated = false;
    if (b->exec) {
      cudaGraphExecUpdateResultInfo info;
      updated = cudaGraphExecUpdate(b->exec, graph, &info) == cudaSuccess;
      if (!updated) {
        cudaGetLastError();
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
      }
    }
    if (!updated) ec = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(b, ec);
    b->key = key;
    b->graph_launches = launch_count() - l0;
  }
  CK(b, cudaEventRecord(b->stop, b->cs));
  CK(b, cudaGraphLaunch(b->exec, b->cs));
  CK(b, cudaEventRecord(b->done, b->cs));
  CK(b, cudaStreamWaitEvent(caller, b->done, 0));
  b->last_launches = b->graph_launches;
  CK(b, cudaStreamSynchronize(b->cs));
  for (int i = 0; i < n; ++i) {
    sparc_context* c = b->hs[i];
    int rc = read_status(c, b->cs);
    if (rc) {
      b->err = "system " + std::to_string(i) + ": " + c->err;
      return rc;
    }
    double lmax;
    CK(b, cudaMemcpy(&lmax, c->lam + ns[i] - 1, sizeof(double), cudaMemcpyDeviceToHost));
    c->have_prev = true;
    c->prev_max = lmax;
    if (eig && eig[i])
      CK(b, cudaMemcpy(eig[i], c->lam, ns[i] * sizeof(double), cudaMemcpyDeviceToHost));
  }
  return SPARC_OK;
}

}  // namespace

extern "C" {

int sparc_batch_create(const sparc_handle* hs, int n, sparc_batch* out) {
  if (!out) return SPARC_ERR_INVALID_ARG;
  *out = nullptr;
  if (!hs || n < 1) {
    g_create_err = "invalid argument: need n >= 1 handles";
    return SPARC_ERR_INVALID_ARG;
  }
  for (int i = 0; i < n; ++i)
    if (!hs[i] || hs[i]->precision != hs[0]->precision || hs[i]->device != hs[0]->device ||
        hs[i]->kpt) {
      g_create_err = "invalid argument: handles must be non-null real (Gamma-point) handles of "
                     "one precision and device";
      return SPARC_ERR_INVALID_ARG;
    }
  sparc_batch_context* b = new sparc_batch_context();
  b->hs.assign(hs, hs + n);
  b->precision = hs[0]->precision;
  b->device = hs[0]->device;
  auto fail = [&](const char* what, cudaError_t e) {
    g_create_err = std::string(what) + ": " + cudaGetErrorString(e);
    batch_free(b);
    return cuda_status(e);
  };
  cudaError_t e = cudaSetDevice(b->device);
  if (e != cudaSuccess) return fail("cudaSetDevice", e);
  if ((e = cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking)) != cudaSuccess)
    return fail("cudaStreamCreate", e);
  const int nw = std::min(kBatchWorkers, n);
  for (int k = 0; k < nw; ++k) {
    cudaStream_t s;
    cudaEvent_t j;
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess)
      return fail("cudaStreamCreate", e);
    b->workers.push_back(s);
    if ((e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming)) != cudaSuccess)
      return fail("cudaEventCreate", e);
    b->joins.push_back(j);
  }
  for (cudaEvent_t* ev : {&b->fork, &b->start, &b->done})
    if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess)
      return fail("cudaEventCreate", e);
  if ((e = cudaEventCreate(&b->stop)) != cudaSuccess) return fail("cudaEventCreate", e);
  // the step's batched eigensolve: each member solves its ns_max problem in
  // its own subspace buffers and eigensolver workspace
  std::vector<int> nsz(n), order;
  for (int i = 0; i < n; ++i) nsz[i] = hs[i]->ns_max;
  eig_plan(nsz, &order, &b->eig_groups, &b->eig_large);
  std::vector<EigBatchItem> tab;
  for (int i : order) {
    sparc_context* c = hs[i];
    tab.push_back(eig_batch_item(c->eig, c->Hs, c->Ms, c->ns_max, c->lam, c->Z));
  }
  const size_t tb = std::max<size_t>(1, (size_t)n) * sizeof(EigBatchItem);
  if ((e = cudaMalloc(&b->d_eig_items, tb)) != cudaSuccess) return fail("cudaMalloc", e);
  if ((e = cudaMalloc(&b->d_eig_call, tb)) != cudaSuccess) return fail("cudaMalloc", e);
  if (!tab.empty() &&
      (e = cudaMemcpy(b->d_eig_items, tab.data(), tab.size() * sizeof(EigBatchItem),
                      cudaMemcpyHostToDevice)) != cudaSuccess)
    return fail("cudaMemcpy", e);
  *out = b;
  return SPARC_OK;
}

int sparc_batch_destroy(sparc_batch b) {
  if (!b) return SPARC_OK;
  cudaSetDevice(b->device);
  batch_free(b);
  return SPARC_OK;
}

const char* sparc_batch_last_error(sparc_batch b) { return b ? b->err.c_str() : ""; }

int sparc_batch_chefsi_step(sparc_batch b, void* const* X, const int* ns, const int64_t* ld,
                            int dtype, const int* degree, const double* bounds,
                            double* const* eig, void* stream) {
  if (!b) return SPARC_ERR_INVALID_ARG;
  ARG(b, X && ns && ld && degree, "null argument");
  const int n = (int)b->hs.size();
  for (int i = 0; i < n; ++i) {
    sparc_context* c = b->hs[i];
    ARG(b, X[i] && is_device_ptr(X[i]), "batched blocks must be device pointers");
    ARG(b, ns[i] == c->ns_max, "batch members run with ns equal to their handle's ns_max");
    ARG(b, ld[i] >= c->nd, "ld must be >= Nd");
    ARG(b, degree[i] >= 1 && degree[i] <= 1000, "degree must be in [1, 1000]");
  }
  const int want = b->precision == SPARC_PREC_MIXED ? SPARC_F32 : SPARC_F64;
  ARG(b, dtype == want, "dtype does not match the handles' precision");
  CK(b, cudaSetDevice(b->device));
  // the members' kernels wait as long as the first member's handle allows
  set_wait_cycles(b->hs.empty() ? 4000000000LL : b->hs[0]->wait_cycles);
  if (dtype == SPARC_F64)
    return batch_step_impl<double>(b, X, ns, ld, degree, bounds, eig, (cudaStream_t)stream);
  return batch_step_impl<float>(b, X, ns, ld, degree, bounds, eig, (cudaStream_t)stream);
}

int sparc_batch_get_info(sparc_batch b, int64_t* launches_per_step) {
  if (!b || !launches_per_step) return SPARC_ERR_INVALID_ARG;
  *launches_per_step = b->last_launches;
  return SPARC_OK;
}

int sparc_batch_subspace_eig(sparc_batch b, const double* const* Hs, const double* const* Ms,
                             const int* ns, double* const* lam, double* const* Z,
                             void* stream) {
  if (!b) return SPARC_ERR_INVALID_ARG;
  ARG(b, Hs && Ms && ns && lam && Z, "null argument");
  const int n = (int)b->hs.size();
  std::vector<int> nsz(n);
  for (int i = 0; i < n; ++i) {
    sparc_context* c = b->hs[i];
    ARG(b, ns[i] >= 1 && ns[i] <= c->ns_max, "ns[i] must be in [1, member i's ns_max]");
    ARG(b, is_device_ptr(Hs[i]) && is_device_ptr(Ms[i]) && is_device_ptr(lam[i]) &&
               is_device_ptr(Z[i]),
        "Hs, Ms, lam and Z must be device pointers");
    nsz[i] = ns[i];
  }
  CK(b, cudaSetDevice(b->device));
  set_wait_cycles(b->hs[0]->wait_cycles);
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int> order, large;
  std::vector<sparc_batch_context::EigGroup> groups;
  eig_plan(nsz, &order, &groups, &large);
  std::vector<EigBatchItem> tab;
  for (int i : order)
    tab.push_back(eig_batch_item(b->hs[i]->eig, Hs[i], Ms[i], ns[i], lam[i], Z[i]));
  for (int i = 0; i < n; ++i)
    CK(b, cudaMemsetAsync(b->hs[i]->eig.status, 0, 5 * sizeof(int), st));
  if (!tab.empty())
    CK(b, cudaMemcpyAsync(b->d_eig_call, tab.data(), tab.size() * sizeof(EigBatchItem),
                          cudaMemcpyHostToDevice, st));
  for (const auto& g : groups)
    CK(b, eig_batch(static_cast<const EigBatchItem*>(b->d_eig_call) + g.first, g.count,
                    g.cluster, g.nmax, st));
  for (int i : large) {
    const EigGemm eg = eig_gemm_of(b->hs[i]);
    CK(b, gen_eig(b->hs[i]->eig, Hs[i], Ms[i], ns[i], lam[i], Z[i], st, &eg));
  }
  CK(b, cudaStreamSynchronize(st));
  for (int i = 0; i < n; ++i) {
    sparc_context* c = b->hs[i];
    int rc = read_status(c, st);
    if (rc) {
      b->err = "system " + std::to_string(i) + ": " + c->err;
      return rc;
    }
  }
  return SPARC_OK;
}

}  // extern "C"
