// Internal declarations shared by the CUDA translation units of libsparc.so.
// Nothing here is part of the public C ABI (see include/sparc.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sparc.h"

namespace sparc {

// Counts kernel launches made by the library (host side, every launch site).
void note_launch();
long long launch_count();

// Message returned by sparc_last_error(NULL) (calls made without a handle).
void set_global_error(const std::string& msg);

// Number of SMs of the current device (queried once per device; 1 if the query
// fails, so grid sizing stays valid).
int sm_count();
// Bound of every device-side wait (SM clock cycles) for the kernels the calling
// host thread launches next; set by each C entry point from its handle.
long long wait_cycles();
void set_wait_cycles(long long cycles);
// Lower bound of the waits with which a stopping kernel lets its own copies
// and tensor-core operations in flight land before it exits (about 0.1 s),
// whatever the wait bound above: those complete on their own.
constexpr long long kDrainCycles = 200000000LL;

// Largest dynamic shared memory a CTA may opt into on the current device.
int smem_optin();
// Sets a kernel's dynamic shared-memory limit on the current device, once per
// device per `bits` word (one word per kernel instantiation).
cudaError_t smem_limit_once(unsigned long long* bits, const void* func, int bytes);

constexpr int kRadius = 6;  // 12th-order central FD Laplacian (radius 6)

struct Grid {
  int nx, ny, nz;
  int bc[3];  // SPARC_PERIODIC / SPARC_DIRICHLET
};

// -1/2 Laplacian coefficients: diag = -1/2 * 3 w0 / h^2, off[p] = -1/2 w_p / h^2.
struct LapCoef {
  double diag;
  double off[kRadius + 1];  // off[0] unused
};

// Nonlocal tables on the device.
//  Gather form (per atom): support indices and the n_supp x nproj chi block,
//  used to form D[n][k] = gamma_k h^3 sum_s chi[s][k] x[idx_s] for all
//  projectors k (global numbering proj_ptr[J] + q).
//  Pull form (per grid point i): entries pull_ptr[i]..pull_ptr[i+1]-1 hold
//  (k, chi_k(i)) so that (V_nl x)_i = sum_e chi_e D[k_e].
// One pull-table entry: projector index k and chi_k(i) in one aligned load.
template <typename T>
struct PullEntry {
  int k;
  T chi;
};

template <typename T>
struct Nonlocal {
  int natoms = 0;
  int kp = 0;  // total projector count
  const int64_t* supp_ptr = nullptr;
  const int* supp_idx = nullptr;
  const int* nproj = nullptr;
  const int64_t* chi_ptr = nullptr;
  const T* chi = nullptr;
  const int* proj_ptr = nullptr;  // int32 copy of proj_ptr
  const double* gamma = nullptr;
  const int* pull_ptr = nullptr;
  const int* pull_k = nullptr;
  const T* pull_chi = nullptr;
  const PullEntry<T>* pull_pk = nullptr;  // packed (k, chi) entries, same order
  // The same entries by groups of `grp` consecutive grid points (grp = 4 for
  // FP32, 2 for FP64): group q owns slots grp_ptr[q] .. grp_ptr[q + 1] - 1, as
  // many as its fullest point has entries; slot s holds for each point v of
  // the group its s-th (k, chi), or (0, 0) where the point has fewer.
  int grp = 0;
  const int* grp_ptr = nullptr;
  const int* grp_k = nullptr;   // slots x grp
  const T* grp_chi = nullptr;   // slots x grp
  const float2* grp_chi_df = nullptr;  // FP64 tables: chi as (hi, lo) FP32 pairs
};

// Launchers (stencil.cu) -------------------------------------------------
// Generic form: y = s_h * ((H - shift) x) + s_p * prev   (prev may be null: s_p
// ignored) with D the nonlocal coefficients of x (computed by nl_coefficients),
// the nonlocal pull-add fused in.
template <typename T>
cudaError_t apply_h(const Grid& g, const LapCoef& lc, const T* veff, const Nonlocal<T>& nl,
                    const T* D, const T* x, int64_t ldx, T* y, int64_t ldy, const T* prev,
                    int64_t ldp, int ns, double shift, double s_h, double s_p, cudaStream_t st);
// Generic local part only (stencil.cu), any grid with nx >= kRadius:
// y = s_h ((-1/2 Lap + Veff - shift) x) + s_p prev by y-slabs of whole rows;
// the nonlocal term follows with nl_apply.  *used = false when the grid does
// not fit it (nx < kRadius or too wide a row).
template <typename T>
cudaError_t apply_h_local(const Grid& g, const LapCoef& lc, const T* veff, const T* x,
                          int64_t ldx, T* y, int64_t ldy, const T* prev, int64_t ldp, int ns,
                          double shift, double s_h, double s_p, cudaStream_t st, bool* used);
// The same in double-FP32 arithmetic for FP64 blocks (stencil_df.cu), the
// local part of the FP64 H application where the double-FP32 ring does not
// fit the grid (veff_df: Veff as pairs).
cudaError_t apply_h_local_df(const Grid& g, const LapCoef& lc, const float2* veff_df,
                             const double* x, int64_t ldx, double* y, int64_t ldy,
                             const double* prev, int64_t ldp, int ns, double shift, double s_h,
                             double s_p, cudaStream_t st, bool* used);
// TMA plane-ring form (stencil_tma.cu) of the local part only:
// y = s_h ((-1/2 Lap + Veff - shift) x) + s_p prev; the nonlocal term follows
// with nl_apply.  *used = false when the grid or the buffers do not fit it.
// `status` (device int) receives SPARC_ERR_TIMEOUT if a bounded wait (of
// `wait_cycles` SM clock cycles) runs out.
// `shape` selects one of ring_num_shapes<T>() thread shapes (rows per thread,
// planes per step, CTA size); all give bit-identical results.
template <typename T>
cudaError_t apply_h_ring(const Grid& g, const LapCoef& lc, const T* veff, const T* x, int64_t ldx,
                         T* y, int64_t ldy, const T* prev, int64_t ldp, int ns, double shift,
                         double s_h, double s_p, long long wait_cycles, int* status,
                         cudaStream_t st, int shape, bool stall, bool* used);
// Whether the ring form runs for these buffers on this grid (some shape fits,
// vector alignment, the tensor-map encoder is available).
template <typename T>
bool ring_applicable(const Grid& g, const T* x, int64_t ldx, const T* y, int64_t ldy,
                     const T* prev, int64_t ldp, const T* veff);
template <typename T>
int ring_num_shapes();
// rows per thread, planes per step, slab rows and threads of a shape on a grid
// (false if that shape does not fit the grid)
template <typename T>
bool ring_shape_info(const Grid& g, int shape, int* vy, int* u, int* by, int* threads);
// Ring plan (stencil_tma.cu): slab rows, ring slots, slot bytes and threads for
// a grid and element type, or false when the generic kernel must run.
template <typename T>
bool ring_plan(const Grid& g, int kp, int& by, int& slots, uint32_t& slot_bytes, int& threads);
// FP64 blocks in double-FP32 arithmetic (stencil_df.cu); *used = false when
// the grid or the buffers do not fit the ring form.
cudaError_t apply_h_ring_df(const Grid& g, const LapCoef& lc, const float2* veff_df,
                            const Nonlocal<double>& nl, const double* D, const double* x,
                            int64_t ldx, double* y, int64_t ldy, const double* prev, int64_t ldp,
                            int ns, double shift, double s_h, double s_p, int* status,
                            cudaStream_t st, bool* used);

// Nonlocal term by tiles of support points (nonlocal.cu) -----------------
constexpr int kTilePts = 256;  // support points per tile (= threads per CTA)
template <typename T>
struct NlTiles {
  int ntiles = 0, npairs = 0, kt_max = 0, et_max = 0;  // projectors, entries per tile (max)
  const int* tile_ptr = nullptr;      // ntiles + 1: each tile's range in pts
  const int* pts = nullptr;           // support points (grid indices), ascending
  const int* ent_ptr = nullptr;       // per support point: range of its entries
  const uint16_t* ent_kl = nullptr;   // entry's tile-local projector index
  const T* ent_chi = nullptr;         // entry's chi_k(i)
  const int* kset_ptr = nullptr;      // ntiles + 1: each tile's (tile, k) pairs
  const int* kset_k = nullptr;        // global projector index of each pair
  const int* kent_ptr = nullptr;      // npairs + 1: entries of each pair
  const uint16_t* kent_pt = nullptr;  // tile-local point index (ascending)
  const T* kent_chi = nullptr;
  const int* kpair_ptr = nullptr;     // kp + 1: pairs of each projector
  const int* kpair = nullptr;         // pair indices, ascending (tile order)
};
struct NlTilesHost {
  int tp = 0, kt_max = 0, et_max = 0;
  std::vector<int> tile_ptr, pts, ent_ptr, kset_ptr, kset_k, kent_ptr, kpair_ptr, kpair;
  std::vector<uint16_t> ent_kl, kent_pt;
  std::vector<double> ent_chi, kent_chi;
};
// Tiles of the support points of the pull table (per grid point: entries
// pull_ptr[i] .. pull_ptr[i + 1] - 1 of (pull_k, pull_chi)).
void nl_tiles_build(int64_t nd, const int* pull_ptr, const int* pull_k, const double* pull_chi,
                    int kp, NlTilesHost& out);
template <typename T>
size_t nl_apply_smem(const NlTiles<T>& t);
// y_i += s_h sum_k chi_k(i) D[k ns + n] (projector-major D) at the support
// points of all ns orbitals; with `part` (npairs x ns) also the per-tile
// partial sums of chi_k^T y for nl_reduce.
template <typename T>
cudaError_t nl_apply(const NlTiles<T>& t, const T* D, int kp, T* y, int64_t ldy, int ns,
                     double s_h, T* part, cudaStream_t st);
// D[k ns + n] = gamma_k h3 sum over the tiles of k of part (tile order)
template <typename T>
cudaError_t nl_reduce(const NlTiles<T>& t, const T* part, int ns, int kp, const double* gamma,
                      double h3, T* D, cudaStream_t st);

// D = gamma_k h^3 sum_s chi[s][k] x[idx_s + n ldx], orbital-major at
// D[n * kp + k] (the fused stencils), or projector-major at D[k * ns + n] with
// `kmajor` (the nonlocal pass by support-point tiles)
template <typename T>
cudaError_t nl_coefficients(const Nonlocal<T>& nl, double h3, const T* x, int64_t ldx, int ns,
                            T* D, cudaStream_t st, bool kmajor = false);

// Small vector kernels (stencil.cu): deterministic two-pass reductions.
cudaError_t dot_f64(const double* u, const double* v, int64_t n, double* partial, double* out,
                    cudaStream_t st);
cudaError_t fill_uniform_f64(double* v, int64_t n, uint64_t seed, cudaStream_t st);
// n complex entries (interleaved): real part u(seed, i) - 1/2, imaginary part 0
cudaError_t fill_uniform_re_c128(double* v, int64_t n, uint64_t seed, cudaStream_t st);
cudaError_t lanczos_update(double* w, const double* v, double* vp, const double* alpha_beta,
                           int j, int64_t n, cudaStream_t st);
cudaError_t lanczos_normalize(double* v, double* w, double* vp, double* alpha_beta, int j,
                              int64_t n, double* partial, cudaStream_t st);
cudaError_t lanczos_bounds(const double* alpha_beta, int k, double* out2, cudaStream_t st);
// dst = src column by column (the element type may widen, e.g. FP32 -> FP64)
template <typename T, typename U = T>
cudaError_t copy_block(const T* src, int64_t lds, U* dst, int64_t ldd, int64_t nd, int ns,
                       cudaStream_t st);

// Dense FP64 kernels (dense.cu) -------------------------------------------
// Hs = Xt^T Yt, Ms = Xt^T Xt (upper tiles + mirror), split-K with a
// deterministic reduction.  `work` holds nsplit * ns * ns * 2 doubles.
template <typename T>
cudaError_t project_simt(const T* Xt, const T* Yt, int64_t ld, int64_t nd, int ns, double* Hs,
                         double* Ms, double* work, int nsplit, cudaStream_t st);
int project_nsplit(int64_t nd, int ns);
// Sum the nsplit partials work[s][{H, M}][ns x ns] of the upper elements, mirror.
cudaError_t project_reduce(const double* work, int nsplit, int ns, double* Hs, double* Ms,
                           cudaStream_t st);

// Split-precision tensor-core GEMMs (tc_gemm.cu): FP32 operands take 4 BF16
// digits (mixed precision), FP64 operands 6 digits (FP64-accurate).
int tc_digits(bool fp64);
size_t tc_slice_elems(int64_t ld, int64_t nd, int ns_max, bool fp64);
size_t tc_esc_bytes(int64_t ld, int64_t nd, int ns_max);
int tc_project_nsplit(int ns);
// `esc`: workspace of tc_esc_bytes() bytes (block exponents).
cudaError_t tc_project(const float* Xt, const float* Yt, int64_t ld, int64_t nd, int ns,
                       double* Hs, double* Ms, double* work, int nsplit, __nv_bfloat16* SX,
                       __nv_bfloat16* SY, int* esc, int* status, cudaStream_t st);
// mixed precision with an FP64 Yt (4 digits of each operand)
cudaError_t tc_project(const float* Xt, int64_t ldx, const double* Yt, int64_t ldy, int64_t nd,
                       int ns, double* Hs, double* Ms, double* work, int nsplit,
                       __nv_bfloat16* SX, __nv_bfloat16* SY, int* esc, int* status,
                       cudaStream_t st);
cudaError_t tc_project(const double* Xt, const double* Yt, int64_t ld, int64_t nd, int ns,
                       double* Hs, double* Ms, double* work, int nsplit, __nv_bfloat16* SX,
                       __nv_bfloat16* SY, int* esc, int* status, cudaStream_t st);
cudaError_t tc_rotate(const float* Xt, int64_t ld, int64_t nd, int ns, const double* Z,
                      float* Xout, int64_t ldo, __nv_bfloat16* SA, __nv_bfloat16* SZ, int* esc,
                      int* status, cudaStream_t st);
cudaError_t tc_rotate(const double* Xt, int64_t ld, int64_t nd, int ns, const double* Z,
                      double* Xout, int64_t ldo, __nv_bfloat16* SA, __nv_bfloat16* SZ, int* esc,
                      int* status, cudaStream_t st);
// C (m x n, ldc) = A (m x k, lda) B (k x n, ldb), FP64-accurate six-digit split
// (SA: 6 MP ldk digits, MP = m rounded up to 128, ldk = k rounded up to 8; SZ:
// 6 n ldk digits; esc: exponent tables of the rotation form)
cudaError_t tc_gemm_f64(const double* A, int64_t lda, int64_t m, int k, const double* B,
                        int64_t ldb, int n, double* C, int64_t ldc, __nv_bfloat16* SA,
                        __nv_bfloat16* SZ, int* esc, int* status, cudaStream_t st);

// density.cu: Fermi occupations (one block) and rho = (2/h^3) sum f_n x_n^2.
cudaError_t fermi_occupations(const double* lam, int ns, double ne, double kT, double* occ,
                              double* mu, cudaStream_t st);
// Nonlocal forces F (natoms x 3 doubles) of the orbitals X (forces.cu); `part`
// is scratch of natoms * ns * 3 doubles.
template <typename T>
cudaError_t nonlocal_forces(const Grid& g, double h, const Nonlocal<double>& nl, const T* X,
                            int64_t ld, int ns, const double* occ, double* F, double* part,
                            cudaStream_t st);
cudaError_t density(const void* X, int64_t ld, int64_t nd, int ns, bool fp32, const double* occ,
                    double h, double* rho, double* work, int64_t work_elems, cudaStream_t st);
// Xout = Xt Z (Z column-major ns x ns)
template <typename T>
cudaError_t rotate_simt(const T* Xt, int64_t ld, int64_t nd, int ns, const double* Z, T* Xout,
                        int64_t ldo, cudaStream_t st);

// Generalised symmetric eigensolver workspace and driver (eig.cu).
struct EigWork {
  int nmax = 0;
  double* L = nullptr;     // Cholesky factor (col-major)
  double* A = nullptr;     // reduced matrix / Householder vectors (row-major)
  double* W = nullptr;     // scratch n x n
  double* V = nullptr;     // eigenvectors of T then of A (row-major)
  double* d = nullptr;     // tridiagonal diagonal
  double* e = nullptr;     // tridiagonal off-diagonal
  double* tau = nullptr;   // Householder scalars
  double* lu = nullptr;    // inverse-iteration factors (4 n x n)
  double* scal = nullptr;  // small scalars
  int* status = nullptr;   // device status word
  int* clus = nullptr;     // cluster bookkeeping (2 n ints)
  int* piv = nullptr;      // inverse-iteration pivot flags (n x n ints)
  double* X0 = nullptr;    // tensor-core mode: triangular inverses (n x n each)
  double* X1 = nullptr;
};
cudaError_t eig_alloc(EigWork& w, int nmax);
void eig_free(EigWork& w);
// Digit buffers of the FP64-accurate tensor-core GEMM (tc_rotate) that the
// eigensolver may borrow for its O(n^3) products (the handle's projection /
// rotation workspace); sa_elems / sz_elems are their sizes in BF16 elements.
struct EigGemm {
  __nv_bfloat16* SA = nullptr;
  __nv_bfloat16* SZ = nullptr;
  int* esc = nullptr;
  size_t sa_elems = 0, sz_elems = 0, esc_bytes = 0;
  int* status = nullptr;  // status word of the GEMM's bounded waits
};
// lam ascending, Z column-major with Z^T M Z = I. Writes *dev_status (device).
// With `g` (and n >= 256, buffers large enough) the reduction to standard form,
// the re-orthonormalisation and the back-substitution run as tensor-core GEMMs
// with an explicit triangular inverse.
cudaError_t gen_eig(EigWork& w, const double* Hs, const double* Ms, int n, double* lam, double* Z,
                    cudaStream_t st, const EigGemm* g = nullptr);

// Batched form of gen_eig: one launch solves many independent problems, each
// by one thread-block cluster (eig_batch_cluster(n) CTAs) that runs all steps
// of gen_eig with cluster barriers between them.  Every problem of one launch
// uses the same cluster size; n <= kEigBatchMax.  The table lives in device
// memory; each entry's work buffers come from an EigWork of nmax >= n.
constexpr int kEigBatchMax = 512;
struct EigBatchItem {
  const double* Hs;
  const double* Ms;
  double* lam;
  double* Z;
  double* L;
  double* A;
  double* W;
  double* V;
  double* lu;
  double* d;
  double* e;
  double* tau;
  double* scal;
  int* status;
  int* clus;
  int* piv;
  int n;
  int pad;
};
EigBatchItem eig_batch_item(const EigWork& w, const double* Hs, const double* Ms, int n,
                            double* lam, double* Z);
// CTAs per problem of size n, reduced if the device cannot co-schedule them
int eig_batch_cluster(int n);
// items: device table of `count` entries, largest n first; nmax = max n
cudaError_t eig_batch(const EigBatchItem* items, int count, int cluster, int nmax,
                      cudaStream_t st);

// Complex step at a Bloch wavevector (kpoint.cu) ---------------------------
struct KpointState;
// builds the phased projector tables and complex workspaces of a k-point handle
int kpoint_init(sparc_context* c, const double kvec[3], const double* positions,
                const sparc_nonlocal* nl);
void kpoint_free(sparc_context* c);
int kpoint_hpsi(sparc_context* c, const void* X, void* Y, int ns, int64_t ld, cudaStream_t st);
int kpoint_bounds(sparc_context* c, int iters, uint64_t seed, double* a0, double* b,
                  cudaStream_t st);
int kpoint_filter(sparc_context* c, void* X, int ns, int64_t ld, int m, double a, double b,
                  double a0, cudaStream_t st);
int kpoint_project(sparc_context* c, const void* Xt, const void* Yt, int ns, int64_t ld, double* Hs,
                   double* Ms, cudaStream_t st);
int kpoint_eig(sparc_context* c, const double* Hs, const double* Ms, int ns, double* lam, double* Z,
               cudaStream_t st);
int kpoint_rotate(sparc_context* c, const void* Xt, void* Xout, const double* Z, int ns, int64_t ld,
                  cudaStream_t st);
int kpoint_step(sparc_context* c, void* X, int ns, int64_t ldx, int m, double a, double b,
                double a0, double* eig, int eig_on_host, cudaStream_t st);

}  // namespace sparc

// Handle ------------------------------------------------------------------
struct sparc_context {
  int device = 0;
  sparc::Grid grid{};
  double h = 0.0;
  int64_t nd = 0, ld = 0;  // internal leading dimension (padded)
  int precision = SPARC_PREC_FP64;
  int ns_max = 1;
  sparc::LapCoef lap{};
  // potentials
  double* veff64 = nullptr;
  float* veff32 = nullptr;
  // nonlocal tables
  sparc::Nonlocal<double> nl64;
  sparc::Nonlocal<float> nl32;
  void* nl_mem[64] = {};
  int nl_nmem = 0;
  // workspaces
  void* W1 = nullptr;
  void* W2 = nullptr;
  void* Wstage = nullptr;  // host-pointer staging (lazy)
  __nv_bfloat16* S1 = nullptr;  // BF16 operand slices (mixed precision)
  __nv_bfloat16* S2 = nullptr;
  __nv_bfloat16* SZ = nullptr;
  int* esc = nullptr;  // per-row exponents of the digit slices (mixed precision)
  void* D = nullptr;       // nonlocal coefficients kp x ns_max
  double* Hs = nullptr;
  double* Ms = nullptr;
  double* Z = nullptr;
  double* lam = nullptr;
  double* proj_work = nullptr;
  int64_t proj_work_elems = 0;
  sparc::EigWork eig;
  // Lanczos
  double* lz = nullptr;  // 3 vectors + coefficients + partials
  bool have_bounds = false;
  double a0 = 0.0, b = 0.0;
  bool have_prev = false;
  double prev_max = 0.0;
  // timings
  cudaEvent_t ev[7] = {};
  cudaEvent_t ev_stage[4] = {};  // host-buffer staging: in start/end, out start/end
  cudaEvent_t ev_tune[2] = {};   // the stencil shape tuner's launches
  // per filter degree on the ring path: before the stencil, after it, after the
  // nonlocal pass (recorded while kev_on)
  std::vector<cudaEvent_t> kev;
  int kev_n = 0;
  bool kev_on = false;
  bool timed = false;
  bool staged = false;           // the last step staged a host block
  double host_ms = 0.0;          // wall time of the last sparc_chefsi_step call
  long long step_launches = 0;
  bool ring_enabled = true;  // TMA-ring stencil (options.reserved[0] bit 0 turns it off)
  bool tc_gemm = true;       // tensor-core projection/rotation (FP64: reserved[0] bit 1 off)
  // nonlocal term by support-point tiles (ring stencil path); tables of the
  // handle's working precision, partial sums npairs x ns_max
  sparc::NlTiles<double> tiles64;
  sparc::NlTiles<float> tiles32;
  bool tiles32_ok = false, tiles64_ok = false;  // tiles built and within shared memory
  size_t part_bytes = 0;                         // size of `part`
  void* part = nullptr;
  long long wait_cycles = 4000000000LL;  // bound of every device wait (SM clock cycles)
  // ring stencil thread shape: fixed (>= 0) or tuned per ns (-1)
  int shape_fixed = -1;
  bool stall_test = false;  // options flag bit 3 (test hook, see sparc.h)
  sparc::KpointState* kpt = nullptr;  // set on handles of a Bloch wavevector (complex)
  std::vector<std::pair<int, int>> shape_by_ns;  // (ns, shape) tuned so far
  sparc_tuning tuning{};
  double* Y64 = nullptr;     // mixed handles: FP64 Yt = H Xt of a step (ld x ns_max)
  float2* veff_df = nullptr; // Veff as (hi, lo) FP32 pairs for the double-FP32 stencil
  bool df_stencil = false;   // FP64 H x in double-FP32 arithmetic (mixed Yt; reserved[0] bit 2)
  double nl_density = 0.0;   // projector entries per grid point (pull table size / Nd)
  std::string err;
};
