// Nonlocal projector term of H (paper Sec. II A: per atom, a dense projector
// block applied to the components of X on the atom's support) for blocks of
// orbitals, after the local stencil (stencil_tma.cu):
//
//   nl_apply:  y_i += s_h sum_k chi_k(i) D[k]            (i a support point)
//              and, from the same updated values, the partial sums
//              C_t[k] = sum_{i in tile t} chi_k(i) y_i    (next degree's D)
//   nl_reduce: D[k] = gamma_k h^3 sum_t C_t[k]           (fixed tile order)
//
// D is projector-major here (D[k ns + n]), so a tile stages the coefficients
// of its projectors for NB orbitals as contiguous rows.
//
// The support points (grid points inside at least one atom's cut-off sphere)
// are cut into tiles of kTilePts consecutive points.  A CTA takes one tile and
// NB orbitals: each thread owns one support point, loads its (k, chi) entries
// once and applies them to all NB orbitals, with the tile's projector
// coefficients D for those orbitals staged in shared memory.  The projector
// tables therefore stream once per NB orbitals instead of once per orbital, and
// every orbital's values move in coalesced rows.  The partial sums C_t are
// taken per (tile, projector) pair in point order (one thread per projector
// and eight orbitals), and the reduction adds the tiles of a projector in tile
// order: no floating-point atomics, so results are bit-reproducible.
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace sparc {

void nl_tiles_build(int64_t nd, const int* pull_ptr, const int* pull_k, const double* pull_chi,
                    int kp, NlTilesHost& o) {
  o = NlTilesHost{};
  o.tp = kTilePts;
  // support points and their entries (pull order: atom, then projector)
  for (int64_t i = 0; i < nd; ++i)
    if (pull_ptr[i + 1] > pull_ptr[i]) o.pts.push_back((int)i);
  const int npts = (int)o.pts.size();
  const int ntiles = (npts + o.tp - 1) / o.tp;
  o.tile_ptr.resize(ntiles + 1);
  for (int t = 0; t <= ntiles; ++t) o.tile_ptr[t] = std::min(t * o.tp, npts);
  o.ent_ptr.assign(npts + 1, 0);
  o.kset_ptr.assign(ntiles + 1, 0);
  std::vector<int> local(kp, -1);
  std::vector<std::vector<std::pair<int, double>>> bykl;  // per tile-local k: (point, chi)
  for (int t = 0; t < ntiles; ++t) {
    std::vector<int> ks;
    bykl.clear();
    for (int pl = o.tile_ptr[t]; pl < o.tile_ptr[t + 1]; ++pl) {
      const int i = o.pts[pl];
      for (int e = pull_ptr[i]; e < pull_ptr[i + 1]; ++e) {
        const int k = pull_k[e];
        if (local[k] < 0) {
          local[k] = (int)ks.size();
          ks.push_back(k);
          bykl.emplace_back();
        }
        o.ent_kl.push_back((uint16_t)local[k]);
        o.ent_chi.push_back(pull_chi[e]);
        bykl[local[k]].emplace_back(pl - o.tile_ptr[t], pull_chi[e]);
      }
      o.ent_ptr[pl + 1] = (int)o.ent_kl.size();
    }
    o.kt_max = std::max(o.kt_max, (int)ks.size());
    o.et_max = std::max(o.et_max, o.ent_ptr[o.tile_ptr[t + 1]] - o.ent_ptr[o.tile_ptr[t]]);
    for (size_t kl = 0; kl < ks.size(); ++kl) {
      o.kset_k.push_back(ks[kl]);
      for (const auto& pc : bykl[kl]) {
        o.kent_pt.push_back((uint16_t)pc.first);
        o.kent_chi.push_back(pc.second);
      }
      o.kent_ptr.push_back((int)o.kent_pt.size());
      local[ks[kl]] = -1;
    }
    o.kset_ptr[t + 1] = (int)o.kset_k.size();
  }
  o.kent_ptr.insert(o.kent_ptr.begin(), 0);
  // pairs of each projector, in tile order
  o.kpair_ptr.assign(kp + 1, 0);
  for (int k : o.kset_k) ++o.kpair_ptr[k + 1];
  for (int k = 0; k < kp; ++k) o.kpair_ptr[k + 1] += o.kpair_ptr[k];
  o.kpair.resize(o.kset_k.size());
  std::vector<int> fill(o.kpair_ptr.begin(), o.kpair_ptr.end() - 1);
  for (int pr = 0; pr < (int)o.kset_k.size(); ++pr) o.kpair[fill[o.kset_k[pr]]++] = pr;
}

namespace {

template <typename T>
struct Vec4;
template <>
struct Vec4<float> { using t = float4; };
template <>
struct Vec4<double> { using t = double2; };

template <typename T>
struct NbOf;
template <>
struct NbOf<float> { static constexpr int v = 16; };
template <>
struct NbOf<double> { static constexpr int v = 16; };

template <typename T, int NB>
__global__ void __launch_bounds__(kTilePts)
    k_nl_apply(const NlTiles<T> t, const T* __restrict__ D, int kp, T* __restrict__ Y,
               int64_t ldy, int ns, T s_h, T* __restrict__ part) {
  extern __shared__ __align__(16) uint8_t nl_smem[];
  // the orbital blocks of one tile run back to back, so the tile's tables are
  // read from DRAM once and from L2 by the other blocks
  const int nblk = (ns + NB - 1) / NB;
  const int tile = blockIdx.x / nblk;
  const int nb0 = (blockIdx.x - tile * nblk) * NB;
  const int nb = min(NB, ns - nb0);
  const int p0 = t.tile_ptr[tile], np = t.tile_ptr[tile + 1] - p0;
  const int k0 = t.kset_ptr[tile], nk = t.kset_ptr[tile + 1] - k0;
  const int e0t = t.ent_ptr[p0], ne = t.ent_ptr[p0 + np] - e0t;
  const int ke0 = t.kent_ptr[k0];
  // Dsh[kl][DS]: one projector's NB orbital values as a row, read with vector
  // loads; the row stride DS = NB + 16 bytes puts the rows of eight
  // consecutive projectors on distinct bank groups
  using V = typename Vec4<T>::t;
  constexpr int VW = 16 / sizeof(T);  // elements per 16-byte load
  constexpr int DS = NB + 16 / (int)sizeof(T);
  // shared layout: Dsh[nk][DS], ysh[kTilePts][DS] (a point's NB updated values
  // as a row), the tile's entries (chi, then projector / point indices) in both
  // orders
  T* const Dsh = reinterpret_cast<T*>(nl_smem);
  T* const ysh = Dsh + t.kt_max * DS;
  T* const echi = ysh + kTilePts * DS;
  T* const kchi = echi + t.et_max;
  uint16_t* const ekl = reinterpret_cast<uint16_t*>(kchi + t.et_max);
  uint16_t* const kpt = ekl + t.et_max;
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    echi[e] = t.ent_chi[e0t + e];
    ekl[e] = t.ent_kl[e0t + e];
    kchi[e] = t.kent_chi[ke0 + e];
    kpt[e] = t.kent_pt[ke0 + e];
  }
  // projector-major D: the NB values of one projector are contiguous
  for (int idx = threadIdx.x; idx < NB * nk; idx += blockDim.x) {
    const int kl = idx / NB, j = idx - kl * NB;
    Dsh[kl * DS + j] = j < nb ? D[(int64_t)t.kset_k[k0 + kl] * ns + nb0 + j] : T(0);
  }
  const int pl = threadIdx.x;
  int64_t i = 0;
  int pe0 = 0, pe1 = 0;
  T y[NB];
  if (pl < np) {
    i = t.pts[p0 + pl];
    pe0 = t.ent_ptr[p0 + pl] - e0t;
    pe1 = t.ent_ptr[p0 + pl + 1] - e0t;
#pragma unroll
    for (int j = 0; j < NB; ++j) y[j] = j < nb ? Y[(int64_t)(nb0 + j) * ldy + i] : T(0);
  }
  __syncthreads();
  if (pl < np) {
    T acc[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) acc[j] = T(0);
    for (int e = pe0; e < pe1; ++e) {
      const V* row = reinterpret_cast<const V*>(Dsh + ekl[e] * DS);
      const T c = echi[e];
#pragma unroll
      for (int q = 0; q < NB / VW; ++q) {
        const V d = row[q];
        const T* dv = reinterpret_cast<const T*>(&d);
#pragma unroll
        for (int w = 0; w < VW; ++w) acc[q * VW + w] += c * dv[w];
      }
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      y[j] += s_h * acc[j];
      if (j < nb) Y[(int64_t)(nb0 + j) * ldy + i] = y[j];
    }
    V* yrow = reinterpret_cast<V*>(ysh + pl * DS);
#pragma unroll
    for (int q = 0; q < NB / VW; ++q) {
      V v;
      T* vv = reinterpret_cast<T*>(&v);
#pragma unroll
      for (int w = 0; w < VW; ++w) vv[w] = y[q * VW + w];
      yrow[q] = v;
    }
  }
  if (!part) return;
  __syncthreads();
  // C_t[k] for this tile's projectors: each thread takes one projector and PW
  // orbitals and sums over the projector's entries in point order
  constexpr int PW = 8;
  constexpr int NQ = NB / PW;
  for (int idx = threadIdx.x; idx < nk * NQ; idx += blockDim.x) {
    const int kl = idx / NQ, j0 = (idx - kl * NQ) * PW;
    if (j0 >= nb) continue;
    const int e1 = t.kent_ptr[k0 + kl + 1] - ke0;
    T sacc[PW];
#pragma unroll
    for (int w = 0; w < PW; ++w) sacc[w] = T(0);
    for (int e = t.kent_ptr[k0 + kl] - ke0; e < e1; ++e) {
      const T c = kchi[e];
      const V* yr = reinterpret_cast<const V*>(ysh + kpt[e] * DS + j0);
#pragma unroll
      for (int q = 0; q < PW / VW; ++q) {
        const V v = yr[q];
        const T* vv = reinterpret_cast<const T*>(&v);
#pragma unroll
        for (int w = 0; w < VW; ++w) sacc[q * VW + w] += c * vv[w];
      }
    }
#pragma unroll
    for (int w = 0; w < PW; ++w)
      if (j0 + w < nb) part[(int64_t)(k0 + kl) * ns + nb0 + j0 + w] = sacc[w];
  }
}

template <typename T>
__global__ void k_nl_reduce(const int* __restrict__ kpair_ptr, const int* __restrict__ kpair,
                            const T* __restrict__ part, int ns, int kp,
                            const double* __restrict__ gamma, double h3, T* __restrict__ D) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)kp * ns) return;
  const int k = (int)(idx / ns), n = (int)(idx - (int64_t)k * ns);
  T s = T(0);
  for (int p = kpair_ptr[k]; p < kpair_ptr[k + 1]; ++p) s += part[(int64_t)kpair[p] * ns + n];
  D[(int64_t)k * ns + n] = T(s * (gamma[k] * h3));
}

}  // namespace

template <typename T>
size_t nl_apply_smem(const NlTiles<T>& t) {
  constexpr int NB = NbOf<T>::v;
  constexpr int DS = NB + 16 / (int)sizeof(T);
  return ((size_t)t.kt_max * DS + (size_t)kTilePts * DS) * sizeof(T) +
         (size_t)t.et_max * 2 * (sizeof(T) + sizeof(uint16_t)) + 16;
}

template <typename T>
cudaError_t nl_apply(const NlTiles<T>& t, const T* D, int kp, T* y, int64_t ldy, int ns,
                     double s_h, T* part, cudaStream_t st) {
  if (t.ntiles == 0 || ns < 1) return cudaSuccess;
  constexpr int NB = NbOf<T>::v;
  const size_t smem = nl_apply_smem(t);
  static unsigned long long attr_bits = 0;
  if (smem > 48 * 1024) {
    // the device's whole opt-in limit, so that handles with larger tiles later
    // need no second setting
    const cudaError_t e = smem_limit_once(&attr_bits, (const void*)k_nl_apply<T, NB>, smem_optin());
    if (e != cudaSuccess) return e;
  }
  const dim3 grid((unsigned)((int64_t)t.ntiles * ((ns + NB - 1) / NB)));
  note_launch(), k_nl_apply<T, NB><<<grid, kTilePts, smem, st>>>(t, D, kp, y, ldy, ns, T(s_h), part);
  return cudaGetLastError();
}

template <typename T>
cudaError_t nl_reduce(const NlTiles<T>& t, const T* part, int ns, int kp, const double* gamma,
                      double h3, T* D, cudaStream_t st) {
  if (t.ntiles == 0 || ns < 1 || kp < 1) return cudaSuccess;
  const int64_t total = (int64_t)kp * ns;
  note_launch(), k_nl_reduce<T><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
      t.kpair_ptr, t.kpair, part, ns, kp, gamma, h3, D);
  return cudaGetLastError();
}

template size_t nl_apply_smem<float>(const NlTiles<float>&);
template size_t nl_apply_smem<double>(const NlTiles<double>&);
template cudaError_t nl_apply<float>(const NlTiles<float>&, const float*, int, float*, int64_t, int,
                                     double, float*, cudaStream_t);
template cudaError_t nl_apply<double>(const NlTiles<double>&, const double*, int, double*, int64_t,
                                      int, double, double*, cudaStream_t);
template cudaError_t nl_reduce<float>(const NlTiles<float>&, const float*, int, int, const double*,
                                      double, float*, cudaStream_t);
template cudaError_t nl_reduce<double>(const NlTiles<double>&, const double*, int, int,
                                       const double*, double, double*, cudaStream_t);

}  // namespace sparc
