// CUDA kernels of the PIT/PIDT particle step for sm_103a (arXiv:1508.02435).
//
// Step structure (Section 3 PIC cycle + Section 5 re-binning):
//   deposit   k_leaf_partials -> k_vertex_charge -> k_sum_blocks        (item 1)
//   solve     k_rhs -> k_jacobi x sweeps (auxiliary)                    (item 2)
//   field     k_efield                                                  (item 3)
//   push      k_push64 / k_push32: gather E_i = R^T(x_i) E, leapfrog kick
//             and drift, wrap, re-location (descent / split resolve), new
//             key, moved flag (warp ballot), bucket counts               (items 3-4)
//   re-bin    scan(counts) -> k_stayers (stable ranks of stayers) ->
//             k_compact_movers (ballot words -> mover list in storage
//             order) -> k_mover_slots -> k_sort_segments -> k_gather_*
//             (stable: stayers first, then movers in storage order)
//
// Determinism: no floating-point atomics.  Every sum has a fixed order (bucket
// order within a leaf, ascending leaf-corner order per vertex); integer atomics
// only count, and the one order they decide (mover slots) is re-sorted.
#include <cuda_runtime.h>

#include <atomic>

#include "dev.cuh"
#include "launch.hpp"
#include "segsort.cuh"

namespace pic {

__constant__ double c_kref64[8][8];
__constant__ float c_kref32[8][8];

constexpr int kBlock = 256;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;
static_assert(kScanTile == kScanTileElems, "scan tile size disagrees with launch.hpp");

static std::atomic<int64_t> g_launches{0};
int64_t launches() { return g_launches.load(); }
void count_launches(int64_t k) { g_launches.fetch_add(k); }
#define COUNT(k) g_launches.fetch_add(k)

static inline int bsz(int32_t b) { return b > 0 ? b : kBlock; }

static inline unsigned grid_for(int64_t n, int block = kBlock) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// ---------------------------------------------------------------------------
// tree view helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ void leaf_info(const DevTree &t, int32_t L, int *lev, int32_t *c) {
  *lev = t.leaf_level[L];
  for (int a = 0; a < t.d; ++a) c[a] = t.leaf_coords[(int64_t)L * t.d + a];
}

// The same with the dimension known at compile time (the loop unrolls).
template <int D>
__device__ __forceinline__ void leaf_info_d(const DevTree &t, int32_t L, int *lev, int32_t *c) {
  *lev = t.leaf_level[L];
#pragma unroll
  for (int a = 0; a < D; ++a) c[a] = t.leaf_coords[(int64_t)L * D + a];
}

__device__ __forceinline__ const InstInfo &inst_of_leaf(const DevTree &t, int32_t L) {
  return t.inst[t.n_inst > 1 ? t.inst_of_leaf[L] : 0];
}
__device__ __forceinline__ const InstInfo &inst_of_vertex(const DevTree &t, int64_t v) {
  return t.inst[t.n_inst > 1 ? t.inst_of_vert[v] : 0];
}

// Global vertex ids of the corners of uniform-grid cell c of instance I.
__device__ __forceinline__ void corner_vertices(const InstInfo &I, const int32_t *c, int d, int32_t *vid) {
  uniform_corner_vertices(c, d, I.M, vid);
  for (int e = 0; e < (1 << d); ++e) vid[e] += I.vert_off;
}

// PIDT owner vertex of corner a of leaf L (uniform grids: the FE vertex).
__device__ __forceinline__ int32_t pidt_vertex(const DevTree &t, int32_t L, int a) {
  if (t.uniform) {
    int32_t c[3] = {0, 0, 0};
    for (int k = 0; k < t.d; ++k) c[k] = t.leaf_coords[(int64_t)L * t.d + k];
    int32_t vid[8];
    corner_vertices(inst_of_leaf(t, L), c, t.d, vid);
    return vid[a];
  }
  return t.corner_pv[(int64_t)L * t.nc + a];
}

// Sort key of a particle in leaf L owned through corner a: PIT = leaf; PIDT =
// owner vertex * 2^d + quadrant of the leaf seen from the vertex.
__device__ __forceinline__ int32_t key_of(const DevTree &t, int32_t L, int a) {
  if (t.scheme == 0) return L;
  return pidt_vertex(t, L, a) * t.nc + (t.nc - 1 - a);
}

// Value of a vertex field at corner e of leaf L (hanging corners interpolated
// from their masters, in ascending master order).
__device__ __forceinline__ double corner_value(const DevTree &t, int32_t L, const int32_t *c, int e,
                                               const double *F) {
  if (t.uniform) return F[inst_of_leaf(t, L).vert_off + uniform_corner_vertex(c, e, t.d, inst_of_leaf(t, L).M)];
  int64_t i = (int64_t)L * t.nc + e;
  double s = 0.0;
  for (int32_t j = t.cexp_ptr[i]; j < t.cexp_ptr[i + 1]; ++j) s = s + t.cexp_w64[j] * F[t.cexp_vid[j]];
  return s;
}

__device__ __forceinline__ float corner_value(const DevTree &t, int32_t L, const int32_t *c, int e,
                                              const float *F) {
  if (t.uniform) return F[inst_of_leaf(t, L).vert_off + uniform_corner_vertex(c, e, t.d, inst_of_leaf(t, L).M)];
  int64_t i = (int64_t)L * t.nc + e;
  float s = 0.0f;
  for (int32_t j = t.cexp_ptr[i]; j < t.cexp_ptr[i + 1]; ++j) s = s + t.cexp_w32[j] * F[t.cexp_vid[j]];
  return s;
}

__device__ __forceinline__ const double *inc_weights(const DevTree &t, double) { return t.inc_w64; }
__device__ __forceinline__ const float *inc_weights(const DevTree &t, float) { return t.inc_w32; }
__device__ __forceinline__ double kref_val(int e, int f, double) { return c_kref64[e][f]; }
__device__ __forceinline__ float kref_val(int e, int f, float) { return c_kref32[e][f]; }
__device__ __forceinline__ double ion_load(const DevTree &t, int64_t v, double) {
  return t.uniform ? inst_of_vertex(t, v).ion_load : t.ion64[v];
}
__device__ __forceinline__ float ion_load(const DevTree &t, int64_t v, float) {
  return t.uniform ? inst_of_vertex(t, v).ion_load32 : t.ion32[v];
}
__device__ __forceinline__ double diag_val(const DevTree &t, int64_t v, double) {
  return t.uniform ? inst_of_vertex(t, v).diag : t.diag64[v];
}
__device__ __forceinline__ float diag_val(const DevTree &t, int64_t v, float) {
  return t.uniform ? inst_of_vertex(t, v).diag32 : t.diag32[v];
}

// Visit the incident leaf corners (lc = leaf * 2^d + corner, ascending) of
// vertex v with their constraint weights: fn(lc, w).
template <typename T, typename Fn>
__device__ __forceinline__ void for_incidences(const DevTree &t, int64_t v, Fn fn) {
  if (t.uniform) {
    int32_t lc[8];
    int m = uniform_incidences(v, t.d, inst_of_vertex(t, v), t.spread, lc);
    for (int i = 0; i < m; ++i) fn(lc[i], (T)1);
  } else {
    const T *ww = inc_weights(t, (T)0);
    for (int32_t j = t.inc_ptr[v]; j < t.inc_ptr[v + 1]; ++j) fn(t.inc_lc[j], ww[j]);
  }
}

// Block partial FP64 sums (fixed reduction tree) for deterministic totals.
__device__ __forceinline__ void block_sum_store(double v, double *block_out) {
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    v = lane < nw ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) block_out[blockIdx.x] = v;
  }
}

__global__ void k_sum_blocks(const double *in, int64_t n, double *out) {
  double v = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v += in[i];
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) *out = v;
  }
}

// ---------------------------------------------------------------------------
// a7 deposit
// ---------------------------------------------------------------------------

__device__ __forceinline__ void local_coords(const double *x, int64_t n, int64_t p, int lev, const int32_t *c,
                                             int d, double *tl) {
  double s = (double)c_pow3[lev];
  for (int a = 0; a < d; ++a) {
    double u = x[a * n + p] * s - (double)c[a];
    tl[a] = u < 0.0 ? 0.0 : (u > 1.0 ? 1.0 : u);
  }
}

// Per leaf: partial sums of the 2^d shape functions over the leaf's particles
// in bucket order (PIDT: the leaf's 2^d sub-buckets in corner order).
template <bool kSplit, int D>
__global__ void k_leaf_partials(DevTree t, const int32_t *__restrict__ start, const void *pos, int64_t n,
                                void *part_out) {
  int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= t.n_leaves) return;
  int lev;
  int32_t c[3] = {0, 0, 0};
  leaf_info_d<D>(t, (int32_t)L, &lev, c);
  constexpr int nc = 1 << D, d = D;
  const int na = t.scheme == 0 ? 1 : nc;
  if (kSplit) {
    const float *o = (const float *)pos;
    float acc[nc];
    for (int e = 0; e < nc; ++e) acc[e] = 0.0f;
    for (int a = 0; a < na; ++a) {
      int32_t k = key_of(t, (int32_t)L, a);
      for (int32_t p = start[k]; p < start[k + 1]; ++p) {
        float tl[d];
        for (int b = 0; b < d; ++b) tl[b] = o[b * n + p];
        for (int e = 0; e < nc; ++e) acc[e] = acc[e] + shape<float>(tl, e, d);
      }
    }
    float *part = (float *)part_out;
    for (int e = 0; e < nc; ++e) part[L * nc + e] = acc[e];
  } else {
    const double *x = (const double *)pos;
    double acc[nc];
    for (int e = 0; e < nc; ++e) acc[e] = 0.0;
    for (int a = 0; a < na; ++a) {
      int32_t k = key_of(t, (int32_t)L, a);
      for (int32_t p = start[k]; p < start[k + 1]; ++p) {
        double tl[d];
        local_coords(x, n, p, lev, c, d, tl);
        for (int e = 0; e < nc; ++e) acc[e] = acc[e] + shape<double>(tl, e, d);
      }
    }
    double *part = (double *)part_out;
    for (int e = 0; e < nc; ++e) part[L * nc + e] = acc[e];
  }
}

// Per vertex: S = sum of w * partial over incident leaf corners (ascending),
// Q = q S + ion * integral(phi_v); block partial sums of Q in FP64.
__device__ __forceinline__ double inst_q(const InstInfo &I, double) { return I.q; }
__device__ __forceinline__ float inst_q(const InstInfo &I, float) { return I.q32; }
__device__ __forceinline__ double inst_ion(const InstInfo &I, double) { return I.ion; }
__device__ __forceinline__ float inst_ion(const InstInfo &I, float) { return I.ion32; }

template <typename T>
__global__ void k_vertex_charge(DevTree t, const T *__restrict__ part, T *Q, double *block_sum) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double mine = 0.0;
  if (v < t.n_vert) {
    const InstInfo &I = inst_of_vertex(t, v);
    const T q = inst_q(I, (T)0), ion = inst_ion(I, (T)0);
    T S = (T)0;
    if (t.uniform) {
      int32_t lc[8];
      int m = uniform_incidences(v, t.d, I, t.spread, lc);
      for (int i = 0; i < m; ++i) S = S + part[lc[i]];
    } else {
      const T *w = inc_weights(t, (T)0);
      for (int32_t j = t.inc_ptr[v]; j < t.inc_ptr[v + 1]; ++j) S = S + w[j] * part[t.inc_lc[j]];
    }
    T val = q * S + ion * ion_load(t, v, (T)0);
    Q[v] = val;
    mine = (double)val;
  }
  block_sum_store(mine, block_sum);
}

// ---------------------------------------------------------------------------
// a8 solve (auxiliary): b = Q - (sum Q) integral(phi); damped Jacobi
// ---------------------------------------------------------------------------

template <typename T>
__global__ void k_rhs(DevTree t, const T *Q, const double *total, T *b) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= t.n_vert) return;
  T tot = (T)(t.n_inst > 1 ? total[1 + t.inst_of_vert[v]] : *total);
  b[v] = Q[v] - tot * ion_load(t, v, (T)0);
}

// (A V)_v assembled leaf by leaf: sum over incident leaf corners (L, e) of
// w * sum_f K_ef h^(d-2) V(L, f).
template <typename T>
__device__ __forceinline__ T apply_row(const DevTree &t, int64_t v, const T *V) {
  T y = (T)0;
  for_incidences<T>(t, v, [&](int32_t lc, T w) {
    int32_t L = lc / t.nc;
    int e = lc - L * t.nc;
    int lev;
    int32_t c[3] = {0, 0, 0};
    leaf_info(t, L, &lev, c);
    T hs = t.d == 2 ? (T)1 : (T)(1.0 / (double)c_pow3[lev]);
    T yc = (T)0;
    for (int f = 0; f < t.nc; ++f) yc = yc + (kref_val(e, f, (T)0) * hs) * corner_value(t, L, c, f, V);
    y = y + w * yc;
  });
  return y;
}

// One sweep V_out = V_in + omega (b - A V_in) / diag; with r2 != NULL also
// block sums of (b - A V_in)^2 in FP64.
template <typename T>
__global__ void k_jacobi(DevTree t, const T *b, const T *Vin, T *Vout, T omega, double *r2) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double rr = 0.0;
  if (v < t.n_vert) {
    T y = apply_row<T>(t, v, Vin);
    T r = b[v] - y;
    if (Vout) Vout[v] = Vin[v] + omega * r / diag_val(t, v, (T)0);
    rr = (double)r * (double)r;
  }
  if (r2) block_sum_store(rr, r2);
}

// E = -grad V at the vertices: minus the mean over leaves that have v as an
// unconstrained corner of the leaf's edge difference along each axis.
template <typename T>
__global__ void k_efield(DevTree t, const T *V, T *E) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= t.n_vert) return;
  T acc[3] = {(T)0, (T)0, (T)0};
  for_incidences<T>(t, v, [&](int32_t lc, T) {
    int32_t L = lc / t.nc;
    int e = lc - L * t.nc;
    if (!t.uniform) {
      if (t.cexp_ptr[lc + 1] - t.cexp_ptr[lc] != 1 || t.cexp_w64[t.cexp_ptr[lc]] != 1.0) return;
    }
    int lev;
    int32_t c[3] = {0, 0, 0};
    leaf_info(t, L, &lev, c);
    T h = (T)(1.0 / (double)c_pow3[lev]);
    for (int a = 0; a < t.d; ++a) {
      T hi = corner_value(t, L, c, e | (1 << a), V);
      T lo = corner_value(t, L, c, e & ~(1 << a), V);
      acc[a] = acc[a] + (hi - lo) / h;
    }
  });
  T cn = (T)(t.uniform ? t.nc : t.dcnt[v]);
  for (int a = 0; a < t.d; ++a) E[a * t.n_vert + v] = -(acc[a] / cn);
}

// ---------------------------------------------------------------------------
// a1/a2 initial keys and split conversion
// ---------------------------------------------------------------------------

__device__ __forceinline__ int pidt_corner_q(const uint32_t *Q, int lev, int d) {
  uint32_t s = c_pow3[18 - lev];
  int a_idx = 0;
  for (int a = 0; a < d; ++a)
    if (Q[a] % (2u * s) >= s) a_idx |= 1 << a;
  return a_idx;
}

__device__ __forceinline__ int pidt_corner_o(const float *o, int d) {
  int a_idx = 0;
  for (int a = 0; a < d; ++a)
    if (o[a] >= 0.5f) a_idx |= 1 << a;
  return a_idx;
}

// Instance of input particle p (binary search over the first particles).
__device__ __forceinline__ int inst_of_particle(const DevTree &t, int64_t p) {
  int lo = 0, hi = t.n_inst;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (t.inst[mid].poff <= p) lo = mid; else hi = mid;
  }
  return lo;
}

// FP64: wrap x in place, covering leaf and key.
__global__ void k_init64(DevTree t, double *x, int64_t n, int32_t *leaf, int32_t *key, int32_t *err) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int root = t.inst[inst_of_particle(t, p)].tab_root;
  uint32_t Q[3] = {0u, 0u, 0u};
  for (int a = 0; a < t.d; ++a) {
    double xa = x[a * n + p];
    if (!isfinite(xa)) { atomicOr(err, 1); xa = 0.0; }
    double y = wrap01(xa);
    x[a * n + p] = y;
    Q[a] = quantise(y);
  }
  int lev;
  int32_t L = descend_q(t.tab, t.d, Q, &lev, root);
  leaf[p] = L;
  key[p] = key_of(t, L, pidt_corner_q(Q, lev, t.d));
}

// Split: leaf by the FP64 owner, o = RN32(clamp(RN64(x 3^l) - c)), v = RN32(v).
__global__ void k_init32(DevTree t, const double *x, const double *v, int64_t n, int32_t *leaf, float *o,
                         float *vf, int32_t *key, int32_t *err) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int root = t.inst[inst_of_particle(t, p)].tab_root;
  uint32_t Q[3] = {0u, 0u, 0u};
  double y[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < t.d; ++a) {
    double xa = x[a * n + p];
    if (!isfinite(xa) || !isfinite(v[a * n + p])) { atomicOr(err, 1); xa = 0.0; }
    y[a] = wrap01(xa);
    Q[a] = quantise(y[a]);
  }
  int lev;
  int32_t L = descend_q(t.tab, t.d, Q, &lev, root);
  leaf[p] = L;
  double s = (double)c_pow3[lev];
  float oo[3] = {0.f, 0.f, 0.f};
  for (int a = 0; a < t.d; ++a) {
    double u = y[a] * s - (double)t.leaf_coords[(int64_t)L * t.d + a];
    if (u < 0.0) u = 0.0;
    oo[a] = clamp_off((float)u);
    o[a * n + p] = oo[a];
    vf[a * n + p] = (float)v[a * n + p];
  }
  key[p] = key_of(t, L, pidt_corner_o(oo, t.d));
}

// Keys of a given split state (leaf + offsets); flags offsets outside [0,1).
__global__ void k_rekey32(DevTree t, const int32_t *leaf, const float *o, int64_t n, int32_t *key, int32_t *err) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  int32_t L = leaf[p];
  if (L < 0 || L >= t.n_leaves) { atomicOr(err, 2); L = 0; }
  float oo[3] = {0.f, 0.f, 0.f};
  for (int a = 0; a < t.d; ++a) {
    oo[a] = o[a * n + p];
    if (!(oo[a] >= 0.0f && oo[a] < 1.0f)) atomicOr(err, 2);
  }
  key[p] = key_of(t, L, pidt_corner_o(oo, t.d));
}

// ---------------------------------------------------------------------------
// a3 + a4 + a1/a2 + a5: fused gather, push, re-location, key, moved flag
// ---------------------------------------------------------------------------

// Adds to count[key] the length of every run of equal keys in adjacent
// active lanes, one atomic per run (particles in bucket order mostly share
// their new bucket with their neighbours; equal keys apart count as separate
// runs).  Active lanes are a prefix of the warp or all of it.
__device__ __forceinline__ void add_runs(int32_t *count, int32_t key, bool act) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int32_t prev = __shfl_up_sync(full, key, 1);
  const unsigned acts = __ballot_sync(full, act);
  const bool head = act && (lane == 0 || prev != key);
  const unsigned heads = __ballot_sync(full, head);
  if (head) {
    const unsigned after = ~((2u << lane) - 1u);  // lanes above this one (none for lane 31)
    const unsigned stop = (heads | ~acts) & after;
    const int end = stop ? __ffs(stop) - 1 : 32;
    atomicAdd(&count[key], end - lane);
  }
}

// Bucket counts, mover ballot word and per-block mover count.  kRuns: one
// atomic per run of equal adjacent keys (3D, where most particles of a warp
// take distinct new keys); else one per distinct key of the warp (2D, where
// repeats of a key are often apart; measured faster on each).
template <bool kRuns>
__device__ __forceinline__ void count_and_ballot(bool act, int32_t knew, bool moved, int32_t *count,
                                                 uint32_t *mover_words, int32_t *block_movers) {
  const unsigned full = 0xffffffffu;
  int lane = threadIdx.x & 31;
  if (kRuns) {
    add_runs(count, knew, act);
  } else {
    const unsigned peers = __match_any_sync(full, act ? knew : -1);
    if (act && lane == __ffs(peers) - 1) atomicAdd(&count[knew], __popc(peers));
  }
  unsigned mv = __ballot_sync(full, act && moved);
  int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (lane == 0) mover_words[gw] = mv;
  __shared__ int sh[32];
  if (lane == 0) sh[threadIdx.x >> 5] = __popc(mv);
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    block_movers[blockIdx.x] = s;
  }
}

// Artificial work of the paper's experiments (Section 6): `flops` floating
// point operations per particle move (fused multiply-adds, two each), on a
// value the move does not use; the never-taken test keeps them.
template <typename T>
__device__ __forceinline__ void artificial_flops(T seed, int32_t flops, int32_t *err) {
  T acc = seed;
  for (int32_t i = 0; i < flops; i += 2) acc = fma(acc, (T)0.999, (T)1e-3);
  if (acc == (T)-12345.0) atomicOr(err, 0);
}

// Reflection at the walls of the unit box, FP64 (the oracle's reading): the
// free path y folds into [0, 2); y >= 1 mirrors to 2 - y with the velocity
// component negated; the far wall itself goes to the largest double below 1.
__device__ __forceinline__ double fold64(double y, bool *flip) {
  double m = y - 2.0 * floor(y * 0.5);
  *flip = false;
  if (m >= 1.0) {
    m = 2.0 - m;
    *flip = true;
    if (m >= 1.0) m = 0x1.fffffffffffffp-1;
  }
  return m;
}

// D = t.d as a compile-time constant: the per-axis loops unroll and the
// per-particle arrays stay in registers.
template <int D>
__global__ void k_push64(DevTree t, Push64Args a) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool act = p < a.n;
  int32_t knew = 0;
  bool moved = false;
  if (act) {
    constexpr int d = D, nc = 1 << D;
    const int64_t n = a.n, nv = t.n_vert;
    int32_t L = a.leaf[p];
    int lev;
    int32_t c[3] = {0, 0, 0};
    leaf_info_d<D>(t, L, &lev, c);
    double tl[3];
    local_coords(a.x, n, p, lev, c, d, tl);
    double E[3] = {0.0, 0.0, 0.0};
    const InstInfo &I = inst_of_leaf(t, L);
    if (!a.E) {
      // the particle-handling move: no field, no kick
    } else if (t.uniform) {
      int32_t vid[8];
      corner_vertices(I, c, d, vid);
      for (int e = 0; e < nc; ++e) {
        double w = shape<double>(tl, e, d);
        for (int ax = 0; ax < d; ++ax) E[ax] = E[ax] + w * a.E[ax * nv + vid[e]];
      }
    } else {
      for (int e = 0; e < nc; ++e) {
        double w = shape<double>(tl, e, d);
        for (int ax = 0; ax < d; ++ax) E[ax] = E[ax] + w * corner_value(t, L, c, e, a.E + ax * nv);
      }
    }
    uint32_t Q[3] = {0u, 0u, 0u};
    double x0n = 0.0, x1n = 0.0, x2n = 0.0, v0n = 0.0, v1n = 0.0, v2n = 0.0;  // record path
    bool bad = false;
    for (int ax = 0; ax < d; ++ax) {
      double vn = a.E ? a.v[ax * n + p] + a.qmdt * E[ax] : a.v[ax * n + p];
      const double y = a.x[ax * n + p] + vn * a.dt;
      double xn;
      if (a.reflect) {
        bool flip;
        xn = fold64(y, &flip);
        if (flip) vn = -vn;
      } else {
        xn = wrap01(y);
      }
      if (!isfinite(vn) || !isfinite(xn)) { bad = true; xn = 0.0; }
      if (a.rec) {
        if (ax == 0) { x0n = xn; v0n = vn; }
        if (ax == 1) { x1n = xn; v1n = vn; }
        if (ax == 2) { x2n = xn; v2n = vn; }
      } else {
        a.tv[ax * n + p] = vn;
        a.tx[ax * n + p] = xn;
      }
      Q[ax] = quantise(xn);
    }
    if (a.flops > 0) artificial_flops<double>(tl[0], a.flops, a.err);
    if (bad) atomicOr(a.err, 1);
    int lev2;
    int32_t L2;
    if (t.uniform) {
      uint32_t step = 2u * c_pow3[18 - I.depth];
      int32_t cc[3] = {(int32_t)(Q[0] / step), (int32_t)(Q[1] / step), d == 3 ? (int32_t)(Q[2] / step) : 0};
      L2 = I.leaf_off + uniform_leaf_of_cell(t.spread + I.spread_off, I.M, cc, d);
      lev2 = I.depth;
    } else {
      // still inside its leaf (the radius of operation of Section 5.3): the
      // covering leaf is the old one, no descent
      const uint32_t step = 2u * c_pow3[18 - lev];
      bool inside = true;
      for (int ax = 0; ax < d; ++ax) inside &= Q[ax] / step == (uint32_t)c[ax];
      if (inside) {
        L2 = L;
        lev2 = lev;
      } else {
        L2 = descend_q(t.tab, d, Q, &lev2, I.tab_root);
      }
    }
    knew = key_of(t, L2, pidt_corner_q(Q, lev2, d));
    int32_t kold = t.scheme == 0 ? L : a.key[p];
    moved = knew != kold;
    if (a.rec) {  // one 64-byte record per particle: the re-bin gathers it whole
      double2 *r = a.rec + 4 * p;
      r[0] = make_double2(x0n, x1n);
      r[1] = make_double2(x2n, v0n);
      r[2] = make_double2(v1n, v2n);
      r[3] = make_double2(__longlong_as_double((long long)(((uint64_t)(uint32_t)knew << 32) | (uint32_t)L2)), 0.0);
    } else {
      a.tleaf[p] = L2;
    }
    if (a.rec || t.scheme != 0) a.keyn[p] = knew;  // PIT rows: the key array is the leaf array
  }
  count_and_ballot<D == 3>(act, knew, moved, a.count, a.mover_words, a.block_movers);
}

template <int D>
__global__ void __launch_bounds__(512, 3) k_push32(DevTree t, Push32Args a) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool act = p < a.n;
  int32_t knew = 0;
  bool moved = false;
  if (act) {
    constexpr int d = D, nc = 1 << D;
    const int64_t n = a.n, nv = t.n_vert;
    int32_t L = a.leaf[p];
    int lev;
    int32_t c[3] = {0, 0, 0};
    leaf_info_d<D>(t, L, &lev, c);
    float o[3] = {0.f, 0.f, 0.f};
    for (int ax = 0; ax < d; ++ax) o[ax] = a.o[ax * n + p];
    float E[3] = {0.f, 0.f, 0.f};
    const InstInfo &Ins = inst_of_leaf(t, L);
    if (!a.E && !a.Ec) {
      // the particle-handling move: no field, no kick
    } else if (t.uniform) {
      int32_t vid[8];
      corner_vertices(Ins, c, d, vid);
      for (int e = 0; e < nc; ++e) {
        float w = shape<float>(o, e, d);
        for (int ax = 0; ax < d; ++ax) E[ax] = E[ax] + w * a.E[ax * nv + vid[e]];
      }
    } else if (a.Ec) {  // the corner values, expanded once per field
      const float4 *ec = a.Ec + (int64_t)L * nc;
      for (int e = 0; e < nc; ++e) {
        float w = shape<float>(o, e, d);
        const float4 q = ec[e];
        const float qv[3] = {q.x, q.y, q.z};
        for (int ax = 0; ax < d; ++ax) E[ax] = E[ax] + w * qv[ax];
      }
    } else {
      for (int e = 0; e < nc; ++e) {
        float w = shape<float>(o, e, d);
        for (int ax = 0; ax < d; ++ax) E[ax] = E[ax] + w * corner_value(t, L, c, e, a.E + ax * nv);
      }
    }
    const int32_t per = (int32_t)c_pow3[lev];
    const float sl = a.sl[lev];
    int32_t I[3] = {0, 0, 0};
    float f[3] = {0.f, 0.f, 0.f}, vnew[3] = {0.f, 0.f, 0.f};
    bool bad = false;
    const bool field = a.E || a.Ec;
    for (int ax = 0; ax < d; ++ax) {
      float vn = field ? a.v[ax * n + p] + a.qmdt * E[ax] : a.v[ax * n + p];
      float tt = o[ax] + vn * sl;
      if (!isfinite(vn) || !isfinite(tt)) { bad = true; tt = 0.0f; }
      float fl = floorf(tt);
      f[ax] = tt - fl;
      int32_t cc;
      if (!a.reflect) {
        if (fabsf(fl) < 1.0e9f) {
          cc = c[ax] + (int32_t)fl;               // periodic wrap, 32-bit
          if (cc < 0 || cc >= per) {
            cc %= per;
            if (cc < 0) cc += per;
          }
        } else {
          int64_t c64 = ((int64_t)c[ax] + (int64_t)fminf(fmaxf(fl, -1.0e15f), 1.0e15f)) % per;
          cc = (int32_t)(c64 < 0 ? c64 + per : c64);
        }
      } else {
        // reflecting walls (the oracle's reading): cell index folded modulo
        // 2 per; the mirrored half maps to (2 per - 1 - Im, 1 - f), or to
        // (2 per - Im, 0) when f = 0, with the velocity component negated
        const int64_t p2 = 2 * (int64_t)per;
        int64_t im = ((int64_t)c[ax] + (int64_t)fminf(fmaxf(fl, -1.0e15f), 1.0e15f)) % p2;
        if (im < 0) im += p2;
        if (im < per) {
          cc = (int32_t)im;
        } else {
          vn = -vn;
          if (f[ax] > 0.0f) {
            cc = (int32_t)(p2 - 1 - im);
            f[ax] = clamp_off(1.0f - f[ax]);
          } else {
            cc = (int32_t)(p2 - im);
            if (cc >= per) {
              cc = per - 1;
              f[ax] = 0x1.fffffep-1f;
            }
          }
        }
      }
      I[ax] = cc;
      if (a.rec) vnew[ax] = vn;
      else a.tv[ax * n + p] = vn;
    }
    if (a.flops > 0) artificial_flops<float>(o[0], a.flops, a.err);
    if (bad) atomicOr(a.err, 1);
    float o2[3] = {0.f, 0.f, 0.f};
    int lev2;
    int32_t L2;
    bool inside = true;  // target cell == the particle's own leaf cell
    for (int ax = 0; ax < d; ++ax) inside &= I[ax] == c[ax];
    if (t.uniform) {  // the covering leaf is the target cell itself; o = f
      L2 = Ins.leaf_off + uniform_leaf_of_cell(t.spread + Ins.spread_off, Ins.M, I, d);
      for (int ax = 0; ax < d; ++ax) o2[ax] = clamp_off(f[ax]);
    } else if (inside) {
      // still inside its leaf (the radius of operation of Section 5.3): no
      // lift, no drop -- the covering leaf is the old one and o = f
      L2 = L;
      lev2 = lev;
      for (int ax = 0; ax < d; ++ax) o2[ax] = clamp_off(f[ax]);
    } else {
      L2 = descend_split(t.tab, d, lev, I, f, o2, &lev2, Ins.tab_root);
    }
    knew = key_of(t, L2, pidt_corner_o(o2, d));
    int32_t kold = t.scheme == 0 ? L : a.key[p];
    moved = knew != kold;
    if (a.rec) {  // one 32-byte record per particle: the re-bin gathers it whole
      a.rec[2 * p] = make_float4(o2[0], o2[1], o2[2], vnew[0]);
      a.rec[2 * p + 1] = make_float4(vnew[1], vnew[2], __int_as_float(L2), __int_as_float(knew));
    } else {
      for (int ax = 0; ax < d; ++ax) a.to[ax * n + p] = o2[ax];
      a.tleaf[p] = L2;
    }
    if (a.rec || t.scheme != 0) a.keyn[p] = knew;  // PIT rows: the key array is the leaf array
  }
  count_and_ballot<D == 3>(act, knew, moved, a.count, a.mover_words, a.block_movers);
}

// Key counts of freshly converted particles (every particle a mover).
__global__ void k_count_all(const int32_t *key, int64_t n, int32_t *count, uint32_t *mover_words,
                            int32_t *block_movers) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool act = p < n;
  int32_t k = act ? key[p] : 0;
  count_and_ballot<false>(act, k, true, count, mover_words, block_movers);
}

// ---------------------------------------------------------------------------
// a6 stable counting sort
// ---------------------------------------------------------------------------

// Exclusive scan of int32 values: tiles of kScanTile elements.
__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t *total) {
  __shared__ int32_t sh[32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    int32_t s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    sh[lane] = s;
  }
  __syncthreads();
  int32_t before = w > 0 ? sh[w - 1] : 0;
  if (total) *total = sh[(blockDim.x >> 5) - 1];
  int32_t r = before + x - v;
  __syncthreads();
  return r;
}

__global__ void k_scan_reduce(const int32_t *in, int64_t n, int32_t *tile_sums) {
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int32_t s = 0;
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) s += in[base + i];
  int32_t tot;
  block_exclusive_scan(s, &tot);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// Single block: exclusive scan of the tile sums in place, total to *total.
__global__ void k_scan_tiles(int32_t *tile_sums, int64_t nt, int32_t *total) {
  int32_t carry = 0;
  for (int64_t base = 0; base < nt; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    int32_t v = i < nt ? tile_sums[i] : 0;
    int32_t tot;
    int32_t ex = block_exclusive_scan(v, &tot);
    if (i < nt) tile_sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_apply(const int32_t *in, int64_t n, const int32_t *tile_offsets, int32_t *out,
                             const int32_t *total) {
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int32_t vals[kScanItems];
  int32_t s = 0;
  for (int i = 0; i < kScanItems; ++i) {
    vals[i] = base + i < n ? in[base + i] : 0;
    s += vals[i];
  }
  int32_t ex = block_exclusive_scan(s, nullptr) + tile_offsets[blockIdx.x];
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = ex;
    ex += vals[i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = *total;
}

// Stayers of old bucket k keep their storage order at the head of new bucket k.
// The largest new bucket goes to *max_bucket with one atomic per block.
__global__ void k_stayers(const int32_t *old_start, const int32_t *keyn, const int32_t *new_start,
                          int64_t n_keys, int32_t *perm, int32_t *n_stay, int32_t *max_bucket) {
  __shared__ int32_t wmax[32];
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int32_t sz = 0;
  if (k < n_keys) {
    int32_t r = 0, dst = new_start[k];
    for (int32_t i = old_start[k]; i < old_start[k + 1]; ++i)
      if (keyn[i] == (int32_t)k) perm[dst + r++] = i;
    n_stay[k] = r;
    sz = new_start[k + 1] - new_start[k];
  }
  const int32_t m = __reduce_max_sync(0xffffffffu, sz);
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = b > wmax[w] ? b : wmax[w];
    if (b > 0) atomicMax(max_bucket, b);
  }
}

// Ballot words -> mover list in storage order.
__global__ void k_compact_movers(const uint32_t *mover_words, const int32_t *block_offsets, int64_t n,
                                 int32_t *movers) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t w0 = ((int64_t)blockIdx.x * blockDim.x) >> 5;
  int32_t off = block_offsets[blockIdx.x];
  for (int k = 0; k < w; ++k) off += __popc(mover_words[w0 + k]);
  uint32_t word = mover_words[w0 + w];
  if (p < n && ((word >> lane) & 1u)) movers[off + __popc(word & ((1u << lane) - 1u))] = (int32_t)p;
}

__global__ void k_mover_slots(const int32_t *movers, const int32_t *n_movers, const int32_t *keyn,
                              const int32_t *new_start, const int32_t *n_stay, int32_t *cursor,
                              int32_t *perm) {
  int32_t m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= *n_movers) return;
  int32_t p = movers[m];
  int32_t k = keyn[p];
  int32_t slot = atomicAdd(&cursor[k], 1);
  perm[new_start[k] + n_stay[k] + slot] = p;
}

// The movers of every bucket in storage order (undoes the atomic slot order).
// Segments of kSmallSeg movers or fewer are sorted here by one thread; longer
// ones are listed for k_sort_medium (up to kMedSeg: one warp each) or
// k_sort_large (one block each).
constexpr int kSmallSeg = 32;
constexpr int kMedSeg = 2048;        // longest segment one warp sorts in shared memory
constexpr int kMedThreads = 256;
constexpr int kLargeSeg = 16384;     // chunk of a long segment sorted in shared memory
constexpr int kLargeThreads = 1024;
__global__ void k_sort_segments(const int32_t *new_start, const int32_t *n_stay, int64_t n_keys, int32_t *perm,
                                int32_t *large, int32_t *n_large, int32_t *med, int32_t *n_med) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_keys) return;
  int32_t b = new_start[k] + n_stay[k], e = new_start[k + 1];
  if (e - b > kSmallSeg) {
    if (e - b <= kMedSeg) med[atomicAdd(n_med, 1)] = (int32_t)k;
    else large[atomicAdd(n_large, 1)] = (int32_t)k;
    return;
  }
  for (int32_t i = b + 1; i < e; ++i) {
    int32_t x = perm[i];
    int32_t j = i - 1;
    while (j >= b && perm[j] > x) {
      perm[j + 1] = perm[j];
      --j;
    }
    perm[j + 1] = x;
  }
}

// One warp per listed segment of at most kMedSeg movers (grid-stride over the
// list): the segment is copied into the warp's shared slice, sorted by the
// bitonic network of segsort.cuh and copied back.
__global__ void __launch_bounds__(kMedThreads) k_sort_medium(const int32_t *new_start, const int32_t *n_stay,
                                                             const int32_t *med, const int32_t *n_med,
                                                             int32_t *perm) {
  extern __shared__ int32_t sw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = kMedThreads / 32;
  int32_t *v = sw + wib * kMedSeg;
  const int nm = *n_med;
  for (int li = blockIdx.x * wpb + wib; li < nm; li += gridDim.x * wpb) {
    const int32_t k = med[li];
    const int32_t b = new_start[k] + n_stay[k], m = new_start[k + 1] - b;
    for (int i = lane; i < m; i += 32) v[i] = perm[b + i];
    __syncwarp();
    warp_sort_direct<int32_t>(v, m);
    for (int i = lane; i < m; i += 32) perm[b + i] = v[i];
    __syncwarp();
  }
}

// One block per long segment (grid-stride over the list): the in-place
// bitonic network of segsort.cuh, chunks of kLargeSeg in shared memory, so a
// bucket of any size sorts in O(m log^2 m).
__global__ void __launch_bounds__(kLargeThreads) k_sort_large(const int32_t *new_start, const int32_t *n_stay,
                                                              const int32_t *large, const int32_t *n_large,
                                                              int32_t *perm) {
  extern __shared__ int32_t sv[];
  const int nl = *n_large;
  for (int li = blockIdx.x; li < nl; li += gridDim.x) {
    const int32_t k = large[li];
    const int32_t b = new_start[k] + n_stay[k], m = new_start[k + 1] - b;
    block_sort_global<int32_t, int32_t>(perm + b, nullptr, m, sv, nullptr, kLargeSeg);
    __syncthreads();
  }
}

// The whole particle state into bucket order in one pass: positions and
// velocities ([d][n]), leaves, and keys and ids where given.
template <typename T>
__global__ void k_gather_state(const int32_t *perm, int64_t n, int d, const T *x, T *x2, const T *v, T *v2,
                               const int32_t *leaf, int32_t *leaf2, const int32_t *key, int32_t *key2,
                               const int32_t *ids, int32_t *ids2) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int32_t i = perm[p];
  for (int a = 0; a < d; ++a) x2[a * n + p] = x[a * n + i];
  for (int a = 0; a < d; ++a) v2[a * n + p] = v[a * n + i];
  leaf2[p] = leaf[i];
  if (key) key2[p] = key[i];
  if (ids) ids2[p] = ids[i];
}

// The pushed-state records in bucket order (two or four 16-byte loads per
// particle instead of one scattered 4- or 8-byte load per array).
__global__ void k_gather_rec32(const int32_t *perm, int64_t n, int d, const float4 *rec, float *x2, float *v2,
                               int32_t *leaf2, int32_t *key2, const int32_t *ids, int32_t *ids2) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int32_t i = perm[p];
  const float4 r0 = rec[2 * (int64_t)i], r1 = rec[2 * (int64_t)i + 1];
  x2[p] = r0.x;
  x2[n + p] = r0.y;
  if (d == 3) {
    x2[2 * n + p] = r0.z;
    v2[p] = r0.w;
    v2[n + p] = r1.x;
    v2[2 * n + p] = r1.y;
  } else {
    v2[p] = r0.w;
    v2[n + p] = r1.x;
  }
  leaf2[p] = __float_as_int(r1.z);
  if (key2) key2[p] = __float_as_int(r1.w);
  if (ids) ids2[p] = ids[i];
}

__global__ void k_gather_rec64(const int32_t *perm, int64_t n, int d, const double2 *rec, double *x2, double *v2,
                               int32_t *leaf2, int32_t *key2, const int32_t *ids, int32_t *ids2) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int32_t i = perm[p];
  const double2 *r = rec + 4 * (int64_t)i;
  const double2 r0 = r[0], r1 = r[1], r2 = r[2], r3 = r[3];
  x2[p] = r0.x;
  x2[n + p] = r0.y;
  if (d == 3) x2[2 * n + p] = r1.x;
  v2[p] = r1.y;
  v2[n + p] = r2.x;
  if (d == 3) v2[2 * n + p] = r2.y;
  const uint64_t lk = (uint64_t)__double_as_longlong(r3.x);
  leaf2[p] = (int32_t)(uint32_t)lk;
  if (key2) key2[p] = (int32_t)(uint32_t)(lk >> 32);
  if (ids) ids2[p] = ids[i];
}

template <typename T>
__global__ void k_gather_vec(const int32_t *perm, int64_t n, int d, const T *src, T *dst) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  int32_t i = perm[p];
  for (int a = 0; a < d; ++a) dst[a * n + p] = src[a * n + i];
}

// ---------------------------------------------------------------------------
// misc
// ---------------------------------------------------------------------------

__global__ void k_absolute_split(DevTree t, const int32_t *leaf, const float *o, int64_t n, double *x) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  int32_t L = leaf[p];
  int lev = t.leaf_level[L];
  double s = (double)c_pow3[lev];
  for (int a = 0; a < t.d; ++a)
    x[a * n + p] = ((double)t.leaf_coords[(int64_t)L * t.d + a] + (double)o[a * n + p]) / s;
}

__global__ void k_widen(const float *in, int64_t n, double *out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (double)in[i];
}

__global__ void k_half_kick64(const double *Ep, int64_t n, double c, double *v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = v[i] - c * Ep[i];
}

__global__ void k_half_kick32(const float *Ep, int64_t n, float c, float *v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = v[i] - c * Ep[i];
}

// Gather only (leapfrog start): E at the particles, [d][n].
__global__ void k_gather_only64(DevTree t, const double *x, const int32_t *leaf, int64_t n, const double *Ev,
                                double *Ep) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  int32_t L = leaf[p];
  int lev;
  int32_t c[3] = {0, 0, 0};
  leaf_info(t, L, &lev, c);
  double tl[3];
  local_coords(x, n, p, lev, c, t.d, tl);
  double E[3] = {0.0, 0.0, 0.0};
  for (int e = 0; e < t.nc; ++e) {
    double w = shape<double>(tl, e, t.d);
    for (int ax = 0; ax < t.d; ++ax) E[ax] = E[ax] + w * corner_value(t, L, c, e, Ev + ax * t.n_vert);
  }
  for (int ax = 0; ax < t.d; ++ax) Ep[ax * n + p] = E[ax];
}

__global__ void k_gather_only32(DevTree t, const float *o, const int32_t *leaf, int64_t n, const float *Ev,
                                float *Ep) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  int32_t L = leaf[p];
  int lev;
  int32_t c[3] = {0, 0, 0};
  leaf_info(t, L, &lev, c);
  float tl[3] = {0.f, 0.f, 0.f};
  for (int a = 0; a < t.d; ++a) tl[a] = o[a * n + p];
  float E[3] = {0.f, 0.f, 0.f};
  for (int e = 0; e < t.nc; ++e) {
    float w = shape<float>(tl, e, t.d);
    for (int ax = 0; ax < t.d; ++ax) E[ax] = E[ax] + w * corner_value(t, L, c, e, Ev + ax * t.n_vert);
  }
  for (int ax = 0; ax < t.d; ++ax) Ep[ax * n + p] = E[ax];
}

// ---------------------------------------------------------------------------
// a9 re-refinement: depth-first cell index on the finest admissible level
// ---------------------------------------------------------------------------

// FP64: cell of the quantised position on level dmax.
__global__ void k_fine_key64(DevTree t, const double *x, int64_t n, int dmax, uint32_t *key) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  uint32_t step = 2u * c_pow3[18 - dmax];
  uint32_t c[3] = {0u, 0u, 0u};
  for (int a = 0; a < t.d; ++a) c[a] = quantise(x[a * n + p]) / step;
  key[p] = (uint32_t)local_index(c[0], c[1], c[2], t.d, dmax);
}

// Split: cell of leaf + offset on level dmax; below the leaf the offset
// digits follow the drop rule of the split re-location.
__global__ void k_fine_key32(DevTree t, const int32_t *leaf, const float *o, int64_t n, int dmax, uint32_t *key) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int32_t L = leaf[p];
  const int lev = t.leaf_level[L];
  uint32_t c[3] = {0u, 0u, 0u};
  for (int a = 0; a < t.d; ++a) {
    uint32_t I = (uint32_t)t.leaf_coords[(int64_t)L * t.d + a];
    if (lev >= dmax) {
      I /= c_pow3[lev - dmax];
    } else {
      float f = o[a * n + p];
      for (int m = lev; m < dmax; ++m) {
        float u = 3.0f * f;
        int dg = (int)floorf(u);
        dg = dg > 2 ? 2 : dg;
        f = clamp_off(u - (float)dg);
        I = 3u * I + (uint32_t)dg;
      }
    }
    c[a] = I;
  }
  key[p] = (uint32_t)local_index(c[0], c[1], c[2], t.d, dmax);
}

// Particles per cell on one level (warp-aggregated).
__global__ void k_level_count(const uint32_t *key, int64_t n, uint32_t div, int32_t *count) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = p < n;
  const uint32_t c = act ? key[p] / div : 0xffffffffu;
  add_runs(count, (int32_t)c, act);
}

__global__ void k_threshold_bits(const int32_t *count, int64_t ncells, int64_t ppc, uint32_t *bits) {
  int64_t wd = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (wd * 32 >= ncells) return;
  uint32_t b = 0;
  for (int i = 0; i < 32; ++i) {
    int64_t c = wd * 32 + i;
    if (c < ncells && count[c] > ppc) b |= 1u << i;
  }
  bits[wd] = b;
}

// Cell counts of one level from those of the level below: the sum over the
// 3^d children (child ch of cell c is cell c 3^d + ch).
__global__ void k_count_parent(const int32_t *fine, int64_t ncoarse, int nch, int32_t *coarse) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncoarse) return;
  int32_t t = 0;
  for (int ch = 0; ch < nch; ++ch) t += fine[c * nch + ch];
  coarse[c] = t;
}

// Whether the particles-per-cell criterion keeps the installed tree: every
// leaf on level l needs dmin <= l <= dmax and (l == dmax or its count <= ppc),
// every ancestor on levels dmin .. l-1 a count > ppc.  Any leaf that fails
// sets *changed.  Counts of level m at count + coff[m].
struct AdaptCheck {
  const int32_t *count;
  int64_t coff[11];
  int dmin, dmax;
  int64_t ppc;
};

__global__ void k_adapt_check(DevTree t, AdaptCheck ac, int32_t *changed) {
  const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= t.n_leaves) return;
  int l;
  int32_t c[3] = {0, 0, 0};
  leaf_info(t, (int32_t)L, &l, c);
  bool bad = l < ac.dmin || l > ac.dmax;
  for (int m = ac.dmin; !bad && m <= l && m < ac.dmax; ++m) {
    const uint32_t sh = c_pow3[l - m];
    const int32_t idx = local_index((uint32_t)c[0] / sh, (uint32_t)c[1] / sh, t.d == 3 ? (uint32_t)c[2] / sh : 0u,
                                    t.d, m);
    const int32_t cnt = ac.count[ac.coff[m] + idx];
    bad = m < l ? cnt <= ac.ppc : cnt > ac.ppc;
  }
  if (bad) *changed = 1;
}

// Split particles of tree `from` re-located in tree `to` (same positions):
// the resolver of the split push with zero displacement.
__global__ void k_relocate32(DevTree from, DevTree to, const int32_t *leaf, const float *o, const float *v,
                             int64_t n, int32_t *leaf2, float *o2, float *v2) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int32_t L = leaf[p];
  const int lev = from.leaf_level[L];
  int32_t I[3] = {0, 0, 0};
  float f[3] = {0.f, 0.f, 0.f};
  for (int a = 0; a < from.d; ++a) {
    I[a] = from.leaf_coords[(int64_t)L * from.d + a];
    f[a] = o[a * n + p];
  }
  float on[3] = {0.f, 0.f, 0.f};
  int lev2;
  leaf2[p] = descend_split(to.tab, to.d, lev, I, f, on, &lev2);
  for (int a = 0; a < from.d; ++a) {
    o2[a * n + p] = on[a];
    v2[a * n + p] = v[a * n + p];
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

cudaError_t set_constants(cudaStream_t s) {
  uint32_t p3[21];
  p3[0] = 1;
  for (int i = 1; i < 21; ++i) p3[i] = p3[i - 1] * 3u;
  cudaError_t e = cudaFuncSetAttribute(k_sort_large, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(int32_t) * kLargeSeg));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_sort_medium, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(int32_t) * kMedSeg * (kMedThreads / 32)));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbolAsync(c_pow3, p3, sizeof(p3), 0, cudaMemcpyHostToDevice, s);
}

cudaError_t set_kref(int d, cudaStream_t s) {
  double k64[8][8];
  float k32[8][8];
  int nc = 1 << d;
  for (int e = 0; e < 8; ++e)
    for (int f = 0; f < 8; ++f) {
      double v = 0.0;
      if (e < nc && f < nc) {
        int diff = __builtin_popcount((unsigned)(e ^ f));
        if (d == 2) {
          const double k2[3] = {4.0 / 6.0, -1.0 / 6.0, -2.0 / 6.0};
          v = k2[diff];
        } else {
          const double k3[4] = {4.0 / 12.0, 0.0, -1.0 / 12.0, -1.0 / 12.0};
          v = k3[diff];
        }
      }
      k64[e][f] = v;
      k32[e][f] = (float)v;
    }
  cudaError_t err = cudaMemcpyToSymbolAsync(c_kref64, k64, sizeof(k64), 0, cudaMemcpyHostToDevice, s);
  if (err != cudaSuccess) return err;
  return cudaMemcpyToSymbolAsync(c_kref32, k32, sizeof(k32), 0, cudaMemcpyHostToDevice, s);
}

void launch_init64(const DevTree &t, double *x, int64_t n, int32_t *leaf, int32_t *key, int32_t *err,
                   cudaStream_t s) {
  if (n > 0) { COUNT(1); k_init64<<<grid_for(n), kBlock, 0, s>>>(t, x, n, leaf, key, err); }
}

void launch_init32(const DevTree &t, const double *x, const double *v, int64_t n, int32_t *leaf, float *o,
                   float *vf, int32_t *key, int32_t *err, cudaStream_t s) {
  if (n > 0) { COUNT(1); k_init32<<<grid_for(n), kBlock, 0, s>>>(t, x, v, n, leaf, o, vf, key, err); }
}

void launch_rekey32(const DevTree &t, const int32_t *leaf, const float *o, int64_t n, int32_t *key, int32_t *err,
                    cudaStream_t s) {
  if (n > 0) { COUNT(1); k_rekey32<<<grid_for(n), kBlock, 0, s>>>(t, leaf, o, n, key, err); }
}

void launch_count_all(const int32_t *key, int64_t n, int32_t *count, uint32_t *mover_words,
                      int32_t *block_movers, int block, cudaStream_t s) {
  const int b = bsz(block);
  { COUNT(1); k_count_all<<<grid_for(n, b), b, 0, s>>>(key, n, count, mover_words, block_movers); }
}

// Flag = 1 if keys are not in ascending order.
__global__ void k_check_sorted(const int32_t *key, int64_t n, int32_t *flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool bad = i + 1 < n && key[i] > key[i + 1];
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

void launch_check_sorted(const int32_t *key, int64_t n, int32_t *flag, cudaStream_t s) {
  if (n > 1) { COUNT(1); k_check_sorted<<<grid_for(n), kBlock, 0, s>>>(key, n, flag); }
}

void launch_fine_keys(const DevTree &t, bool split, const void *pos, const int32_t *leaf, int64_t n, int dmax,
                      uint32_t *key, cudaStream_t s) {
  if (n <= 0) return;
  COUNT(1);
  if (split)
    k_fine_key32<<<grid_for(n), kBlock, 0, s>>>(t, leaf, (const float *)pos, n, dmax, key);
  else
    k_fine_key64<<<grid_for(n), kBlock, 0, s>>>(t, (const double *)pos, n, dmax, key);
}

void launch_adapt_bits(const uint32_t *key, int64_t n, int nch, int dmin, int dmax, int64_t ppc, int32_t *count,
                       const int64_t *cnt_off, uint32_t *bits, const int64_t *bit_off, cudaStream_t s) {
  if (dmax <= dmin) return;
  int64_t ncells = 1;
  for (int m = 0; m < dmax - 1; ++m) ncells *= nch;
  int32_t *fine = count + cnt_off[dmax - 1];
  cudaMemsetAsync(fine, 0, sizeof(int32_t) * ncells, s);
  if (n > 0) { COUNT(1); k_level_count<<<grid_for(n), kBlock, 0, s>>>(key, n, (uint32_t)nch, fine); }
  for (int m = dmax - 1; m >= dmin; --m) {
    if (m < dmax - 1) {
      COUNT(1);
      k_count_parent<<<grid_for(ncells), kBlock, 0, s>>>(count + cnt_off[m + 1], ncells, nch, count + cnt_off[m]);
    }
    COUNT(1);
    k_threshold_bits<<<grid_for((ncells + 31) / 32), kBlock, 0, s>>>(count + cnt_off[m], ncells, ppc,
                                                                    bits + bit_off[m]);
    ncells /= nch;
  }
}

void launch_adapt_check(const DevTree &t, const int32_t *count, const int64_t *coff, int dmin, int dmax, int64_t ppc,
                        int32_t *changed, cudaStream_t s) {
  AdaptCheck ac{};
  ac.count = count;
  for (int m = 0; m <= dmax && m < 11; ++m) ac.coff[m] = coff[m];
  ac.dmin = dmin;
  ac.dmax = dmax;
  ac.ppc = ppc;
  if (t.n_leaves > 0) { COUNT(1); k_adapt_check<<<grid_for(t.n_leaves), kBlock, 0, s>>>(t, ac, changed); }
}

void launch_relocate32(const DevTree &from, const DevTree &to, const int32_t *leaf, const float *o, const float *v,
                       int64_t n, int32_t *leaf2, float *o2, float *v2, cudaStream_t s) {
  if (n <= 0) return;
  COUNT(1);
  k_relocate32<<<grid_for(n), kBlock, 0, s>>>(from, to, leaf, o, v, n, leaf2, o2, v2);
}

// Per-instance FP64 sums of the vertex charges, one block per instance (fixed order).
template <typename T>
__global__ void k_inst_sum(DevTree t, const T *Q, double *out) {
  const InstInfo &I = t.inst[blockIdx.x];
  double v = 0.0;
  for (int64_t i = threadIdx.x; i < I.n_vert; i += blockDim.x) v += (double)Q[I.vert_off + i];
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) out[blockIdx.x] = v;
  }
}

void launch_vertex_charge(const DevTree &t, bool split, const void *part, void *Q, double *block_sum,
                          double *total, cudaStream_t s) {
  if (split) {
    { COUNT(1); k_vertex_charge<float><<<grid_for(t.n_vert, bsz(t.block_vert)), bsz(t.block_vert), 0, s>>>(t, (const float *)part, (float *)Q, block_sum); }
  } else {
    { COUNT(1); k_vertex_charge<double><<<grid_for(t.n_vert, bsz(t.block_vert)), bsz(t.block_vert), 0, s>>>(t, (const double *)part, (double *)Q, block_sum); }
  }
  if (t.n_inst > 1) {
    COUNT(2);
    if (split)
      k_inst_sum<float><<<t.n_inst, 256, 0, s>>>(t, (const float *)Q, total + 1);
    else
      k_inst_sum<double><<<t.n_inst, 256, 0, s>>>(t, (const double *)Q, total + 1);
    k_sum_blocks<<<1, 1024, 0, s>>>(total + 1, t.n_inst, total);
  } else {
    COUNT(1);
    k_sum_blocks<<<1, 1024, 0, s>>>(block_sum, grid_for(t.n_vert, bsz(t.block_vert)), total);
  }
}

void launch_deposit(const DevTree &t, bool split, const int32_t *start, const void *pos, int64_t n, void *part,
                    void *Q, double *block_sum, double *total, cudaStream_t s) {
  if (split) {
    { COUNT(1); if (t.d == 3) k_leaf_partials<true, 3><<<grid_for(t.n_leaves, bsz(t.block_leaf)), bsz(t.block_leaf), 0, s>>>(t, start, pos, n, part);
      else k_leaf_partials<true, 2><<<grid_for(t.n_leaves, bsz(t.block_leaf)), bsz(t.block_leaf), 0, s>>>(t, start, pos, n, part); }
  } else {
    { COUNT(1); if (t.d == 3) k_leaf_partials<false, 3><<<grid_for(t.n_leaves, bsz(t.block_leaf)), bsz(t.block_leaf), 0, s>>>(t, start, pos, n, part);
      else k_leaf_partials<false, 2><<<grid_for(t.n_leaves, bsz(t.block_leaf)), bsz(t.block_leaf), 0, s>>>(t, start, pos, n, part); }
  }
  launch_vertex_charge(t, split, part, Q, block_sum, total, s);
}

void launch_solve(const DevTree &t, bool split, const void *Q, const double *total, void *b, void *V, void *Vtmp,
                  int sweeps, double omega, double *block_sum, double *resid2, cudaStream_t s) {
  unsigned g = grid_for(t.n_vert);
  if (split) {
    { COUNT(1); k_rhs<float><<<g, kBlock, 0, s>>>(t, (const float *)Q, total, (float *)b); }
    float *a = (float *)V, *c = (float *)Vtmp;
    for (int it = 0; it < sweeps; ++it) {
      { COUNT(1); k_jacobi<float><<<g, kBlock, 0, s>>>(t, (const float *)b, a, c, (float)omega, nullptr); }
      float *tmp = a; a = c; c = tmp;
    }
    if (a != (float *)V) cudaMemcpyAsync(V, a, sizeof(float) * t.n_vert, cudaMemcpyDeviceToDevice, s);
    { COUNT(1); k_jacobi<float><<<g, kBlock, 0, s>>>(t, (const float *)b, (const float *)V, nullptr, (float)omega, block_sum); }
  } else {
    { COUNT(1); k_rhs<double><<<g, kBlock, 0, s>>>(t, (const double *)Q, total, (double *)b); }
    double *a = (double *)V, *c = (double *)Vtmp;
    for (int it = 0; it < sweeps; ++it) {
      { COUNT(1); k_jacobi<double><<<g, kBlock, 0, s>>>(t, (const double *)b, a, c, omega, nullptr); }
      double *tmp = a; a = c; c = tmp;
    }
    if (a != (double *)V) cudaMemcpyAsync(V, a, sizeof(double) * t.n_vert, cudaMemcpyDeviceToDevice, s);
    { COUNT(1); k_jacobi<double><<<g, kBlock, 0, s>>>(t, (const double *)b, (const double *)V, nullptr, omega, block_sum); }
  }
  { COUNT(1); k_sum_blocks<<<1, 1024, 0, s>>>(block_sum, g, resid2); }
}

void launch_efield(const DevTree &t, bool split, const void *V, void *E, cudaStream_t s) {
  if (split)
    { COUNT(1); k_efield<float><<<grid_for(t.n_vert), kBlock, 0, s>>>(t, (const float *)V, (float *)E); }
  else
    { COUNT(1); k_efield<double><<<grid_for(t.n_vert), kBlock, 0, s>>>(t, (const double *)V, (double *)E); }
}

void launch_push64(const DevTree &t, const Push64Args &a, cudaStream_t s) {
  COUNT(1);
  if (t.d == 3) k_push64<3><<<grid_for(a.n, bsz(t.block_push)), bsz(t.block_push), 0, s>>>(t, a);
  else k_push64<2><<<grid_for(a.n, bsz(t.block_push)), bsz(t.block_push), 0, s>>>(t, a);
}

// Field at every leaf corner: the same expansion sums the push would form
// per particle (corner_value), once per leaf corner.
__global__ void k_corner_field32(DevTree t, const float *__restrict__ E, float4 *__restrict__ Ec) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.n_leaves * t.nc) return;
  const int32_t L = (int32_t)(i / t.nc);
  const int e = (int)(i - (int64_t)L * t.nc);
  int lev;
  int32_t c[3] = {0, 0, 0};
  leaf_info(t, L, &lev, c);
  float q[3] = {0.f, 0.f, 0.f};
  for (int ax = 0; ax < t.d; ++ax) q[ax] = corner_value(t, L, c, e, E + ax * t.n_vert);
  Ec[i] = make_float4(q[0], q[1], q[2], 0.f);
}

void launch_corner_field32(const DevTree &t, const float *E, float4 *Ec, cudaStream_t s) {
  const int64_t m = t.n_leaves * t.nc;
  { COUNT(1); k_corner_field32<<<grid_for(m, 256), 256, 0, s>>>(t, E, Ec); }
}

void launch_push32(const DevTree &t, const Push32Args &a, cudaStream_t s) {
  COUNT(1);
  if (t.d == 3) k_push32<3><<<grid_for(a.n, bsz(t.block_push)), bsz(t.block_push), 0, s>>>(t, a);
  else k_push32<2><<<grid_for(a.n, bsz(t.block_push)), bsz(t.block_push), 0, s>>>(t, a);
}

int64_t scan_tiles_needed(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

void launch_exclusive_scan(const int32_t *in, int64_t n, int32_t *out, int32_t *tile_sums, int32_t *total,
                           cudaStream_t s) {
  int64_t nt = scan_tiles_needed(n);
  if (nt < 1) nt = 1;
  { COUNT(1); k_scan_reduce<<<(unsigned)nt, kScanThreads, 0, s>>>(in, n, tile_sums); }
  { COUNT(1); k_scan_tiles<<<1, kScanThreads, 0, s>>>(tile_sums, nt, total); }
  { COUNT(1); k_scan_apply<<<(unsigned)nt, kScanThreads, 0, s>>>(in, n, tile_sums, out, total); }
}

void launch_rebin(const RebinArgs &r, cudaStream_t s) {
  // bucket offsets
  launch_exclusive_scan(r.count, r.n_keys, r.new_start, r.tile_sums, r.scalars + 0, s);
  // mover list in storage order
  const int bp = bsz(r.block);
  unsigned gp = grid_for(r.n, bp);
  launch_exclusive_scan(r.block_movers, gp, r.block_offsets, r.tile_sums2, r.scalars + 1, s);
  if (r.old_start)
    { COUNT(1); k_stayers<<<grid_for(r.n_keys), kBlock, 0, s>>>(r.old_start, r.keyn, r.new_start, r.n_keys, r.perm, r.n_stay,
                                                    r.scalars + 2); }
  else
    cudaMemsetAsync(r.n_stay, 0, sizeof(int32_t) * r.n_keys, s);
  { COUNT(1); k_compact_movers<<<gp, bp, 0, s>>>(r.mover_words, r.block_offsets, r.n, r.movers); }
  cudaMemsetAsync(r.cursor, 0, sizeof(int32_t) * r.n_keys, s);
  { COUNT(1); k_mover_slots<<<gp, bp, 0, s>>>(r.movers, r.scalars + 1, r.keyn, r.new_start, r.n_stay, r.cursor, r.perm); }
  cudaMemsetAsync(r.scalars + 5, 0, sizeof(int32_t), s);
  cudaMemsetAsync(r.scalars + 7, 0, sizeof(int32_t), s);
  // the mover list is no longer needed: it holds the list of medium segments
  { COUNT(1); k_sort_segments<<<grid_for(r.n_keys), kBlock, 0, s>>>(r.new_start, r.n_stay, r.n_keys, r.perm, r.cursor,
                                                                      r.scalars + 5, r.movers, r.scalars + 7); }
  { COUNT(1); k_sort_medium<<<456, kMedThreads, sizeof(int32_t) * kMedSeg * (kMedThreads / 32), s>>>(
      r.new_start, r.n_stay, r.movers, r.scalars + 7, r.perm); }
  { COUNT(1); k_sort_large<<<304, kLargeThreads, sizeof(int32_t) * kLargeSeg, s>>>(r.new_start, r.n_stay, r.cursor,
                                                                                  r.scalars + 5, r.perm); }
}

void launch_gather_state(bool split, const int32_t *perm, int64_t n, int d, const void *x, void *x2, const void *v,
                         void *v2, const int32_t *leaf, int32_t *leaf2, const int32_t *key, int32_t *key2,
                         const int32_t *ids, int32_t *ids2, cudaStream_t s) {
  if (n <= 0) return;
  COUNT(1);
  if (split)
    k_gather_state<float><<<grid_for(n), kBlock, 0, s>>>(perm, n, d, (const float *)x, (float *)x2, (const float *)v,
                                                          (float *)v2, leaf, leaf2, key, key2, ids, ids2);
  else
    k_gather_state<double><<<grid_for(n), kBlock, 0, s>>>(perm, n, d, (const double *)x, (double *)x2,
                                                           (const double *)v, (double *)v2, leaf, leaf2, key, key2,
                                                           ids, ids2);
}

void launch_gather_records(bool split, const int32_t *perm, int64_t n, int d, const void *rec, void *x2, void *v2,
                           int32_t *leaf2, int32_t *key2, const int32_t *ids, int32_t *ids2, cudaStream_t s) {
  if (n <= 0) return;
  COUNT(1);
  if (split)
    k_gather_rec32<<<grid_for(n), kBlock, 0, s>>>(perm, n, d, (const float4 *)rec, (float *)x2, (float *)v2, leaf2,
                                                   key2, ids, ids2);
  else
    k_gather_rec64<<<grid_for(n), kBlock, 0, s>>>(perm, n, d, (const double2 *)rec, (double *)x2, (double *)v2,
                                                   leaf2, key2, ids, ids2);
}

void launch_gather_f64(const int32_t *perm, int64_t n, int d, const double *src, double *dst, cudaStream_t s) {
  if (n > 0) { COUNT(1); k_gather_vec<double><<<grid_for(n), kBlock, 0, s>>>(perm, n, d, src, dst); }
}
void launch_gather_f32(const int32_t *perm, int64_t n, int d, const float *src, float *dst, cudaStream_t s) {
  if (n > 0) { COUNT(1); k_gather_vec<float><<<grid_for(n), kBlock, 0, s>>>(perm, n, d, src, dst); }
}
void launch_gather_i32(const int32_t *perm, int64_t n, const int32_t *src, int32_t *dst, cudaStream_t s) {
  if (n > 0) { COUNT(1); k_gather_vec<int32_t><<<grid_for(n), kBlock, 0, s>>>(perm, n, 1, src, dst); }
}

void launch_absolute_split(const DevTree &t, const int32_t *leaf, const float *o, int64_t n, double *x,
                           cudaStream_t s) {
  if (n > 0) { COUNT(1); k_absolute_split<<<grid_for(n), kBlock, 0, s>>>(t, leaf, o, n, x); }
}

void launch_widen(const float *in, int64_t n, double *out, cudaStream_t s) {
  if (n > 0) { COUNT(1); k_widen<<<grid_for(n), kBlock, 0, s>>>(in, n, out); }
}

void launch_gather_only(const DevTree &t, bool split, const void *pos, const int32_t *leaf, int64_t n,
                        const void *Ev, void *Ep, cudaStream_t s) {
  if (n <= 0) return;
  if (split)
    { COUNT(1); k_gather_only32<<<grid_for(n), kBlock, 0, s>>>(t, (const float *)pos, leaf, n, (const float *)Ev, (float *)Ep); }
  else
    { COUNT(1); k_gather_only64<<<grid_for(n), kBlock, 0, s>>>(t, (const double *)pos, leaf, n, (const double *)Ev,
                                                   (double *)Ep); }
}

// ---------------------------------------------------------------------------
// Lift and drop counts of Algorithm 1 (diagnostic, PIT)
// ---------------------------------------------------------------------------

// The leaf of every particle before a step, by particle id.
__global__ void k_scatter_by_id(const int32_t *ids, const int32_t *leaf, int64_t n, int32_t *by_id) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int32_t id = ids[p];
  if (id >= 0 && id < n) by_id[id] = leaf[p];
}

// True when the closed boxes of leaves L1 and L2 share a point (periodic),
// compared on the finer of the two levels.
__device__ __forceinline__ bool leaves_touch(const DevTree &t, int32_t L1, int32_t L2) {
  const int l1 = t.leaf_level[L1], l2 = t.leaf_level[L2];
  const int lm = l1 > l2 ? l1 : l2;
  const int64_t s1 = c_pow3[lm - l1], s2 = c_pow3[lm - l2], P = c_pow3[lm];
  for (int a = 0; a < t.d; ++a) {
    const int64_t lo1 = (int64_t)t.leaf_coords[(int64_t)L1 * t.d + a] * s1;
    const int64_t lo2 = (int64_t)t.leaf_coords[(int64_t)L2 * t.d + a] * s2;
    int64_t d12 = (lo2 - lo1) % P, d21 = (lo1 - lo2) % P;
    if (d12 < 0) d12 += P;
    if (d21 < 0) d21 += P;
    if (d12 > s1 && d21 > s2) return false;
  }
  return true;
}

// Warp sums of (lifts, drops, tunnellers) into counts[0..2].
__device__ __forceinline__ void add_counts(unsigned lifts, unsigned drops, unsigned tun, unsigned long long *counts) {
  for (int off = 16; off > 0; off >>= 1) {
    lifts += __shfl_down_sync(0xffffffffu, lifts, off);
    drops += __shfl_down_sync(0xffffffffu, drops, off);
    tun += __shfl_down_sync(0xffffffffu, tun, off);
  }
  if ((threadIdx.x & 31) == 0) {
    if (lifts) atomicAdd(&counts[0], (unsigned long long)lifts);
    if (drops) atomicAdd(&counts[1], (unsigned long long)drops);
    if (tun) atomicAdd(&counts[2], (unsigned long long)tun);
  }
}

// A particle that went from leaf L1 (level l1, coordinates c1) to leaf L2 is
// lifted out of every cell from L1 up to the deepest ancestor that contains
// L2, then dropped down to L2: lifts = l1 - m, drops = l2 - m with m the level
// of that ancestor (levels and coordinates of one instance's tree).  It
// tunnelled when L2 does not touch L1.  Warp sums go to counts[0] (lifts),
// counts[1] (drops) and counts[2] (tunnellers).
__global__ void k_lift_drop(DevTree t, const int32_t *ids, const int32_t *leaf, const int32_t *old_by_id, int64_t n,
                            unsigned long long *counts) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned lifts = 0, drops = 0, tun = 0;
  if (p < n) {
    const int32_t id = ids[p];
    const int32_t L2 = leaf[p];
    const int32_t L1 = (id >= 0 && id < n) ? old_by_id[id] : -1;
    if (L1 >= 0 && L1 < t.n_leaves && L2 >= 0 && L2 < t.n_leaves) {
      const int l1 = t.leaf_level[L1], l2 = t.leaf_level[L2];
      int m = l1 < l2 ? l1 : l2;
      uint32_t a1[3] = {0u, 0u, 0u}, a2[3] = {0u, 0u, 0u};
      for (int a = 0; a < t.d; ++a) {
        a1[a] = (uint32_t)t.leaf_coords[(int64_t)L1 * t.d + a] / c_pow3[l1 - m];
        a2[a] = (uint32_t)t.leaf_coords[(int64_t)L2 * t.d + a] / c_pow3[l2 - m];
      }
      while (m > 0 && (a1[0] != a2[0] || a1[1] != a2[1] || a1[2] != a2[2])) {
        for (int a = 0; a < 3; ++a) {
          a1[a] /= 3u;
          a2[a] /= 3u;
        }
        --m;
      }
      lifts = (unsigned)(l1 - m);
      drops = (unsigned)(l2 - m);
      tun = leaves_touch(t, L1, L2) ? 0u : 1u;
    }
  }
  add_counts(lifts, drops, tun, counts);
}

// Owner vertex (level, j) of PIDT key k (owner vertex id = k / 2^d): the
// finite-element vertex of a uniform tree (row-major on the finest level),
// else the owner-vertex table.
__device__ __forceinline__ int pidt_owner(const DevTree &t, const int32_t *pv_level, const int32_t *pv_j, int32_t k,
                                          int64_t *j) {
  const int32_t pv = k / t.nc;
  if (t.uniform) {
    int64_t v = pv;
    for (int a = 0; a < t.d; ++a) {
      j[a] = v % t.M;
      v /= t.M;
    }
    return t.depth;
  }
  for (int a = 0; a < t.d; ++a) j[a] = pv_j[(int64_t)pv * t.d + a];
  return pv_level[pv];
}

// Lifts and drops of PIDT (reading of Algorithms 2-3 as a count): a particle
// whose new owner is a vertex of its old leaf on that leaf's level is handed
// over inside the cell (none); any other is lifted from its old vertex to the
// deepest dual ancestor whose dual cell holds both owners' dual cells and
// dropped to the new owner, the dual parent of (l, j) being
// (l - 1, (j + 1) div 3).  Tunnellers as for PIT, from the leaves.
__global__ void k_lift_drop_pidt(DevTree t, const int32_t *pv_level, const int32_t *pv_j, const int32_t *ids,
                                 const int32_t *leaf, const int32_t *key, const int32_t *old_leaf_by_id,
                                 const int32_t *old_key_by_id, int64_t n, unsigned long long *counts) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned lifts = 0, drops = 0, tun = 0;
  if (p < n) {
    const int32_t id = ids[p];
    const int32_t L2 = leaf[p], k2 = key[p];
    const bool ok = id >= 0 && id < n;
    const int32_t L1 = ok ? old_leaf_by_id[id] : -1, k1 = ok ? old_key_by_id[id] : -1;
    if (L1 >= 0 && L1 < t.n_leaves && L2 >= 0 && L2 < t.n_leaves && k1 >= 0 && k1 < t.n_keys && k2 >= 0 &&
        k2 < t.n_keys) {
      tun = leaves_touch(t, L1, L2) ? 0u : 1u;
      if (k1 / t.nc != k2 / t.nc) {
        int64_t j1[3] = {0, 0, 0}, j2[3] = {0, 0, 0};
        const int l1 = pidt_owner(t, pv_level, pv_j, k1, j1);
        const int l2 = pidt_owner(t, pv_level, pv_j, k2, j2);
        const int ll = t.leaf_level[L1];
        const int64_t per = c_pow3[ll];
        bool handed = l2 == ll;
        for (int a = 0; a < t.d && handed; ++a) {
          int64_t r = (j2[a] - t.leaf_coords[(int64_t)L1 * t.d + a]) % per;
          if (r < 0) r += per;
          handed = r <= 1;
        }
        if (!handed) {
          int m = l1 < l2 ? l1 : l2;
          for (int l = l1; l > m; --l)
            for (int a = 0; a < t.d; ++a) j1[a] = ((j1[a] + 1) / 3) % (int64_t)c_pow3[l - 1];
          for (int l = l2; l > m; --l)
            for (int a = 0; a < t.d; ++a) j2[a] = ((j2[a] + 1) / 3) % (int64_t)c_pow3[l - 1];
          while (m > 0 && (j1[0] != j2[0] || j1[1] != j2[1] || j1[2] != j2[2])) {
            for (int a = 0; a < t.d; ++a) {
              j1[a] = ((j1[a] + 1) / 3) % (int64_t)c_pow3[m - 1];
              j2[a] = ((j2[a] + 1) / 3) % (int64_t)c_pow3[m - 1];
            }
            --m;
          }
          lifts = (unsigned)(l1 - m);
          drops = (unsigned)(l2 - m);
        }
      }
    }
  }
  add_counts(lifts, drops, tun, counts);
}

void launch_scatter_by_id(const int32_t *ids, const int32_t *leaf, int64_t n, int32_t *by_id, cudaStream_t s) {
  if (n > 0) { COUNT(1); k_scatter_by_id<<<grid_for(n), kBlock, 0, s>>>(ids, leaf, n, by_id); }
}

void launch_lift_drop(const DevTree &t, const int32_t *ids, const int32_t *leaf, const int32_t *old_by_id, int64_t n,
                      unsigned long long *counts, cudaStream_t s) {
  if (n > 0) { COUNT(1); k_lift_drop<<<grid_for(n), kBlock, 0, s>>>(t, ids, leaf, old_by_id, n, counts); }
}

void launch_lift_drop_pidt(const DevTree &t, const int32_t *pv_level, const int32_t *pv_j, const int32_t *ids,
                           const int32_t *leaf, const int32_t *key, const int32_t *old_leaf_by_id,
                           const int32_t *old_key_by_id, int64_t n, unsigned long long *counts, cudaStream_t s) {
  if (n > 0) {
    COUNT(1);
    k_lift_drop_pidt<<<grid_for(n), kBlock, 0, s>>>(t, pv_level, pv_j, ids, leaf, key, old_leaf_by_id, old_key_by_id,
                                                    n, counts);
  }
}

// ---------------------------------------------------------------------------
// raPIDT tree attribute v_max (Section 5.4)
// ---------------------------------------------------------------------------

// Per leaf: the largest velocity component magnitude of its particles -- PIT:
// the leaf's bucket; PIDT: the buckets of the leaf's 2^d vertices, i.e. every
// dual cell intersecting the leaf (the paper's definition).
template <typename T>
__global__ void k_leaf_vmax(DevTree t, const int32_t *__restrict__ start, const T *__restrict__ v, int64_t n,
                            double *leaf_vmax) {
  const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= t.n_leaves) return;
  double m = 0.0;
  const int na = t.scheme == 0 ? 1 : t.nc;
  for (int a = 0; a < na; ++a) {
    int32_t k0, k1;
    if (t.scheme == 0) {
      k0 = (int32_t)L;
      k1 = k0 + 1;
    } else {
      k0 = pidt_vertex(t, (int32_t)L, a) * t.nc;
      k1 = k0 + t.nc;
    }
    for (int32_t p = start[k0]; p < start[k1]; ++p)
      for (int ax = 0; ax < t.d; ++ax) {
        const double x = fabs((double)v[ax * n + p]);
        m = x > m ? x : m;
      }
  }
  leaf_vmax[L] = m;
}

// Per tree node of one level (level order): a leaf takes its leaf's value,
// a refined node the largest of its 3^d children's (Eq. v_max).
__global__ void k_node_vmax(const int32_t *child0, const int32_t *leaf_of_node, int64_t b, int64_t e, int nch,
                            const double *leaf_vmax, double *node_vmax) {
  const int64_t i = b + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= e) return;
  if (leaf_of_node[i] >= 0) {
    node_vmax[i] = leaf_vmax[leaf_of_node[i]];
    return;
  }
  double m = 0.0;
  for (int k = 0; k < nch; ++k) {
    const double x = node_vmax[child0[i] + k];
    m = x > m ? x : m;
  }
  node_vmax[i] = m;
}

void launch_vmax(const DevTree &t, bool split, const int32_t *start, const void *v, int64_t n, const int32_t *child0,
                 const int32_t *leaf_of_node, const int64_t *level_begin, int depth, double *leaf_vmax,
                 double *node_vmax, cudaStream_t s) {
  COUNT(1);
  if (split)
    k_leaf_vmax<float><<<grid_for(t.n_leaves), kBlock, 0, s>>>(t, start, (const float *)v, n, leaf_vmax);
  else
    k_leaf_vmax<double><<<grid_for(t.n_leaves), kBlock, 0, s>>>(t, start, (const double *)v, n, leaf_vmax);
  for (int l = depth; l >= 0; --l) {
    const int64_t b = level_begin[l], e = level_begin[l + 1];
    if (e <= b) continue;
    COUNT(1);
    k_node_vmax<<<grid_for(e - b), kBlock, 0, s>>>(child0, leaf_of_node, b, e, t.nch, leaf_vmax, node_vmax);
  }
}

void launch_half_kick(bool split, const void *Ep, int64_t n_total, double c, void *v, cudaStream_t s) {
  if (n_total <= 0) return;
  if (split)
    { COUNT(1); k_half_kick32<<<grid_for(n_total), kBlock, 0, s>>>((const float *)Ep, n_total, (float)c, (float *)v); }
  else
    { COUNT(1); k_half_kick64<<<grid_for(n_total), kBlock, 0, s>>>((const double *)Ep, n_total, c, (double *)v); }
}

}  // namespace pic
