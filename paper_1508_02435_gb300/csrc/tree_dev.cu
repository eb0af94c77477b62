// Device tabulation of an adaptive spacetree: the d-linear finite-element
// grid of Section 3 on the leaves of the Section 4 tree (grid points, hanging
// points and their constraint expansions, leaf-corner -> vertex expansions,
// their transpose, per-vertex ion load, stiffness diagonal and direct-corner
// count) and the PIDT owner vertices of Section 5.2 (the distinct (level, j)
// pairs of leaf corners).  The tables equal those of the host tabulation
// (csrc/tree.cpp): the same points, numbering, expansion order and floating-
// point operations in the same order.
//
// Points are marked in a dense bitmap over the finest lattice (one bit per
// row-major point key), so a point's id is the number of marked keys below
// it; the PIDT owners use one bitmap per level.  Hanging points are expanded
// level by level of their coarsest incident leaf: the masters of a hanging
// point are corners of a coarser leaf, so their expansions are complete when
// it is expanded.
//
// Device code is compiled with --fmad=false: every + - * / is one IEEE
// round-to-nearest operation in program order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "dev.cuh"
#include "launch.hpp"
#include "segsort.cuh"
#include "tree_dev.hpp"

namespace pic {

namespace {

constexpr int kTB = 256;
constexpr int kHexCap = 64;          // entries of one hanging point's expansion
constexpr int kSmallSeg = 32;        // vertex incidence lists sorted by one thread up to this length

unsigned grid_of(int64_t n) {
  int64_t g = (n + kTB - 1) / kTB;
  return (unsigned)(g < 1 ? 1 : g);
}

// Per leaf level l: the corner integral of a unit density, (3^-l)^d / 2^d,
// and the stiffness scale (1 in 2D, 3^-l in 3D), formed on the host by the
// same operations as the host tabulation forms them per leaf.
__constant__ double c_tg_cint[kMaxLevel + 1], c_tg_hs[kMaxLevel + 1];

struct HexEntry {
  int32_t pid;
  int32_t pad;
  double w;
};

// View of the tree and the point bitmap shared by the kernels.
struct TV {
  int d, nc, depth;
  int64_t M;
  const TabEntry *tab;
  const uint8_t *leaf_level;
  const int32_t *leaf_coords;
  const uint32_t *bits;     // one bit per finest-lattice point key
  const int32_t *wpre;      // marked bits before each word
};

__device__ __forceinline__ int64_t p3_64(int k) {
  int64_t r = 1;
  for (int i = 0; i < k; ++i) r *= 3;
  return r;
}

__device__ __forceinline__ int32_t point_rank(const TV &v, uint64_t key) {
  const uint64_t w = key >> 5;
  const uint32_t below = v.bits[w] & ((1u << (key & 31u)) - 1u);
  return v.wpre[w] + __popc(below);
}

// Row-major key of leaf corner e of leaf L on the finest lattice (periodic).
__device__ __forceinline__ uint64_t corner_key(const TV &v, int64_t L, int e) {
  const int lev = v.leaf_level[L];
  const int64_t s = p3_64(v.depth - lev);
  uint64_t k = 0, m = 1;
  for (int a = 0; a < v.d; ++a) {
    int64_t q = ((int64_t)v.leaf_coords[L * v.d + a] + ((e >> a) & 1)) * s;
    if (q >= v.M) q -= v.M;
    k += (uint64_t)q * m;
    m *= (uint64_t)v.M;
  }
  return k;
}

__global__ void k_tg_mark(TV v, int64_t nlc, uint64_t *ckey, uint32_t *bits) {
  const int64_t lc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (lc >= nlc) return;
  const uint64_t k = corner_key(v, lc / v.nc, (int)(lc % v.nc));
  ckey[lc] = k;
  atomicOr(&bits[k >> 5], 1u << (k & 31u));
}

__global__ void k_tg_popc(const uint32_t *bits, int64_t nw, int32_t *cnt) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w < nw) cnt[w] = __popc(bits[w]);
}

// The marked keys in ascending order (the point keys); base_bit is the bit
// index of bits[0] (PIDT levels keep their keys relative to their level).
__global__ void k_tg_keys(const uint32_t *bits, const int32_t *wpre, int64_t nw, int64_t base_bit, uint64_t *out) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nw) return;
  uint32_t b = bits[w];
  int32_t at = wpre[w];
  while (b) {
    const int pos = __ffs(b) - 1;
    out[at++] = (uint64_t)(w * 32 + pos) - (uint64_t)base_bit;
    b &= b - 1u;
  }
}

__global__ void k_tg_corner_pt(TV v, const uint64_t *ckey, int64_t nlc, int32_t *corner_pt) {
  const int64_t lc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (lc < nlc) corner_pt[lc] = point_rank(v, ckey[lc]);
}

// Per point: the coarsest leaf whose closure holds it (the first of minimal
// level among the leaves of the 2^d finest cells around it) and whether the
// point is one of that leaf's corners (non-hanging) or not (hanging).
__global__ void k_tg_hanging(TV v, const uint64_t *pkey, int64_t np, uint8_t *hanging, int32_t *best_leaf,
                             uint8_t *best_level) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= np) return;
  int64_t p[3] = {0, 0, 0};
  uint64_t k = pkey[id];
  for (int a = 0; a < v.d; ++a) {
    p[a] = (int64_t)(k % (uint64_t)v.M);
    k /= (uint64_t)v.M;
  }
  const uint32_t half = c_pow3[18 - v.depth];
  int32_t best = -1;
  int blev = 0;
  for (int e = 0; e < v.nc; ++e) {
    uint32_t Q[3] = {0u, 0u, 0u};
    for (int a = 0; a < v.d; ++a) {
      const int64_t c = ((e >> a) & 1) ? p[a] : (p[a] == 0 ? v.M - 1 : p[a] - 1);
      Q[a] = (uint32_t)(2 * c + 1) * half;
    }
    int lev;
    const int32_t L = descend_q(v.tab, v.d, Q, &lev);
    if (best < 0 || lev < blev) {
      best = L;
      blev = lev;
    }
  }
  const int64_t s = p3_64(v.depth - blev);
  bool corner = true;
  for (int a = 0; a < v.d; ++a) {
    int64_t rr = p[a] - (int64_t)v.leaf_coords[(int64_t)best * v.d + a] * s;
    if (rr < 0) rr += v.M;
    if (rr != 0 && rr != s) corner = false;
  }
  hanging[id] = corner ? 0 : 1;
  best_leaf[id] = best;
  best_level[id] = (uint8_t)blev;
}

// Hanging points by the level of their coarsest leaf.
__global__ void k_tg_level_count(const uint8_t *hanging, const uint8_t *best_level, int64_t np, int32_t *lcount) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id < np && hanging[id]) atomicAdd(&lcount[best_level[id]], 1);
}

__global__ void k_tg_level_lists(const uint8_t *hanging, const uint8_t *best_level, int64_t np,
                                 const int32_t *loff, int32_t *lcursor, int32_t *list) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id < np && hanging[id]) {
    const int l = best_level[id];
    list[loff[l] + atomicAdd(&lcursor[l], 1)] = (int32_t)id;
  }
}

// The constraint expansion of hanging point id onto non-hanging points, in
// the order of the host tabulation: the corners e of its coarsest leaf in
// order, each weighted by the d-linear shape value at the point (products of
// the per-axis fractions in axis order); a non-hanging corner contributes
// itself, a hanging one its own expansion scaled by that weight; entries of
// the same point are summed in that order.  Returns the length, or -1 when it
// would exceed cap.
__device__ int expand_point(const TV &v, const uint64_t *pkey, const uint8_t *hanging, const int32_t *best_leaf,
                            const uint8_t *best_level, HexEntry *const *hx_ptr, const int32_t *hx_len,
                            int32_t id, HexEntry *buf, int cap) {
  int64_t p[3] = {0, 0, 0};
  uint64_t k = pkey[id];
  for (int a = 0; a < v.d; ++a) {
    p[a] = (int64_t)(k % (uint64_t)v.M);
    k /= (uint64_t)v.M;
  }
  const int32_t best = best_leaf[id];
  const int64_t s = p3_64(v.depth - best_level[id]);
  int64_t r[3] = {0, 0, 0}, cb[3] = {0, 0, 0};
  for (int a = 0; a < v.d; ++a) {
    cb[a] = v.leaf_coords[(int64_t)best * v.d + a];
    int64_t rr = p[a] - cb[a] * s;
    if (rr < 0) rr += v.M;
    r[a] = rr;
  }
  int n = 0;
  bool over = false;
  auto add = [&](int32_t pid, double val) {
    for (int i = 0; i < n; ++i)
      if (buf[i].pid == pid) {
        buf[i].w += val;
        return;
      }
    if (n < cap) {
      buf[n].pid = pid;
      buf[n].w = val;
      ++n;
    } else {
      over = true;
    }
  };
  for (int e = 0; e < v.nc; ++e) {
    double w = 1.0;
    uint64_t key = 0, m = 1;
    for (int a = 0; a < v.d; ++a) {
      const int ea = (e >> a) & 1;
      w *= ea ? (double)r[a] / (double)s : (double)(s - r[a]) / (double)s;
      const int64_t q = ((cb[a] + ea) * s) % v.M;
      key += (uint64_t)q * m;
      m *= (uint64_t)v.M;
    }
    if (w == 0.0) continue;
    const int32_t cid = point_rank(v, key);
    if (!hanging[cid]) {
      add(cid, w * 1.0);
    } else {
      const HexEntry *src = hx_ptr[cid];
      for (int i = 0; i < hx_len[cid]; ++i) add(src[i].pid, w * src[i].w);
    }
  }
  return over ? -1 : n;
}

__global__ void k_tg_hex_size(TV v, const uint64_t *pkey, const uint8_t *hanging, const int32_t *best_leaf,
                              const uint8_t *best_level, HexEntry *const *hx_ptr, int32_t *hx_len,
                              const int32_t *list, int32_t n, int32_t *len_out, int32_t *err) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  HexEntry buf[kHexCap];
  const int m = expand_point(v, pkey, hanging, best_leaf, best_level, hx_ptr, hx_len, list[t], buf, kHexCap);
  if (m < 0) atomicOr(err, 1);
  len_out[t] = m < 0 ? 0 : m;
}

__global__ void k_tg_hex_fill(TV v, const uint64_t *pkey, const uint8_t *hanging, const int32_t *best_leaf,
                              const uint8_t *best_level, HexEntry **hx_ptr, int32_t *hx_len, const int32_t *list,
                              int32_t n, const int32_t *off, HexEntry *pool) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  HexEntry buf[kHexCap];
  const int32_t id = list[t];
  const int m = expand_point(v, pkey, hanging, best_leaf, best_level, hx_ptr, hx_len, id, buf, kHexCap);
  HexEntry *dst = pool + off[t];
  for (int i = 0; i < m; ++i) dst[i] = buf[i];
  hx_ptr[id] = dst;
  hx_len[id] = m;
}

__global__ void k_tg_flag_direct(const uint8_t *hanging, int64_t np, int32_t *flag) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id < np) flag[id] = hanging[id] ? 0 : 1;
}

__global__ void k_tg_vertices(const uint8_t *hanging, const int32_t *vpre, const uint64_t *pkey, int64_t np,
                              int64_t *vert_key) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id < np && !hanging[id]) vert_key[vpre[id]] = (int64_t)pkey[id];
}

__global__ void k_tg_cexp_size(const int32_t *corner_pt, const uint8_t *hanging, const int32_t *hx_len, int64_t nlc,
                               int32_t *size) {
  const int64_t lc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (lc >= nlc) return;
  const int32_t pt = corner_pt[lc];
  size[lc] = hanging[pt] ? hx_len[pt] : 1;
}

// Leaf corner -> (vertex, weight), ascending vertex.
__global__ void k_tg_cexp_fill(const int32_t *corner_pt, const uint8_t *hanging, HexEntry *const *hx_ptr,
                               const int32_t *hx_len, const int32_t *vpre, int64_t nlc, const int32_t *cexp_ptr,
                               int32_t *vid, double *w) {
  const int64_t lc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (lc >= nlc) return;
  const int32_t pt = corner_pt[lc];
  const int32_t o = cexp_ptr[lc];
  if (!hanging[pt]) {
    vid[o] = vpre[pt];
    w[o] = 1.0;
    return;
  }
  const HexEntry *src = hx_ptr[pt];
  const int m = hx_len[pt];
  for (int i = 0; i < m; ++i) {  // insertion by vertex (the vertices are distinct)
    const int32_t v = vpre[src[i].pid];
    const double x = src[i].w;
    int j = i;
    while (j > 0 && vid[o + j - 1] > v) {
      vid[o + j] = vid[o + j - 1];
      w[o + j] = w[o + j - 1];
      --j;
    }
    vid[o + j] = v;
    w[o + j] = x;
  }
}

__global__ void k_tg_inc_count(const int32_t *cexp_vid, int64_t nnz, int32_t *cnt) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nnz) atomicAdd(&cnt[cexp_vid[j]], 1);
}

__global__ void k_tg_inc_scatter(const int32_t *cexp_ptr, const int32_t *cexp_vid, const double *cexp_w, int64_t nlc,
                                 const int32_t *inc_ptr, int32_t *cursor, int32_t *inc_lc, double *inc_w) {
  const int64_t lc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (lc >= nlc) return;
  for (int32_t j = cexp_ptr[lc]; j < cexp_ptr[lc + 1]; ++j) {
    const int32_t v = cexp_vid[j];
    const int32_t slot = inc_ptr[v] + atomicAdd(&cursor[v], 1);
    inc_lc[slot] = (int32_t)lc;
    inc_w[slot] = cexp_w[j];
  }
}

// Incidences of every vertex in leaf-corner order (the atomic slots above are
// in arbitrary order): short lists by one thread, long ones listed for a warp.
__global__ void k_tg_inc_sort_small(const int32_t *inc_ptr, int64_t nv, int32_t *inc_lc, double *inc_w,
                                    int32_t *long_list, int32_t *n_long) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  const int32_t b = inc_ptr[v], e = inc_ptr[v + 1];
  if (e - b > kSmallSeg) {
    long_list[atomicAdd(n_long, 1)] = (int32_t)v;
    return;
  }
  for (int32_t i = b + 1; i < e; ++i) {
    const int32_t k = inc_lc[i];
    const double x = inc_w[i];
    int32_t j = i;
    while (j > b && inc_lc[j - 1] > k) {
      inc_lc[j] = inc_lc[j - 1];
      inc_w[j] = inc_w[j - 1];
      --j;
    }
    inc_lc[j] = k;
    inc_w[j] = x;
  }
}

// One warp per long list: (leaf corner, position) packed into 64-bit keys,
// sorted, then the weights follow their keys.
__global__ void k_tg_inc_sort_long(const int32_t *inc_ptr, const int32_t *long_list, const int32_t *n_long,
                                   int32_t *inc_lc, double *inc_w, uint64_t *kscratch, double *wscratch) {
  const int lane = threadIdx.x & 31;
  const int32_t warp = (int32_t)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int32_t nw = (int32_t)(((int64_t)gridDim.x * blockDim.x) >> 5);
  for (int32_t t = warp; t < *n_long; t += nw) {
    const int32_t v = long_list[t];
    const int32_t b = inc_ptr[v], m = inc_ptr[v + 1] - b;
    uint64_t *kk = kscratch + b;
    double *ww = wscratch + b;
    for (int32_t i = lane; i < m; i += 32) {
      kk[i] = ((uint64_t)(uint32_t)inc_lc[b + i] << 32) | (uint32_t)i;
      ww[i] = inc_w[b + i];
    }
    __syncwarp();
    warp_sort_direct<uint64_t>(kk, m);
    for (int32_t i = lane; i < m; i += 32) {
      inc_lc[b + i] = (int32_t)(kk[i] >> 32);
      inc_w[b + i] = ww[(uint32_t)kk[i]];
    }
    __syncwarp();
  }
}

__device__ __forceinline__ double kref_dev(int d, int e, int f) {
  const int diff = __popc((unsigned)(e ^ f));
  if (d == 2) return diff == 0 ? 4.0 / 6.0 : (diff == 1 ? -1.0 / 6.0 : -2.0 / 6.0);
  return diff == 0 ? 4.0 / 12.0 : (diff == 1 ? 0.0 : -1.0 / 12.0);
}

// Per vertex: ion load, stiffness diagonal and the number of leaf corners that
// are the vertex itself, summed over the incident corners in leaf-corner
// order, pairs of corners of one leaf in (e, f) order.  Vertices with up to
// kSmallSeg incidences take one thread each; longer lists (the masters of
// many hanging points) are listed for one warp each.
__global__ void k_tg_vertex_aux(TV v, const int32_t *inc_ptr, const int32_t *inc_lc, const double *inc_w,
                                const int32_t *cexp_ptr, const int32_t *corner_pt, const uint8_t *hanging,
                                int64_t nv, double *ion_load, double *diag, int32_t *dcnt, int32_t *long_list,
                                int32_t *n_long) {
  const int64_t vx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (vx >= nv) return;
  const int nc = v.nc, d = v.d;
  const int32_t end = inc_ptr[vx + 1];
  if (end - inc_ptr[vx] > kSmallSeg) {
    long_list[atomicAdd(n_long, 1)] = (int32_t)vx;
    return;
  }
  double ion = 0.0, dg = 0.0;
  int32_t dc = 0;
  for (int32_t j = inc_ptr[vx]; j < end;) {
    const int64_t leaf = inc_lc[j] / nc;
    int32_t k = j;
    while (k < end && inc_lc[k] / nc == leaf) ++k;
    const int lev = v.leaf_level[leaf];
    const double cint = c_tg_cint[lev], hs = c_tg_hs[lev];
    for (int32_t a1 = j; a1 < k; ++a1) {
      const int64_t i = inc_lc[a1];
      ion += inc_w[a1] * cint;
      if (cexp_ptr[i + 1] - cexp_ptr[i] == 1 && !hanging[corner_pt[i]]) ++dc;
      const int e = (int)(i % nc);
      for (int32_t a2 = j; a2 < k; ++a2) {
        const int f = (int)(inc_lc[a2] % nc);
        dg += kref_dev(d, e, f) * hs * inc_w[a1] * inc_w[a2];
      }
    }
    j = k;
  }
  ion_load[vx] = ion;
  diag[vx] = dg;
  dcnt[vx] = dc;
}

// The same for one long list per warp: 32 incidences at a time, each lane
// forms the terms of one incidence (its ion term, its direct-corner flag and
// its pair terms with the corners of the same leaf), then lane 0 adds them
// in the order of the one-thread loop.
__global__ void __launch_bounds__(kTB) k_tg_vertex_aux_long(TV v, const int32_t *inc_ptr, const int32_t *inc_lc,
                                                            const double *inc_w, const int32_t *cexp_ptr,
                                                            const int32_t *corner_pt, const uint8_t *hanging,
                                                            const int32_t *long_list, const int32_t *n_long,
                                                            double *ion_load, double *diag, int32_t *dcnt) {
  __shared__ double s_ion[kTB], s_pair[kTB * 8];
  __shared__ uint8_t s_np[kTB], s_dir[kTB];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int32_t warp = (int32_t)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int32_t nw = (int32_t)(((int64_t)gridDim.x * blockDim.x) >> 5);
  const int nc = v.nc, d = v.d;
  double *pi = s_ion + wib * 32, *pp = s_pair + wib * 32 * 8;
  uint8_t *np = s_np + wib * 32, *dir = s_dir + wib * 32;
  for (int32_t t = warp; t < *n_long; t += nw) {
    const int32_t vx = long_list[t];
    const int32_t b = inc_ptr[vx], end = inc_ptr[vx + 1];
    double ion = 0.0, dg = 0.0;
    int32_t dc = 0;
    for (int32_t c0 = b; c0 < end; c0 += 32) {
      const int32_t a1 = c0 + lane;
      if (a1 < end) {
        const int64_t i = inc_lc[a1];
        const int64_t leaf = i / nc;
        int32_t j = a1, k = a1 + 1;  // the run of incidences of the same leaf
        while (j > b && inc_lc[j - 1] / nc == leaf) --j;
        while (k < end && inc_lc[k] / nc == leaf) ++k;
        const int lev = v.leaf_level[leaf];
        const double cint = c_tg_cint[lev], hs = c_tg_hs[lev];
        pi[lane] = inc_w[a1] * cint;
        dir[lane] = cexp_ptr[i + 1] - cexp_ptr[i] == 1 && !hanging[corner_pt[i]];
        const int e = (int)(i % nc);
        np[lane] = (uint8_t)(k - j);
        for (int32_t a2 = j; a2 < k; ++a2) {
          const int f = (int)(inc_lc[a2] % nc);
          pp[lane * 8 + (a2 - j)] = kref_dev(d, e, f) * hs * inc_w[a1] * inc_w[a2];
        }
      }
      __syncwarp();
      if (lane == 0) {
        const int m = end - c0 < 32 ? end - c0 : 32;
        for (int q = 0; q < m; ++q) {
          ion += pi[q];
          dc += dir[q];
          for (int r = 0; r < np[q]; ++r) dg += pp[q * 8 + r];
        }
      }
      __syncwarp();
    }
    if (lane == 0) {
      ion_load[vx] = ion;
      diag[vx] = dg;
      dcnt[vx] = dc;
    }
  }
}

__global__ void k_tg_to32(const double *in, int64_t n, float *out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)in[i];
}

// PIDT owners: leaf corner -> (level, row-major index on that level), one
// bitmap per level starting at word lword[level].
__global__ void k_tg_pv_mark(TV v, int64_t nlc, const int64_t *lword, uint32_t *bits, uint64_t *cbit) {
  const int64_t lc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (lc >= nlc) return;
  const int64_t L = lc / v.nc;
  const int e = (int)(lc % v.nc);
  const int lev = v.leaf_level[L];
  const int64_t per = p3_64(lev);
  int64_t rm = 0, m = 1;
  for (int a = 0; a < v.d; ++a) {
    int64_t c = (int64_t)v.leaf_coords[L * v.d + a] + ((e >> a) & 1);
    if (c == per) c = 0;
    rm += c * m;
    m *= per;
  }
  const uint64_t b = (uint64_t)lword[lev] * 32u + (uint64_t)rm;
  cbit[lc] = b;
  atomicOr(&bits[b >> 5], 1u << (b & 31u));
}

__global__ void k_tg_pv_corner(const uint64_t *cbit, const uint32_t *bits, const int32_t *wpre, int64_t nlc,
                               int32_t *corner_pv) {
  const int64_t lc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (lc >= nlc) return;
  const uint64_t b = cbit[lc];
  corner_pv[lc] = wpre[b >> 5] + __popc(bits[b >> 5] & ((1u << (b & 31u)) - 1u));
}

// Owner vertices of one level: (level, j) from the marked bits.
__global__ void k_tg_pv_decode(const uint32_t *bits, const int32_t *wpre, int64_t w0, int64_t nw, int lev, int d,
                               int32_t *pv_level, int32_t *pv_j) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nw) return;
  const int64_t w = w0 + t;
  uint32_t b = bits[w];
  int32_t at = wpre[w];
  const int64_t per = p3_64(lev);
  while (b) {
    const int pos = __ffs(b) - 1;
    int64_t rm = t * 32 + pos;
    pv_level[at] = lev;
    for (int a = 0; a < d; ++a) {
      pv_j[(int64_t)at * d + a] = (int32_t)(rm % per);
      rm /= per;
    }
    ++at;
    b &= b - 1u;
  }
}

}  // namespace

bool grid_on_device_fits(const HostTree &ht) {
  if (ht.uniform || ht.depth > 12) return false;
  double bits = 1.0;
  for (int a = 0; a < ht.d; ++a) bits *= (double)ht.M;
  return bits <= 8589934592.0;  // 2^33 bits: a 1 GiB bitmap
}

int tabulate_on_device(const HostTree &ht, const TabEntry *tab, const uint8_t *leaf_level, const int32_t *leaf_coords,
                       bool pidt, cudaStream_t s, const GridAlloc &A, DeviceGrid *out) {
  *out = DeviceGrid{};
  std::vector<void *> scratch;
  auto take = [&](void **p, size_t bytes, bool keep) -> int {
    const int rc = A.alloc(A.ctx, p, bytes > 0 ? bytes : 16, keep);
    if (!rc && !keep) scratch.push_back(*p);
    return rc;
  };
  auto done = [&](int rc) {
    cudaStreamSynchronize(s);
    for (void *p : scratch) A.release(A.ctx, p);
    return rc;
  };
#define TG_TAKE(ptr, type, count, keep) \
  if (take((void **)&(ptr), sizeof(type) * (size_t)(count), keep)) return done(kTabNoMemory)
#define TG_CK(call) \
  if ((call) != cudaSuccess) return done(kTabCuda)

  {
    uint32_t p3[21];
    p3[0] = 1;
    for (int i = 1; i < 21; ++i) p3[i] = p3[i - 1] * 3u;
    TG_CK(cudaMemcpyToSymbolAsync(c_pow3, p3, sizeof(p3), 0, cudaMemcpyHostToDevice, s));
    double cint[kMaxLevel + 1], hs[kMaxLevel + 1];
    for (int l = 0; l <= kMaxLevel; ++l) {
      const double h = 1.0 / (double)pow3(l);
      double vol = 1.0;
      for (int a = 0; a < ht.d; ++a) vol *= h;
      cint[l] = vol / (double)ht.nc;
      hs[l] = ht.d == 2 ? 1.0 : h;
    }
    TG_CK(cudaMemcpyToSymbolAsync(c_tg_cint, cint, sizeof(cint), 0, cudaMemcpyHostToDevice, s));
    TG_CK(cudaMemcpyToSymbolAsync(c_tg_hs, hs, sizeof(hs), 0, cudaMemcpyHostToDevice, s));
  }
  const int d = ht.d, nc = ht.nc;
  const int64_t nl = ht.n_leaves, nlc = nl * nc;
  uint64_t lattice = 1;
  for (int a = 0; a < d; ++a) lattice *= (uint64_t)ht.M;
  const int64_t nw = (int64_t)((lattice + 31) / 32);

  int64_t launched = 0;  // this file's kernels (the scans count their own)
  TV v{};
  v.d = d;
  v.nc = nc;
  v.depth = ht.depth;
  v.M = ht.M;
  v.tab = tab;
  v.leaf_level = leaf_level;
  v.leaf_coords = leaf_coords;

  int32_t *scal;  // [0] scan total, [1] error, [2] long lists
  TG_TAKE(scal, int32_t, 8, false);
  TG_CK(cudaMemsetAsync(scal, 0, sizeof(int32_t) * 8, s));
  const int64_t max_scan = std::max<int64_t>({nw, nlc, (int64_t)1}) + 1;
  int32_t *tiles;
  TG_TAKE(tiles, int32_t, scan_tiles_needed(max_scan) + 1, false);

  // 1. points: the distinct leaf corners, ranked by key
  uint32_t *bits;
  uint64_t *ckey;
  int32_t *wcnt, *wpre;
  TG_TAKE(bits, uint32_t, nw, false);
  TG_TAKE(ckey, uint64_t, nlc, false);
  TG_TAKE(wcnt, int32_t, nw, false);
  TG_TAKE(wpre, int32_t, nw + 1, false);
  TG_CK(cudaMemsetAsync(bits, 0, sizeof(uint32_t) * nw, s));
  ++launched;
  k_tg_mark<<<grid_of(nlc), kTB, 0, s>>>(v, nlc, ckey, bits);
  ++launched;
  k_tg_popc<<<grid_of(nw), kTB, 0, s>>>(bits, nw, wcnt);
  launch_exclusive_scan(wcnt, nw, wpre, tiles, scal, s);
  int32_t np32 = 0;
  TG_CK(cudaMemcpyAsync(&np32, scal, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  TG_CK(cudaStreamSynchronize(s));
  const int64_t np = np32;
  v.bits = bits;
  v.wpre = wpre;
  uint64_t *pkey;
  int32_t *corner_pt;
  TG_TAKE(pkey, uint64_t, np, false);
  TG_TAKE(corner_pt, int32_t, nlc, false);
  ++launched;
  k_tg_keys<<<grid_of(nw), kTB, 0, s>>>(bits, wpre, nw, 0, pkey);
  ++launched;
  k_tg_corner_pt<<<grid_of(nlc), kTB, 0, s>>>(v, ckey, nlc, corner_pt);

  // 2. hanging points and their coarsest leaves
  uint8_t *hanging, *best_level;
  int32_t *best_leaf;
  TG_TAKE(hanging, uint8_t, np, false);
  TG_TAKE(best_level, uint8_t, np, false);
  TG_TAKE(best_leaf, int32_t, np, false);
  ++launched;
  k_tg_hanging<<<grid_of(np), kTB, 0, s>>>(v, pkey, np, hanging, best_leaf, best_level);

  // 3. expansions of the hanging points, coarsest leaf level by level
  const int nlev = ht.depth + 1;
  int32_t *lcount, *lcursor, *hlist;
  HexEntry **hx_ptr;
  int32_t *hx_len;
  TG_TAKE(lcount, int32_t, nlev, false);
  TG_TAKE(lcursor, int32_t, nlev, false);
  TG_TAKE(hx_ptr, HexEntry *, np, false);
  TG_TAKE(hx_len, int32_t, np, false);
  TG_CK(cudaMemsetAsync(lcount, 0, sizeof(int32_t) * nlev, s));
  TG_CK(cudaMemsetAsync(lcursor, 0, sizeof(int32_t) * nlev, s));
  TG_CK(cudaMemsetAsync(hx_len, 0, sizeof(int32_t) * std::max<int64_t>(np, 1), s));
  ++launched;
  k_tg_level_count<<<grid_of(np), kTB, 0, s>>>(hanging, best_level, np, lcount);
  std::vector<int32_t> lc_host(nlev), loff_host(nlev + 1, 0);
  TG_CK(cudaMemcpyAsync(lc_host.data(), lcount, sizeof(int32_t) * nlev, cudaMemcpyDeviceToHost, s));
  TG_CK(cudaStreamSynchronize(s));
  for (int l = 0; l < nlev; ++l) loff_host[l + 1] = loff_host[l] + lc_host[l];
  const int64_t n_hang = loff_host[nlev];
  int32_t *loff;
  TG_TAKE(loff, int32_t, nlev + 1, false);
  TG_TAKE(hlist, int32_t, n_hang, false);
  TG_CK(cudaMemcpyAsync(loff, loff_host.data(), sizeof(int32_t) * (nlev + 1), cudaMemcpyHostToDevice, s));
  ++launched;
  k_tg_level_lists<<<grid_of(np), kTB, 0, s>>>(hanging, best_level, np, loff, lcursor, hlist);
  int32_t *hlen, *hoff;
  TG_TAKE(hlen, int32_t, n_hang, false);
  TG_TAKE(hoff, int32_t, n_hang + 1, false);
  for (int l = 0; l < nlev; ++l) {
    const int32_t n = lc_host[l];
    if (n == 0) continue;
    const int32_t *list = hlist + loff_host[l];
    int32_t *len = hlen + loff_host[l], *off = hoff + loff_host[l];
    ++launched;
    k_tg_hex_size<<<grid_of(n), kTB, 0, s>>>(v, pkey, hanging, best_leaf, best_level, hx_ptr, hx_len, list, n, len,
                                             scal + 1);
    launch_exclusive_scan(len, n, off, tiles, scal, s);
    int32_t tot[2] = {0, 0};
    TG_CK(cudaMemcpyAsync(tot, scal, sizeof(tot), cudaMemcpyDeviceToHost, s));
    TG_CK(cudaStreamSynchronize(s));
    if (tot[1]) return done(kTabUnsupported);  // an expansion longer than kHexCap
    HexEntry *pool;
    TG_TAKE(pool, HexEntry, tot[0], false);
    ++launched;
    k_tg_hex_fill<<<grid_of(n), kTB, 0, s>>>(v, pkey, hanging, best_leaf, best_level, hx_ptr, hx_len, list, n, off,
                                             pool);
  }

  // 4. vertices: the non-hanging points in key order
  int32_t *vflag, *vpre;
  TG_TAKE(vflag, int32_t, np, false);
  TG_TAKE(vpre, int32_t, np + 1, false);
  ++launched;
  k_tg_flag_direct<<<grid_of(np), kTB, 0, s>>>(hanging, np, vflag);
  launch_exclusive_scan(vflag, np, vpre, tiles, scal, s);
  int32_t nv32 = 0;
  TG_CK(cudaMemcpyAsync(&nv32, scal, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  TG_CK(cudaStreamSynchronize(s));
  const int64_t nv = nv32;
  TG_TAKE(out->vert_key, int64_t, nv, true);
  ++launched;
  k_tg_vertices<<<grid_of(np), kTB, 0, s>>>(hanging, vpre, pkey, np, out->vert_key);

  // 5. leaf corner -> (vertex, weight)
  int32_t *csize;
  TG_TAKE(csize, int32_t, nlc, false);
  TG_TAKE(out->cexp_ptr, int32_t, nlc + 1, true);
  ++launched;
  k_tg_cexp_size<<<grid_of(nlc), kTB, 0, s>>>(corner_pt, hanging, hx_len, nlc, csize);
  launch_exclusive_scan(csize, nlc, out->cexp_ptr, tiles, scal, s);
  int32_t nnz32 = 0;
  TG_CK(cudaMemcpyAsync(&nnz32, scal, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  TG_CK(cudaStreamSynchronize(s));
  const int64_t nnz = nnz32;
  TG_TAKE(out->cexp_vid, int32_t, nnz, true);
  TG_TAKE(out->cexp_w64, double, nnz, true);
  TG_TAKE(out->cexp_w32, float, nnz, true);
  ++launched;
  k_tg_cexp_fill<<<grid_of(nlc), kTB, 0, s>>>(corner_pt, hanging, hx_ptr, hx_len, vpre, nlc, out->cexp_ptr,
                                              out->cexp_vid, out->cexp_w64);

  // 6. vertex -> (leaf corner, weight), stable in leaf-corner order
  int32_t *vcnt, *cursor, *long_list;
  TG_TAKE(vcnt, int32_t, nv, false);
  TG_TAKE(cursor, int32_t, nv, false);
  TG_TAKE(long_list, int32_t, nv, false);
  TG_TAKE(out->inc_ptr, int32_t, nv + 1, true);
  TG_TAKE(out->inc_lc, int32_t, nnz, true);
  TG_TAKE(out->inc_w64, double, nnz, true);
  TG_TAKE(out->inc_w32, float, nnz, true);
  TG_CK(cudaMemsetAsync(vcnt, 0, sizeof(int32_t) * std::max<int64_t>(nv, 1), s));
  TG_CK(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * std::max<int64_t>(nv, 1), s));
  ++launched;
  k_tg_inc_count<<<grid_of(nnz), kTB, 0, s>>>(out->cexp_vid, nnz, vcnt);
  launch_exclusive_scan(vcnt, nv, out->inc_ptr, tiles, scal, s);
  ++launched;
  k_tg_inc_scatter<<<grid_of(nlc), kTB, 0, s>>>(out->cexp_ptr, out->cexp_vid, out->cexp_w64, nlc, out->inc_ptr,
                                                cursor, out->inc_lc, out->inc_w64);
  TG_CK(cudaMemsetAsync(scal + 2, 0, sizeof(int32_t), s));
  ++launched;
  k_tg_inc_sort_small<<<grid_of(nv), kTB, 0, s>>>(out->inc_ptr, nv, out->inc_lc, out->inc_w64, long_list, scal + 2);
  {
    uint64_t *kscr;
    double *wscr;
    TG_TAKE(kscr, uint64_t, nnz, false);
    TG_TAKE(wscr, double, nnz, false);
    ++launched;
    k_tg_inc_sort_long<<<304, kTB, 0, s>>>(out->inc_ptr, long_list, scal + 2, out->inc_lc, out->inc_w64, kscr, wscr);
  }

  // 7. per-vertex ion load, stiffness diagonal, direct corners; FP32 copies
  TG_TAKE(out->ion64, double, nv, true);
  TG_TAKE(out->diag64, double, nv, true);
  TG_TAKE(out->ion32, float, nv, true);
  TG_TAKE(out->diag32, float, nv, true);
  TG_TAKE(out->dcnt, int32_t, nv, true);
  TG_CK(cudaMemsetAsync(scal + 3, 0, sizeof(int32_t), s));
  ++launched;
  k_tg_vertex_aux<<<grid_of(nv), kTB, 0, s>>>(v, out->inc_ptr, out->inc_lc, out->inc_w64, out->cexp_ptr, corner_pt,
                                              hanging, nv, out->ion64, out->diag64, out->dcnt, long_list, scal + 3);
  ++launched;
  k_tg_vertex_aux_long<<<304, kTB, 0, s>>>(v, out->inc_ptr, out->inc_lc, out->inc_w64, out->cexp_ptr, corner_pt,
                                           hanging, long_list, scal + 3, out->ion64, out->diag64, out->dcnt);
  ++launched;
  k_tg_to32<<<grid_of(nnz), kTB, 0, s>>>(out->cexp_w64, nnz, out->cexp_w32);
  ++launched;
  k_tg_to32<<<grid_of(nnz), kTB, 0, s>>>(out->inc_w64, nnz, out->inc_w32);
  ++launched;
  k_tg_to32<<<grid_of(nv), kTB, 0, s>>>(out->ion64, nv, out->ion32);
  ++launched;
  k_tg_to32<<<grid_of(nv), kTB, 0, s>>>(out->diag64, nv, out->diag32);

  // 8. PIDT owner vertices: distinct (level, j) of leaf corners, level-major
  int64_t npv = 0;
  if (pidt) {
    std::vector<int64_t> lword(nlev + 1, 0);
    for (int l = 0; l < nlev; ++l) {
      uint64_t cells = 1;
      for (int a = 0; a < d; ++a) cells *= (uint64_t)pow3(l);
      lword[l + 1] = lword[l] + (int64_t)((cells + 31) / 32);
    }
    const int64_t pw = lword[nlev];
    int64_t *lword_d;
    uint32_t *pbits;
    uint64_t *cbit;
    int32_t *pcnt, *ppre;
    TG_TAKE(lword_d, int64_t, nlev + 1, false);
    TG_TAKE(pbits, uint32_t, pw, false);
    TG_TAKE(cbit, uint64_t, nlc, false);
    TG_TAKE(pcnt, int32_t, pw, false);
    TG_TAKE(ppre, int32_t, pw + 1, false);
    TG_CK(cudaMemcpyAsync(lword_d, lword.data(), sizeof(int64_t) * (nlev + 1), cudaMemcpyHostToDevice, s));
    TG_CK(cudaMemsetAsync(pbits, 0, sizeof(uint32_t) * pw, s));
    ++launched;
    k_tg_pv_mark<<<grid_of(nlc), kTB, 0, s>>>(v, nlc, lword_d, pbits, cbit);
    ++launched;
    k_tg_popc<<<grid_of(pw), kTB, 0, s>>>(pbits, pw, pcnt);
    int32_t *ptiles;
    TG_TAKE(ptiles, int32_t, scan_tiles_needed(pw + 1) + 1, false);
    launch_exclusive_scan(pcnt, pw, ppre, ptiles, scal, s);
    int32_t npv32 = 0;
    TG_CK(cudaMemcpyAsync(&npv32, scal, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    TG_CK(cudaStreamSynchronize(s));
    npv = npv32;
    TG_TAKE(out->corner_pv, int32_t, nlc, true);
    TG_TAKE(out->pv_level, int32_t, npv, true);
    TG_TAKE(out->pv_j, int32_t, npv * d, true);
    ++launched;
    k_tg_pv_corner<<<grid_of(nlc), kTB, 0, s>>>(cbit, pbits, ppre, nlc, out->corner_pv);
    for (int l = 0; l < nlev; ++l) {
      ++launched;
      k_tg_pv_decode<<<grid_of(lword[l + 1] - lword[l]), kTB, 0, s>>>(pbits, ppre, lword[l], lword[l + 1] - lword[l],
                                                                        l, d, out->pv_level, out->pv_j);
    }
  }
  count_launches(launched);
  TG_CK(cudaGetLastError());
  TG_CK(cudaStreamSynchronize(s));
  out->n_vert = nv;
  out->n_pv = npv;
  out->n_entries = nnz;
#undef TG_TAKE
#undef TG_CK
  return done(0);
}

}  // namespace pic
