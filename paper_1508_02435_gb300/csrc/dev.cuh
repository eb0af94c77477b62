// Device view of a tabulated spacetree and the per-particle primitives of
// the PIT/PIDT step (arXiv:1508.02435): quantisation, descent of the
// flattened level-ordered table (the end state of the lifts and drops of
// Algorithm 1 / Theorem 1), the split-precision re-location, d-linear shape
// functions (Section 3) and leaf-corner to vertex maps.
//
// Device code is compiled with --fmad=false: every + - * / below is one IEEE
// round-to-nearest operation in program order.
#pragma once
#include <cstdint>

#include "tree.hpp"

namespace pic {

__constant__ uint32_t c_pow3[21];

// One plasma instance of a batch: its tree occupies the leaves, vertices and
// sort keys [*_off, *_off + count) of the concatenated arrays.  A single
// handle is a batch of one with every offset zero.
struct InstInfo {
  int32_t depth, M;            // uniform trees: level of every leaf, 3^depth
  int32_t leaf_off, vert_off, key_off, spread_off, tab_root, n_vert;
  int64_t poff;                // first particle of the instance in input order
  double q, ion, ion_load, diag;
  float q32, ion32, ion_load32, diag32;
};

struct DevTree {
  int d, nch, nc, depth, uniform, scheme;
  int32_t n_inst;
  int32_t block_push, block_leaf, block_vert;  // threads per block (autotuned; 0 = 256)
  const InstInfo *inst;
  const int32_t *inst_of_leaf, *inst_of_vert;
  int64_t n_leaves, n_vert, n_pv, n_keys;
  int32_t M;  // 3^depth
  const TabEntry *tab;
  int32_t n_tab;
  // uniform trees: spread[a * M + c] = base-3 digits of c interleaved on axis a,
  // so the depth-first leaf id of cell c is the sum over the axes
  const int32_t *spread;
  const uint8_t *leaf_level;
  const int32_t *leaf_coords;
  // adaptive grids
  const int32_t *cexp_ptr, *cexp_vid, *inc_ptr, *inc_lc, *dcnt, *corner_pv;
  const double *cexp_w64, *inc_w64, *ion64, *diag64;
  const float *cexp_w32, *inc_w32, *ion32, *diag32;
  // uniform grids
  double ion_u64, diag_u64;
  float ion_u32, diag_u32;
};

// ---- quantisation ---------------------------------------------------------

__device__ __forceinline__ double wrap01(double x) {
  double y = x - floor(x);
  return y >= 1.0 ? 0.0 : y;
}

__device__ __forceinline__ uint32_t quantise(double y) {  // y already in [0,1)
  double s = y * 774840978.0;
  double f = floor(s);
  if (f < 0.0) f = 0.0;
  if (f > 774840977.0) f = 774840977.0;
  return (uint32_t)f;
}

// ---- descent ----------------------------------------------------------------

__device__ __forceinline__ int digit_q(const uint32_t Q[3], int d, int m) {
  uint32_t step = 2u * c_pow3[18 - m];
  int dg = (int)((Q[0] / step) % 3u) + 3 * (int)((Q[1] / step) % 3u);
  if (d == 3) dg += 9 * (int)((Q[2] / step) % 3u);
  return dg;
}

// Local depth-first index inside a complete subtree of depth k whose leaves
// have coordinates J (on the leaves' level): base-3^d digits, bottom-up.
__device__ __forceinline__ int32_t local_index(uint32_t J0, uint32_t J1, uint32_t J2, int d, int k) {
  int32_t local = 0, mul = 1, nch = d == 3 ? 27 : 9;
  for (int i = 0; i < k; ++i) {
    int dg = (int)(J0 % 3u) + 3 * (int)(J1 % 3u);
    if (d == 3) dg += 9 * (int)(J2 % 3u);
    J0 /= 3u; J1 /= 3u; J2 /= 3u;
    local += dg * mul;
    mul *= nch;
  }
  return local;
}

// Covering leaf of the quantised position Q (PIT owner, Theorem 1), from the
// table entry `root` of the instance's tree.
__device__ __forceinline__ int32_t descend_q(const TabEntry *tab, int d, const uint32_t Q[3], int *lev_out,
                                             int root = 0) {
  int ent = root, lev = 0;
  for (;;) {
    TabEntry e = tab[ent];
    if (e.a < 0) {
      int k = -e.a - 1;
      int L = lev + k;
      uint32_t step = 2u * c_pow3[18 - L];
      *lev_out = L;
      return e.b + local_index(Q[0] / step, Q[1] / step, d == 3 ? Q[2] / step : 0u, d, k);
    }
    ent = e.a + digit_q(Q, d, lev + 1);
    ++lev;
  }
}

__device__ __forceinline__ float clamp_off(float f) {
  const float one_minus = 0x1.fffffep-1f;
  return f < 0.0f ? 0.0f : (f > one_minus ? one_minus : f);
}

// One drop below the integer level: u = RN32(3 f), digit = min(floor u, 2),
// f = u - digit (the split-precision rule of the design notes).
__device__ __forceinline__ int drop_digit(float *f, int d) {
  int dg = 0, mul = 1;
  for (int a = 0; a < d; ++a) {
    float u = 3.0f * f[a];
    int g = (int)floorf(u);
    g = g > 2 ? 2 : g;
    f[a] = clamp_off(u - (float)g);
    dg += g * mul;
    mul *= 3;
  }
  return dg;
}

// Split-precision re-location: the leaf covering integer cell I on level lev
// plus fraction f.  Writes the leaf's offsets; returns the leaf id.
__device__ __forceinline__ int32_t descend_split(const TabEntry *tab, int d, int lev, const int32_t I[3],
                                                 float f[3], float o_out[3], int *lev_out, int root = 0) {
  int ent = root, m = 0, nch = d == 3 ? 27 : 9;
  for (;;) {
    TabEntry e = tab[ent];
    if (e.a < 0) {
      int k = -e.a - 1;
      int L = m + k;
      *lev_out = L;
      if (L <= lev) {  // lift: the covering leaf is on a level <= lev
        uint32_t sh = c_pow3[lev - L];
        uint32_t J[3] = {0u, 0u, 0u};
        for (int a = 0; a < d; ++a) {
          J[a] = (uint32_t)I[a] / sh;
          uint32_t r = (uint32_t)I[a] - J[a] * sh;
          o_out[a] = clamp_off(((float)r + f[a]) / (float)sh);
        }
        return e.b + local_index(J[0], J[1], J[2], d, k);
      }
      // digits from I down to lev, then drops from the fraction
      int32_t local = 0;
      for (int mm = m + 1; mm <= L; ++mm) {
        int dg;
        if (mm <= lev) {
          uint32_t sh = c_pow3[lev - mm];
          dg = (int)(((uint32_t)I[0] / sh) % 3u) + 3 * (int)(((uint32_t)I[1] / sh) % 3u);
          if (d == 3) dg += 9 * (int)(((uint32_t)I[2] / sh) % 3u);
        } else {
          dg = drop_digit(f, d);
        }
        local = local * nch + dg;
      }
      for (int a = 0; a < d; ++a) o_out[a] = clamp_off(f[a]);
      return e.b + local;
    }
    int dg;
    if (m + 1 <= lev) {
      uint32_t sh = c_pow3[lev - m - 1];
      dg = (int)(((uint32_t)I[0] / sh) % 3u) + 3 * (int)(((uint32_t)I[1] / sh) % 3u);
      if (d == 3) dg += 9 * (int)(((uint32_t)I[2] / sh) % 3u);
    } else {
      dg = drop_digit(f, d);
    }
    ent = e.a + dg;
    ++m;
  }
}

// ---- grid maps ---------------------------------------------------------------

// Row-major vertex ids of the 2^d corners of uniform-grid cell c (periodic).
__device__ __forceinline__ void uniform_corner_vertices(const int32_t *c, int d, int32_t M, int32_t *vid) {
  int32_t x0 = c[0], x1 = c[0] + 1 == M ? 0 : c[0] + 1;
  int32_t y0 = c[1] * M, y1 = (c[1] + 1 == M ? 0 : c[1] + 1) * M;
  vid[0] = x0 + y0; vid[1] = x1 + y0; vid[2] = x0 + y1; vid[3] = x1 + y1;
  if (d == 3) {
    int32_t z0 = c[2] * M * M, z1 = (c[2] + 1 == M ? 0 : c[2] + 1) * M * M;
    for (int e = 0; e < 4; ++e) { vid[e + 4] = vid[e] + z1; vid[e] += z0; }
  }
}

// Row-major vertex of corner e of the uniform-grid cell c (periodic).
__device__ __forceinline__ int32_t uniform_corner_vertex(const int32_t *c, int e, int d, int32_t M) {
  int64_t v = 0, mul = 1;
  for (int a = 0; a < d; ++a) {
    int32_t j = c[a] + ((e >> a) & 1);
    if (j >= M) j -= M;
    v += (int64_t)j * mul;
    mul *= M;
  }
  return (int32_t)v;
}

// Depth-first leaf id of cell c on a uniform tree (digit-interleave tables).
__device__ __forceinline__ int32_t uniform_leaf_of_cell(const int32_t *spread, int32_t M, const int32_t *c, int d) {
  int32_t l = __ldg(spread + c[0]) + __ldg(spread + M + c[1]);
  if (d == 3) l += __ldg(spread + 2 * M + c[2]);
  return l;
}

// d-linear shape function of corner e at local coordinates t.
template <typename T>
__device__ __forceinline__ T shape(const T *t, int e, int d) {
  T w = (T)1;
  for (int a = 0; a < d; ++a) {
    T f = ((e >> a) & 1) ? t[a] : (T)1 - t[a];
    w = w * f;
  }
  return w;
}

// Ascending bitonic sorting network over N register values (N a power of two).
template <int N, typename T>
__device__ __forceinline__ void bitonic_sort(T *r) {
#pragma unroll
  for (int k = 2; k <= N; k <<= 1)
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int l = i ^ j;
        if (l > i) {
          const T x = r[i], y = r[l];
          const bool up = (i & k) == 0;
          r[i] = up ? (x < y ? x : y) : (x < y ? y : x);
          r[l] = up ? (x < y ? y : x) : (x < y ? x : y);
        }
      }
}

// Incident leaf corners of uniform vertex v (global id) in ascending
// leaf-corner order, for the instance I.  The cell of corner f is
// j - bits(f) per axis (periodic); its leaf id is a sum of per-axis spread values.
template <int D>
__device__ __forceinline__ void uniform_incidences_d(int64_t v, const InstInfo &I, const int32_t *spread,
                                                     int32_t *lc) {
  const int32_t M = I.M;
  int32_t r = (int32_t)(v - I.vert_off);  // < 3^(d depth) <= 3^18
  int32_t s_hi[3] = {0, 0, 0}, s_lo[3] = {0, 0, 0};
  const int32_t *sp = spread + I.spread_off;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const int32_t qt = r / M, j = r - qt * M;
    r = qt;
    s_hi[a] = __ldg(sp + a * M + j);
    s_lo[a] = __ldg(sp + a * M + (j == 0 ? M - 1 : j - 1));
  }
  constexpr int NC = 1 << D;
  int32_t k[NC];
#pragma unroll
  for (int f = 0; f < NC; ++f) {
    int32_t leaf = I.leaf_off;
#pragma unroll
    for (int a = 0; a < D; ++a) leaf += ((f >> a) & 1) ? s_lo[a] : s_hi[a];
    k[f] = leaf * NC + f;
  }
  bitonic_sort<NC>(k);
#pragma unroll
  for (int f = 0; f < NC; ++f) lc[f] = k[f];
}

__device__ __forceinline__ int uniform_incidences(int64_t v, int d, const InstInfo &I, const int32_t *spread,
                                                  int32_t *lc) {
  if (d == 3) {
    uniform_incidences_d<3>(v, I, spread, lc);
    return 8;
  }
  uniform_incidences_d<2>(v, I, spread, lc);
  return 4;
}

}  // namespace pic
