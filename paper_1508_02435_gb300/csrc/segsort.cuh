// In-place sorts of one segment of distinct keys, for the places where a
// segment can be long (a crowded bucket, a leaf that collects many arrivals)
// and a per-thread insertion sort would be quadratic.
//
// The network is the all-ascending form of Batcher's bitonic sort over
// P = 2^p >= m positions: stage k (k = 2, 4, ..., P) starts with the pairs
// (i, i ^ (k - 1)) for i in the lower half of every aligned block of k, then
// applies the pairs (i, i + j) with bit j of i clear for j = k/4, ..., 1.
// Every comparator moves the smaller element to the lower position, so a
// segment of any length m sorts as if padded with +infinity up to P: a
// comparator that reaches past m would never swap and is skipped.  The work is
// O(m log^2 m) compare-exchanges with no data-dependent trip counts and no
// memory beyond the segment (and a shared-memory chunk for the block form).
#pragma once
#include <cstdint>

namespace pic {

// Positions (i, l), i < l, of comparator c of the step with distance j in
// stage k (j == k / 2 is the stage's first step); j and k are powers of two.
// In both kinds i = 2c - (c mod j); l >= 2c - j + 2.
__device__ __forceinline__ void bitonic_pair(int64_t c, int64_t k, int64_t j, int64_t *i, int64_t *l) {
  const int64_t r = c & (j - 1);
  *i = 2 * c - r;
  *l = 2 * j == k ? (*i ^ (k - 1)) : *i + j;
}

// One warp sorts idx[0..m) (shared memory) ascending by key[idx[.]]; the keys
// are distinct.  All 32 lanes must call it.
template <typename Idx, typename Key>
__device__ void warp_sort_indirect(Idx *idx, int m, const Key *key) {
  if (m <= 1) return;
  const int lane = threadIdx.x & 31;
  int P = 1;
  while (P < m) P <<= 1;
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int c = lane; c < (P >> 1); c += 32) {
        int64_t i, l;
        bitonic_pair(c, k, j, &i, &l);
        if (l < m) {
          const Idx a = idx[i], b = idx[l];
          if (key[b] < key[a]) {
            idx[i] = b;
            idx[l] = a;
          }
        }
      }
      __syncwarp();
    }
}

// One warp sorts v[0..m) (shared memory) ascending; the values are distinct.
// All 32 lanes must call it.
template <typename T>
__device__ void warp_sort_direct(T *v, int m) {
  if (m <= 1) return;
  const int lane = threadIdx.x & 31;
  int P = 1;
  while (P < m) P <<= 1;
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      // comparator c reaches l >= 2c - j + 2: none past (m + j) / 2 has both positions valid
      for (int c = lane; c <= (m + j) / 2; c += 32) {
        int64_t i, l;
        bitonic_pair(c, k, j, &i, &l);
        if (l < m) {
          const T a = v[i], b = v[l];
          if (b < a) {
            v[i] = b;
            v[l] = a;
          }
        }
      }
      __syncwarp();
    }
}

// Compare-exchange of positions i < l of (key, val) arrays; val may be null.
template <typename K, typename V>
__device__ __forceinline__ void cmpx(K *key, V *val, int64_t i, int64_t l) {
  const K a = key[i], b = key[l];
  if (b < a) {
    key[i] = b;
    key[l] = a;
    if (val) {
      const V t = val[i];
      val[i] = val[l];
      val[l] = t;
    }
  }
}

// The steps j = j_hi, j_hi / 2, ..., 1 of stage k on the chunk of cs (a power
// of two, j_hi < cs unless the chunk is the whole stage) positions starting at
// c0 of the segment, in shared memory (sk / sv); mm = valid positions of the
// chunk.  Block-wide, one barrier per step.
template <typename K, typename V>
__device__ void chunk_steps(K *sk, V *sv, int mm, int64_t k, int64_t j_hi) {
  for (int64_t j = j_hi; j > 0; j >>= 1) {
    // comparator c reaches l >= 2c - j + 2: none past (mm + j) / 2 has both positions valid
    for (int64_t c = threadIdx.x; c <= (mm + j) / 2; c += blockDim.x) {
      int64_t i, l;
      bitonic_pair(c, k, j, &i, &l);
      if (l < mm) cmpx<K, V>(sk, sv, i, l);
    }
    __syncthreads();
  }
}

// One block sorts key[0..m) ascending (distinct keys), carrying val[0..m)
// along when val is not null, in place in global memory.  sk / sv are shared
// buffers of cs elements (cs a power of two; sv unused when val is null).
// Every thread of the block must call it; it ends with a block barrier.
// Stages that fit one chunk run in shared memory; longer-distance steps run
// in global memory with eight comparators in flight per thread.
template <typename K, typename V>
__device__ void block_sort_global(K *key, V *val, int64_t m, K *sk, V *sv, int cs) {
  if (m <= 1) return;
  int64_t P = 1;
  while (P < m) P <<= 1;
  const int64_t C = P < cs ? P : cs;
  auto load = [&](int64_t c0, int mm) {
    for (int t = threadIdx.x; t < mm; t += blockDim.x) {
      sk[t] = key[c0 + t];
      if (val) sv[t] = val[c0 + t];
    }
    __syncthreads();
  };
  auto store = [&](int64_t c0, int mm) {
    for (int t = threadIdx.x; t < mm; t += blockDim.x) {
      key[c0 + t] = sk[t];
      if (val) val[c0 + t] = sv[t];
    }
    __syncthreads();
  };
  // stages 2 .. C: every aligned chunk of C is sorted on its own
  for (int64_t c0 = 0; c0 < m; c0 += C) {
    const int mm = (int)(m - c0 < C ? m - c0 : C);
    load(c0, mm);
    for (int64_t k = 2; k <= C; k <<= 1) chunk_steps<K, V>(sk, val ? sv : nullptr, mm, k, k >> 1);
    store(c0, mm);
  }
  // stages 2C .. P: steps of distance >= C in global memory, the rest per chunk
  for (int64_t k = 2 * C; k <= P; k <<= 1) {
    for (int64_t j = k >> 1; j >= C; j >>= 1) {
      const int64_t ncmp = P >> 1;
      for (int64_t c0 = (int64_t)threadIdx.x * 8; c0 < ncmp; c0 += (int64_t)blockDim.x * 8) {
        int64_t ii[8], ll[8];
        K a[8], b[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          bitonic_pair(c0 + u, k, j, &ii[u], &ll[u]);
          const bool ok = c0 + u < ncmp && ll[u] < m;
          if (!ok) ll[u] = -1;
          a[u] = ok ? key[ii[u]] : K(0);
          b[u] = ok ? key[ll[u]] : K(0);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (ll[u] >= 0 && b[u] < a[u]) {
            key[ii[u]] = b[u];
            key[ll[u]] = a[u];
            if (val) {
              const V t = val[ii[u]];
              val[ii[u]] = val[ll[u]];
              val[ll[u]] = t;
            }
          }
      }
      __syncthreads();
    }
    for (int64_t c0 = 0; c0 < m; c0 += C) {
      const int mm = (int)(m - c0 < C ? m - c0 : C);
      load(c0, mm);
      chunk_steps<K, V>(sk, val ? sv : nullptr, mm, k, C >> 1);
      store(c0, mm);
    }
  }
}

}  // namespace pic
