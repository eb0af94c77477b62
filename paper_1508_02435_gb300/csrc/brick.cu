// Brick path of the PIT split-precision step on uniform trees (sm_103a).
//
// A brick is the subtree of one cell kb levels above the leaves: B = 3^kb
// leaves per axis, LB = B^d leaves, contiguous in depth-first leaf order and so
// contiguous in the bucket-sorted particle arrays.  One step re-bins every
// particle (PIT, Algorithm 1 end state) in two passes over the particles:
//
//   K1 k_brick_push_st  two CTAs per SM, one per half brick: the half's
//                       particle rows land in shared memory by bulk copies,
//                       the brick's vertex field is staged, every particle is
//                       gathered, kicked, drifted and re-located (integer
//                       arithmetic, split rule); each warp then reserves one
//                       run per destination unit (half brick) it sends to and
//                       appends its particles there, with their canonical
//                       key: moved bit, storage index.
//   K2 k_brick_pull_st  two CTAs per SM, one per destination unit: its
//                       staging area lands by bulk copies; leaf counts, scan,
//                       slots, and a per-leaf sort by key restore the canonical
//                       order -- stayers first, then movers, each in storage
//                       order -- before the coalesced writes of the new bucket
//                       order and the leaf-corner deposit partials.
//
// Bricks over the shared-memory capacity (K1) and units over their staging
// capacity (K2) take global-memory kernels with the same arithmetic.  The
// result is bit-identical to the generic path.
#include <cuda_runtime.h>

#include <algorithm>

#include "dev.cuh"
#include "launch.hpp"
#include "segsort.cuh"

namespace pic {

void count_launches(int64_t k);

constexpr int kFarSlot = 27;
constexpr int kSelfDir = 13;         // (0, 0, 0)
constexpr uint16_t kStayBit = 0x8000;
constexpr uint16_t kMoverCode = 0;   // leaf code flags of an arrival from another leaf
constexpr int kPushThreads = 512;
constexpr unsigned kFallbackBlocks = 608;  // blocks of the global-memory fallback kernels (4 per SM)
constexpr unsigned kPersistBlocks = 304;   // CTAs of K1's shared-memory kernel (2 per SM, each taking half bricks in turn)
constexpr int kPullThreads = 256;

// Compile-time brick shape: B = 9 leaves per axis (two levels).
template <int D>
struct BK {
  static constexpr int B = 9, V1 = 10;
  static constexpr int LB = D == 3 ? 729 : 81;
  static constexpr int NVB = D == 3 ? 1000 : 100;
  static constexpr int LSW = (LB + 4 + 3) & ~3;   // leaf-offset words in shared memory (head + LB + 1)
  static constexpr int DECW = (LB + 3) & ~3;      // decode-table words (a multiple of four)
  static constexpr int NC = 1 << D;
  static constexpr int LH = (LB + 1) / 2;  // leaves of the first destination half (local leaves [0, LH))
};

// Destination unit of local leaf lidx of brick b: the brick's leaves are split
// in two halves, each re-binned by its own CTA.
template <int D>
__device__ __forceinline__ int32_t unit_of(int32_t b, int lidx) { return 2 * b + (lidx >= BK<D>::LH); }

// Asynchronous 4-byte global -> shared copies (no register round trip); the
// issuing thread waits for all of its copies with cp_async_wait_all().
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// One-dimensional bulk copies (TMA) global -> shared, completed on an
// mbarrier: both addresses 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
// Bounded wait for phase `parity` of the mbarrier: false if it did not
// complete within about `cycles` SM clocks.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, long long cycles) {
  const long long t0 = clock64();
  unsigned done = 0;
  do {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
  } while (!done && clock64() - t0 < cycles);
  return done != 0;
}
// Limit of the wait that lets copies still in flight land before a CTA that
// gave up returns (its shared memory must outlive them): about two seconds at
// the maximum SM clock, whatever limit the first wait had.
constexpr long long kWaitCycles = 4000000000LL;

constexpr int kErrTimeout = 8;                   // error bit: a bounded device wait gave up
constexpr int kErrCode = 16;                     // error bit: a staged leaf code outside its unit, or counts that disagree

__device__ __forceinline__ int dir_delta(int dir, int a) {
  return a == 0 ? dir % 3 - 1 : (a == 1 ? (dir / 3) % 3 - 1 : dir / 9 - 1);
}

template <int D>
__device__ __forceinline__ int32_t brick_of_coords(const DevTree &t, const int32_t *bc) {
  int32_t c[3] = {bc[0] * 9, bc[1] * 9, D == 3 ? bc[2] * 9 : 0};
  return uniform_leaf_of_cell(t.spread, t.M, c, D) / BK<D>::LB;
}

// ---------------------------------------------------------------------------
// K1
// ---------------------------------------------------------------------------

// Gather + kick + drift + re-location of one particle -- the arithmetic of
// the generic split push, field values from the staged brick field.  o and v
// are the particle's offset and velocity; returns the destination direction
// slot and writes the new offset, velocity and leaf.
template <int D>
__device__ __forceinline__ int push_core(const DevTree &t, const BrickGeom &g, const BrickPushArgs &a,
                                         const float *o, const float *vin, const int32_t *lc,
                                         const int32_t *origin, const int32_t *bc, const float *Eb, float *on,
                                         float *vn, int32_t &L2, bool &bad) {
  using K = BK<D>;
  float om[D];
#pragma unroll
  for (int ax = 0; ax < D; ++ax) om[ax] = 1.0f - o[ax];
  float E[D];
#pragma unroll
  for (int ax = 0; ax < D; ++ax) E[ax] = 0.0f;
  const int base = lc[0] + K::V1 * (lc[1] + (D == 3 ? K::V1 * lc[2] : 0));
#pragma unroll
  for (int e = 0; e < K::NC; ++e) {
    float w = 1.0f;
#pragma unroll
    for (int ax = 0; ax < D; ++ax) w = w * (((e >> ax) & 1) ? o[ax] : om[ax]);
    const int lv = base + (e & 1) + ((e >> 1) & 1) * K::V1 + ((e >> 2) & 1) * K::V1 * K::V1;
#pragma unroll
    for (int ax = 0; ax < D; ++ax) E[ax] = E[ax] + w * Eb[ax * K::NVB + lv];
  }
  int32_t I[3] = {0, 0, 0};
  const int32_t per = t.M;
  int dir = 0, mul = 1;
  bool far = false;
#pragma unroll
  for (int ax = 0; ax < D; ++ax) {
    float v = vin[ax] + a.qmdt * E[ax];
    float tt = o[ax] + v * a.sl;
    if (!isfinite(v) || !isfinite(tt)) { bad = true; tt = 0.0f; }
    float fl = floorf(tt);
    float f = tt - fl;
    int32_t c = origin[ax] + lc[ax], cc;
    if (fabsf(fl) < 1.0e9f) {
      cc = c + (int32_t)fl;
      if (cc < 0 || cc >= per) {
        cc %= per;
        if (cc < 0) cc += per;
      }
    } else {
      int64_t c64 = ((int64_t)c + (int64_t)fminf(fmaxf(fl, -1.0e15f), 1.0e15f)) % per;
      cc = (int32_t)(c64 < 0 ? c64 + per : c64);
    }
    I[ax] = cc;
    vn[ax] = v;
    on[ax] = clamp_off(f);
    int32_t db = cc / K::B - bc[ax];
    if (db < 0) db += g.nbx;
    int dl = db == 0 ? 0 : (db == 1 ? 1 : (db == g.nbx - 1 ? -1 : 2));
    far |= dl == 2;
    dir += (dl + 1) * mul;
    mul *= 3;
  }
  if (D == 2) dir += 9;
  L2 = uniform_leaf_of_cell(t.spread, t.M, I, D);
  return far ? kFarSlot : dir;
}

template <int D>
__device__ __forceinline__ int brick_push_one(const DevTree &t, const BrickGeom &g, const BrickPushArgs &a,
                                              int32_t p, const int32_t *lc, const int32_t *origin,
                                              const int32_t *bc, const float *Eb, float *on, float *vn,
                                              int32_t &L2, bool &bad) {
  const int64_t n = a.n;
  float o[D], v[D];
#pragma unroll
  for (int ax = 0; ax < D; ++ax) {
    o[ax] = a.o[ax * n + p];
    v[ax] = a.v[ax * n + p];
  }
  return push_core<D>(t, g, a, o, v, lc, origin, bc, Eb, on, vn, L2, bad);
}

// Stage the brick's vertex field: (B+1)^D vertices, periodic.
template <int D>
__device__ __forceinline__ void stage_field(const DevTree &t, const BrickPushArgs &a, const int32_t *origin,
                                            float *Eb) {
  using K = BK<D>;
  for (int i = threadIdx.x; i < K::NVB; i += blockDim.x) {
    int lx = i % K::V1, ly = (i / K::V1) % K::V1, lz = D == 3 ? i / (K::V1 * K::V1) : 0;
    int32_t gx = origin[0] + lx, gy = origin[1] + ly, gz = D == 3 ? origin[2] + lz : 0;
    if (gx >= t.M) gx -= t.M;
    if (gy >= t.M) gy -= t.M;
    if (gz >= t.M) gz -= t.M;
    int64_t vid = gx + (int64_t)t.M * (gy + (int64_t)t.M * gz);
#pragma unroll
    for (int ax = 0; ax < D; ++ax) Eb[ax * K::NVB + i] = a.E[ax * t.n_vert + vid];
  }
}

// ---------------------------------------------------------------------------
// K1, shared-memory form
// ---------------------------------------------------------------------------

// Two independent FP32 products in one instruction, each rounded to nearest.
__device__ __forceinline__ float2 mul2_rn(float2 a, float2 b) {
  float2 r;
  asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " mul.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}\n"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}

// Staged field entry of one vertex: the D components side by side, so one
// vector shared-memory load serves a corner.
template <int D> struct EVec;
template <> struct EVec<3> { using T = float4; };
template <> struct EVec<2> { using T = float2; };

__device__ __forceinline__ float ecomp(const float4 &e, int ax) { return ax == 0 ? e.x : (ax == 1 ? e.y : e.z); }
__device__ __forceinline__ float ecomp(const float2 &e, int ax) { return ax == 0 ? e.x : e.y; }

// Contribution of local cell coordinate x (0 <= x < 9) on axis ax to the
// depth-first index of a leaf inside its brick (two base-3 digits per axis).
template <int D>
__device__ __forceinline__ int lidx_axis(int x, int ax) {
  const int hi = (x * 11) >> 5, lo = x - 3 * hi;  // x / 3 and x % 3 for 0 <= x < 9
  const int p = ax == 0 ? 1 : (ax == 1 ? 3 : 9);
  return (lo + hi * (D == 3 ? 27 : 9)) * p;
}

// Re-location when some axis leaves the [-9, 18) window around the brick
// (wrap-around, tunnelling): global cell, brick delta modulo the brick grid.
struct SlowIn {
  int32_t lc[3], origin[3], bc[3];
  float fl[3];
};
struct SlowOut {
  int dir, lidx;
  int32_t dest;
};

template <int D>
__device__ __noinline__ SlowOut relocate_slow(const DevTree &t, const BrickGeom &g, const SlowIn in) {
  const int32_t *lc = in.lc, *origin = in.origin, *bc = in.bc;
  const float *fl = in.fl;
  const int32_t per = t.M;
  int dir = 0, mul = 1, li = 0;
  bool far = false;
  int32_t dbc[3] = {0, 0, 0};
#pragma unroll
  for (int ax = 0; ax < D; ++ax) {
    const int32_t c = origin[ax] + lc[ax];
    int32_t cc;
    if (fabsf(fl[ax]) < 1.0e9f) {
      cc = c + (int32_t)fl[ax];
      if (cc < 0 || cc >= per) {
        cc %= per;
        if (cc < 0) cc += per;
      }
    } else {
      const int64_t c64 = ((int64_t)c + (int64_t)fminf(fmaxf(fl[ax], -1.0e15f), 1.0e15f)) % per;
      cc = (int32_t)(c64 < 0 ? c64 + per : c64);
    }
    dbc[ax] = cc / 9;
    li += lidx_axis<D>(cc - 9 * dbc[ax], ax);
    int32_t db = dbc[ax] - bc[ax];
    if (db < 0) db += g.nbx;
    const int dl = db == 0 ? 0 : (db == 1 ? 1 : (db == g.nbx - 1 ? -1 : 2));
    far |= dl == 2;
    dir += (dl + 1) * mul;
    mul *= 3;
  }
  if (D == 2) dir += 9;
  return SlowOut{far ? kFarSlot : dir, li, brick_of_coords<D>(t, dbc)};
}

// K1 runs two CTAs per SM, each on one half of a brick's particles (storage
// order); bricks with more than 2 kHalfCap particles take k_brick_push.
constexpr int kHThreads = 512;
constexpr int kUnitSlots = 56;       // destination units by direction: 27 neighbour bricks x 2 halves (+ pad)
constexpr int kHalfCap = 3200;       // particles of one half held in shared memory (two CTAs still fit an SM)
constexpr int kHS = kHalfCap + 8;    // shared row stride (room for a 16-byte aligned head)

// First storage offset (within the brick) of half h of a brick holding nb particles.
__host__ __device__ __forceinline__ int32_t half_start(int32_t nb, int h) { return h == 0 ? 0 : (nb + 1) / 2; }

// Shared-memory offsets of K1's bulk-copy targets must be multiples of 16 bytes.
template <int D>
constexpr size_t push_st_off_field() { return sizeof(float) * 2 * D * kHS + sizeof(uint16_t) * kHalfCap; }
static_assert(push_st_off_field<3>() % 16 == 0 && push_st_off_field<2>() % 16 == 0, "field staging misaligned");
static_assert((push_st_off_field<3>() + 16 * BK<3>::NVB) % 16 == 0 && (push_st_off_field<2>() + 8 * BK<2>::NVB) % 16 == 0,
              "leaf offsets misaligned");
static_assert(BK<3>::LSW % 4 == 0 && BK<2>::LSW % 4 == 0 && BK<3>::DECW % 4 == 0 && BK<2>::DECW % 4 == 0,
              "decode table misaligned");

template <int D>
size_t push_st_smem() {
  using K = BK<D>;
  return sizeof(float) * 2 * D * kHS + sizeof(uint16_t) * kHalfCap + sizeof(typename EVec<D>::T) * K::NVB +
         sizeof(int32_t) * K::LSW + sizeof(uint32_t) * K::DECW + sizeof(int32_t) * (3 * 32 + 32) +
         sizeof(uint8_t) * kHalfCap + sizeof(int32_t) * (kHThreads / 32) * kUnitSlots;
}

// Writes one arrival into slot `slot` of brick dest's staging area, or into
// the overflow list when the area is full.
template <int D>
__device__ __forceinline__ void stage_put(const BrickStage &st, int32_t dest, int32_t slot, const float *on,
                                          const float *vn, uint16_t code, uint32_t key, int32_t id, bool with_id,
                                          int32_t *err) {
  if (slot < st.cap) {
    const uint32_t at = (uint32_t)dest * (uint32_t)st.cap + (uint32_t)slot;  // < 2^31 (checked at set-up)
    float *r = st.rec + (size_t)at * (2 * D);  // 8-byte aligned (3D) / 16-byte aligned (2D)
    if constexpr (D == 3) {
      reinterpret_cast<float2 *>(r)[0] = make_float2(on[0], on[1]);
      reinterpret_cast<float2 *>(r)[1] = make_float2(on[2], vn[0]);
      reinterpret_cast<float2 *>(r)[2] = make_float2(vn[1], vn[2]);
    } else {
      *reinterpret_cast<float4 *>(r) = make_float4(on[0], on[1], vn[0], vn[1]);
    }
    st.code[at] = code;
    st.key[at] = key;
    if (with_id) st.id[at] = id;
  } else {
    const int32_t k = atomicAdd(st.ovf_n, 1);
    if (k >= st.ovf_cap) {
      atomicOr(err, 4);
      return;
    }
    st.ovf_dest[k] = dest;
#pragma unroll
    for (int ax = 0; ax < D; ++ax) {
      st.ovf_o[ax * (int64_t)st.ovf_cap + k] = on[ax];
      st.ovf_v[ax * (int64_t)st.ovf_cap + k] = vn[ax];
    }
    st.ovf_code[k] = code;
    st.ovf_key[k] = key;
    if (with_id) st.ovf_id[k] = id;
  }
}

// Appends the pushed particles of one warp to the staging areas of their
// destination units (the global-memory K1): one global atomic per distinct
// destination of the warp, lanes in lane order; arrivals beyond the area's
// capacity go to the overflow list.  Inactive lanes pass dest < 0.
template <int D>
__device__ __forceinline__ void stage_append(const BrickStage &st, int32_t dest, const float *on, const float *vn,
                                             uint16_t code, uint32_t key, int32_t id, bool with_id,
                                             int32_t *err) {
  const int lane = threadIdx.x & 31;
  unsigned todo = __ballot_sync(0xffffffffu, dest >= 0);
  int32_t slot = -1;
  while (todo) {
    const int leader = __ffs(todo) - 1;
    const int32_t dd = __shfl_sync(0xffffffffu, dest, leader);
    const unsigned m = __ballot_sync(0xffffffffu, dest == dd);
    int32_t base = 0;
    if (lane == leader) base = atomicAdd(&st.fill[dd], __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (dest == dd) slot = base + __popc(m & ((1u << lane) - 1u));
    todo &= ~m;
  }
  if (dest >= 0) stage_put<D>(st, dest, slot, on, vn, code, key, id, with_id, err);
}

// A half brick in shared memory, as one warp of K1 sees it.
template <int D>
struct HalfView {
  float *so, *sv;                   // offset and velocity rows (row r starts at so + r kHS)
  int32_t offO[D], offV[D];         // index of the half's particle 0 in each row
  uint16_t *pos;                    // local leaf of every particle, then its destination code
  uint8_t *lslot;                   // rank within (warp, unit slot)
  const typename EVec<D>::T *Eb;    // the brick's field, one vector per vertex
  const uint32_t *dec;              // local leaf -> x | y << 10 | z << 20
  const int32_t *rel, *nbr;         // per-axis re-location table; neighbour bricks by direction
  int32_t nb, hs;                   // particles of the half; storage index of its first
  int32_t origin[3], bc[3];         // first leaf cell of the brick; brick coordinates
};

// One warp's share of a half brick in K1: pass A pushes the warp's chunks
// (chunk c = first, first + stride, ...), pass B appends them to the
// destination units' staging areas after one reservation per unit.  wc holds
// the warp's kUnitSlots counters (zero on entry).  Same arithmetic as
// push_core (gather in corner order, kick, drift, split re-location), with
// the destination found from the brick-local cell through a per-axis table.
template <int D, bool kAligned>
__device__ __forceinline__ void push_half_warp(const DevTree &t, const BrickGeom &g, const BrickPushArgs &a,
                                               const HalfView<D> &hv, int first, int stride, int32_t *wc,
                                               bool &bad, int &movers) {
  using K = BK<D>;
  using EV = typename EVec<D>::T;
  const int lane = threadIdx.x & 31;
  const int32_t nb = hv.nb, hs = hv.hs;
  const int32_t h0 = hv.offO[0];
  auto O = [&](int ax, int32_t q) -> float & { return kAligned ? hv.so[ax * kHS + h0 + q] : hv.so[hv.offO[ax] + q]; };
  auto V = [&](int ax, int32_t q) -> float & { return kAligned ? hv.sv[ax * kHS + h0 + q] : hv.sv[hv.offV[ax] + q]; };
  uint16_t *pos = hv.pos;
  // pass A: push every particle once; the new state goes back to its shared
  // slot and its leaf code gains the destination direction (bits 10-14).  Its
  // unit slot (direction, destination half) and its rank among the arrivals
  // of its warp for that slot are noted; per-warp counts go to wc[].  The
  // pull restores the canonical order, so any order of the slots will do.
  // Arrivals beyond the neighbour bricks are appended at once.
  const int nc32 = (nb + 31) >> 5;
  for (int c = first; c < nc32; c += stride) {
    const int32_t q = c * 32 + lane;
    const bool act = q < nb;
    int uslot = -1;  // unit slot 2 direction + destination half; -1: none (idle lane, far arrival)
    if (act) {
      float on[D], vn[D];
      int dir;
      const int l = pos[q];
      const uint32_t pk = hv.dec[l];
      const int32_t lc[3] = {(int32_t)(pk & 1023u), (int32_t)((pk >> 10) & 1023u), (int32_t)(pk >> 20)};
      float o[D], om[D];
#pragma unroll
      for (int ax = 0; ax < D; ++ax) {
        o[ax] = O(ax, q);
        om[ax] = 1.0f - o[ax];
      }
      const int base = lc[0] + K::V1 * (lc[1] + (D == 3 ? K::V1 * lc[2] : 0));
      // corner weights (1 * f0) * f1 [* f2], f = o or 1 - o by corner bit,
      // two corners per paired multiply; then E = sum over corners of w * E_corner
      // in corner order.  (Paired adds are not used: the compiler fuses a paired
      // multiply and add into one rounding, which would change the result.)
      float wgt[K::NC];
      {
        const float2 f0 = make_float2(om[0], o[0]);
        const float2 a01 = mul2_rn(f0, make_float2(om[1], om[1]));  // corners 0, 1
        const float2 a23 = mul2_rn(f0, make_float2(o[1], o[1]));    // corners 2, 3
        if constexpr (D == 3) {
          const float2 w01 = mul2_rn(a01, make_float2(om[2], om[2]));
          const float2 w23 = mul2_rn(a23, make_float2(om[2], om[2]));
          const float2 w45 = mul2_rn(a01, make_float2(o[2], o[2]));
          const float2 w67 = mul2_rn(a23, make_float2(o[2], o[2]));
          wgt[0] = w01.x; wgt[1] = w01.y; wgt[2] = w23.x; wgt[3] = w23.y;
          wgt[4] = w45.x; wgt[5] = w45.y; wgt[6] = w67.x; wgt[7] = w67.y;
        } else {
          wgt[0] = a01.x; wgt[1] = a01.y; wgt[2] = a23.x; wgt[3] = a23.y;
        }
      }
      float E[D];
#pragma unroll
      for (int ax = 0; ax < D; ++ax) E[ax] = 0.0f;
#pragma unroll
      for (int e = 0; e < K::NC; ++e) {
        const EV ev = hv.Eb[base + (e & 1) + ((e >> 1) & 1) * K::V1 + ((e >> 2) & 1) * K::V1 * K::V1];
#pragma unroll
        for (int ax = 0; ax < D; ++ax) E[ax] = E[ax] + wgt[e] * ecomp(ev, ax);
      }
      // kick and drift: v += (q/m) dt E, t = o + v s_l.  t is non-finite
      // whenever the new velocity is (s_l is finite), so checking t suffices.
      float fl[D];
      int32_t packed = D == 2 ? (9 << 16) : 0;
      bool win = true;
#pragma unroll
      for (int ax = 0; ax < D; ++ax) {
        vn[ax] = V(ax, q) + a.qmdt * E[ax];
        float tt = o[ax] + vn[ax] * a.sl;
        if (!isfinite(tt)) {
          bad = true;
          tt = 0.0f;
        }
        fl[ax] = floorf(tt);
        on[ax] = clamp_off(tt - fl[ax]);
        const uint32_t li = (uint32_t)(lc[ax] + K::B + (int32_t)fmaxf(fminf(fl[ax], 64.0f), -64.0f));
        win &= li < 3u * K::B;
        packed += hv.rel[ax * 32 + (li < 3u * K::B ? li : 0u)];
      }
      int lidx;
      int32_t dest = -1;
      if (win) {
        dir = packed >> 16;
        lidx = packed & 0xffff;
      } else {
        SlowIn in{};
#pragma unroll
        for (int ax = 0; ax < D; ++ax) {
          in.lc[ax] = lc[ax];
          in.origin[ax] = hv.origin[ax];
          in.bc[ax] = hv.bc[ax];
          in.fl[ax] = fl[ax];
        }
        const SlowOut r = relocate_slow<D>(t, g, in);
        dir = r.dir;
        lidx = r.lidx;
        dest = r.dest;
      }
      const bool stay = dir == kSelfDir && lidx == l;
      movers += !stay;
      if (dir == kFarSlot) {  // beyond the neighbour bricks: its own slot now
        const int32_t u = unit_of<D>(dest, lidx);
        const int32_t slot = atomicAdd(&a.st.fill[u], 1);
        stage_put<D>(a.st, u, slot, on, vn, (uint16_t)(lidx | kMoverCode), 0x80000000u | (uint32_t)(hs + q),
                     a.ids ? a.ids[hs + q] : 0, a.ids != nullptr, a.err);
      }
#pragma unroll
      for (int ax = 0; ax < D; ++ax) {
        O(ax, q) = on[ax];
        V(ax, q) = vn[ax];
      }
      pos[q] = (uint16_t)(lidx | (dir << 10) | (stay ? kStayBit : 0));
      if (dir != kFarSlot) uslot = 2 * dir + (lidx >= K::LH);
    }
    // lanes of the chunk with the same unit slot
    const unsigned peers = __match_any_sync(0xffffffffu, uslot);
    const int leader = uslot >= 0 ? __ffs(peers) - 1 : lane;
    int32_t r0 = 0;
    if (uslot >= 0 && lane == leader) {  // one leader per distinct slot: distinct words
      r0 = wc[uslot];
      wc[uslot] = r0 + __popc(peers);
    }
    r0 = __shfl_sync(0xffffffffu, r0, leader);
    if (uslot >= 0) hv.lslot[q] = (uint8_t)(r0 + __popc(peers & ((1u << lane) - 1u)));
    __syncwarp();  // the counts are read by other lanes in the next chunk
  }
  // the warp reserves its runs in the destination units' staging areas (one
  // atomic per unit it sends to; the count becomes the run's first slot)
  {  // both of a lane's atomics in flight at once
    const int us1 = lane + 32;
    const int32_t c0 = wc[lane], c1 = us1 < 54 ? wc[us1] : 0;
    int32_t r0 = 0, r1 = 0;
    if (c0 > 0) r0 = atomicAdd(&a.st.fill[2 * hv.nbr[lane >> 1] + (lane & 1)], c0);
    if (c1 > 0) r1 = atomicAdd(&a.st.fill[2 * hv.nbr[us1 >> 1] + (us1 & 1)], c1);
    if (c0 > 0) wc[lane] = r0;
    if (c1 > 0) wc[us1] = r1;
  }
  __syncwarp();
  // pass B, the warp's own chunks: every arrival to its reserved slot
  // (consecutive particles of a chunk hold consecutive ranks, so the stores
  // coalesce)
  for (int c = first; c < nc32; c += stride) {
    const int32_t q = c * 32 + lane;
    if (q >= nb) break;
    const uint16_t cd = pos[q];
    const int dir = (cd >> 10) & 31;
    if (dir == kFarSlot) continue;
    const int hh = (cd & 0x3ff) >= K::LH;
    const int us = 2 * dir + hh;
    const int32_t slot = wc[us] + hv.lslot[q];
    float on[D], vn[D];
#pragma unroll
    for (int ax = 0; ax < D; ++ax) {
      on[ax] = O(ax, q);
      vn[ax] = V(ax, q);
    }
    const bool stay = (cd & kStayBit) != 0;
    stage_put<D>(a.st, 2 * hv.nbr[dir] + hh, slot, on, vn, (uint16_t)(cd & (kStayBit | 0x3ff)),
                 (stay ? 0u : 0x80000000u) | (uint32_t)(hs + q), a.ids ? a.ids[hs + q] : 0, a.ids != nullptr,
                 a.err);
  }
  __syncwarp();
  for (int us = lane; us < kUnitSlots; us += 32) wc[us] = 0;  // ready for the warp's next half brick
  __syncwarp();
}

// Per-axis re-location table of K1: for local cell l - 9 (l = 0 .. 26) on
// axis ax, (direction digit + 1) 3^ax << 16 | the cell's part of the leaf
// index; computed by threads 0 .. 80.
template <int D>
__device__ __forceinline__ void fill_rel(int32_t *rel, int tid) {
  using K = BK<D>;
  if (tid < 3 * 27) {
    const int ax = tid / 27, loc = tid % 27 - K::B;
    const int dl = (loc >= K::B) - (loc < 0);
    const int p3 = ax == 0 ? 1 : (ax == 1 ? 3 : 9);
    rel[ax * 32 + tid % 27] = ((dl + 1) * p3 << 16) | lidx_axis<D>(loc - K::B * dl, ax);
  }
}

// Neighbour brick of brick coordinates bc in direction dir (-1 for the
// directions a 2D brick does not have).
template <int D>
__device__ __forceinline__ int32_t neighbour_brick(const DevTree &t, const BrickGeom &g, const int32_t *bc, int dir) {
  int32_t sc[3] = {0, 0, 0};
  for (int ax = 0; ax < D; ++ax) {
    const int32_t x = bc[ax] + dir_delta(dir, ax);
    sc[ax] = x < 0 ? x + g.nbx : (x >= g.nbx ? x - g.nbx : x);
  }
  return (D == 2 && dir_delta(dir, 2) != 0) ? -1 : brick_of_coords<D>(t, sc);
}

// K1, shared-memory form: every CTA takes half bricks in turn (a grid of two
// CTAs per SM); per half brick its copies land, the leaf map is built, and
// every warp pushes its share (push_half_warp).  The next half brick's leaf
// offsets are read while the current one is pushed, so its copies go out as
// soon as the shared memory is free.
template <int D, bool kAligned>
__global__ void __launch_bounds__(kHThreads, 2) k_brick_push_st(DevTree t, BrickGeom g, BrickPushArgs a) {
  using K = BK<D>;
  using EV = typename EVec<D>::T;
  constexpr int kW = kHThreads / 32;
  extern __shared__ __align__(128) float smf[];
  float *so = smf;                                   // D rows of kHS offsets
  float *sv = so + D * kHS;                          // D rows of kHS velocities
  uint16_t *pos = (uint16_t *)(sv + D * kHS);        // local leaf of every particle of the half
  EV *Eb = (EV *)(pos + kHalfCap);                   // NVB staged field vectors (16-byte aligned)
  int32_t *lsb = (int32_t *)(Eb + K::NVB);           // LB + 1 absolute leaf offsets after a head of < 4
  uint32_t *dec = (uint32_t *)(lsb + K::LSW);        // LB (padded to DECW words)
  int32_t *rel = (int32_t *)(dec + K::DECW);         // 3 x 32: per-axis direction | leaf-index parts
  int32_t *nbr = rel + 3 * 32;                       // 27 neighbour bricks by direction
  int32_t *wc = nbr + 32;                            // [warp][unit slot] arrivals, then first slot
  uint8_t *lslot = (uint8_t *)(wc + kW * kUnitSlots); // rank within (warp, unit slot)
  __shared__ int32_t s_movers;
  __shared__ uint64_t s_bar;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t n = a.n;
  const int32_t nh = 2 * g.n_bricks;
  // brick-independent tables, once per CTA
  fill_rel<D>(rel, tid);
  for (int i = tid; i < K::DECW; i += blockDim.x) dec[i] = g.decodeL[i];
  for (int i = tid; i < kW * kUnitSlots; i += blockDim.x) wc[i] = 0;  // each warp leaves its counts at zero
  if (tid == 0) {
    s_movers = 0;
    mbar_init(&s_bar, 1);
  }
  bool bad = false;
  int movers = 0;
  unsigned parity = 0;  // phase of s_bar the current half brick's copies complete
  int32_t hb = blockIdx.x;
  int32_t ps = 0, pe = 0;
  if (hb < nh) {
    ps = a.start[(hb >> 1) * K::LB];
    pe = a.start[(hb >> 1) * K::LB + K::LB];
  }
  __syncthreads();  // tables written, barrier initialised
  for (; hb < nh; hb += gridDim.x) {
    const int32_t b = hb >> 1, h = hb & 1, L0 = b * K::LB;
    const int32_t nbr_n = pe - ps;
    const int32_t q0 = half_start(nbr_n, h), q1 = h ? nbr_n : half_start(nbr_n, 1), nb = q1 - q0;
    const int32_t hs = ps + q0;  // storage index of this half's first particle
    // the next half brick's offsets, read now and used after this one
    const int32_t hn = hb + (int32_t)gridDim.x;
    int32_t ps_next = 0, pe_next = 0;
    if (hn < nh) {
      ps_next = a.start[(hn >> 1) * K::LB];
      pe_next = a.start[(hn >> 1) * K::LB + K::LB];
    }
    // bricks over 2 kHalfCap particles: listed for the global-memory kernel;
    // empty halves: nothing to push
    if (nbr_n > 2 * kHalfCap && h == 0 && tid == 0) a.st.over_bricks[atomicAdd(&a.st.over[0], 1)] = b;
    if (nbr_n <= 2 * kHalfCap && nb > 0) {
      HalfView<D> hv;
      hv.so = so;
      hv.sv = sv;
      hv.pos = pos;
      hv.lslot = lslot;
      hv.Eb = Eb;
      hv.dec = dec;
      hv.rel = rel;
      hv.nbr = nbr;
      hv.nb = nb;
      hv.hs = hs;
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        hv.origin[ax] = ax < D ? t.leaf_coords[(int64_t)L0 * D + ax] : 0;
        hv.bc[ax] = hv.origin[ax] / K::B;
      }
      if (tid >= 128 && tid < 128 + 27) nbr[tid - 128] = neighbour_brick<D>(t, g, hv.bc, tid - 128);
      // the half's particle rows: one bulk copy per row from the 16-byte
      // boundary at or below its first particle; row r holds particle q at
      // index off[r] + q
#pragma unroll
      for (int r = 0; r < 2 * D; ++r) {
        const float *src = (r < D ? a.o + r * n : a.v + (r - D) * n) + hs;
        const int32_t head = (int32_t)(((uintptr_t)src & 15u) >> 2);
        if (r < D) hv.offO[r] = r * kHS + head;
        else hv.offV[r - D] = (r - D) * kHS + head;
      }
      // the brick's leaf offsets start at the 16-byte boundary at or below L0
      const int32_t lhead = (int32_t)(((uintptr_t)(a.start + L0) & 15u) >> 2);
      const int32_t *ls = lsb + lhead;
      if (tid == 0) {
        // every global -> shared copy of the half brick is one bulk copy,
        // issued before any is awaited: the particle rows of the half, the
        // brick's leaf offsets and the brick's field (one vector per vertex,
        // laid out brick by brick when the field was set).  The shared memory
        // they overwrite was last read and written by the generic proxy.
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        uint32_t total = 0, bytes[2 * D];
        const float *src[2 * D];
#pragma unroll
        for (int r = 0; r < 2 * D; ++r) {
          const float *p = (r < D ? a.o + r * n : a.v + (r - D) * n) + hs;
          const uintptr_t a0 = (uintptr_t)p & ~(uintptr_t)15;
          src[r] = (const float *)a0;
          bytes[r] = (uint32_t)(((uintptr_t)(p + nb) - a0 + 15u) & ~(uintptr_t)15);
          total += bytes[r];
        }
        const int32_t *ls0 = a.start + L0 - lhead;
        const uint32_t lbytes = (uint32_t)(((lhead + K::LB + 1) * 4 + 15) & ~15);
        constexpr uint32_t ebytes = K::NVB * sizeof(EV);
        total += lbytes + ebytes;
        mbar_expect_tx(&s_bar, total);
#pragma unroll
        for (int r = 0; r < 2 * D; ++r)
          bulk_g2s(r < D ? so + r * kHS : sv + (r - D) * kHS, src[r], bytes[r], &s_bar);
        bulk_g2s(lsb, ls0, lbytes, &s_bar);
        bulk_g2s(Eb, (const EV *)a.Ebrick + (int64_t)b * K::NVB, ebytes, &s_bar);
      }
      const bool landed = mbar_wait(&s_bar, parity, a.wait_cycles);
      if (__syncthreads_or(!landed)) {
        if (!landed) mbar_wait(&s_bar, parity, kWaitCycles);  // let copies in flight land before leaving
        if (tid == 0) atomicOr(a.err, kErrTimeout);
        return;
      }
      parity ^= 1u;
      for (int l = tid; l < K::LB; l += blockDim.x) {
        const int32_t lo = max(ls[l] - hs, 0), hi = min(ls[l + 1] - hs, nb);
        for (int32_t q = lo; q < hi; ++q) pos[q] = (uint16_t)l;
      }
      __syncthreads();  // leaf map and neighbour bricks written
      push_half_warp<D, kAligned>(t, g, a, hv, w, kW, wc + w * kUnitSlots, bad, movers);
      __syncthreads();  // the shared memory is free for the next half brick's copies
    }
    ps = ps_next;
    pe = pe_next;
  }
  if (bad) atomicOr(a.err, 1);
  for (int o = 16; o > 0; o >>= 1) movers += __shfl_down_sync(0xffffffffu, movers, o);
  if (lane == 0 && movers) atomicAdd(&s_movers, movers);
  __syncthreads();
  if (tid == 0 && s_movers) atomicAdd(a.n_movers, s_movers);
}

// K1 for bricks over 2 kHalfCap particles: the same arithmetic (push_core),
// particles and field read from global memory, one thread per particle.
template <int D>
__device__ __forceinline__ void brick_push_fallback(const DevTree &t, const BrickGeom &g, const BrickPushArgs &a,
                                                    const int32_t b) {
  using K = BK<D>;
  __shared__ int32_t ls[K::LB + 1];
  __shared__ uint32_t dec[K::LB];
  __shared__ float Eb[D * K::NVB];
  __shared__ int32_t s_movers;
  const int tid = threadIdx.x, lane = tid & 31;
  const int32_t L0 = b * K::LB;
  const int32_t ps = a.start[L0], pe = a.start[L0 + K::LB], nb = pe - ps;
  if (nb <= 2 * kHalfCap) return;  // the shared-memory kernel took this brick
  int32_t origin[3] = {0, 0, 0}, bc[3] = {0, 0, 0};
  for (int ax = 0; ax < D; ++ax) {
    origin[ax] = t.leaf_coords[(int64_t)L0 * D + ax];
    bc[ax] = origin[ax] / K::B;
  }
  for (int i = tid; i <= K::LB; i += blockDim.x) ls[i] = a.start[L0 + i] - ps;
  for (int i = tid; i < K::LB; i += blockDim.x) dec[i] = g.decodeL[i];
  stage_field<D>(t, a, origin, Eb);
  if (tid == 0) s_movers = 0;
  __syncthreads();
  bool bad = false;
  int movers = 0;
  for (int32_t base = 0; base < nb; base += blockDim.x) {
    const int32_t q = base + tid;
    const bool act = q < nb;
    int32_t dest = -1;
    float on[D], vn[D];
    uint16_t code = 0;
    uint32_t key = 0;
    if (act) {
      int lo = 0, hi = K::LB - 1;  // leaf of storage position q: last l with ls[l] <= q
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ls[mid] <= q) lo = mid;
        else hi = mid - 1;
      }
      const int l = lo;
      const uint32_t pk = dec[l];
      const int32_t lc[3] = {(int32_t)(pk & 1023u), (int32_t)((pk >> 10) & 1023u), (int32_t)(pk >> 20)};
      int32_t L2;
      const int dir = brick_push_one<D>(t, g, a, ps + q, lc, origin, bc, Eb, on, vn, L2, bad);
      (void)dir;
      const bool stay = L2 == L0 + l;
      movers += !stay;
      dest = unit_of<D>(L2 / K::LB, L2 % K::LB);
      code = (uint16_t)((L2 % K::LB) | (stay ? kStayBit : 0));
      key = (stay ? 0u : 0x80000000u) | (uint32_t)(ps + q);
    }
    stage_append<D>(a.st, dest, on, vn, code, key, (a.ids && act) ? a.ids[ps + q] : 0, a.ids != nullptr, a.err);
  }
  if (bad) atomicOr(a.err, 1);
  for (int o = 16; o > 0; o >>= 1) movers += __shfl_down_sync(0xffffffffu, movers, o);
  if (lane == 0) atomicAdd(&s_movers, movers);
  __syncthreads();
  if (tid == 0 && s_movers) atomicAdd(a.n_movers, s_movers);
}

// Bricks too large for the shared-memory kernel (listed by it), from global
// memory; the blocks take the listed bricks in turn.
template <int D>
__global__ void __launch_bounds__(kPushThreads) k_brick_push(DevTree t, BrickGeom g, BrickPushArgs a) {
  const int32_t m = min(*a.st.over, (int32_t)g.n_bricks);
  for (int32_t i = blockIdx.x; i < m; i += gridDim.x) {
    brick_push_fallback<D>(t, g, a, a.st.over_bricks[i]);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// between K1 and K2: overflow arrivals grouped by destination, brick totals
// ---------------------------------------------------------------------------

__global__ void k_ovf_count(const int32_t *ovf_n, int32_t ovf_cap, const int32_t *ovf_dest, int32_t *fcount) {
  const int32_t nf = min(*ovf_n, ovf_cap);
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x)
    atomicAdd(&fcount[ovf_dest[i]], 1);
}

__global__ void k_ovf_scatter(const int32_t *ovf_n, int32_t ovf_cap, const int32_t *ovf_dest, const int32_t *fstart,
                              int32_t *fcursor, int32_t *sorted) {
  const int32_t nf = min(*ovf_n, ovf_cap);
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x) {
    const int32_t db = ovf_dest[i];
    sorted[fstart[db] + atomicAdd(&fcursor[db], 1)] = i;
  }
}

__global__ void k_brick_totals(int64_t n_units, int32_t cap, const int32_t *fill, const int32_t *fstart,
                               int32_t *tot) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n_units) return;
  tot[u] = min(fill[u], cap) + (fstart[u + 1] - fstart[u]);
}

// ---------------------------------------------------------------------------
// K2: one CTA per destination unit (half brick), two CTAs per SM
// ---------------------------------------------------------------------------

constexpr int kStThreads = 512;
constexpr int kStCap = 3456;  // arrivals per unit held in shared memory (the largest staging capacity)

template <int D>
size_t pull_st_smem() {
  return (sizeof(float) * 2 * D + sizeof(uint32_t) + 2 * sizeof(uint16_t)) * kStCap;
}

// Sorts the m <= N arrival indices mp[0..m) of one leaf by their keys
// (distinct) with Batcher's odd-even merge network (5, 19 and 63 comparators
// for N = 4, 8, 16) over (key, index) pairs in registers.
template <int N>
__device__ __forceinline__ void sort_leaf_net(uint16_t *mp, int m, const uint32_t *key) {
  uint32_t k[N], v[N];
#pragma unroll
  for (int t = 0; t < N; ++t) {
    v[t] = t < m ? mp[t] : 0u;
    k[t] = t < m ? key[v[t]] : 0xffffffffu;
  }
#pragma unroll
  for (int p = 1; p < N; p <<= 1)
#pragma unroll
    for (int c = p; c >= 1; c >>= 1)
#pragma unroll
      for (int j = c % p; j + c < N; j += 2 * c)
#pragma unroll
        for (int i = 0; i < N; ++i)
          if (i < c && i < N - j - c && (i + j) / (2 * p) == (i + j + c) / (2 * p)) {
            const int x = i + j, y = i + j + c;
            const bool sw = k[x] > k[y];
            const uint32_t tk = k[x], tv = v[x];
            k[x] = sw ? k[y] : tk;
            v[x] = sw ? v[y] : tv;
            k[y] = sw ? tk : k[y];
            v[y] = sw ? tv : v[y];
          }
#pragma unroll
  for (int t = 0; t < N; ++t)
    if (t < m) mp[t] = (uint16_t)v[t];
}

// Size class of a leaf's sort: -1 nothing to sort, 0..2 networks of 4, 8
// and 16, 3 a warp.
__device__ __forceinline__ int leaf_class(int32_t m) {
  return m <= 1 ? -1 : (m <= 4 ? 0 : (m <= 8 ? 1 : (m <= 16 ? 2 : 3)));
}

// Exclusive scan of c over the first nl <= blockDim.x threads of the block
// (c = 0 beyond); returns this thread's offset.  wsum holds one word per warp.
__device__ __forceinline__ int32_t block_excl_scan(int32_t c, int32_t *wsum) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int32_t x = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  int32_t before = 0;
  for (int k = 0; k < nw; ++k)
    if (k < w) before += wsum[k];
  return before + x - c;
}

template <int D>
__global__ void __launch_bounds__(kStThreads, 2) k_brick_pull_st(DevTree t, BrickGeom g, BrickPullArgs a) {
  using K = BK<D>;
  extern __shared__ __align__(128) float smf[];
  float *srec = smf;                                 // kStCap records of 2 D floats (arrival order)
  uint32_t *key = (uint32_t *)(srec + 2 * D * kStCap);  // canonical keys
  uint16_t *code = (uint16_t *)(key + kStCap);       // local leaf | stayer bit; later the final position
  uint16_t *map = code + kStCap;                     // bucket position -> arrival
  __shared__ int32_t cnt[K::LH + 1];
  __shared__ int32_t cur[K::LH];
  __shared__ int32_t wsum[kStThreads / 32];
  __shared__ int32_t s_max, s_ccount[4];
  __shared__ uint64_t s_bar, s_bar2;  // keys and codes; offsets and velocities
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const BrickStage &st = a.st;
  const int32_t u = blockIdx.x, b = u >> 1;
  const int lf0 = (u & 1) ? K::LH : 0, nlf = (u & 1) ? K::LB - K::LH : K::LH;
  const int32_t L0 = b * K::LB + lf0;  // first leaf of the unit
  const int64_t n = a.n;
  const int32_t nin = st.fill[u];
  if (nin > st.cap) {  // listed for the global-memory kernel
    if (tid == 0) st.over_units[atomicAdd(&st.over[1], 1)] = u;
    return;
  }
  const int64_t at = (int64_t)u * st.cap;
  if (tid < 4) s_ccount[tid] = 0;
  if (tid == 0) {
    s_max = 0;
    if (nin > 0) {
      // keys and codes on one barrier, the state rows on another: the counts,
      // offsets and per-leaf sorts need only the former, so they start while
      // the state (24 of the 30 bytes per arrival) is still landing
      mbar_init(&s_bar, 1);
      mbar_init(&s_bar2, 1);
      const uint32_t rb = (uint32_t)((nin * 4 + 15) & ~15), cb = (uint32_t)((nin * 2 + 15) & ~15);
      mbar_expect_tx(&s_bar, rb + cb);
      bulk_g2s(key, st.key + at, rb, &s_bar);
      bulk_g2s(code, st.code + at, cb, &s_bar);
      const uint32_t sb = (uint32_t)((nin * 8 * D + 15) & ~15);
      mbar_expect_tx(&s_bar2, sb);
      bulk_g2s(srec, st.rec + at * (2 * D), sb, &s_bar2);
    }
  }
  for (int i = tid; i <= nlf; i += blockDim.x) cnt[i] = 0;
  __syncthreads();  // the barriers are initialised and armed before anyone waits on them
  {
    const bool landed = nin == 0 || mbar_wait(&s_bar, 0, a.wait_cycles);
    if (__syncthreads_or(!landed)) {
      if (nin > 0) {  // let copies in flight land before leaving
        if (!landed) mbar_wait(&s_bar, 0, kWaitCycles);
        mbar_wait(&s_bar2, 0, kWaitCycles);
      }
      if (tid == 0) atomicOr(a.err, kErrTimeout);
      return;
    }
  }
  // leaf counts: four consecutive arrivals per thread (one 8-byte load of
  // their codes), one shared atomic per run
  bool badc = false;
  for (int32_t r0 = 4 * tid; r0 < nin; r0 += 4 * kStThreads) {
    int leaf = -1, run = 0;
    const uint2 c4 = *reinterpret_cast<const uint2 *>(code + r0);
    const uint32_t cw[2] = {c4.x, c4.y};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (r0 + k >= nin) break;
      const int lf = (int)((cw[k >> 1] >> (16 * (k & 1))) & 0x3ffu) - lf0;
      if (lf < 0 || lf >= nlf) {
        badc = true;
        continue;
      }
      if (lf == leaf) {
        ++run;
      } else {
        if (run) atomicAdd(&cnt[leaf], run);
        leaf = lf;
        run = 1;
      }
    }
    if (run) atomicAdd(&cnt[leaf], run);
  }
  if (__syncthreads_or(badc)) {  // a staged code names no leaf of the unit
    if (nin > 0) mbar_wait(&s_bar2, 0, kWaitCycles);  // let the state copy land before leaving
    if (tid == 0) atomicOr(a.err, kErrCode);
    return;
  }
  // leaf offsets (nlf <= blockDim.x), cursors, largest leaf count; the
  // thread of leaf tid notes its sort class and its rank within the class
  int cls = -1, crank = 0;
  {
    const int32_t c = tid < nlf ? cnt[tid] : 0;
    const int32_t off = block_excl_scan(c, wsum);
    if (tid < nlf) {
      cnt[tid] = off;
      cur[tid] = off;
    }
    const int32_t wmax = __reduce_max_sync(0xffffffffu, c);
    if (lane == 0 && wmax > 0) atomicMax(&s_max, wmax);
    if (tid == 0) cnt[nlf] = nin;
    cls = leaf_class(c);
    const unsigned peers = __match_any_sync(0xffffffffu, cls);
    const int leader = __ffs(peers) - 1;
    int32_t base = 0;
    if (cls >= 0 && lane == leader) base = atomicAdd(&s_ccount[cls], __popc(peers));
    crank = __shfl_sync(0xffffffffu, base, leader) + __popc(peers & ((1u << lane) - 1u));
  }
  __syncthreads();
  // bucket positions in any order
  for (int32_t i = tid; i < nin; i += blockDim.x) map[atomicAdd(&cur[(code[i] & 0x3ff) - lf0], 1)] = (uint16_t)i;
  __syncthreads();
  // leaves to sort, grouped by size class (the cursors are free now), so that
  // the threads of a warp run the same network
  uint16_t *list = (uint16_t *)cur;
  const int32_t nA = s_ccount[0], nB = s_ccount[1], nC = s_ccount[2], nD = s_ccount[3];
  if (cls >= 0) list[(cls > 0 ? nA : 0) + (cls > 1 ? nB : 0) + (cls > 2 ? nC : 0) + crank] = (uint16_t)tid;
  __syncthreads();
  // every leaf's arrivals sorted by canonical key, in place
  const int32_t nABC = nA + nB + nC;
  for (int32_t t = tid; t < nABC; t += blockDim.x) {
    const int lf = list[t];
    const int32_t lo = cnt[lf], m = cnt[lf + 1] - lo;
    if (m <= 4) sort_leaf_net<4>(map + lo, m, key);
    else if (m <= 8) sort_leaf_net<8>(map + lo, m, key);
    else sort_leaf_net<16>(map + lo, m, key);
  }
  for (int32_t dd = w; dd < nD; dd += blockDim.x >> 5) {  // a warp per leaf over 16 arrivals
    const int lf = list[nABC + dd];
    const int32_t lo = cnt[lf], m = cnt[lf + 1] - lo;
    if (m <= 32) {
      const int32_t i = lane < m ? map[lo + lane] : 0;
      const uint32_t kx = lane < m ? key[i] : 0xffffffffu;
      int32_t r = 0;
      for (int t2 = 0; t2 < m; ++t2) r += __shfl_sync(0xffffffffu, kx, t2) < kx;
      __syncwarp();
      if (lane < m) map[lo + r] = (uint16_t)i;
    } else {  // crowded leaves: the warp runs a bitonic network over the leaf's slots
      warp_sort_indirect<uint16_t, uint32_t>(map + lo, m, key);
    }
    __syncwarp();
  }
  const int32_t bstart = a.bstart[u];
  for (int l = tid; l < nlf; l += blockDim.x) a.new_start[L0 + l] = bstart + cnt[l];
  if (u == 2 * g.n_bricks - 1 && tid == 0) a.new_start[(int64_t)g.n_bricks * K::LB] = bstart + nin;
  if (tid == 0 && s_max > 0) atomicMax(a.max_bucket, s_max);
  {
    const bool landed = nin == 0 || mbar_wait(&s_bar2, 0, a.wait_cycles);
    if (__syncthreads_or(!landed)) {
      if (!landed) mbar_wait(&s_bar2, 0, kWaitCycles);  // let copies in flight land before leaving
      if (tid == 0) atomicOr(a.err, kErrTimeout);
      return;
    }
  }
  // coalesced writes in destination order
  {
    float *gO[D], *gV[D];
#pragma unroll
    for (int ax = 0; ax < D; ++ax) {
      gO[ax] = a.o + ax * n + bstart;
      gV[ax] = a.v + ax * n + bstart;
    }
    for (int32_t j = tid; j < nin; j += blockDim.x) {
      const float *r = srec + 2 * D * map[j];
      if constexpr (D == 3) {
        const float2 r0 = reinterpret_cast<const float2 *>(r)[0], r1 = reinterpret_cast<const float2 *>(r)[1],
                     r2 = reinterpret_cast<const float2 *>(r)[2];
        gO[0][j] = r0.x; gO[1][j] = r0.y; gO[2][j] = r1.x;
        gV[0][j] = r1.y; gV[1][j] = r2.x; gV[2][j] = r2.y;
      } else {
        const float4 r0 = *reinterpret_cast<const float4 *>(r);
        gO[0][j] = r0.x; gO[1][j] = r0.y;
        gV[0][j] = r0.z; gV[1][j] = r0.w;
      }
    }
    if (a.ids)
      for (int32_t j = tid; j < nin; j += blockDim.x) a.ids[bstart + j] = st.id[at + map[j]];
  }
  // deposit partials of the new positions, per leaf in bucket order; the
  // next particle's offsets are fetched while the current one is summed
  if (a.part) {
    for (int l = tid; l < nlf; l += blockDim.x) {
      float acc[K::NC];
#pragma unroll
      for (int e = 0; e < K::NC; ++e) acc[e] = 0.0f;
      const int32_t lo = cnt[l], hi = cnt[l + 1];
      float on[D];
      if (lo < hi) {
        const float *r = srec + 2 * D * map[lo];
#pragma unroll
        for (int ax = 0; ax < D; ++ax) on[ax] = r[ax];
      }
      for (int32_t j = lo; j < hi; ++j) {
        float o[D], om[D];
#pragma unroll
        for (int ax = 0; ax < D; ++ax) {
          o[ax] = on[ax];
          om[ax] = 1.0f - o[ax];
        }
        if (j + 1 < hi) {
          const float *r = srec + 2 * D * map[j + 1];
#pragma unroll
          for (int ax = 0; ax < D; ++ax) on[ax] = r[ax];
        }
        // corner weights (f0 * f1) [* f2] as in the push, two corners per
        // paired multiply, then summed per corner in bucket order
        const float2 f0 = make_float2(om[0], o[0]);
        const float2 a01 = mul2_rn(f0, make_float2(om[1], om[1]));
        const float2 a23 = mul2_rn(f0, make_float2(o[1], o[1]));
        if constexpr (D == 3) {
          const float2 w01 = mul2_rn(a01, make_float2(om[2], om[2]));
          const float2 w23 = mul2_rn(a23, make_float2(om[2], om[2]));
          const float2 w45 = mul2_rn(a01, make_float2(o[2], o[2]));
          const float2 w67 = mul2_rn(a23, make_float2(o[2], o[2]));
          acc[0] = acc[0] + w01.x; acc[1] = acc[1] + w01.y; acc[2] = acc[2] + w23.x; acc[3] = acc[3] + w23.y;
          acc[4] = acc[4] + w45.x; acc[5] = acc[5] + w45.y; acc[6] = acc[6] + w67.x; acc[7] = acc[7] + w67.y;
        } else {
          acc[0] = acc[0] + a01.x; acc[1] = acc[1] + a01.y; acc[2] = acc[2] + a23.x; acc[3] = acc[3] + a23.y;
        }
      }
      float *gp = a.part + (int64_t)(L0 + l) * K::NC;
#pragma unroll
      for (int e = 0; e < K::NC; ++e) gp[e] = acc[e];
    }
  }
}

// K2 for units over their staging capacity: the staging area (first cap
// arrivals) and the unit's overflow arrivals; a counting sort by leaf in
// global scratch (fb_key / fb_idx at the unit's output range), a per-leaf
// sort by key (insertion by one thread up to kPullSmallLeaf arrivals, the
// block's bitonic network above), then gathers in bucket order.  Arrival r < cap is
// staging slot r, arrival cap + k the unit's k-th overflow entry.
constexpr int kPullSmallLeaf = 32;  // leaves up to this many arrivals: one thread's insertion sort
constexpr int kPullChunk = 2048;    // (key, index) pairs of a crowded leaf sorted at once in shared memory

template <int D>
__device__ __forceinline__ void brick_pull_fallback(const DevTree &t, const BrickGeom &g, const BrickPullArgs &a,
                                                    const int32_t u) {
  using K = BK<D>;
  __shared__ uint32_t sk[kPullChunk];
  __shared__ int32_t sv[kPullChunk];
  __shared__ int32_t cnt[K::LH + 1];
  __shared__ int32_t cur[K::LH];
  __shared__ int32_t wsum[kPullThreads / 32];
  __shared__ int32_t s_max;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  const BrickStage &st = a.st;
  const int32_t b = u >> 1;
  const int lf0 = (u & 1) ? K::LH : 0, nlf = (u & 1) ? K::LB - K::LH : K::LH;
  const int32_t L0 = b * K::LB + lf0;
  const int64_t n = a.n;
  if (st.fill[u] <= st.cap) return;  // the shared-memory kernel took this unit
  const int32_t nf = st.cap;
  const int32_t f0 = a.fstart[u], nov = a.fstart[u + 1] - f0, nin = nf + nov;
  const int64_t at = (int64_t)u * st.cap;
  auto code_of = [&](int32_t r) -> uint16_t {
    return r < nf ? st.code[at + r] : st.ovf_code[a.ovf_sorted[f0 + r - nf]];
  };
  auto key_of = [&](int32_t r) -> uint32_t {
    return r < nf ? st.key[at + r] : st.ovf_key[a.ovf_sorted[f0 + r - nf]];
  };
  auto leaf_of = [&](int32_t r) -> int { return min(max((code_of(r) & 0x3ff) - lf0, 0), nlf - 1); };
  for (int i = tid; i <= nlf; i += blockDim.x) cnt[i] = 0;
  if (tid == 0) s_max = 0;
  __syncthreads();
  for (int32_t r = tid; r < nin; r += blockDim.x) atomicAdd(&cnt[leaf_of(r)], 1);
  __syncthreads();
  int32_t carry = 0;
  for (int base = 0; base < nlf; base += blockDim.x) {
    const int l = base + tid;
    const int32_t c = l < nlf ? cnt[l] : 0;
    int32_t x = c;
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    int32_t before = 0, all = 0;
    for (int k = 0; k < nw; ++k) {
      if (k < w) before += wsum[k];
      all += wsum[k];
    }
    if (l < nlf) {
      cnt[l] = carry + before + x - c;
      cur[l] = cnt[l];
      if (c > 0) atomicMax(&s_max, c);
    }
    carry += all;
    __syncthreads();
  }
  if (tid == 0) cnt[nlf] = carry;
  __syncthreads();
  const int32_t bstart = a.bstart[u];
  for (int32_t r = tid; r < nin; r += blockDim.x) {
    const int32_t p = bstart + atomicAdd(&cur[leaf_of(r)], 1);
    a.fb_key[p] = key_of(r);
    a.fb_idx[p] = r;
  }
  __syncthreads();
  for (int l = tid; l < nlf; l += blockDim.x) {
    a.new_start[L0 + l] = bstart + cnt[l];
    const int32_t lo = bstart + cnt[l], hi = bstart + cnt[l + 1];
    if (hi - lo > kPullSmallLeaf) continue;  // crowded: sorted by the whole block below
    for (int32_t i = lo + 1; i < hi; ++i) {
      const uint32_t kx = a.fb_key[i];
      const int32_t vx = a.fb_idx[i];
      int32_t j = i - 1;
      while (j >= lo && a.fb_key[j] > kx) {
        a.fb_key[j + 1] = a.fb_key[j];
        a.fb_idx[j + 1] = a.fb_idx[j];
        --j;
      }
      a.fb_key[j + 1] = kx;
      a.fb_idx[j + 1] = vx;
    }
  }
  __syncthreads();
  for (int l = 0; l < nlf; ++l) {  // crowded leaves, one at a time, by the whole block
    const int32_t lo = bstart + cnt[l], m = cnt[l + 1] - cnt[l];
    if (m > kPullSmallLeaf) block_sort_global<uint32_t, int32_t>(a.fb_key + lo, a.fb_idx + lo, m, sk, sv, kPullChunk);
  }
  if (u == 2 * g.n_bricks - 1 && tid == 0) a.new_start[(int64_t)g.n_bricks * K::LB] = bstart + nin;
  if (tid == 0 && s_max > 0) atomicMax(a.max_bucket, s_max);
  __syncthreads();
  for (int32_t j = tid; j < nin; j += blockDim.x) {
    const int32_t r = a.fb_idx[bstart + j];
    const int32_t dst = bstart + j;
    if (r < nf) {
      const float *rr = st.rec + (at + r) * (2 * D);
#pragma unroll
      for (int ax = 0; ax < D; ++ax) {
        a.o[ax * n + dst] = rr[ax];
        a.v[ax * n + dst] = rr[D + ax];
      }
      if (a.ids) a.ids[dst] = st.id[at + r];
    } else {
      const int32_t k = a.ovf_sorted[f0 + r - nf];
#pragma unroll
      for (int ax = 0; ax < D; ++ax) {
        a.o[ax * n + dst] = st.ovf_o[ax * (int64_t)st.ovf_cap + k];
        a.v[ax * n + dst] = st.ovf_v[ax * (int64_t)st.ovf_cap + k];
      }
      if (a.ids) a.ids[dst] = st.ovf_id[k];
    }
  }
  __syncthreads();
  // deposit partials of the new positions, per leaf in bucket order
  if (a.part) {
    for (int l = tid; l < nlf; l += blockDim.x) {
      float acc[K::NC];
#pragma unroll
      for (int e = 0; e < K::NC; ++e) acc[e] = 0.0f;
      for (int32_t p = bstart + cnt[l]; p < bstart + cnt[l + 1]; ++p) {
        float o[D], om[D];
#pragma unroll
        for (int ax = 0; ax < D; ++ax) {
          o[ax] = a.o[ax * n + p];
          om[ax] = 1.0f - o[ax];
        }
#pragma unroll
        for (int e = 0; e < K::NC; ++e) {
          float wgt = 1.0f;
#pragma unroll
          for (int ax = 0; ax < D; ++ax) wgt = wgt * (((e >> ax) & 1) ? o[ax] : om[ax]);
          acc[e] = acc[e] + wgt;
        }
      }
#pragma unroll
      for (int e = 0; e < K::NC; ++e) a.part[(int64_t)(L0 + l) * K::NC + e] = acc[e];
    }
  }
}

// Destination units whose arrivals overflow their staging area (listed by
// the shared-memory kernel), from global memory; the blocks take the listed
// units in turn.
template <int D>
__global__ void __launch_bounds__(kPullThreads) k_brick_pull(DevTree t, BrickGeom g, BrickPullArgs a) {
  const int32_t m = min(a.st.over[1], (int32_t)(2 * g.n_bricks));
  for (int32_t i = blockIdx.x; i < m; i += gridDim.x) {
    brick_pull_fallback<D>(t, g, a, a.st.over_units[i]);
    __syncthreads();
  }
}

__global__ void k_expand_leaves(const int32_t *start, int64_t n_leaves, int32_t *leaf) {
  int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n_leaves) return;
  for (int32_t p = start[l]; p < start[l + 1]; ++p) leaf[p] = (int32_t)l;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

void launch_brick_push(const DevTree &t, const BrickGeom &g, const BrickPushArgs &pa, cudaStream_t s) {
  cudaMemsetAsync(pa.st.fill, 0, sizeof(int32_t) * 2 * g.n_bricks, s);
  cudaMemsetAsync(pa.st.ovf_n, 0, sizeof(int32_t), s);
  cudaMemsetAsync(pa.st.over, 0, 2 * sizeof(int32_t), s);
  const unsigned nb = (unsigned)g.n_bricks;
  const bool al = pa.n % 4 == 0;
  const unsigned np = std::min(2 * nb, kPersistBlocks);
  if (g.d == 3) {
    if (al) k_brick_push_st<3, true><<<np, kHThreads, push_st_smem<3>(), s>>>(t, g, pa);
    else k_brick_push_st<3, false><<<np, kHThreads, push_st_smem<3>(), s>>>(t, g, pa);
  } else {
    if (al) k_brick_push_st<2, true><<<np, kHThreads, push_st_smem<2>(), s>>>(t, g, pa);
    else k_brick_push_st<2, false><<<np, kHThreads, push_st_smem<2>(), s>>>(t, g, pa);
  }
  const unsigned nf = std::min(nb, kFallbackBlocks);  // the fallback visits every brick with fewer blocks
  if (g.d == 3) k_brick_push<3><<<nf, kPushThreads, 0, s>>>(t, g, pa);
  else k_brick_push<2><<<nf, kPushThreads, 0, s>>>(t, g, pa);
  count_launches(2);
}

void launch_brick_pull(const DevTree &t, const BrickGeom &g, const BrickPullArgs &qa, int32_t *fcount,
                       int32_t *fcursor, int32_t *tile_sums, int32_t *scratch_total, cudaStream_t s) {
  const int64_t nu = 2 * g.n_bricks;  // destination units
  cudaMemsetAsync(fcount, 0, sizeof(int32_t) * nu, s);
  cudaMemsetAsync(fcursor, 0, sizeof(int32_t) * nu, s);
  k_ovf_count<<<64, 256, 0, s>>>(qa.st.ovf_n, qa.st.ovf_cap, qa.st.ovf_dest, fcount);
  launch_exclusive_scan(fcount, nu, qa.fstart_w, tile_sums, scratch_total, s);
  k_ovf_scatter<<<64, 256, 0, s>>>(qa.st.ovf_n, qa.st.ovf_cap, qa.st.ovf_dest, qa.fstart, fcursor, qa.ovf_sorted_w);
  k_brick_totals<<<(unsigned)((nu + 255) / 256), 256, 0, s>>>(nu, qa.st.cap, qa.st.fill, qa.fstart, qa.tot_w);
  launch_exclusive_scan(qa.tot_w, nu, qa.bstart_w, tile_sums, scratch_total, s);
  if (g.d == 3) {
    k_brick_pull_st<3><<<(unsigned)nu, kStThreads, pull_st_smem<3>(), s>>>(t, g, qa);
    k_brick_pull<3><<<std::min((unsigned)nu, kFallbackBlocks), kPullThreads, 0, s>>>(t, g, qa);
  } else {
    k_brick_pull_st<2><<<(unsigned)nu, kStThreads, pull_st_smem<2>(), s>>>(t, g, qa);
    k_brick_pull<2><<<std::min((unsigned)nu, kFallbackBlocks), kPullThreads, 0, s>>>(t, g, qa);
  }
  count_launches(5);  // overflow count, overflow scatter, totals, two pull kernels (the scans count themselves)
}

// Self-test of the bounded wait: the barrier expects 16 bytes and no copy is
// ever issued, so the wait must give up after `cycles` and the kernel return.
__global__ void k_wait_selftest(long long cycles, int32_t *flag) {
  __shared__ uint64_t s_bar;
  if (threadIdx.x == 0) {
    mbar_init(&s_bar, 1);
    mbar_expect_tx(&s_bar, 16);
  }
  __syncthreads();  // initialised and armed before anyone waits
  const bool done = mbar_wait(&s_bar, 0, cycles);
  if (__syncthreads_or(!done)) {
    if (threadIdx.x == 0) *flag = 1;
  } else if (threadIdx.x == 0) {
    *flag = 2;
  }
}

void launch_wait_selftest(long long cycles, int32_t *flag, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(cycles, flag);
  count_launches(1);
}

template <int D>
__global__ void k_brick_field(DevTree t, BrickGeom g, const float *__restrict__ E,
                              typename EVec<D>::T *__restrict__ out) {
  using K = BK<D>;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n_bricks * K::NVB) return;
  const int64_t b = i / K::NVB;
  const int v = (int)(i - b * K::NVB);
  const int lx = v % K::V1, ly = (v / K::V1) % K::V1, lz = D == 3 ? v / (K::V1 * K::V1) : 0;
  const int64_t L0 = b * K::LB;
  int32_t gx = t.leaf_coords[L0 * D + 0] + lx, gy = t.leaf_coords[L0 * D + 1] + ly;
  int32_t gz = D == 3 ? t.leaf_coords[L0 * D + 2] + lz : 0;
  if (gx >= t.M) gx -= t.M;
  if (gy >= t.M) gy -= t.M;
  if (gz >= t.M) gz -= t.M;
  const int64_t vid = gx + (int64_t)t.M * (gy + (int64_t)t.M * gz);
  if constexpr (D == 3)
    out[i] = make_float4(E[vid], E[t.n_vert + vid], E[2 * t.n_vert + vid], 0.0f);
  else
    out[i] = make_float2(E[vid], E[t.n_vert + vid]);
}

void launch_brick_field(const DevTree &t, const BrickGeom &g, const float *E, float *Ebrick, cudaStream_t s) {
  const int64_t m = g.n_bricks * (g.d == 3 ? BK<3>::NVB : BK<2>::NVB);
  const unsigned grid = (unsigned)((m + 255) / 256);
  if (g.d == 3)
    k_brick_field<3><<<grid, 256, 0, s>>>(t, g, E, (float4 *)Ebrick);
  else
    k_brick_field<2><<<grid, 256, 0, s>>>(t, g, E, (float2 *)Ebrick);
  count_launches(1);
}

void launch_expand_leaves(const int32_t *start, int64_t n_leaves, int32_t *leaf, cudaStream_t s) {
  k_expand_leaves<<<(unsigned)((n_leaves + 255) / 256), 256, 0, s>>>(start, n_leaves, leaf);
  count_launches(1);
}

int32_t brick_stage_cap(int64_t n, int64_t n_units) {
  // four times the mean arrivals per unit and some slack, a multiple of 8
  // (every unit's area then starts on a 16-byte boundary in each row), at most
  // what the shared-memory kernel holds; fuller units take the overflow list
  const int64_t want = 4 * (n / (n_units > 0 ? n_units : 1)) + 256;
  return (int32_t)std::min<int64_t>(kStCap, (want + 7) & ~(int64_t)7);
}

cudaError_t brick_configure(const BrickGeom &g) {
  cudaError_t e = cudaSuccess;
  if (g.d == 3) {
    for (auto fn : {k_brick_push_st<3, true>, k_brick_push_st<3, false>}) {
      if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)push_st_smem<3>());
      if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_brick_pull_st<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pull_st_smem<3>());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_brick_pull_st<3>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  } else {
    for (auto fn : {k_brick_push_st<2, true>, k_brick_push_st<2, false>}) {
      if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)push_st_smem<2>());
      if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_brick_pull_st<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pull_st_smem<2>());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_brick_pull_st<2>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  }
  return e;
}

}  // namespace pic
