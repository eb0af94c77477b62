// Brick path of the PIT split-precision step on uniform trees (sm_103a).
//
// A brick is the subtree of one cell kb levels above the leaves: B = 3^kb
// leaves per axis, LB = B^d leaves, contiguous in depth-first leaf order and so
// contiguous in the bucket-sorted particle arrays.  One step re-bins every
// particle (PIT, Algorithm 1 end state) in two passes over the particles:
//
//   K1 k_brick_push   one CTA per source brick: stage the brick's vertex
//                     field in shared memory, gather + kick + drift every
//                     particle, re-locate it (integer arithmetic, split rule),
//                     and stably partition it by destination brick direction
//                     (27 neighbours + "far") into a temporary array.
//   K2 k_brick_pull   one CTA per destination brick: pull the 27 incoming
//                     segments (+ far arrivals) in canonical order -- stayers
//                     first in storage order, then movers in storage order --
//                     rank them per leaf with per-warp histograms, write the
//                     new bucket order and the leaf offsets.
//
// The result is bit-identical to the generic path (same arithmetic, same
// canonical bucket order), with each particle read twice and written twice
// and no global atomics on the hot path.
#include <cuda_runtime.h>

#include "dev.cuh"
#include "launch.hpp"

namespace pic {

void count_launches(int64_t k);

constexpr int kSlots = 28;           // 27 neighbour directions + far
constexpr int kFarSlot = 27;
constexpr int kSelfDir = 13;         // (0, 0, 0)
constexpr uint16_t kStayBit = 0x8000;
constexpr int kPushThreads = 512;
constexpr int kPullThreads = 256;
constexpr int kPullWarps = kPullThreads / 32;
constexpr int kMaxPieces = 128;      // round-1 pieces + 2 x 27 segments + 55 runs of far arrivals
constexpr int kLidxCap = 8192;       // particles per brick with a shared-memory leaf index
constexpr int kStageCap = 6144;      // particles per brick staged in shared memory

// Compile-time brick shape: B = 9 leaves per axis (two levels).
template <int D>
struct BK {
  static constexpr int B = 9, V1 = 10;
  static constexpr int LB = D == 3 ? 729 : 81;
  static constexpr int NVB = D == 3 ? 1000 : 100;
  static constexpr int NC = 1 << D;
};

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
constexpr long long kWaitCycles = 4000000000LL;  // about two seconds at the maximum SM clock
constexpr int kErrTimeout = 8;                   // error bit: a bounded device wait gave up

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
// K1, shared-memory form: the brick's particles are loaded once, pushed once
// and kept on chip until their partitioned positions are known.
// ---------------------------------------------------------------------------

constexpr int kStThreads = 1024;
constexpr int kLoadBatch = 4;        // particles whose loads one thread keeps in flight
constexpr int kStCap = 7168;         // particles per brick held in shared memory
constexpr int kStS = kStCap + 8;     // shared row stride of the K1 stash (room for a 16-byte aligned head)

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

// K1 runs two CTAs per SM: each takes one half of a brick's particles
// (storage order) and partitions that half by direction on its own, so a
// brick's segment towards one neighbour is two runs, half 0 then half 1.
constexpr int kHThreads = 512;
constexpr int kHalfCap = 3040;       // particles of one half held in shared memory
constexpr int kHS = kHalfCap + 8;    // shared row stride (room for a 16-byte aligned head)
constexpr int kHChunks = (kHalfCap + kHThreads - 1) / kHThreads;
constexpr int kH32 = (kHalfCap + 31) / 32;  // 32-particle chunks of one half

// First storage offset (within the brick) of half h of a brick holding nb
// particles: halves of the shared-memory kernel, or everything in half 0 for
// bricks that the global-memory kernel takes.
__host__ __device__ __forceinline__ int32_t half_start(int32_t nb, int h) {
  if (h == 0) return 0;
  return nb <= 2 * kHalfCap ? (nb + 1) / 2 : nb;
}

template <int D>
size_t push_st_smem() {
  using K = BK<D>;
  return sizeof(float) * 2 * D * kHS + sizeof(uint16_t) * 2 * kHalfCap + sizeof(typename EVec<D>::T) * K::NVB +
         sizeof(int32_t) * (K::LB + 1) + sizeof(uint32_t) * K::LB + sizeof(uint16_t) * kH32 * kSlots +
         sizeof(int32_t) * 2 * kSlots + sizeof(int32_t) * 3 * 32;
}

// K1, shared-memory form, one CTA per half brick.  Same arithmetic as
// push_core (gather in corner order, kick, drift, split re-location), with
// the brick's field staged as one vector per vertex and the destination found
// from the brick-local cell through a per-axis table.
template <int D, bool kAligned>
__global__ void __launch_bounds__(kHThreads, 2) k_brick_push_st(DevTree t, BrickGeom g, BrickPushArgs a) {
  using K = BK<D>;
  using EV = typename EVec<D>::T;
  constexpr int kW = kHThreads / 32;
  extern __shared__ __align__(128) float smf[];
  float *so = smf;                                   // D rows of kHS offsets
  float *sv = so + D * kHS;                          // D rows of kHS velocities
  uint16_t *code = (uint16_t *)(sv + D * kHS);       // new local leaf | dir << 10 | stay << 15
  uint16_t *pos = code + kHalfCap;                   // local leaf, rank in (chunk, dir), then inverse map
  EV *Eb = (EV *)(pos + kHalfCap);                   // NVB staged field vectors
  int32_t *ls = (int32_t *)(Eb + K::NVB);            // LB + 1 absolute leaf offsets
  uint32_t *dec = (uint32_t *)(ls + K::LB + 1);      // LB
  uint16_t *cw = (uint16_t *)(dec + K::LB);          // kH32 x kSlots: per 32-particle chunk and
                                                     // direction counts, then exclusive offsets
  int32_t *seg = (int32_t *)(cw + kH32 * kSlots);    // kSlots
  int32_t *dtot = seg + kSlots;                      // kSlots
  int32_t *rel = dtot + kSlots;                      // 3 x 32: per-axis direction | leaf-index parts
  __shared__ int32_t s_movers;
  __shared__ uint64_t s_bar;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int32_t b = blockIdx.x >> 1, h = blockIdx.x & 1, L0 = b * K::LB;
  const int32_t ps = a.start[L0], pe = a.start[L0 + K::LB], nbr = pe - ps;
  if (nbr > 2 * kHalfCap) return;  // the global-memory kernel takes this brick
  const int32_t q0 = half_start(nbr, h), q1 = h ? nbr : half_start(nbr, 1), nb = q1 - q0;
  const int32_t hs = ps + q0;  // storage index of this half's first particle
  const int64_t n = a.n;
  int32_t origin[3] = {0, 0, 0}, bc[3] = {0, 0, 0};
#pragma unroll
  for (int ax = 0; ax < D; ++ax) {
    origin[ax] = t.leaf_coords[(int64_t)L0 * D + ax];
    bc[ax] = origin[ax] / K::B;
  }
  // every global -> shared copy is issued before any is awaited
  for (int i = tid; i <= K::LB; i += blockDim.x) cp_async4(ls + i, a.start + L0 + i);
  for (int i = tid; i < K::LB; i += blockDim.x) cp_async4(dec + i, g.decodeL + i);
  for (int i = tid; i < K::NVB; i += blockDim.x) {
    int lx = i % K::V1, ly = (i / K::V1) % K::V1, lz = D == 3 ? i / (K::V1 * K::V1) : 0;
    int32_t gx = origin[0] + lx, gy = origin[1] + ly, gz = D == 3 ? origin[2] + lz : 0;
    if (gx >= t.M) gx -= t.M;
    if (gy >= t.M) gy -= t.M;
    if (gz >= t.M) gz -= t.M;
    const int64_t vid = gx + (int64_t)t.M * (gy + (int64_t)t.M * gz);
    float *slot = (float *)(Eb + i);
#pragma unroll
    for (int ax = 0; ax < D; ++ax) cp_async4(slot + ax, a.E + ax * t.n_vert + vid);
  }
  if (tid < 3 * 27) {  // local cell l - 9 on axis tid / 27: (direction digit + 1) 3^axis << 16 | leaf part
    const int ax = tid / 27, loc = tid % 27 - K::B;
    const int dl = (loc >= K::B) - (loc < 0);
    const int p3 = ax == 0 ? 1 : (ax == 1 ? 3 : 9);
    rel[ax * 32 + tid % 27] = ((dl + 1) * p3 << 16) | lidx_axis<D>(loc - K::B * dl, ax);
  }
  for (int i = tid; i < kH32 * kSlots / 2; i += blockDim.x) reinterpret_cast<uint32_t *>(cw)[i] = 0u;
  // the half's particle rows: one bulk copy per row from the 16-byte boundary
  // at or below its first particle; row r holds particle q at index off[r] + q
  int32_t offO[D], offV[D];
#pragma unroll
  for (int r = 0; r < 2 * D; ++r) {
    const float *src = (r < D ? a.o + r * n : a.v + (r - D) * n) + hs;
    const int32_t head = (int32_t)(((uintptr_t)src & 15u) >> 2);
    if (r < D) offO[r] = r * kHS + head;
    else offV[r - D] = (r - D) * kHS + head;
  }
  // with n a multiple of 4 every row has the same head, so row ax of particle
  // q sits a compile-time distance from row 0
  const int32_t h0 = offO[0];
  auto O = [&](int ax, int32_t q) -> float & { return kAligned ? so[ax * kHS + h0 + q] : so[offO[ax] + q]; };
  auto V = [&](int ax, int32_t q) -> float & { return kAligned ? sv[ax * kHS + h0 + q] : sv[offV[ax] + q]; };
  if (tid == 0) {
    s_movers = 0;
    if (nb > 0) {
      mbar_init(&s_bar, 1);
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
      mbar_expect_tx(&s_bar, total);
#pragma unroll
      for (int r = 0; r < 2 * D; ++r)
        bulk_g2s(r < D ? so + r * kHS : sv + (r - D) * kHS, src[r], bytes[r], &s_bar);
    }
  }
  cp_async_wait_all();
  __syncthreads();  // the barrier is initialised and armed before anyone waits on it
  const bool landed = nb == 0 || mbar_wait(&s_bar, 0, kWaitCycles);
  if (__syncthreads_or(!landed)) {
    if (!landed) mbar_wait(&s_bar, 0, kWaitCycles);  // let copies in flight land before leaving
    if (tid == 0) atomicOr(a.err, kErrTimeout);
    return;
  }
  for (int l = tid; l < K::LB; l += blockDim.x) {
    const int32_t lo = max(ls[l] - hs, 0), hi = min(ls[l + 1] - hs, nb);
    for (int32_t q = lo; q < hi; ++q) pos[q] = (uint16_t)l;
  }
  __syncthreads();

  // push every particle once, warp by warp over chunks of 32 consecutive
  // particles: rank within (chunk, direction) by a warp match, chunk counts
  // into cw[]; no block barrier until every particle is pushed
  bool bad = false;
  const int nc32 = (nb + 31) >> 5;
  for (int c = w; c < nc32; c += kW) {
    const int32_t q = c * 32 + lane;
    const bool act = q < nb;
    int dir = 255;
    if (act) {
      const int l = pos[q];
      const uint32_t pk = dec[l];
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
        const EV ev = Eb[base + (e & 1) + ((e >> 1) & 1) * K::V1 + ((e >> 2) & 1) * K::V1 * K::V1];
#pragma unroll
        for (int ax = 0; ax < D; ++ax) E[ax] = E[ax] + wgt[e] * ecomp(ev, ax);
      }
      // kick and drift: v += (q/m) dt E, t = o + v s_l
      float vv[D], tt[D];
#pragma unroll
      for (int ax = 0; ax < D; ++ax) {
        vv[ax] = V(ax, q) + a.qmdt * E[ax];
        tt[ax] = o[ax] + vv[ax] * a.sl;
      }
      float fl[D];
      int32_t packed = D == 2 ? (9 << 16) : 0;
      bool win = true;
#pragma unroll
      for (int ax = 0; ax < D; ++ax) {
        if (!isfinite(vv[ax]) || !isfinite(tt[ax])) {
          bad = true;
          tt[ax] = 0.0f;
        }
        fl[ax] = floorf(tt[ax]);
        O(ax, q) = clamp_off(tt[ax] - fl[ax]);
        V(ax, q) = vv[ax];
        const uint32_t li = (uint32_t)(lc[ax] + K::B + (int32_t)fmaxf(fminf(fl[ax], 64.0f), -64.0f));
        win &= li < 3u * K::B;
        packed += rel[ax * 32 + (li < 3u * K::B ? li : 0u)];
      }
      int lidx;
      if (win) {
        dir = packed >> 16;
        lidx = packed & 0xffff;
      } else {
        SlowIn in{};
#pragma unroll
        for (int ax = 0; ax < D; ++ax) {
          in.lc[ax] = lc[ax];
          in.origin[ax] = origin[ax];
          in.bc[ax] = bc[ax];
          in.fl[ax] = fl[ax];
        }
        const SlowOut r = relocate_slow<D>(t, g, in);
        dir = r.dir;
        lidx = r.lidx;
        if (dir == kFarSlot) a.far_scratch[hs + q] = r.dest;
      }
      const bool stay = dir == kSelfDir && lidx == l;
      code[q] = (uint16_t)(lidx | (dir << 10) | (stay ? kStayBit : 0));
    }
    const unsigned peers = __match_any_sync(0xffffffffu, dir);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (act) {
      pos[q] = (uint16_t)rank;
      if (rank == 0) cw[c * kSlots + dir] = (uint16_t)__popc(peers);
    }
  }
  __syncthreads();
  // exclusive offsets of every (chunk, direction) over the chunks; direction totals
  for (int d = w; d < kSlots; d += kW) {
    int32_t carry = 0;
    for (int c0 = 0; c0 < nc32; c0 += 32) {
      const int c = c0 + lane;
      const int32_t v = c < nc32 ? cw[c * kSlots + d] : 0;
      int32_t x = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (c < nc32) cw[c * kSlots + d] = (uint16_t)(carry + x - v);
      carry += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) dtot[d] = carry;
  }
  __syncthreads();
  if (tid == 0) {
    int32_t sum = 0;
    const int64_t row = ((int64_t)b * 2 + h) * kSlots;
    for (int k = 0; k < kSlots; ++k) {
      seg[k] = sum;
      a.cnt[row + k] = dtot[k];
      a.segoff[row + k] = sum;
      sum += dtot[k];
    }
  }
  __syncthreads();
  // final position of every particle (registers), then the inverse map in
  // pos[] so that the writes walk the destination order (coalesced)
  int32_t fin[kHChunks];
  int movers = 0;
#pragma unroll
  for (int u = 0; u < kHChunks; ++u) {
    const int32_t q = u * kHThreads + tid;
    fin[u] = -1;
    if (q < nb) {
      const uint16_t cd = code[q];
      const int dir = (cd >> 10) & 31;
      fin[u] = seg[dir] + cw[(q >> 5) * kSlots + dir] + pos[q];
      movers += !(cd & kStayBit);
      if (dir == kFarSlot) {
        int32_t k = atomicAdd(a.far_n, 1);
        if (k < a.far_cap) {
          a.far_tidx[k] = hs + fin[u];
          a.far_src[k] = b;
          a.far_dest[k] = a.far_scratch[hs + q];
        } else {
          atomicOr(a.err, 4);
        }
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < kHChunks; ++u)
    if (fin[u] >= 0) pos[fin[u]] = (uint16_t)(u * kHThreads + tid);
  __syncthreads();
  {
    float *tO[D], *tV[D];
#pragma unroll
    for (int ax = 0; ax < D; ++ax) {
      tO[ax] = a.to + ax * n + hs;
      tV[ax] = a.tv + ax * n + hs;
    }
    uint16_t *tC = a.tcode + hs;
    auto put = [&](int32_t p) {
      const int32_t q = pos[p];
#pragma unroll
      for (int ax = 0; ax < D; ++ax) {
        tO[ax][p] = O(ax, q);
        tV[ax][p] = V(ax, q);
      }
      tC[p] = (uint16_t)(code[q] & (kStayBit | 0x3ffu));
      if (a.ids) a.tids[hs + p] = a.ids[hs + q];
    };
    if (kAligned && !a.ids) {
      // 16-byte stores: positions p with hs + p a multiple of 4 start a group
      const int32_t p0 = min((int32_t)((4 - (hs & 3)) & 3), nb);
      const int32_t ng = (nb - p0) >> 2;
      if (tid < p0) put(tid);
      for (int32_t gi = tid; gi < ng; gi += blockDim.x) {
        const int32_t p = p0 + 4 * gi;
        int32_t qq[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) qq[k] = pos[p + k];
#pragma unroll
        for (int ax = 0; ax < D; ++ax) {
          *reinterpret_cast<float4 *>(tO[ax] + p) = make_float4(O(ax, qq[0]), O(ax, qq[1]), O(ax, qq[2]), O(ax, qq[3]));
          *reinterpret_cast<float4 *>(tV[ax] + p) = make_float4(V(ax, qq[0]), V(ax, qq[1]), V(ax, qq[2]), V(ax, qq[3]));
        }
        const uint32_t c01 = (uint32_t)(code[qq[0]] & (kStayBit | 0x3ffu)) |
                             ((uint32_t)(code[qq[1]] & (kStayBit | 0x3ffu)) << 16);
        const uint32_t c23 = (uint32_t)(code[qq[2]] & (kStayBit | 0x3ffu)) |
                             ((uint32_t)(code[qq[3]] & (kStayBit | 0x3ffu)) << 16);
        *reinterpret_cast<uint2 *>(tC + p) = make_uint2(c01, c23);
      }
      for (int32_t p = p0 + 4 * ng + tid; p < nb; p += blockDim.x) put(p);
    } else {
      for (int32_t p = tid; p < nb; p += blockDim.x) put(p);
    }
  }
  if (bad) atomicOr(a.err, 1);
  for (int o = 16; o > 0; o >>= 1) movers += __shfl_down_sync(0xffffffffu, movers, o);
  if (lane == 0) atomicAdd(&s_movers, movers);
  __syncthreads();
  if (tid == 0 && s_movers) atomicAdd(a.n_movers, s_movers);
}

template <int D>
__global__ void __launch_bounds__(kPushThreads) k_brick_push(DevTree t, BrickGeom g, BrickPushArgs a) {
  using K = BK<D>;
  __shared__ int32_t ls[K::LB + 1];
  __shared__ uint32_t dec[K::LB];
  __shared__ float Eb[D * K::NVB];
  __shared__ uint16_t lidx[kLidxCap];
  __shared__ int32_t counters[kSlots], seg[kSlots], run[kSlots];
  __shared__ int32_t wcnt[(kPushThreads / 32) * kSlots];
  __shared__ int32_t s_movers;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  const int32_t b = blockIdx.x, L0 = b * K::LB;
  int32_t origin[3] = {0, 0, 0}, bc[3] = {0, 0, 0};
#pragma unroll
  for (int ax = 0; ax < D; ++ax) {
    origin[ax] = t.leaf_coords[(int64_t)L0 * D + ax];
    bc[ax] = origin[ax] / K::B;
  }
  const int32_t ps = a.start[L0], pe = a.start[L0 + K::LB], nb = pe - ps;
  if (nb <= 2 * kHalfCap) return;  // the shared-memory kernel took this brick (in halves)
  for (int i = tid; i <= K::LB; i += blockDim.x) ls[i] = a.start[L0 + i] - ps;
  for (int i = tid; i < K::LB; i += blockDim.x) dec[i] = g.decodeL[i];
  for (int i = tid; i < K::NVB; i += blockDim.x) {
    int lx = i % K::V1, ly = (i / K::V1) % K::V1, lz = D == 3 ? i / (K::V1 * K::V1) : 0;
    int32_t gx = origin[0] + lx, gy = origin[1] + ly, gz = D == 3 ? origin[2] + lz : 0;
    if (gx >= t.M) gx -= t.M;
    if (gy >= t.M) gy -= t.M;
    if (gz >= t.M) gz -= t.M;
    int64_t vid = gx + (int64_t)t.M * (gy + (int64_t)t.M * gz);
#pragma unroll
    for (int ax = 0; ax < D; ++ax) Eb[ax * K::NVB + i] = a.E[ax * t.n_vert + vid];
  }
  if (tid < kSlots) { counters[tid] = 0; run[tid] = 0; }
  if (tid == 0) s_movers = 0;
  __syncthreads();
  // particle -> local leaf index
  for (int l = tid; l < K::LB; l += blockDim.x)
    for (int32_t q = ls[l]; q < ls[l + 1] && q < kLidxCap; ++q) lidx[q] = (uint16_t)l;
  __syncthreads();
  auto local_leaf = [&](int32_t q) -> int {
    if (q < kLidxCap) return lidx[q];
    int lo = 0, hi = K::LB;
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (ls[mid] <= q) lo = mid; else hi = mid;
    }
    return lo;
  };

  // pass A: destination counts (warp-aggregated)
  bool bad = false;
  for (int32_t base = 0; base < nb; base += blockDim.x) {
    const int32_t q = base + tid;
    int dir = 255;
    if (q < nb) {
      const int l = local_leaf(q);
      const uint32_t pk = dec[l];
      const int32_t lc[3] = {(int32_t)(pk & 1023u), (int32_t)((pk >> 10) & 1023u), (int32_t)(pk >> 20)};
      float on[D], vn[D];
      int32_t L2;
      dir = brick_push_one<D>(t, g, a, ps + q, lc, origin, bc, Eb, on, vn, L2, bad);
    }
    unsigned peers = __match_any_sync(0xffffffffu, dir);
    if (dir != 255 && lane == __ffs(peers) - 1) atomicAdd(&counters[dir], __popc(peers));
  }
  __syncthreads();
  if (tid == 0) {  // the whole brick is half 0; half 1 is empty
    int s = 0;
    for (int k = 0; k < kSlots; ++k) {
      seg[k] = s;
      a.cnt[(int64_t)b * 2 * kSlots + k] = counters[k];
      a.segoff[(int64_t)b * 2 * kSlots + k] = s;
      a.cnt[((int64_t)b * 2 + 1) * kSlots + k] = 0;
      a.segoff[((int64_t)b * 2 + 1) * kSlots + k] = s;
      s += counters[k];
    }
  }
  __syncthreads();

  // pass B: stable partition by direction
  int movers = 0;
  const int64_t n = a.n;
  for (int32_t base = 0; base < nb; base += blockDim.x) {
    const int32_t q = base + tid;
    const bool act = q < nb;
    if (lane < kSlots) wcnt[w * kSlots + lane] = 0;
    __syncwarp();
    int dir = 255, l = 0;
    float on[D], vn[D];
    int32_t L2 = 0;
    if (act) {
      l = local_leaf(q);
      const uint32_t pk = dec[l];
      const int32_t lc[3] = {(int32_t)(pk & 1023u), (int32_t)((pk >> 10) & 1023u), (int32_t)(pk >> 20)};
      dir = brick_push_one<D>(t, g, a, ps + q, lc, origin, bc, Eb, on, vn, L2, bad);
    }
    unsigned peers = __match_any_sync(0xffffffffu, dir);
    int rank = __popc(peers & ((1u << lane) - 1u));
    if (act && rank == 0) wcnt[w * kSlots + dir] = __popc(peers);
    __syncthreads();
    if (tid < kSlots) {
      int s = run[tid];
      for (int k = 0; k < nw; ++k) {
        int c = wcnt[k * kSlots + tid];
        wcnt[k * kSlots + tid] = s;
        s += c;
      }
      run[tid] = s;
    }
    __syncthreads();
    if (act) {
      const int32_t pos = ps + seg[dir] + wcnt[w * kSlots + dir] + rank;
#pragma unroll
      for (int ax = 0; ax < D; ++ax) {
        a.to[ax * n + pos] = on[ax];
        a.tv[ax * n + pos] = vn[ax];
      }
      const bool stay = L2 == L0 + l;
      movers += !stay;
      a.tcode[pos] = (uint16_t)(L2 % K::LB) | (stay ? kStayBit : 0);
      if (a.ids) a.tids[pos] = a.ids[ps + q];
      if (dir == kFarSlot) {
        int32_t k = atomicAdd(a.far_n, 1);
        if (k < a.far_cap) {
          a.far_tidx[k] = pos;
          a.far_src[k] = b;
          a.far_dest[k] = L2 / K::LB;
        } else {
          atomicOr(a.err, 4);
        }
      }
    }
    __syncthreads();
  }
  if (bad) atomicOr(a.err, 1);
  for (int o = 16; o > 0; o >>= 1) movers += __shfl_down_sync(0xffffffffu, movers, o);
  if (lane == 0) atomicAdd(&s_movers, movers);
  __syncthreads();
  if (tid == 0 && s_movers) atomicAdd(a.n_movers, s_movers);
}

// ---------------------------------------------------------------------------
// far arrivals: sorted per destination brick by temporary index
// ---------------------------------------------------------------------------

__global__ void k_far_count(const int32_t *far_n, int32_t far_cap, const int32_t *far_dest, int32_t *fcount) {
  int32_t nf = min(*far_n, far_cap);
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x)
    atomicAdd(&fcount[far_dest[i]], 1);
}

__global__ void k_far_scatter(const int32_t *far_n, int32_t far_cap, const int32_t *far_dest,
                              const int32_t *far_tidx, const int32_t *far_src, const int32_t *fstart,
                              int32_t *fcursor, int32_t *sorted_tidx, int32_t *sorted_src) {
  int32_t nf = min(*far_n, far_cap);
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x) {
    int32_t db = far_dest[i];
    int32_t k = fstart[db] + atomicAdd(&fcursor[db], 1);
    sorted_tidx[k] = far_tidx[i];
    sorted_src[k] = far_src[i];
  }
}

// Per destination brick: far arrivals sorted by temporary index (storage
// order), and the brick's total incoming count.
template <int D>
__global__ void k_brick_totals(DevTree t, BrickGeom g, const int32_t *cnt, const int32_t *segoff,
                               const int32_t *old_start, const int32_t *fstart, int32_t *sorted_tidx,
                               int32_t *sorted_src, int32_t *tot, int4 *bpiece) {
  // one warp per destination brick, lane = direction of the source brick
  const int lane = threadIdx.x & 31;
  const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (b >= g.n_bricks) return;
  const int32_t fb = fstart[b], fe = fstart[b + 1];
  if (lane == 0)
    for (int32_t i = fb + 1; i < fe; ++i) {
      int32_t x = sorted_tidx[i], y = sorted_src[i], j = i - 1;
      while (j >= fb && sorted_tidx[j] > x) {
        sorted_tidx[j + 1] = sorted_tidx[j];
        sorted_src[j + 1] = sorted_src[j];
        --j;
      }
      sorted_tidx[j + 1] = x;
      sorted_src[j + 1] = y;
    }
  const int32_t L0 = (int32_t)b * BK<D>::LB;
  int32_t len = 0;
  if (lane < 27) {
    const int dir = lane;
    int4 pc0 = make_int4(0, 0, INT32_MAX, 0), pc1 = make_int4(0, 0, INT32_MAX, 1);
    if (!(D == 2 && dir_delta(dir, 2) != 0)) {
      int32_t sc[3] = {0, 0, 0};
      for (int ax = 0; ax < D; ++ax) {
        const int32_t x = t.leaf_coords[(int64_t)L0 * D + ax] / 9 - dir_delta(dir, ax);
        sc[ax] = x < 0 ? x + g.nbx : (x >= g.nbx ? x - g.nbx : x);
      }
      const int32_t src = brick_of_coords<D>(t, sc);
      const int32_t s0 = old_start[(int64_t)src * BK<D>::LB];
      const int32_t nbs = old_start[(int64_t)(src + 1) * BK<D>::LB] - s0;
      const int64_t k0 = (int64_t)src * 2 * kSlots + dir, k1 = k0 + kSlots;
      pc0 = make_int4(s0 + segoff[k0], cnt[k0], src, 0);
      pc1 = make_int4(s0 + half_start(nbs, 1) + segoff[k1], cnt[k1], src, 1);
      len = pc0.y + pc1.y;
    }
    bpiece[((int64_t)b * 27 + dir) * 2] = pc0;
    bpiece[((int64_t)b * 27 + dir) * 2 + 1] = pc1;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) len += __shfl_down_sync(0xffffffffu, len, o);
  if (lane == 0) tot[b] = len + (fe - fb);
}

// ---------------------------------------------------------------------------
// K2
// ---------------------------------------------------------------------------

struct Piece {
  int32_t tstart, len, src;
  int16_t round1;    // 1: keep stayers only; 0: keep movers only
  int16_t indirect;  // 1: positions tstart.. index the sorted far arrivals
};

// Round-2 piece holding stage index si: the largest k in [1, np) with
// spfx[k] <= si (empty pieces share their successor's prefix).
__device__ __forceinline__ int piece_of(const int32_t *spfx, int np, int32_t si) {
  int lo = 1, hi = np - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (spfx[mid] <= si) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int D>
__global__ void __launch_bounds__(kPullThreads) k_brick_pull(DevTree t, BrickGeom g, BrickPullArgs a) {
  using K = BK<D>;
  extern __shared__ float stage[];                      // kStageCap staged values
  uint16_t *map = (uint16_t *)(stage + kStageCap);      // slot -> raw position -> stage index
  __shared__ int32_t cnt[K::LB + 1];                    // counts, then offsets
  __shared__ int32_t cur[K::LB];
  __shared__ Piece pieces[kMaxPieces];
  __shared__ Piece sdesc[54];
  __shared__ int32_t pfx[kMaxPieces + 1];
  __shared__ int32_t spfx[kMaxPieces + 1];              // stage offset of round-2 pieces
  __shared__ int32_t wsum[kPullThreads / 32];
  __shared__ int32_t s_np, s_self, s_max;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  const int32_t b = blockIdx.x, L0 = b * K::LB;
  const int64_t n = a.n;
  if (a.tot[b] <= kStCap) return;  // the shared-memory kernel took this brick

  // neighbour segments (two halves each), one thread per direction, placed by
  // source-brick rank; round 1 = the stayers of this brick's own two halves
  __shared__ int32_t s_src[27];
  Piece m0{0, 0, INT32_MAX, 0, 0}, m1{0, 0, INT32_MAX, 0, 0};
  if (tid < 27) {
    const int4 p0 = a.bpiece[((int64_t)b * 27 + tid) * 2], p1 = a.bpiece[((int64_t)b * 27 + tid) * 2 + 1];
    m0 = Piece{p0.x, p0.y, p0.z, 0, 0};
    m1 = Piece{p1.x, p1.y, p1.z, 0, 0};
    s_src[tid] = m0.src;
  }
  for (int i = tid; i < K::LB + 1; i += blockDim.x) cnt[i] = 0;
  __syncthreads();
  if (tid < 27 && m0.src != INT32_MAX) {
    int rank = 0;
    for (int k = 0; k < 27; ++k) rank += s_src[k] < m0.src;
    sdesc[2 * rank] = m0;
    sdesc[2 * rank + 1] = m1;
    if (tid == kSelfDir) {
      pieces[0] = Piece{m0.tstart, m0.len, m0.src, 1, 0};
      pieces[1] = Piece{m1.tstart, m1.len, m1.src, 1, 0};
    }
  }
  __syncthreads();
  if (tid == 0) {
    const int ns = 2 * (D == 3 ? 27 : 9);
    // far arrivals (sorted by storage index, so by source brick) go between
    // the neighbour segments as runs of the sorted far list
    int np = 2;
    int32_t fi = a.fstart[b];
    const int32_t fe = a.fstart[b + 1];
    for (int k = 0; k < ns; ++k) {
      if (fi < fe) {
        int32_t f0 = fi;
        while (fi < fe && a.far_src[fi] < sdesc[k].src) ++fi;
        if (fi > f0) pieces[np++] = Piece{f0, fi - f0, -1, 0, 1};
      }
      if (sdesc[k].src == b && (k & 1) == 0) s_self = np;
      pieces[np++] = sdesc[k];
    }
    if (fi < fe) pieces[np++] = Piece{fi, fe - fi, -1, 0, 1};
    int32_t s = 0;
    for (int k = 0; k < np; ++k) {
      pfx[k] = s;
      spfx[k] = k < 2 ? 0 : s - pieces[0].len - pieces[1].len;
      s += pieces[k].len;
    }
    pfx[np] = s;
    s_np = np;
    s_max = 0;
  }
  __syncthreads();
  const int np = s_np;
  const int32_t self_stage = spfx[s_self];

  // every raw position of every piece: fn(raw position, temporary index, keep, leaf)
  auto each = [&](auto fn) {
    for (int k = 0; k < np; ++k) {
      const Piece pc = pieces[k];
      const int32_t r0 = pfx[k];
      for (int32_t i = tid; i < pc.len; i += blockDim.x) {
        const int32_t tidx = pc.indirect ? a.far_tidx[pc.tstart + i] : pc.tstart + i;
        const uint16_t code = a.tcode[tidx];
        const bool stay = (code & kStayBit) != 0;
        if (pc.round1 ? stay : !stay) fn(r0 + i, code & 0x7fff);
      }
    }
  };
  // counts per leaf
  each([&](int32_t, int leaf) { atomicAdd(&cnt[leaf], 1); });
  __syncthreads();
  // exclusive scan of the counts (in place), cursors
  int32_t carry = 0;
  for (int base = 0; base < K::LB; base += blockDim.x) {
    const int l = base + tid;
    const int32_t c = l < K::LB ? cnt[l] : 0;
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
    if (l < K::LB) {
      cnt[l] = carry + before + x - c;
      cur[l] = cnt[l];
      if (c > 0) atomicMax(&s_max, c);
    }
    carry += all;
    __syncthreads();
  }
  if (tid == 0) cnt[K::LB] = carry;
  __syncthreads();
  const int32_t bstart = a.bstart[b];
  const int32_t nin = cnt[K::LB];
  for (int l = tid; l < K::LB; l += blockDim.x) a.new_start[L0 + l] = bstart + cnt[l];
  if (b == g.n_bricks - 1 && tid == 0) a.new_start[(int64_t)g.n_bricks * K::LB] = bstart + nin;
  if (tid == 0 && s_max > 0) atomicMax(a.max_bucket, s_max);

  if (nin <= kStageCap) {
    // slots (any order), then every leaf's slots sorted by raw position: the
    // canonical order (stayers first, then movers in storage order)
    each([&](int32_t r, int leaf) { map[atomicAdd(&cur[leaf], 1)] = (uint16_t)r; });
    __syncthreads();
    for (int l = tid; l < K::LB; l += blockDim.x) {
      const int32_t lo = cnt[l], hi = cnt[l + 1];
      for (int32_t i = lo + 1; i < hi; ++i) {
        const uint16_t x = map[i];
        int32_t j = i - 1;
        while (j >= lo && map[j] > x) { map[j + 1] = map[j]; --j; }
        map[j + 1] = x;
      }
      for (int32_t i = lo; i < hi; ++i) {  // raw position -> stage index
        const int32_t r = map[i];
        map[i] = (uint16_t)(r < pfx[2] ? self_stage + r : r - pfx[2]);
      }
    }
    __syncthreads();
    // one array at a time: coalesced reads of the incoming pieces into shared
    // memory, coalesced writes in destination order
    const int na = 2 * D + (a.ids ? 1 : 0);
    for (int arr = 0; arr < na; ++arr) {
      const float *src = arr < D ? a.to + arr * n : (arr < 2 * D ? a.tv + (arr - D) * n : (const float *)a.tids);
      float *dst = arr < D ? a.o + arr * n : (arr < 2 * D ? a.v + (arr - D) * n : (float *)a.ids);
      for (int k = 2; k < np; ++k) {
        const Piece pc = pieces[k];
        const int32_t so = spfx[k];
        for (int32_t i = tid; i < pc.len; i += blockDim.x)
          stage[so + i] = src[pc.indirect ? a.far_tidx[pc.tstart + i] : pc.tstart + i];
      }
      __syncthreads();
      for (int32_t j = tid; j < nin; j += blockDim.x) dst[bstart + j] = stage[map[j]];
      __syncthreads();
    }
  } else {
    // large brick: one thread per leaf walks the raw positions in order
    for (int l = tid; l < K::LB; l += blockDim.x) {
      int32_t dl = cnt[l];
      for (int k = 0; k < np; ++k) {
        const Piece pc = pieces[k];
        for (int32_t i = 0; i < pc.len; ++i) {
          const int32_t tidx = pc.indirect ? a.far_tidx[pc.tstart + i] : pc.tstart + i;
          const uint16_t code = a.tcode[tidx];
          const bool stay = (code & kStayBit) != 0;
          if (!(pc.round1 ? stay : !stay) || (code & 0x7fff) != l) continue;
          const int32_t dst = bstart + dl++;
#pragma unroll
          for (int ax = 0; ax < D; ++ax) {
            a.o[ax * n + dst] = a.to[ax * n + tidx];
            a.v[ax * n + dst] = a.tv[ax * n + tidx];
          }
          if (a.ids) a.ids[dst] = a.tids[tidx];
        }
      }
    }
    __syncthreads();
  }
  // deposit partials of the new positions, per leaf in bucket order (the
  // arithmetic and order of the generic per-leaf deposit)
  if (a.part) {
    for (int l = tid; l < K::LB; l += blockDim.x) {
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

// ---------------------------------------------------------------------------
// K2, shared-memory form: every arrival is loaded once (coalesced), counted,
// ordered, written in destination order and deposited from shared memory.
// ---------------------------------------------------------------------------

template <int D>
size_t pull_st_smem() {
  return sizeof(float) * 2 * D * kStCap + sizeof(uint16_t) * 2 * kStCap;
}

// Canonical position order inside the brick's incoming pieces: round-1 (the
// stayers of the self segment) before round-2 (everything else in source
// order); stage index = position among round-2 pieces.
template <int D>
__device__ __forceinline__ void build_pieces(const DevTree &t, const BrickGeom &g, const BrickPullArgs &a,
                                             int32_t b, Piece *pieces, Piece *sdesc, int32_t *s_src,
                                             int32_t *pfx, int32_t *spfx, int32_t *s_np, int32_t *s_self) {
  (void)t;
  (void)g;
  (void)s_src;
  const int tid = threadIdx.x, lane = tid & 31;
  constexpr unsigned kAll = 0xffffffffu;
  if (tid < 32) {  // warp 0: lane = direction of the source brick, two halves each
    Piece m0{0, 0, INT32_MAX, 0, 0}, m1{0, 0, INT32_MAX, 0, 0};
    if (lane < 27) {
      const int4 p0 = a.bpiece[((int64_t)b * 27 + lane) * 2], p1 = a.bpiece[((int64_t)b * 27 + lane) * 2 + 1];
      m0 = Piece{p0.x, p0.y, p0.z, 0, 0};
      m1 = Piece{p1.x, p1.y, p1.z, 0, 0};
    }
    const int32_t fi0 = a.fstart[b], fe = a.fstart[b + 1];
    int rank = 0;  // sources in ascending brick order = storage order
    for (int k = 0; k < 27; ++k) rank += __shfl_sync(kAll, m0.src, k) < m0.src;
    const bool valid = lane < 27 && m0.src != INT32_MAX;
    const int ns = 2 * (D == 3 ? 27 : 9);
    const int32_t len0 = __shfl_sync(kAll, m0.len + m1.len, kSelfDir);  // stayers come from both halves
    if (lane == 0) pieces[0] = Piece{0, len0, b, 1, 0};
    if (fi0 == fe) {
      // no far arrivals: the neighbour segments in (source, half) order, in parallel
      if (valid) {
        pieces[1 + 2 * rank] = m0;
        pieces[2 + 2 * rank] = m1;
        if (m0.src == b) *s_self = 1 + 2 * rank;
      }
      __syncwarp();
      const int32_t x0 = 2 * lane < ns ? pieces[1 + 2 * lane].len : 0;
      const int32_t x1 = 2 * lane < ns ? pieces[2 + 2 * lane].len : 0;
      const int32_t x = x0 + x1;
      int32_t incl = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(kAll, incl, o);
        if (lane >= o) incl += y;
      }
      if (2 * lane < ns) {
        const int32_t ex = incl - x;
        pfx[1 + 2 * lane] = len0 + ex;
        spfx[1 + 2 * lane] = ex;
        pfx[2 + 2 * lane] = len0 + ex + x0;
        spfx[2 + 2 * lane] = ex + x0;
      }
      if (lane == 0) pfx[0] = spfx[0] = 0;
      if (2 * lane == ns - 2) {
        pfx[ns + 1] = len0 + incl;
        spfx[ns + 1] = incl;
        *s_np = ns + 1;
      }
    } else {
      if (valid) {
        sdesc[2 * rank] = m0;
        sdesc[2 * rank + 1] = m1;
      }
      __syncwarp();
      if (lane == 0) {
        // far arrivals (sorted by storage index, so by source brick) go
        // between the neighbour segments as runs of the sorted far list
        int np = 1;
        int32_t fi = fi0;
        for (int k = 0; k < ns; ++k) {
          if (fi < fe) {
            int32_t f0 = fi;
            while (fi < fe && a.far_src[fi] < sdesc[k].src) ++fi;
            if (fi > f0) pieces[np++] = Piece{f0, fi - f0, -1, 0, 1};
          }
          if (sdesc[k].src == b && (k & 1) == 0) *s_self = np;
          pieces[np++] = sdesc[k];
        }
        if (fi < fe) pieces[np++] = Piece{fi, fe - fi, -1, 0, 1};
        int32_t sum = 0;
        for (int k = 0; k < np; ++k) {
          pfx[k] = sum;
          spfx[k] = k == 0 ? 0 : sum - pieces[0].len;
          sum += pieces[k].len;
        }
        pfx[np] = sum;
        spfx[np] = sum - pieces[0].len;
        *s_np = np;
      }
    }
  }
  __syncthreads();
}

// Sorts the m <= N canonical keys of one leaf (ascending) with a bitonic
// network in registers and replaces each by its stage index.
template <int N>
__device__ __forceinline__ void sort_keys_net(uint16_t *keys, int m, int32_t len0, int32_t self_stage) {
  uint32_t r[N];
#pragma unroll
  for (int i = 0; i < N; ++i) r[i] = i < m ? keys[i] : 0xffffu;
  bitonic_sort<N>(r);
#pragma unroll
  for (int i = 0; i < N; ++i)
    if (i < m) keys[i] = (uint16_t)((int32_t)r[i] < len0 ? self_stage + (int32_t)r[i] : (int32_t)r[i] - len0);
}

// Leaves with 17..32 keys (rare): out of line, so that the 32-entry network
// does not raise the register demand of the calling kernel.
__device__ __noinline__ void sort_keys_net32(uint16_t *keys, int m, int32_t len0, int32_t self_stage) {
  sort_keys_net<32>(keys, m, len0, self_stage);
}

template <int D>
__global__ void __launch_bounds__(kStThreads, 1) k_brick_pull_st(DevTree t, BrickGeom g, BrickPullArgs a) {
  using K = BK<D>;
  extern __shared__ __align__(128) float smf[];
  float *so = smf;                                   // D * kStCap
  float *sv = so + D * kStCap;                       // D * kStCap
  uint16_t *code = (uint16_t *)(sv + D * kStCap);    // kStCap tcode of every arrival (stage order)
  uint16_t *map = code + kStCap;                     // kStCap slot -> key -> stage index
  __shared__ int32_t cnt[K::LB + 1];
  __shared__ int32_t cur[K::LB];
  __shared__ Piece pieces[kMaxPieces];
  __shared__ Piece sdesc[54];
  __shared__ int32_t s_src[27];
  __shared__ int32_t pfx[kMaxPieces + 1], spfx[kMaxPieces + 1];
  __shared__ int32_t wsum[32];
  __shared__ int32_t s_np, s_self, s_max;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  const int32_t b = blockIdx.x, L0 = b * K::LB;
  const int64_t n = a.n;
  if (a.tot[b] > kStCap) return;  // the global-memory kernel takes this brick
  if (tid == 0) s_max = 0;
  for (int i = tid; i < K::LB + 1; i += blockDim.x) cnt[i] = 0;
  build_pieces<D>(t, g, a, b, pieces, sdesc, s_src, pfx, spfx, &s_np, &s_self);
  const int np = s_np;
  const int32_t len0 = pieces[0].len, self_stage = spfx[s_self];
  const int32_t nin = spfx[np];
  // load every arrival once (round-2 pieces cover each exactly once): one
  // thread per arrival over all pieces; payload by asynchronous copies, the
  // codes through registers for the leaf counts
  {
    const float *gO[D], *gV[D];
#pragma unroll
    for (int ax = 0; ax < D; ++ax) {
      gO[ax] = a.to + ax * n;
      gV[ax] = a.tv + ax * n;
    }
    int kp = tid < nin ? piece_of(spfx, np, tid) : 1;  // arrivals only move forward
    for (int32_t base = 0; base < nin; base += kLoadBatch * kStThreads) {
      uint16_t rc[kLoadBatch];
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int32_t si = base + u * kStThreads + tid;
        if (si < nin) {
          while (kp + 1 < np && spfx[kp + 1] <= si) ++kp;
          const Piece pc = pieces[kp];
          const int32_t off = si - spfx[kp];
          const int32_t tx = pc.indirect ? a.far_tidx[pc.tstart + off] : pc.tstart + off;
#pragma unroll
          for (int ax = 0; ax < D; ++ax) {
            cp_async4(so + ax * kStCap + si, gO[ax] + tx);
            cp_async4(sv + ax * kStCap + si, gV[ax] + tx);
          }
          rc[u] = __ldg(a.tcode + tx);
        }
      }
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int32_t si = base + u * kStThreads + tid;
        if (si < nin) {
          code[si] = rc[u];
          atomicAdd(&cnt[rc[u] & 0x3ff], 1);
        }
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();
  // exclusive scan of the leaf counts, cursors
  int32_t carry = 0;
  for (int base = 0; base < K::LB; base += blockDim.x) {
    const int l = base + tid;
    const int32_t c = l < K::LB ? cnt[l] : 0;
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
    if (l < K::LB) {
      cnt[l] = carry + before + x - c;
      cur[l] = cnt[l];
      if (c > 0) atomicMax(&s_max, c);
    }
    carry += all;
    __syncthreads();
  }
  if (tid == 0) cnt[K::LB] = carry;
  __syncthreads();
  // slots in any order, keyed by canonical position
  for (int32_t si = tid; si < nin; si += blockDim.x) {
    const uint16_t cd = code[si];
    const bool stay = (cd & kStayBit) != 0;
    const int32_t key = stay ? si - self_stage : len0 + si;
    map[atomicAdd(&cur[cd & 0x3ff], 1)] = (uint16_t)key;
  }
  __syncthreads();
  const int32_t bstart = a.bstart[b];
  for (int l = tid; l < K::LB; l += blockDim.x) {
    a.new_start[L0 + l] = bstart + cnt[l];
    const int32_t lo = cnt[l], hi = cnt[l + 1];
    if (hi - lo <= 16) {
      sort_keys_net<16>(map + lo, hi - lo, len0, self_stage);
      continue;
    }
    if (hi - lo <= 32) {
      sort_keys_net32(map + lo, hi - lo, len0, self_stage);
      continue;
    }
    for (int32_t i = lo + 1; i < hi; ++i) {
      const uint16_t x = map[i];
      int32_t j = i - 1;
      while (j >= lo && map[j] > x) { map[j + 1] = map[j]; --j; }
      map[j + 1] = x;
    }
    for (int32_t i = lo; i < hi; ++i) {
      const int32_t key = map[i];
      map[i] = (uint16_t)(key < len0 ? self_stage + key : key - len0);
    }
  }
  if (b == g.n_bricks - 1 && tid == 0) a.new_start[(int64_t)g.n_bricks * K::LB] = bstart + nin;
  if (tid == 0 && s_max > 0) atomicMax(a.max_bucket, s_max);
  __syncthreads();
  // coalesced writes in destination order
  {
    float *gO[D], *gV[D];
#pragma unroll
    for (int ax = 0; ax < D; ++ax) {
      gO[ax] = a.o + ax * n + bstart;
      gV[ax] = a.v + ax * n + bstart;
    }
    for (int32_t j = tid; j < nin; j += blockDim.x) {
      const int32_t si = map[j];
#pragma unroll
      for (int ax = 0; ax < D; ++ax) {
        gO[ax][j] = so[ax * kStCap + si];
        gV[ax][j] = sv[ax * kStCap + si];
      }
    }
  }
  if (a.ids) {
    // ids: the source of stage index si is found in the round-2 pieces
    for (int32_t j = tid; j < nin; j += blockDim.x) {
      const int32_t si = map[j];
      const int k = piece_of(spfx, np, si);
      const Piece pc = pieces[k];
      const int32_t off = si - spfx[k];
      a.ids[bstart + j] = a.tids[pc.indirect ? a.far_tidx[pc.tstart + off] : pc.tstart + off];
    }
  }
  // deposit partials of the new positions, per leaf in bucket order; the
  // next particle's offsets are fetched while the current one is summed
  if (a.part) {
    for (int l = tid; l < K::LB; l += blockDim.x) {
      float acc[K::NC];
#pragma unroll
      for (int e = 0; e < K::NC; ++e) acc[e] = 0.0f;
      const int32_t lo = cnt[l], hi = cnt[l + 1];
      float on[D];
      if (lo < hi) {
        const int32_t si = map[lo];
#pragma unroll
        for (int ax = 0; ax < D; ++ax) on[ax] = so[ax * kStCap + si];
      }
      for (int32_t j = lo; j < hi; ++j) {
        float o[D], om[D];
#pragma unroll
        for (int ax = 0; ax < D; ++ax) {
          o[ax] = on[ax];
          om[ax] = 1.0f - o[ax];
        }
        if (j + 1 < hi) {
          const int32_t si = map[j + 1];
#pragma unroll
          for (int ax = 0; ax < D; ++ax) on[ax] = so[ax * kStCap + si];
        }
#pragma unroll
        for (int e = 0; e < K::NC; ++e) {
          float wgt = 1.0f;
#pragma unroll
          for (int ax = 0; ax < D; ++ax) wgt = wgt * (((e >> ax) & 1) ? o[ax] : om[ax]);
          acc[e] = acc[e] + wgt;
        }
      }
      float *gp = a.part + (int64_t)(L0 + l) * K::NC;
#pragma unroll
      for (int e = 0; e < K::NC; ++e) gp[e] = acc[e];
    }
  }
}

// Leaf id of every particle from the bucket offsets (thread per leaf).
__global__ void k_expand_leaves(const int32_t *start, int64_t n_leaves, int32_t *leaf) {
  int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n_leaves) return;
  for (int32_t p = start[l]; p < start[l + 1]; ++p) leaf[p] = (int32_t)l;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

void launch_brick_push(const DevTree &t, const BrickGeom &g, const BrickPushArgs &pa, cudaStream_t s) {
  cudaMemsetAsync(pa.far_n, 0, sizeof(int32_t), s);
  const unsigned nb = (unsigned)g.n_bricks;
  if (g.d == 3) {
    if (pa.n % 4 == 0)
      k_brick_push_st<3, true><<<2 * nb, kHThreads, push_st_smem<3>(), s>>>(t, g, pa);
    else
      k_brick_push_st<3, false><<<2 * nb, kHThreads, push_st_smem<3>(), s>>>(t, g, pa);
    k_brick_push<3><<<nb, kPushThreads, 0, s>>>(t, g, pa);
  } else {
    if (pa.n % 4 == 0)
      k_brick_push_st<2, true><<<2 * nb, kHThreads, push_st_smem<2>(), s>>>(t, g, pa);
    else
      k_brick_push_st<2, false><<<2 * nb, kHThreads, push_st_smem<2>(), s>>>(t, g, pa);
    k_brick_push<2><<<nb, kPushThreads, 0, s>>>(t, g, pa);
  }
  count_launches(2);
}

void launch_brick_pull(const DevTree &t, const BrickGeom &g, const BrickPushArgs &pa, const BrickPullArgs &qa,
                       int32_t *fcount, int32_t *fcursor, int32_t *tile_sums, int32_t *scratch_total,
                       cudaStream_t s) {
  const unsigned nb = (unsigned)g.n_bricks;
  const size_t stage_bytes = (sizeof(float) + sizeof(uint16_t)) * kStageCap;
  cudaMemsetAsync(fcount, 0, sizeof(int32_t) * g.n_bricks, s);
  cudaMemsetAsync(fcursor, 0, sizeof(int32_t) * g.n_bricks, s);
  k_far_count<<<64, 256, 0, s>>>(pa.far_n, pa.far_cap, pa.far_dest, fcount);
  launch_exclusive_scan(fcount, g.n_bricks, qa.fstart_w, tile_sums, scratch_total, s);
  k_far_scatter<<<64, 256, 0, s>>>(pa.far_n, pa.far_cap, pa.far_dest, pa.far_tidx, pa.far_src, qa.fstart,
                                   fcursor, qa.far_tidx_w, qa.far_src_w);
  if (g.d == 3)
    k_brick_totals<3><<<(nb + 7) / 8, 256, 0, s>>>(t, g, pa.cnt, pa.segoff, qa.old_start, qa.fstart,
                                                   qa.far_tidx_w, qa.far_src_w, qa.tot_w, qa.bpiece_w);
  else
    k_brick_totals<2><<<(nb + 7) / 8, 256, 0, s>>>(t, g, pa.cnt, pa.segoff, qa.old_start, qa.fstart,
                                                   qa.far_tidx_w, qa.far_src_w, qa.tot_w, qa.bpiece_w);
  launch_exclusive_scan(qa.tot_w, g.n_bricks, qa.bstart_w, tile_sums, scratch_total, s);
  if (g.d == 3) {
    k_brick_pull_st<3><<<nb, kStThreads, pull_st_smem<3>(), s>>>(t, g, qa);
    k_brick_pull<3><<<nb, kPullThreads, stage_bytes, s>>>(t, g, qa);
  } else {
    k_brick_pull_st<2><<<nb, kStThreads, pull_st_smem<2>(), s>>>(t, g, qa);
    k_brick_pull<2><<<nb, kPullThreads, stage_bytes, s>>>(t, g, qa);
  }
  count_launches(5);  // far count, far scatter, totals, two pull kernels (the scans count themselves)
}

void launch_expand_leaves(const int32_t *start, int64_t n_leaves, int32_t *leaf, cudaStream_t s) {
  k_expand_leaves<<<(unsigned)((n_leaves + 255) / 256), 256, 0, s>>>(start, n_leaves, leaf);
  count_launches(1);
}

cudaError_t brick_configure(const BrickGeom &g) {
  const int bytes = (int)((sizeof(float) + sizeof(uint16_t)) * kStageCap);
  cudaError_t e;
  if (g.d == 3) {
    e = cudaFuncSetAttribute(k_brick_pull<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    for (auto fn : {k_brick_push_st<3, true>, k_brick_push_st<3, false>}) {
      if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)push_st_smem<3>());
      if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_brick_pull_st<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pull_st_smem<3>());
  } else {
    e = cudaFuncSetAttribute(k_brick_pull<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    for (auto fn : {k_brick_push_st<2, true>, k_brick_push_st<2, false>}) {
      if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)push_st_smem<2>());
      if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_brick_pull_st<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pull_st_smem<2>());
  }
  return e;
}

}  // namespace pic
