// Kernel launch interface between the C-ABI layer (pic_api.cu) and the
// kernels (kernels.cu).  All launches are stream-ordered on `s`.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace pic {

struct DevTree;

struct Push64Args {
  int64_t n;
  const double *x, *v;          // current state, bucket-sorted
  const int32_t *leaf, *key;    // key used by PIDT only
  double2 *rec;                 // [n][4] pushed state: x0 x1 | x2 v0 | v1 v2 | (leaf, key as bits), 0, or NULL:
  double *tx, *tv;              // the pushed state in rows [d][n] and tleaf
  int32_t *tleaf, *keyn;        // keyn: new key per particle (PIT: the leaf)
  const double *E;              // [d][n_vert]; NULL: no field (the particle-handling move, no kick)
  double qmdt, dt;
  int32_t *count;               // per key, zeroed before the launch
  uint32_t *mover_words;        // one ballot word per warp
  int32_t *block_movers;        // movers per block
  int32_t *err;
  int32_t reflect;              // 1: reflecting walls of the unit box; 0: periodic
  int32_t flops;                // artificial floating-point operations per particle move
};

struct Push32Args {
  int64_t n;
  const float *o, *v;
  const int32_t *leaf, *key;
  float4 *rec;                  // [n][2] pushed state: o0 o1 o2 v0 | v1 v2 leaf key (leaf, key as bits), or NULL:
  float *to, *tv;               // the pushed state in rows [d][n] and tleaf
  int32_t *tleaf, *keyn;        // keyn: new key per particle (PIT: the leaf)
  const float *E;               // NULL (and Ec NULL): no field (the particle-handling move, no kick)
  const float4 *Ec;             // field at every leaf corner [leaf][corner] (adaptive trees), or NULL
  float qmdt;
  double dt;
  float sl[19];                 // RN32(dt * 3^level) per level
  int32_t *count;
  uint32_t *mover_words;
  int32_t *block_movers;
  int32_t *err;
  int32_t reflect;              // 1: reflecting walls of the unit box; 0: periodic
  int32_t flops;                // artificial floating-point operations per particle move
};

struct RebinArgs {
  int64_t n, n_keys;
  const int32_t *count;         // per key
  const int32_t *keyn;          // new key per particle (storage order)
  const int32_t *old_start;     // CSR of the current order, NULL at creation
  int32_t *new_start;           // n_keys + 1
  const uint32_t *mover_words;
  const int32_t *block_movers;
  int32_t *block_offsets, *movers, *n_stay, *cursor, *perm;
  int32_t *tile_sums, *tile_sums2;
  int32_t *scalars;             // [0] n, [1] movers, [2] max bucket
  int block;                     // threads per block of the push (ballot words, block counts)
};

// Elements per tile of launch_exclusive_scan: a scan of n elements writes
// scan_tiles_needed(n) = ceil(n / kScanTileElems) tile sums.
constexpr int64_t kScanTileElems = 8192;

// Kernels launched by this library so far (all handles of the process).
int64_t launches();
void count_launches(int64_t k);

// Brick path (uniform trees, PIT, split precision): see brick.cu.
struct BrickGeom {
  int d, kb, B, LB, nbx, depth;  // B = 3^kb leaves per brick axis, LB = B^d, nbx bricks per axis
  int64_t n_bricks;
  const uint32_t *decodeL;       // local depth-first index -> x | y << 10 | z << 20
};

// Staging between K1 and K2: every pushed particle is appended to the area of
// its destination unit U (half a brick: local leaves below or from (LB+1)/2),
// slots [U cap, U cap + cap) of each row; arrivals beyond cap go to an
// overflow list.
struct BrickStage {
  int32_t cap;                   // slots per destination unit (a multiple of 8)
  int64_t row;                   // slots in all (2 n_bricks cap, padded)
  float *rec;                    // [row][2 D] one record per slot: the D offsets, then the D velocities
  uint16_t *code;                // destination local leaf | stayer bit
  uint32_t *key;                 // moved << 31 | storage index before the step (canonical order)
  int32_t *id;                   // particle ids (tracked ids only)
  int32_t *fill;                 // [2 n_bricks] arrivals per destination unit (may exceed cap)
  int32_t *over;                 // [2] bricks listed for the global-memory K1, units for the global-memory K2
  int32_t *over_bricks;          // [n_bricks] bricks over the shared-memory K1's capacity (any order)
  int32_t *over_units;           // [2 n_bricks] units over their staging capacity (any order)
  int32_t *ovf_n;                // overflow count
  int32_t ovf_cap;
  int32_t *ovf_dest;             // [ovf_cap] destination unit
  float *ovf_o, *ovf_v;          // [D][ovf_cap]
  uint16_t *ovf_code;
  uint32_t *ovf_key;
  int32_t *ovf_id;
};

struct BrickPushArgs {
  int64_t n;
  const float *o, *v;
  const int32_t *start;          // current leaf offsets
  const int32_t *ids;            // NULL unless ids are tracked
  const float *E;
  const void *Ebrick;            // the field brick by brick: (9+1)^d vertices per brick, float4 (3D) / float2 (2D)
  float qmdt, sl;
  BrickStage st;
  int32_t *n_movers;
  int32_t *err;
  long long wait_cycles;         // limit of the bounded wait for the bulk copies (SM clocks)
};

struct BrickPullArgs {
  int64_t n;
  BrickStage st;
  const int32_t *fstart;         // overflow arrivals sorted per destination brick
  int32_t *fstart_w;
  const int32_t *ovf_sorted;     // overflow list positions, grouped by destination brick
  int32_t *ovf_sorted_w;
  int32_t *tot_w;
  const int32_t *tot;            // incoming particles per destination brick
  const int32_t *bstart;
  int32_t *bstart_w;
  float *o, *v;
  int32_t *ids;
  int32_t *new_start;
  int32_t *max_bucket;
  int32_t *err;
  float *part;                   // leaf-corner deposit partials of the new positions, or NULL
  uint32_t *fb_key;              // [n] scratch of the global-memory kernel
  int32_t *fb_idx;
  long long wait_cycles;         // limit of the bounded wait for the bulk copies (SM clocks)
};

cudaError_t brick_configure(const BrickGeom &g);
int32_t brick_stage_cap(int64_t n, int64_t n_units);  // staging slots per destination unit
void launch_brick_push(const DevTree &t, const BrickGeom &g, const BrickPushArgs &pa, cudaStream_t s);
void launch_brick_pull(const DevTree &t, const BrickGeom &g, const BrickPullArgs &qa, int32_t *fcount,
                       int32_t *fcursor, int32_t *tile_sums, int32_t *scratch_total, cudaStream_t s);
void launch_expand_leaves(const int32_t *start, int64_t n_leaves, int32_t *leaf, cudaStream_t s);
// The vertex field E[d][n_vert] re-laid brick by brick for K1: brick b holds
// the (9+1)^d vertices from its origin on (periodic), x fastest, one vector
// (E_x, E_y[, E_z, 0]) per vertex.
void launch_brick_field(const DevTree &t, const BrickGeom &g, const float *E, float *Ebrick, cudaStream_t s);
// One CTA arms an mbarrier for 16 bytes that are never sent and waits for it
// with the bounded wait of the brick kernels (limit `cycles`); *flag becomes
// 1 when the wait gave up (the expected outcome), 2 if it completed.
void launch_wait_selftest(long long cycles, int32_t *flag, cudaStream_t s);

cudaError_t set_constants(cudaStream_t s);
cudaError_t set_kref(int d, cudaStream_t s);
int64_t scan_tiles_needed(int64_t n);

void launch_init64(const DevTree &t, double *x, int64_t n, int32_t *leaf, int32_t *key, int32_t *err,
                   cudaStream_t s);
void launch_init32(const DevTree &t, const double *x, const double *v, int64_t n, int32_t *leaf, float *o,
                   float *vf, int32_t *key, int32_t *err, cudaStream_t s);
void launch_rekey32(const DevTree &t, const int32_t *leaf, const float *o, int64_t n, int32_t *key, int32_t *err,
                    cudaStream_t s);
void launch_check_sorted(const int32_t *key, int64_t n, int32_t *flag, cudaStream_t s);
void launch_count_all(const int32_t *key, int64_t n, int32_t *count, uint32_t *mover_words,
                      int32_t *block_movers, int block, cudaStream_t s);
// Re-refinement: depth-first cell index on level dmax per particle; cells of
// level m (index key / div) holding more than ppc particles as a bitmap.
void launch_fine_keys(const DevTree &t, bool split, const void *pos, const int32_t *leaf, int64_t n, int dmax,
                      uint32_t *key, cudaStream_t s);
// *changed = 1 unless every leaf of t passes the particles-per-cell criterion
// on the counts of levels dmin .. dmax-1 (level m at count + coff[m]), i.e.
// unless the criterion gives back the installed tree.
void launch_adapt_check(const DevTree &t, const int32_t *count, const int64_t *coff, int dmin, int dmax, int64_t ppc,
                        int32_t *changed, cudaStream_t s);
// Threshold bits (count > ppc) of every cell on levels dmin .. dmax-1 from
// the level-dmax cell keys: counts on level dmax-1 summed up child by child;
// level m's counts at count + cnt_off[m], its bits at bits + bit_off[m].
void launch_adapt_bits(const uint32_t *key, int64_t n, int nch, int dmin, int dmax, int64_t ppc, int32_t *count,
                       const int64_t *cnt_off, uint32_t *bits, const int64_t *bit_off, cudaStream_t s);
void launch_relocate32(const DevTree &from, const DevTree &to, const int32_t *leaf, const float *o, const float *v,
                       int64_t n, int32_t *leaf2, float *o2, float *v2, cudaStream_t s);

// Vertex charges and FP64 total from leaf-corner partials already computed.
void launch_vertex_charge(const DevTree &t, bool split, const void *part, void *Q, double *block_sum,
                          double *total, cudaStream_t s);
// Charges per instance: q and ion density come from the instance table;
// total[0] is the FP64 sum over all vertices, total[1 + i] per instance.
void launch_deposit(const DevTree &t, bool split, const int32_t *start, const void *pos, int64_t n, void *part,
                    void *Q, double *block_sum, double *total, cudaStream_t s);
void launch_solve(const DevTree &t, bool split, const void *Q, const double *total, void *b, void *V, void *Vtmp,
                  int sweeps, double omega, double *block_sum, double *resid2, cudaStream_t s);
void launch_efield(const DevTree &t, bool split, const void *V, void *E, cudaStream_t s);
void launch_push64(const DevTree &t, const Push64Args &a, cudaStream_t s);
void launch_push32(const DevTree &t, const Push32Args &a, cudaStream_t s);
// Field at every leaf corner, the corner expansion applied once per field:
// Ec[L nc + e] = (E_x, E_y, E_z, 0) at corner e of leaf L (adaptive trees).
void launch_corner_field32(const DevTree &t, const float *E, float4 *Ec, cudaStream_t s);
void launch_exclusive_scan(const int32_t *in, int64_t n, int32_t *out, int32_t *tile_sums, int32_t *total,
                           cudaStream_t s);
void launch_rebin(const RebinArgs &r, cudaStream_t s);
// dst[p] = src[perm[p]] for positions, velocities ([d][n]), leaves and,
// where not NULL, keys and ids, in one kernel (split: float, else double).
// Bucket order from the pushed-state records: x2/v2 [d][n] rows, leaf2, and
// key2 unless NULL (PIT), ids2 from ids unless NULL.
void launch_gather_records(bool split, const int32_t *perm, int64_t n, int d, const void *rec, void *x2, void *v2,
                           int32_t *leaf2, int32_t *key2, const int32_t *ids, int32_t *ids2, cudaStream_t s);
void launch_gather_state(bool split, const int32_t *perm, int64_t n, int d, const void *x, void *x2, const void *v,
                         void *v2, const int32_t *leaf, int32_t *leaf2, const int32_t *key, int32_t *key2,
                         const int32_t *ids, int32_t *ids2, cudaStream_t s);
void launch_gather_f64(const int32_t *perm, int64_t n, int d, const double *src, double *dst, cudaStream_t s);
void launch_gather_f32(const int32_t *perm, int64_t n, int d, const float *src, float *dst, cudaStream_t s);
void launch_gather_i32(const int32_t *perm, int64_t n, const int32_t *src, int32_t *dst, cudaStream_t s);
void launch_absolute_split(const DevTree &t, const int32_t *leaf, const float *o, int64_t n, double *x,
                           cudaStream_t s);
void launch_widen(const float *in, int64_t n, double *out, cudaStream_t s);
void launch_gather_only(const DevTree &t, bool split, const void *pos, const int32_t *leaf, int64_t n,
                        const void *Ev, void *Ep, cudaStream_t s);
void launch_half_kick(bool split, const void *Ep, int64_t n_total, double c, void *v, cudaStream_t s);
// raPIDT v_max: per leaf (largest |velocity component| of its particles, or
// of its vertices' particles for PIDT), then per node of the level-ordered
// tree bottom-up (level_begin[l] = first node of level l, depth + 2 entries).
void launch_vmax(const DevTree &t, bool split, const int32_t *start, const void *v, int64_t n, const int32_t *child0,
                 const int32_t *leaf_of_node, const int64_t *level_begin, int depth, double *leaf_vmax,
                 double *node_vmax, cudaStream_t s);
// lift and drop counts (diagnostic): counts[0..2] = lifts, drops, tunnellers
void launch_scatter_by_id(const int32_t *ids, const int32_t *leaf, int64_t n, int32_t *by_id, cudaStream_t s);
void launch_lift_drop(const DevTree &t, const int32_t *ids, const int32_t *leaf, const int32_t *old_by_id, int64_t n,
                      unsigned long long *counts, cudaStream_t s);
// PIDT: pv_level / pv_j are the owner-vertex table (adaptive trees; unused on
// uniform ones); counts[0..2] = lifts, drops, tunnellers.
void launch_lift_drop_pidt(const DevTree &t, const int32_t *pv_level, const int32_t *pv_j, const int32_t *ids,
                           const int32_t *leaf, const int32_t *key, const int32_t *old_leaf_by_id,
                           const int32_t *old_key_by_id, int64_t n, unsigned long long *counts, cudaStream_t s);

}  // namespace pic
