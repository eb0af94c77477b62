// C ABI of libpic (include/pic.h): handle management, device memory, and the
// orchestration of one PIT/PIDT particle step on the handle's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/pic.h"
#include "dev.cuh"
#include "launch.hpp"
#include "snapshot.hpp"
#include "tree.hpp"
#include "tree_dev.hpp"

using namespace pic;

namespace {

struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct pic_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  pic_config cfg{};
  // device memory through the caller's allocator (pic_set_allocator at
  // creation); NULL: cudaMalloc / cudaFree
  pic_alloc_fn alloc_fn = nullptr;
  pic_free_fn free_fn = nullptr;
  void *alloc_user = nullptr;
  int d = 0, scheme = 0, split = 0;
  int64_t n = 0;
  std::vector<HostTree> hts;   // every instance
  HostTree &ht0() { return hts[0]; }  // instance 0 (the only one unless batched)
  std::vector<InstInfo> inst;
  DevTree dt{};
  uint64_t tree_gen = 0;  // counts installed trees
  // state_bufs: sized by the particle count (kept across re-trees);
  // grid_bufs: sized by the tree (leaves, vertices, keys)
  std::vector<DevBuf> tree_bufs, state_bufs, grid_bufs;
  int64_t device_bytes = 0;
  // re-refinement (pic_adapt): cell counts of every decision level and their
  // threshold bits, kept between calls
  std::vector<DevBuf> adapt_bufs;
  // device tabulation of adaptive trees: its tables (when grid_dev) and its
  // scratch, kept for the next re-tree while it is small
  DeviceGrid gdev{};
  bool grid_dev = false;
  std::vector<DevBuf> tab_scratch;
  // buffers of superseded trees and grids, reused by the next re-tree
  struct Spare {
    DevBuf b;
    uint64_t gen;
  };
  std::vector<Spare> spare;
  int64_t adapt_cells = 0, adapt_words = 0;
  int32_t *adapt_count = nullptr;
  uint32_t *adapt_bits = nullptr;

  // particle state: [0] current (bucket-sorted), [1] pushed (same index)
  void *pos[2] = {nullptr, nullptr};  // x (double) or o (float), [d][n]
  void *prec = nullptr;               // 3D: pushed-state records of the generic step, 32 (split) or 64 bytes each
  void *vel[2] = {nullptr, nullptr};
  int32_t *leaf[2] = {nullptr, nullptr};
  int32_t *key[2] = {nullptr, nullptr};  // [1] doubles as the new key
  int32_t *ids[2] = {nullptr, nullptr};
  // re-bin scratch
  int32_t *start_cur = nullptr, *start_new = nullptr, *count = nullptr, *n_stay = nullptr, *cursor = nullptr;
  int32_t *perm = nullptr, *movers = nullptr, *block_movers = nullptr, *block_offsets = nullptr;
  int32_t *tile_sums = nullptr, *tile_sums2 = nullptr, *scalars = nullptr, *err = nullptr;
  uint32_t *mover_words = nullptr;
  // grid
  void *part = nullptr, *Q = nullptr, *b = nullptr, *V = nullptr, *Vtmp = nullptr, *E = nullptr;
  double *block_sum = nullptr, *total = nullptr, *resid2 = nullptr;
  void *Ep = nullptr;  // d * n scratch (gather at the particles, FP64 staging)
  float4 *ecorner = nullptr;  // split, adaptive: field at every leaf corner
  bool ecorner_valid = false; // ecorner holds the corners of the current E
  float *ebrick = nullptr;    // brick path: the field brick by brick (float4 / float2 per vertex)
  bool ebrick_valid = false;  // ebrick holds the current E

  int64_t step = 0;
  std::string last_error;
  long long wait_cycles = 4000000000LL;  // bounded device waits of the brick kernels (pic_set_wait_limit)

  // lift and drop counts of the steps (pic_count_lifts; tracked ids)
  bool count_lifts = false;
  int32_t *lift_old = nullptr;             // leaf before the step, by particle id
  int32_t *lift_oldkey = nullptr;          // PIDT: key before the step, by particle id
  int32_t *lift_pvl = nullptr, *lift_pvj = nullptr;  // PIDT, adaptive: owner-vertex levels and indices
  std::vector<DevBuf> lift_tab_bufs;                  // holds lift_pvl / lift_pvj of tree lift_gen
  uint64_t lift_gen = ~0ull;
  unsigned long long *lift_counts = nullptr;  // [0] lifts, [1] drops, [2] tunnellers
  int64_t lift_steps = 0;
  std::vector<DevBuf> diag_bufs;

  // brick path (uniform tree, PIT, split precision)
  bool brick = false;
  bool brick_ok = false;    // the brick path applies (its buffers exist)
  bool leaf_stale = false;  // leaf[0] not yet expanded from the offsets
  bool q_valid = false;     // Q holds the charges of the current positions

  // CUDA graphs of one fixed-field step: [0] from the current buffer
  // assignment, [1] from the swapped one (the step alternates ping-pong offsets)
  struct HostView {  // host-side buffer assignment a step swaps
    int32_t *start_cur, *start_new, *ids0, *ids1;
    bool leaf_stale, q_valid;
  };
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  HostView graph_pre[2]{}, graph_post[2]{};
  int64_t graph_kernels = 0;
  BrickGeom bg{};
  std::vector<DevBuf> brick_bufs;
  BrickStage stage{};      // per-destination staging between the two brick kernels
  int32_t *fcount = nullptr, *fcursor = nullptr, *fstart = nullptr, *ovf_sorted = nullptr;
  int32_t *btot = nullptr, *bstart = nullptr, *fb_idx = nullptr;
  uint32_t *fb_key = nullptr;

  // per-phase event timing (pic_profile / pic_phase_times)
  struct Pending {
    int phase;
    cudaEvent_t a, b;
    int64_t kernels;
  };
  bool prof = false;
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  double phase_ms[PIC_NPHASES] = {0, 0, 0, 0, 0};
  int64_t phase_kernels[PIC_NPHASES] = {0, 0, 0, 0, 0};
};

namespace {

int fail(pic_t h, int code, const std::string &msg) {
  if (h) h->last_error = msg;
  return code;
}

int cuda_fail(pic_t h, cudaError_t e, const char *what) {
  if (h) h->last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return PIC_ECUDA;
}

#define CK(call)                                        \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

// Process-wide allocator that handles created from now on adopt.
std::mutex g_alloc_mu;
pic_alloc_fn g_alloc_fn = nullptr;
pic_free_fn g_free_fn = nullptr;
void *g_alloc_user = nullptr;

template <typename T>
int dalloc(pic_t h, std::vector<DevBuf> &bufs, T **out, size_t count) {
  size_t bytes = sizeof(T) * (count ? count : 1);
  void *p = nullptr;
  *out = nullptr;
  if (h->alloc_fn) {
    p = h->alloc_fn(h->alloc_user, bytes, (void *)h->stream);
    if (!p) return fail(h, PIC_ENOMEM, "the caller's allocator failed for " + std::to_string(bytes) + " bytes");
    if ((uintptr_t)p & 255u) {
      h->free_fn(h->alloc_user, p, bytes, (void *)h->stream);
      return fail(h, PIC_ENOMEM, "the caller's allocator returned a pointer not aligned to 256 bytes");
    }
    // a recycled block may still be in use by work queued on the stream
    // before it was handed over; some uploads copy outside the stream
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      h->free_fn(h->alloc_user, p, bytes, (void *)h->stream);
      return cuda_fail(h, e, "cudaStreamSynchronize");
    }
  } else {
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess)
      return fail(h, PIC_ENOMEM, std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes failed");
  }
  bufs.push_back({p, bytes});
  h->device_bytes += (int64_t)bytes;
  *out = (T *)p;
  return PIC_OK;
}

void free_bufs(pic_t h, std::vector<DevBuf> &bufs) {
  // blocks go back to the caller's allocator only once the stream is done
  // with them (cudaFree synchronises the device itself)
  if (h->free_fn && !bufs.empty()) cudaStreamSynchronize(h->stream);
  for (auto &b : bufs) {
    if (h->free_fn)
      h->free_fn(h->alloc_user, b.p, b.bytes, (void *)h->stream);
    else
      cudaFree(b.p);
    h->device_bytes -= (int64_t)b.bytes;
  }
  bufs.clear();
}

template <typename T, typename A>
int upload(pic_t h, std::vector<DevBuf> &bufs, const T **out, const std::vector<T, A> &v) {
  T *p = nullptr;
  int rc = dalloc(h, bufs, &p, v.size());
  if (rc) return rc;
  if (!v.empty()) CK(cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  *out = p;
  return PIC_OK;
}

// Tree and grid buffers go through a spare list: a superseded tree's or
// grid's buffers are kept, and a request takes the smallest spare buffer that
// holds it (at most twice its size), so re-trees of similar trees need no
// cudaMalloc / cudaFree.  Spares not taken by the next re-tree are freed.
template <typename T>
int galloc(pic_t h, std::vector<DevBuf> &bufs, T **out, size_t count) {
  const size_t bytes = sizeof(T) * (count ? count : 1);
  int best = -1;
  for (size_t i = 0; i < h->spare.size(); ++i) {
    const size_t b = h->spare[i].b.bytes;
    if (b >= bytes && b <= 2 * bytes + 65536 && (best < 0 || b < h->spare[best].b.bytes)) best = (int)i;
  }
  if (best < 0) return dalloc(h, bufs, out, count);
  bufs.push_back(h->spare[best].b);
  *out = (T *)h->spare[best].b.p;
  h->spare.erase(h->spare.begin() + best);
  return PIC_OK;
}

void retire(pic_t h, std::vector<DevBuf> &bufs) {
  for (auto &b : bufs) h->spare.push_back({b, h->tree_gen});
  bufs.clear();
}

// Frees the spares retired before tree generation `gen`.
void drop_spares(pic_t h, uint64_t gen) {
  std::vector<DevBuf> old;
  size_t k = 0;
  for (auto &sp : h->spare) {
    if (sp.gen < gen) old.push_back(sp.b);
    else h->spare[k++] = sp;
  }
  h->spare.resize(k);
  free_bufs(h, old);
}

template <typename T, typename A>
int gupload(pic_t h, std::vector<DevBuf> &bufs, const T **out, const std::vector<T, A> &v) {
  T *p = nullptr;
  int rc = galloc(h, bufs, &p, v.size());
  if (rc) return rc;
  if (!v.empty()) CK(cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  *out = p;
  return PIC_OK;
}

// Tabulate the trees of all instances on the host and upload the device view
// (leaves, vertices and keys concatenated instance by instance).  The previous
// device buffers are handed back in *old (freed by the caller) so particles
// can still be re-located from them.
// Host tabulation instead of the device one (PIC_HOST_TABLES=1), for
// comparing the two; the tables, and so every result, are the same.
bool host_tables_forced() {
  const char *e = std::getenv("PIC_HOST_TABLES");
  return e && e[0] == '1';
}

// Device memory of the device tabulation: its tables go to the tree's
// buffers; its scratch buffers are slots of h->tab_scratch, reused by the
// next re-tree when large enough (the same sequence of requests).
struct TabCtx {
  pic_t h;
  std::vector<DevBuf> *keep;
  size_t next;
};

int tab_alloc(void *c, void **out, size_t bytes, bool keep) {
  TabCtx *ctx = (TabCtx *)c;
  pic_t h = ctx->h;
  char *p = nullptr;
  if (keep) {
    if (galloc(h, *ctx->keep, &p, bytes)) return kTabNoMemory;
    *out = p;
    return 0;
  }
  auto &sc = h->tab_scratch;
  const size_t k = ctx->next++;
  if (k < sc.size() && sc[k].bytes >= bytes) {
    *out = sc[k].p;
    return 0;
  }
  std::vector<DevBuf> fresh;
  if (dalloc(h, fresh, &p, bytes + bytes / 4)) return kTabNoMemory;
  if (k < sc.size()) {
    std::vector<DevBuf> one(1, sc[k]);
    free_bufs(h, one);
    sc[k] = fresh[0];
  } else {
    sc.push_back(fresh[0]);
  }
  *out = p;
  return 0;
}

void tab_release(void *, void *) {}  // slots stay for the next re-tree (trim_tab_scratch)

// Scratch is kept only while it is small (frequent re-trees of small trees).
void trim_tab_scratch(pic_t h) {
  int64_t bytes = 0;
  for (const auto &b : h->tab_scratch) bytes += (int64_t)b.bytes;
  if (bytes > (int64_t)256 << 20) free_bufs(h, h->tab_scratch);
}

int install_forest(pic_t h, const pic_tree_desc *trees, int32_t n_inst, const std::vector<double> &qs,
                   std::vector<DevBuf> *old = nullptr) {
  if (!trees || n_inst < 1) return fail(h, PIC_EINVAL, "tree descriptor is NULL");
  std::vector<HostTree> hts(n_inst);
  for (int32_t i = 0; i < n_inst; ++i) {
    std::string err;
    HostTree &ht = hts[i];
    if (!trees[i].flags) return fail(h, PIC_EINVAL, "tree descriptor is NULL");
    if (ht.build(trees[i].d, trees[i].n_nodes, trees[i].flags, &err))
      return fail(h, PIC_EINVAL, "instance " + std::to_string(i) + ": " + err);
    if ((h->d && trees[i].d != h->d) || trees[i].d != trees[0].d)
      return fail(h, PIC_EINVAL, "tree dimension differs from the handle");
    if (ht.depth > 12 && !ht.uniform) return fail(h, PIC_EINVAL, "adaptive trees deeper than level 12 are not supported");
    if (n_inst > 1 && !ht.uniform) return fail(h, PIC_EINVAL, "batched instances must have uniform trees");
    int64_t mv = 1;
    for (int a = 0; a < ht.d; ++a) mv *= ht.M;
    if (mv > INT32_MAX) return fail(h, PIC_EINVAL, "finest level has more than 2^31 grid points");
    if (n_inst == 1 && grid_on_device_fits(ht) && !host_tables_forced()) continue;  // tabulated on the device below
    ht.build_grid();
    if (h->scheme == PIC_PIDT) ht.build_pidt();  // PIT handles build it on demand
  }
  const bool on_device = n_inst == 1 && grid_on_device_fits(hts[0]) && !host_tables_forced();
  const HostTree &h0 = hts[0];
  const int d = h0.d, nc = h0.nc;
  int64_t nl = 0, nv = 0, npv = 0, ntab = 0, nspread = 0;
  std::vector<InstInfo> inst(n_inst);
  for (int32_t i = 0; i < n_inst; ++i) {
    const HostTree &ht = hts[i];
    InstInfo &I = inst[i];
    I.depth = ht.depth;
    I.M = (int32_t)ht.M;
    I.leaf_off = (int32_t)nl;
    I.vert_off = (int32_t)nv;
    I.key_off = (int32_t)(h->scheme == PIC_PIT ? nl : npv * nc);
    I.spread_off = (int32_t)nspread;
    I.tab_root = (int32_t)ntab;
    I.n_vert = (int32_t)ht.n_vert;
    I.poff = 0;
    I.q = qs[i];
    I.ion = h->cfg.ion;
    I.ion_load = ht.uniform ? ht.ion_load[0] : 0.0;
    I.diag = ht.uniform ? ht.diag[0] : 0.0;
    I.q32 = (float)I.q;
    I.ion32 = (float)I.ion;
    I.ion_load32 = (float)I.ion_load;
    I.diag32 = (float)I.diag;
    nl += ht.n_leaves;
    nv += ht.n_vert;
    npv += ht.n_pv;
    ntab += (int64_t)ht.tab.size();
    if (ht.uniform) nspread += (int64_t)d * ht.M;
  }
  int64_t nkeys = h->scheme == PIC_PIT ? nl : npv * nc;
  if (nl >= INT32_MAX / 8 || nv >= INT32_MAX || nkeys >= INT32_MAX)
    return fail(h, PIC_EINVAL, "more than 2^31 leaves, vertices or sort keys");
  std::vector<TabEntry> tab;
  std::vector<uint8_t> leaf_level;
  std::vector<int32_t> leaf_coords, spread, iol, iov;
  tab.reserve(ntab);
  leaf_level.reserve(nl);
  leaf_coords.reserve(nl * d);
  if (n_inst > 1) {
    iol.reserve(nl);
    iov.reserve(nv);
  }
  for (int32_t i = 0; i < n_inst; ++i) {
    const HostTree &ht = hts[i];
    const InstInfo &I = inst[i];
    for (const TabEntry &e : ht.tab)
      tab.push_back(e.a >= 0 ? TabEntry{e.a + I.tab_root, 0} : TabEntry{e.a, e.b + I.leaf_off});
    leaf_level.insert(leaf_level.end(), ht.leaf_level.begin(), ht.leaf_level.end());
    leaf_coords.insert(leaf_coords.end(), ht.leaf_coords.begin(), ht.leaf_coords.end());
    if (ht.uniform)
      for (int a = 0; a < d; ++a)
        for (int64_t c = 0; c < ht.M; ++c) {
          int64_t v = 0, cc = c, mul = pow3(a);
          for (int k = 0; k < ht.depth; ++k) {
            v += (cc % 3) * mul;
            cc /= 3;
            mul *= ht.nch;
          }
          spread.push_back((int32_t)v);
        }
    if (n_inst > 1) {
      iol.insert(iol.end(), ht.n_leaves, i);
      iov.insert(iov.end(), ht.n_vert, i);
    }
  }
  std::vector<DevBuf> prev;
  prev.swap(h->tree_bufs);
  DevTree dt{};
  dt.d = d;
  dt.nch = h0.nch;
  dt.nc = nc;
  dt.depth = h0.depth;
  dt.uniform = h0.uniform ? 1 : 0;
  dt.scheme = h->scheme;
  dt.n_inst = n_inst;
  dt.n_leaves = nl;
  dt.n_vert = nv;
  dt.n_pv = npv;
  dt.n_keys = nkeys;
  dt.M = (int32_t)h0.M;
  dt.n_tab = (int32_t)tab.size();
  int rc;
  auto &tb = h->tree_bufs;
  if ((rc = gupload(h, tb, &dt.tab, tab))) return rc;
  if ((rc = gupload(h, tb, &dt.leaf_level, leaf_level))) return rc;
  if ((rc = gupload(h, tb, &dt.leaf_coords, leaf_coords))) return rc;
  bool device_tables = false;
  if (on_device) {
    // the grid and owner tables of the adaptive tree, built on the GPU
    HostTree &ht = hts[0];
    TabCtx ctx{h, &tb, 0};
    GridAlloc A{&ctx, tab_alloc, tab_release};
    DeviceGrid G;
    const int trc = tabulate_on_device(ht, dt.tab, dt.leaf_level, dt.leaf_coords, h->scheme == PIC_PIDT, h->stream,
                                       A, &G);
    trim_tab_scratch(h);
    if (trc == kTabNoMemory) return fail(h, PIC_ENOMEM, "device memory for the tree tables");
    if (trc == kTabCuda) return cuda_fail(h, cudaGetLastError(), "device tabulation of the tree");
    if (trc == 0) {
      device_tables = true;
      nv = G.n_vert;
      npv = h->scheme == PIC_PIDT ? G.n_pv : 0;
      nkeys = h->scheme == PIC_PIT ? nl : npv * nc;
      if (nv >= INT32_MAX || nkeys >= INT32_MAX) return fail(h, PIC_EINVAL, "more than 2^31 vertices or sort keys");
      ht.n_vert = nv;
      ht.n_pv = npv;
      ht.pidt_built = h->scheme == PIC_PIDT;  // the owner tables live on the device (gdev)
      inst[0].n_vert = (int32_t)nv;
      dt.n_vert = nv;
      dt.n_pv = npv;
      dt.n_keys = nkeys;
      dt.cexp_ptr = G.cexp_ptr;
      dt.cexp_vid = G.cexp_vid;
      dt.cexp_w64 = G.cexp_w64;
      dt.cexp_w32 = G.cexp_w32;
      dt.inc_ptr = G.inc_ptr;
      dt.inc_lc = G.inc_lc;
      dt.inc_w64 = G.inc_w64;
      dt.inc_w32 = G.inc_w32;
      dt.ion64 = G.ion64;
      dt.ion32 = G.ion32;
      dt.diag64 = G.diag64;
      dt.diag32 = G.diag32;
      dt.dcnt = G.dcnt;
      dt.corner_pv = G.corner_pv;
      h->gdev = G;
    } else {  // an expansion too long for the device path: the host tables
      ht.build_grid();
      if (h->scheme == PIC_PIDT) ht.build_pidt();
      nv = ht.n_vert;
      npv = h->scheme == PIC_PIDT ? ht.n_pv : 0;
      nkeys = h->scheme == PIC_PIT ? nl : npv * nc;
      inst[0].n_vert = (int32_t)nv;
      dt.n_vert = nv;
      dt.n_pv = npv;
      dt.n_keys = nkeys;
    }
  }
  if ((rc = gupload(h, tb, &dt.inst, inst))) return rc;
  if (n_inst > 1) {
    if ((rc = gupload(h, tb, &dt.inst_of_leaf, iol))) return rc;
    if ((rc = gupload(h, tb, &dt.inst_of_vert, iov))) return rc;
  }
  if (h0.uniform) {
    if ((rc = gupload(h, tb, &dt.spread, spread))) return rc;
  } else if (!device_tables) {
    const HostTree &ht = h0;
    std::vector<float> f;
    auto to32 = [&](const table<double> &v) {
      f.assign(v.size(), 0.f);
      for (size_t i = 0; i < v.size(); ++i) f[i] = (float)v[i];
      return f;
    };
    if ((rc = gupload(h, tb, &dt.cexp_ptr, ht.cexp_ptr))) return rc;
    if ((rc = gupload(h, tb, &dt.cexp_vid, ht.cexp_vid))) return rc;
    if ((rc = gupload(h, tb, &dt.cexp_w64, ht.cexp_w))) return rc;
    if ((rc = gupload(h, tb, &dt.cexp_w32, to32(ht.cexp_w)))) return rc;
    if ((rc = gupload(h, tb, &dt.inc_ptr, ht.inc_ptr))) return rc;
    if ((rc = gupload(h, tb, &dt.inc_lc, ht.inc_lc))) return rc;
    if ((rc = gupload(h, tb, &dt.inc_w64, ht.inc_w))) return rc;
    if ((rc = gupload(h, tb, &dt.inc_w32, to32(ht.inc_w)))) return rc;
    if ((rc = gupload(h, tb, &dt.ion64, ht.ion_load))) return rc;
    if ((rc = gupload(h, tb, &dt.ion32, to32(ht.ion_load)))) return rc;
    if ((rc = gupload(h, tb, &dt.diag64, ht.diag))) return rc;
    if ((rc = gupload(h, tb, &dt.diag32, to32(ht.diag)))) return rc;
    if ((rc = gupload(h, tb, &dt.dcnt, ht.direct_cnt))) return rc;
    if ((rc = gupload(h, tb, &dt.corner_pv, ht.corner_pv))) return rc;
  }
  h->d = d;
  h->inst = inst;
  h->hts = std::move(hts);
  h->dt = dt;
  h->grid_dev = device_tables;
  if (!device_tables) h->gdev = DeviceGrid{};
  h->tree_gen++;
  if (old)
    old->swap(prev);
  else
    free_bufs(h, prev);
  return PIC_OK;
}

int install_tree(pic_t h, const pic_tree_desc *tree, std::vector<DevBuf> *old = nullptr) {
  std::vector<double> qs(1, h->cfg.q);
  return install_forest(h, tree, 1, qs, old);
}

// Particle offsets of the instances (input order), uploaded into the table.
int set_particle_offsets(pic_t h, const std::vector<int64_t> &poff) {
  for (size_t i = 0; i < h->inst.size(); ++i) h->inst[i].poff = poff[i];
  CK(cudaMemcpy((void *)h->dt.inst, h->inst.data(), sizeof(InstInfo) * h->inst.size(), cudaMemcpyHostToDevice));
  return PIC_OK;
}

// The solver's warm start, the vertex field and the charge totals start
// from zero (after a new tree is installed, or an unchanged one confirmed).
int reset_grid_state(pic_t h) {
  cudaStream_t s = h->stream;
  const size_t fs = h->split ? sizeof(float) : sizeof(double);
  const int64_t nv = h->dt.n_vert;
  CK(cudaMemsetAsync(h->V, 0, fs * nv, s));
  CK(cudaMemsetAsync(h->E, 0, fs * nv * h->d, s));
  CK(cudaMemsetAsync(h->total, 0, sizeof(double) * (2 + h->dt.n_inst), s));
  CK(cudaMemsetAsync(h->resid2, 0, sizeof(double) * 2, s));
  h->ecorner_valid = false;
  h->ebrick_valid = false;
  h->q_valid = false;
  return PIC_OK;
}

// Per-particle buffers, sized from n alone: a re-tree keeps them.
int alloc_particles(pic_t h) {
  free_bufs(h, h->state_bufs);
  auto &sb = h->state_bufs;
  const int64_t n = h->n, d = h->d;
  const size_t fs = h->split ? sizeof(float) : sizeof(double);
  const int64_t nblk = (n + 127) / 128 + 1;  // blocks of the smallest tuned block size
  int rc;
  for (int s = 0; s < 2; ++s) {
    char *p;
    // + 64 bytes: bulk copies read whole 16-byte units around a particle range
    if ((rc = dalloc(h, sb, &p, fs * d * n + 64))) return rc;
    h->pos[s] = p;
    if ((rc = dalloc(h, sb, &p, fs * d * n + 64))) return rc;
    h->vel[s] = p;
    if ((rc = dalloc(h, sb, &h->leaf[s], n))) return rc;
    if (h->scheme == PIC_PIT) {
      h->key[s] = h->leaf[s];  // PIT keys are the leaves
    } else if ((rc = dalloc(h, sb, &h->key[s], n))) {
      return rc;
    }
    if ((rc = dalloc(h, sb, &h->ids[s], n))) return rc;
  }
  h->prec = nullptr;
  if (d == 3) {  // 3D: eight arrays per particle, gathered as one record (2D keeps the rows)
    char *p;
    if ((rc = dalloc(h, sb, &p, (h->split ? 32 : 64) * n))) return rc;
    h->prec = p;
  }
  if ((rc = dalloc(h, sb, &h->perm, n))) return rc;
  if ((rc = dalloc(h, sb, &h->movers, n))) return rc;
  if ((rc = dalloc(h, sb, &h->block_movers, nblk))) return rc;
  if ((rc = dalloc(h, sb, &h->block_offsets, nblk + 1))) return rc;
  if ((rc = dalloc(h, sb, &h->mover_words, (n + 31) / 32 + 64))) return rc;
  if ((rc = dalloc(h, sb, &h->tile_sums2, scan_tiles_needed(nblk) + 1))) return rc;
  if ((rc = dalloc(h, sb, &h->scalars, 8))) return rc;
  if ((rc = dalloc(h, sb, &h->err, 1))) return rc;
  cudaStream_t s = h->stream;
  CK(cudaMemsetAsync(h->err, 0, sizeof(int32_t), s));
  CK(cudaMemsetAsync(h->scalars, 0, sizeof(int32_t) * 8, s));
  return PIC_OK;
}

// Buffers sized from the installed tree (bucket offsets and counts, leaf
// partials, vertex fields, the FP64 staging area); the solver's warm start
// and the field start from zero.
int alloc_grid(pic_t h) {
  retire(h, h->grid_bufs);  // stream-ordered reuse: every later use is queued after the old one
  auto &sb = h->grid_bufs;
  const int64_t n = h->n, d = h->d;
  const size_t fs = h->split ? sizeof(float) : sizeof(double);
  const int64_t nk = h->dt.n_keys, nv = h->dt.n_vert, nl = h->dt.n_leaves;
  int rc;
  // bucket offsets, padded: the brick kernels copy whole 16-byte units of them
  if ((rc = galloc(h, sb, &h->start_cur, nk + 8))) return rc;
  if ((rc = galloc(h, sb, &h->start_new, nk + 8))) return rc;
  if ((rc = galloc(h, sb, &h->count, nk))) return rc;
  if ((rc = galloc(h, sb, &h->n_stay, nk))) return rc;
  if ((rc = galloc(h, sb, &h->cursor, nk))) return rc;
  if ((rc = galloc(h, sb, &h->tile_sums, scan_tiles_needed(nk) + 1))) return rc;
  char *p;
  if ((rc = galloc(h, sb, &p, fs * nl * h->dt.nc))) return rc;
  h->part = p;
  if ((rc = galloc(h, sb, &p, fs * nv))) return rc;
  h->Q = p;
  if ((rc = galloc(h, sb, &p, fs * nv))) return rc;
  h->b = p;
  if ((rc = galloc(h, sb, &p, fs * nv))) return rc;
  h->V = p;
  if ((rc = galloc(h, sb, &p, fs * nv))) return rc;
  h->Vtmp = p;
  if ((rc = galloc(h, sb, &p, fs * nv * d))) return rc;
  h->E = p;
  if ((rc = galloc(h, sb, &h->block_sum, (nv + 127) / 128 + 1))) return rc;
  if ((rc = galloc(h, sb, &h->total, 2 + h->dt.n_inst))) return rc;
  if ((rc = galloc(h, sb, &h->resid2, 2))) return rc;
  // FP64 staging: particle arrays (d * n) and widened vertex fields (d * n_vert)
  if ((rc = galloc(h, sb, &p, sizeof(double) * d * std::max(n, nv)))) return rc;
  h->Ep = p;
  h->ecorner = nullptr;
  h->ecorner_valid = false;
  h->ebrick_valid = false;
  if (h->split && !h->dt.uniform && (rc = galloc(h, sb, &h->ecorner, nl * h->dt.nc))) return rc;
  return reset_grid_state(h);
}

int alloc_state(pic_t h) {
  int rc;
  if ((rc = alloc_particles(h))) return rc;
  return alloc_grid(h);
}

cudaEvent_t take_event(pic_t h) {
  if (!h->event_pool.empty()) {
    cudaEvent_t e = h->event_pool.back();
    h->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Sums the recorded phase intervals into the per-phase totals.
int drain_profile(pic_t h) {
  CK(cudaStreamSynchronize(h->stream));
  for (auto &p : h->pending) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, p.a, p.b));
    h->phase_ms[p.phase] += ms;
    h->phase_kernels[p.phase] += p.kernels;
    h->event_pool.push_back(p.a);
    h->event_pool.push_back(p.b);
  }
  h->pending.clear();
  return PIC_OK;
}

// Records CUDA events around one phase on the handle's stream when profiling.
struct PhaseScope {
  pic_t h;
  int phase;
  cudaEvent_t a = nullptr;
  int64_t k0 = 0;
  PhaseScope(pic_t h_, int phase_) : h(h_), phase(phase_) {
    if (!h->prof) return;
    a = take_event(h);
    cudaEventRecord(a, h->stream);
    k0 = launches();
  }
  ~PhaseScope() {
    if (!h->prof || !a) return;
    cudaEvent_t b = take_event(h);
    cudaEventRecord(b, h->stream);
    h->pending.push_back({phase, a, b, launches() - k0});
    if (h->pending.size() > 4096) drain_profile(h);
  }
};

// Buffers and tables of the brick path, when it applies.
int setup_brick(pic_t h) {
  free_bufs(h, h->brick_bufs);
  h->brick = false;
  h->brick_ok = false;
  const auto &t = h->ht0();
  if (h->cfg.path != PIC_PATH_AUTO || !t.uniform || h->scheme != PIC_PIT || !h->split || t.depth < 3 ||
      h->dt.n_inst > 1)
    return PIC_OK;
  BrickGeom g{};
  g.d = t.d;
  g.kb = 2;
  g.B = 9;
  g.LB = t.d == 3 ? 729 : 81;
  g.depth = t.depth;
  g.nbx = (int)pow3(t.depth - g.kb);
  g.n_bricks = 1;
  for (int a = 0; a < t.d; ++a) g.n_bricks *= g.nbx;
  std::vector<uint32_t> dec((g.LB + 3) & ~3, 0u);  // padded to whole 16-byte units (one bulk copy)
  for (int l = 0; l < g.LB; ++l) {
    uint32_t c[3] = {0, 0, 0};
    int rest = l;
    uint32_t p3i = 1;
    for (int i = 0; i < g.kb; ++i) {
      int dg = rest % t.nch;
      rest /= t.nch;
      c[0] += (uint32_t)(dg % 3) * p3i;
      c[1] += (uint32_t)((dg / 3) % 3) * p3i;
      c[2] += (uint32_t)(dg / 9) * p3i;
      p3i *= 3;
    }
    dec[l] = c[0] | (c[1] << 10) | (c[2] << 20);
  }
  auto &bb = h->brick_bufs;
  int rc;
  if ((rc = upload(h, bb, &g.decodeL, dec))) return rc;
  const int64_t n = h->n, nu = 2 * g.n_bricks;  // destination units: half bricks
  // staging: cap slots per destination unit (a multiple of 8, so every unit's
  // area starts on a 16-byte boundary in the record array and in the code and
  // key rows), plus a tail for the bulk copies of the last unit, which read
  // whole 16-byte units
  BrickStage &st = h->stage;
  st = BrickStage{};
  st.cap = brick_stage_cap(n, nu);
  st.row = nu * st.cap + 16;
  // a tree with many more bricks than particles would spend more memory on
  // empty staging areas than on the particles: the generic path serves it
  if (nu * st.cap > 16 * n + (int64_t(1) << 24) || st.row >= (int64_t(1) << 31)) return PIC_OK;
  if ((rc = dalloc(h, bb, &st.rec, st.row * 2 * t.d))) return rc;
  if ((rc = dalloc(h, bb, &st.code, st.row))) return rc;
  if ((rc = dalloc(h, bb, &st.key, st.row))) return rc;
  if (h->cfg.track_ids && (rc = dalloc(h, bb, &st.id, st.row))) return rc;
  if ((rc = dalloc(h, bb, &st.fill, nu))) return rc;
  if ((rc = dalloc(h, bb, &st.over, 2))) return rc;
  if ((rc = dalloc(h, bb, &st.over_bricks, g.n_bricks))) return rc;
  if ((rc = dalloc(h, bb, &st.over_units, nu))) return rc;
  // the field laid out brick by brick, one vector per vertex of the brick
  // and its upper faces ((9+1)^d vertices), refreshed whenever E changes
  if ((rc = dalloc(h, bb, &h->ebrick, g.n_bricks * (t.d == 3 ? 1000 * 4 : 100 * 2)))) return rc;
  h->ebrick_valid = false;
  if ((rc = dalloc(h, bb, &st.ovf_n, 1))) return rc;
  // overflow list: one entry per particle at most; offsets, velocities and
  // ids in the pushed-state rows, which the brick step leaves unused (set per
  // step)
  st.ovf_cap = (int32_t)n;
  if ((rc = dalloc(h, bb, &st.ovf_dest, n))) return rc;
  if ((rc = dalloc(h, bb, &st.ovf_code, n))) return rc;
  if ((rc = dalloc(h, bb, &st.ovf_key, n))) return rc;
  if ((rc = dalloc(h, bb, &h->ovf_sorted, n))) return rc;
  if ((rc = dalloc(h, bb, &h->fb_key, n))) return rc;
  if ((rc = dalloc(h, bb, &h->fb_idx, n))) return rc;
  if ((rc = dalloc(h, bb, &h->fcount, nu))) return rc;
  if ((rc = dalloc(h, bb, &h->fcursor, nu))) return rc;
  if ((rc = dalloc(h, bb, &h->fstart, nu + 1))) return rc;
  if ((rc = dalloc(h, bb, &h->btot, nu))) return rc;
  if ((rc = dalloc(h, bb, &h->bstart, nu + 1))) return rc;
  if (scan_tiles_needed(nu) + 1 > scan_tiles_needed(h->dt.n_keys) + 1)
    return fail(h, PIC_EINVAL, "brick count exceeds scan scratch");
  CK(brick_configure(g));
  h->bg = g;
  h->brick = true;
  h->brick_ok = true;
  return PIC_OK;
}

int ensure_leaf(pic_t h) {
  if (!h->leaf_stale) return PIC_OK;
  launch_expand_leaves(h->start_cur, h->dt.n_leaves, h->leaf[0], h->stream);
  CK(cudaGetLastError());
  h->leaf_stale = false;
  return PIC_OK;
}

int brick_push_and_rebin(pic_t h, double dt) {
  cudaStream_t s = h->stream;
  BrickPushArgs pa{};
  pa.n = h->n;
  pa.o = (const float *)h->pos[0];
  pa.v = (const float *)h->vel[0];
  pa.start = h->start_cur;
  pa.ids = h->cfg.track_ids ? h->ids[0] : nullptr;
  pa.E = (const float *)h->E;
  if (!h->ebrick_valid) {
    launch_brick_field(h->dt, h->bg, (const float *)h->E, h->ebrick, s);
    h->ebrick_valid = true;
  }
  pa.Ebrick = h->ebrick;
  pa.qmdt = (float)(h->cfg.qm * dt);
  pa.sl = (float)(dt * (double)pow3(h->ht0().depth));
  pa.st = h->stage;
  pa.st.ovf_o = (float *)h->pos[1];  // the current assignment: re-bins elsewhere swap the rows
  pa.st.ovf_v = (float *)h->vel[1];
  pa.st.ovf_id = h->ids[1];
  pa.n_movers = h->scalars + 1;
  pa.err = h->err;
  pa.wait_cycles = h->wait_cycles;
  // the pull reads only the staging area and the overflow list, so the new
  // bucket order is written over the current state in place
  BrickPullArgs qa{};
  qa.n = h->n;
  qa.st = pa.st;
  qa.fstart = h->fstart;
  qa.fstart_w = h->fstart;
  qa.ovf_sorted = h->ovf_sorted;
  qa.ovf_sorted_w = h->ovf_sorted;
  qa.tot_w = h->btot;
  qa.tot = h->btot;
  qa.bstart = h->bstart;
  qa.bstart_w = h->bstart;
  qa.o = (float *)h->pos[0];
  qa.v = (float *)h->vel[0];
  qa.ids = pa.ids ? h->ids[0] : nullptr;
  qa.new_start = h->start_new;
  qa.max_bucket = h->scalars + 2;
  qa.err = h->err;
  qa.part = (float *)h->part;
  qa.fb_key = h->fb_key;
  qa.fb_idx = h->fb_idx;
  qa.wait_cycles = h->wait_cycles;
  CK(cudaMemsetAsync(h->scalars + 1, 0, sizeof(int32_t) * 2, s));
  {
    PhaseScope ps(h, PIC_PHASE_PUSH);
    launch_brick_push(h->dt, h->bg, pa, s);
  }
  {
    PhaseScope ps(h, PIC_PHASE_REBIN);
    launch_brick_pull(h->dt, h->bg, qa, h->fcount, h->fcursor, h->tile_sums, h->scalars + 3, s);
  }
  {
    // the pull also summed the deposit partials of the new positions
    PhaseScope ps(h, PIC_PHASE_DEPOSIT);
    launch_vertex_charge(h->dt, true, h->part, h->Q, h->block_sum, h->total, s);
  }
  CK(cudaGetLastError());
  std::swap(h->start_cur, h->start_new);
  h->leaf_stale = true;
  h->q_valid = true;
  return PIC_OK;
}

// Stable re-bin of the pushed state into the current state [0]: from the
// records of the generic push (records) or from the rows [1] (fresh state).
// old_start == NULL: fresh particles, every one counted as a mover.
int rebin_and_gather(pic_t h, const int32_t *old_start, bool records = false) {
  cudaStream_t s = h->stream;
  const int64_t n = h->n;
  RebinArgs r{};
  r.n = n;
  r.n_keys = h->dt.n_keys;
  r.count = h->count;
  r.keyn = h->key[1];
  r.old_start = old_start;
  r.new_start = h->start_new;
  r.mover_words = h->mover_words;
  r.block_movers = h->block_movers;
  r.block_offsets = h->block_offsets;
  r.movers = h->movers;
  r.n_stay = h->n_stay;
  r.cursor = h->cursor;
  r.perm = h->perm;
  r.tile_sums = h->tile_sums;
  r.tile_sums2 = h->tile_sums2;
  r.scalars = h->scalars;
  r.block = h->dt.block_push;
  {
    PhaseScope ps(h, PIC_PHASE_REBIN);
    launch_rebin(r, s);
  }
  PhaseScope ps(h, PIC_PHASE_PERMUTE);
  const int d = h->d;
  if (records) {  // the pushed state, one record per particle
    launch_gather_records(h->split, h->perm, n, d, h->prec, h->pos[0], h->vel[0], h->leaf[0],
                          h->scheme == PIC_PIT ? nullptr : h->key[0], h->cfg.track_ids ? h->ids[0] : nullptr,
                          h->cfg.track_ids ? h->ids[1] : nullptr, s);
    if (h->cfg.track_ids) std::swap(h->ids[0], h->ids[1]);
  } else if (h->scheme == PIC_PIT) {
    // one pass over the permutation (measured faster for PIT; PIDT's extra
    // key array makes the separate passes faster: 6.1 against 6.7 ms on the
    // 2e8-particle 3D two-stream step)
    launch_gather_state(h->split, h->perm, n, d, h->pos[1], h->pos[0], h->vel[1], h->vel[0], h->leaf[1],
                        h->leaf[0], nullptr, nullptr, h->cfg.track_ids ? h->ids[0] : nullptr,
                        h->cfg.track_ids ? h->ids[1] : nullptr, s);
    if (h->cfg.track_ids) std::swap(h->ids[0], h->ids[1]);
  } else if (h->split) {
    launch_gather_f32(h->perm, n, d, (const float *)h->pos[1], (float *)h->pos[0], s);
    launch_gather_f32(h->perm, n, d, (const float *)h->vel[1], (float *)h->vel[0], s);
  } else {
    launch_gather_f64(h->perm, n, d, (const double *)h->pos[1], (double *)h->pos[0], s);
    launch_gather_f64(h->perm, n, d, (const double *)h->vel[1], (double *)h->vel[0], s);
  }
  if (!records && h->scheme != PIC_PIT) {
    launch_gather_i32(h->perm, n, h->leaf[1], h->leaf[0], s);
    launch_gather_i32(h->perm, n, h->key[1], h->key[0], s);
    if (h->cfg.track_ids) {
      launch_gather_i32(h->perm, n, h->ids[0], h->ids[1], s);
      std::swap(h->ids[0], h->ids[1]);
    }
  }
  std::swap(h->start_cur, h->start_new);
  h->leaf_stale = false;
  CK(cudaGetLastError());
  return PIC_OK;
}

// Keys of fresh state in [1] -> counts -> re-bin.  Fresh particles are all
// movers, so the canonical order is the stable order by key; when the keys
// already ascend (a state read back by pic_get_state, for example) that is the
// input order and only the bucket offsets are computed.
int bin_fresh(pic_t h) {
  h->q_valid = false;
  cudaStream_t s = h->stream;
  CK(cudaMemsetAsync(h->count, 0, sizeof(int32_t) * h->dt.n_keys, s));
  launch_count_all(h->key[1], h->n, h->count, h->mover_words, h->block_movers, h->dt.block_push, s);
  CK(cudaMemsetAsync(h->scalars + 6, 0, sizeof(int32_t), s));
  launch_check_sorted(h->key[1], h->n, h->scalars + 6, s);
  int32_t unsorted = 1;
  CK(cudaMemcpyAsync(&unsorted, h->scalars + 6, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (unsorted) return rebin_and_gather(h, nullptr);
  launch_exclusive_scan(h->count, h->dt.n_keys, h->start_new, h->tile_sums, h->scalars + 0, s);
  std::swap(h->pos[0], h->pos[1]);
  std::swap(h->vel[0], h->vel[1]);
  std::swap(h->leaf[0], h->leaf[1]);
  if (h->key[0] != h->leaf[1]) std::swap(h->key[0], h->key[1]);  // PIT keys alias the leaves
  else {
    h->key[0] = h->leaf[0];
    h->key[1] = h->leaf[1];
  }
  std::swap(h->start_cur, h->start_new);
  h->leaf_stale = false;
  CK(cudaGetLastError());
  return PIC_OK;
}

int deposit(pic_t h) {
  if (h->q_valid) return PIC_OK;
  PhaseScope ps(h, PIC_PHASE_DEPOSIT);
  h->q_valid = true;
  launch_deposit(h->dt, h->split, h->start_cur, h->pos[0], h->n, h->part, h->Q,
                 h->block_sum, h->total, h->stream);
  CK(cudaGetLastError());
  return PIC_OK;
}

int field(pic_t h, pic_solve_fn hook, void *user) {
  PhaseScope ps(h, PIC_PHASE_SOLVE);
  cudaStream_t s = h->stream;
  h->ecorner_valid = false;  // E changes below
  h->ebrick_valid = false;
  if (hook) {
    int r = hook(user, h->Q, h->E, h->dt.n_vert, h->split ? PIC_FP32_SPLIT : PIC_FP64, (void *)s);
    if (r != 0) return fail(h, PIC_EHOOK, "field-solve hook returned " + std::to_string(r));
    return PIC_OK;
  }
  launch_solve(h->dt, h->split, h->Q, h->total, h->b, h->V, h->Vtmp, h->cfg.sweeps, h->cfg.omega, h->block_sum,
               h->resid2, s);
  launch_efield(h->dt, h->split, h->V, h->E, s);
  CK(cudaGetLastError());
  return PIC_OK;
}

// What moves the particles: the PIC push (gather + kick + drift, periodic)
// or the particle-handling move of the paper's experiments (no field,
// periodic or reflecting walls, artificial flops per move).
struct MoveKind {
  bool field = true;
  int32_t reflect = 0, flops = 0;
};

int push_and_rebin(pic_t h, double dt, MoveKind mk = MoveKind{}) {
  if (h->brick && mk.field) return brick_push_and_rebin(h, dt);
  int rc0 = ensure_leaf(h);
  if (rc0) return rc0;
  h->q_valid = false;
  cudaStream_t s = h->stream;
  CK(cudaMemsetAsync(h->count, 0, sizeof(int32_t) * h->dt.n_keys, s));
  CK(cudaMemsetAsync(h->scalars + 2, 0, sizeof(int32_t), s));
  PhaseScope *ps = new PhaseScope(h, PIC_PHASE_PUSH);
  if (h->split) {
    Push32Args a{};
    a.n = h->n;
    a.o = (const float *)h->pos[0];
    a.v = (const float *)h->vel[0];
    a.leaf = h->leaf[0];
    a.key = h->key[0];
    a.rec = (float4 *)h->prec;
    a.to = (float *)h->pos[1];
    a.tv = (float *)h->vel[1];
    a.tleaf = h->leaf[1];
    a.keyn = h->key[1];
    a.E = mk.field ? (const float *)h->E : nullptr;
    if (h->ecorner && mk.field) {
      if (!h->ecorner_valid) {
        launch_corner_field32(h->dt, (const float *)h->E, h->ecorner, s);
        h->ecorner_valid = true;
      }
      a.Ec = h->ecorner;
    }
    a.reflect = mk.reflect;
    a.flops = mk.flops;
    a.qmdt = (float)(h->cfg.qm * dt);
    a.dt = dt;
    for (int l = 0; l <= 18; ++l) a.sl[l] = (float)(dt * (double)pow3(l));
    a.count = h->count;
    a.mover_words = h->mover_words;
    a.block_movers = h->block_movers;
    a.err = h->err;
    launch_push32(h->dt, a, s);
  } else {
    Push64Args a{};
    a.n = h->n;
    a.x = (const double *)h->pos[0];
    a.v = (const double *)h->vel[0];
    a.leaf = h->leaf[0];
    a.key = h->key[0];
    a.rec = (double2 *)h->prec;
    a.tx = (double *)h->pos[1];
    a.tv = (double *)h->vel[1];
    a.tleaf = h->leaf[1];
    a.keyn = h->key[1];
    a.E = mk.field ? (const double *)h->E : nullptr;
    a.reflect = mk.reflect;
    a.flops = mk.flops;
    a.qmdt = h->cfg.qm * dt;
    a.dt = dt;
    a.count = h->count;
    a.mover_words = h->mover_words;
    a.block_movers = h->block_movers;
    a.err = h->err;
    launch_push64(h->dt, a, s);
  }
  delete ps;
  CK(cudaGetLastError());
  return rebin_and_gather(h, h->start_cur, h->prec != nullptr);
}

int check_handle(pic_t h) { return h ? PIC_OK : PIC_EINVAL; }

void drop_graphs(pic_t h) {
  for (auto &g : h->graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}



int copy_out(pic_t h, void *dst, const void *src, size_t bytes, int32_t where) {
  if (!dst) return PIC_OK;
  if (where == PIC_HOST) {
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  } else {
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, h->stream));
  }
  return PIC_OK;
}

int copy_in(pic_t h, void *dst, const void *src, size_t bytes, int32_t where) {
  CK(cudaMemcpyAsync(dst, src, bytes, where == PIC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                     h->stream));
  return PIC_OK;
}

// Load FP64 particles (host or device, one piece per instance, concatenated
// axis by axis) into state [1] and bin them.
int load_particles64(pic_t h, const pic_particles_desc *parts, int32_t n_inst) {
  cudaStream_t s = h->stream;
  const int d = h->d;
  const int64_t n = h->n;
  int rc;
  double *xs, *vs;
  std::vector<DevBuf> tmp;
  if (h->split) {
    xs = (double *)h->Ep;
    if ((rc = dalloc(h, tmp, &vs, (size_t)d * n))) return rc;
  } else {
    xs = (double *)h->pos[1];
    vs = (double *)h->vel[1];
  }
  int64_t off = 0;
  for (int32_t i = 0; i < n_inst; ++i) {
    const int64_t ni = parts[i].n;
    for (int a = 0; a < d && ni > 0; ++a) {
      if ((rc = copy_in(h, xs + a * n + off, parts[i].x + a * ni, sizeof(double) * ni, parts[i].where)) ||
          (rc = copy_in(h, vs + a * n + off, parts[i].v + a * ni, sizeof(double) * ni, parts[i].where))) {
        free_bufs(h, tmp);
        return rc;
      }
    }
    off += ni;
  }
  if (h->split) {
    launch_init32(h->dt, xs, vs, n, h->leaf[1], (float *)h->pos[1], (float *)h->vel[1], h->key[1], h->err, s);
    cudaError_t e = cudaStreamSynchronize(s);
    free_bufs(h, tmp);
    if (e != cudaSuccess) return cuda_fail(h, e, "particle conversion");
  } else {
    launch_init64(h->dt, xs, n, h->leaf[1], h->key[1], h->err, s);
  }
  CK(cudaGetLastError());
  return bin_fresh(h);
}

int read_err(pic_t h, int32_t *err) {
  CK(cudaMemcpyAsync(err, h->err, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return PIC_OK;
}

}  // namespace

extern "C" {

const char *pic_strerror(int code) {
  switch (code) {
    case PIC_OK: return "ok";
    case PIC_EINVAL: return "invalid argument or malformed tree";
    case PIC_ENOMEM: return "out of memory";
    case PIC_ERANGE: return "non-finite position or velocity";
    case PIC_EHOOK: return "field-solve hook failed";
    case PIC_ETIMEOUT: return "device wait timed out";
    case PIC_ECUDA: return "CUDA runtime error";
    case PIC_ESTATE: return "call not valid in this state";
    case PIC_EIO: return "checkpoint file missing, unreadable, truncated or corrupt";
    default: return "unknown error";
  }
}

// Message of the last failed handle-less call (pic_load) on this thread.
static thread_local std::string t_last_error;

const char *pic_last_error(pic_t h) {
  if (h) return h->last_error.c_str();
  return t_last_error.empty() ? "NULL handle" : t_last_error.c_str();
}

void pic_destroy(pic_t h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  for (auto &p : h->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : h->event_pool) cudaEventDestroy(e);
  drop_graphs(h);
  free_bufs(h, h->diag_bufs);
  free_bufs(h, h->lift_tab_bufs);
  free_bufs(h, h->adapt_bufs);
  free_bufs(h, h->tab_scratch);
  for (auto &sp : h->spare) {
    std::vector<DevBuf> one(1, sp.b);
    free_bufs(h, one);
  }
  h->spare.clear();
  free_bufs(h, h->brick_bufs);
  free_bufs(h, h->grid_bufs);
  free_bufs(h, h->state_bufs);
  free_bufs(h, h->tree_bufs);
  delete h;
}

// Common creation path: n_inst instances (a single handle is a batch of one).
static int create_forest(pic_t *out, int32_t n_inst, const pic_tree_desc *trees, const pic_particles_desc *parts,
                         const double *q, const pic_config *cfg) {
  if (!out) return PIC_EINVAL;
  *out = nullptr;
  if (n_inst < 1 || !trees || !parts || !cfg) return PIC_EINVAL;
  if (cfg->scheme != PIC_PIT && cfg->scheme != PIC_PIDT) return PIC_EINVAL;
  if (cfg->precision != PIC_FP64 && cfg->precision != PIC_FP32_SPLIT) return PIC_EINVAL;
  if (cfg->sweeps < 0) return PIC_EINVAL;
  int64_t n_total = 0;
  std::vector<int64_t> poff(n_inst);
  for (int32_t i = 0; i < n_inst; ++i) {
    const pic_particles_desc &pp = parts[i];
    if (pp.n < 0 || (pp.n > 0 && (!pp.x || !pp.v))) return PIC_EINVAL;
    if (pp.where != PIC_HOST && pp.where != PIC_DEVICE) return PIC_EINVAL;
    if (trees[i].d != 2 && trees[i].d != 3) return PIC_EINVAL;
    if (pp.where == PIC_HOST) {
      size_t m = (size_t)trees[i].d * pp.n;
      for (size_t k = 0; k < m; ++k)
        if (!std::isfinite(pp.x[k]) || !std::isfinite(pp.v[k])) return PIC_ERANGE;
    }
    poff[i] = n_total;
    n_total += pp.n;
  }
  if (n_total >= INT32_MAX) return PIC_EINVAL;
  pic_t h = new (std::nothrow) pic_s();
  if (!h) return PIC_ENOMEM;
  h->cfg = *cfg;
  h->scheme = cfg->scheme;
  h->split = cfg->precision == PIC_FP32_SPLIT;
  h->n = n_total;
  h->stream = (cudaStream_t)cfg->stream;
  {
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    h->alloc_fn = g_alloc_fn;
    h->free_fn = g_free_fn;
    h->alloc_user = g_alloc_user;
  }
  cudaGetDevice(&h->device);
  int rc;
  cudaError_t e = set_constants(h->stream);
  if (e != cudaSuccess) { rc = cuda_fail(h, e, "set_constants"); pic_destroy(h); return rc; }
  std::vector<double> qs(n_inst, cfg->q);
  if (q)
    for (int32_t i = 0; i < n_inst; ++i) qs[i] = q[i];
  if ((rc = install_forest(h, trees, n_inst, qs))) { pic_destroy(h); return rc; }
  if ((rc = set_particle_offsets(h, poff))) { pic_destroy(h); return rc; }
  e = set_kref(h->d, h->stream);
  if (e != cudaSuccess) { rc = cuda_fail(h, e, "set_kref"); pic_destroy(h); return rc; }
  if ((rc = alloc_state(h))) { pic_destroy(h); return rc; }
  if ((rc = setup_brick(h))) { pic_destroy(h); return rc; }
  if (h->n > 0) {
    std::vector<int32_t> iota(h->n);
    for (int64_t i = 0; i < h->n; ++i) iota[i] = (int32_t)i;
    e = cudaMemcpy(h->ids[0], iota.data(), sizeof(int32_t) * h->n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { rc = cuda_fail(h, e, "ids"); pic_destroy(h); return rc; }
  }
  if ((rc = load_particles64(h, parts, n_inst))) { pic_destroy(h); return rc; }
  int32_t err = 0;
  if ((rc = read_err(h, &err))) { pic_destroy(h); return rc; }
  if (err) { pic_destroy(h); return PIC_ERANGE; }
  *out = h;
  return PIC_OK;
}

int pic_create(pic_t *out, const pic_tree_desc *tree, const pic_particles_desc *parts, const pic_config *cfg) {
  return create_forest(out, 1, tree, parts, nullptr, cfg);
}

int pic_create_batch(pic_t *out, int32_t n_inst, const pic_tree_desc *trees, const pic_particles_desc *parts,
                     const double *q, const pic_config *cfg) {
  return create_forest(out, n_inst, trees, parts, q, cfg);
}

int pic_instances(pic_t h, int64_t *particle_start, int64_t *vertex_start, int64_t *bucket_start) {
  if (check_handle(h)) return PIC_EINVAL;
  const int32_t ni = h->dt.n_inst;
  const int stride = h->scheme == PIC_PIT ? 1 : h->dt.nc;
  for (int32_t i = 0; i <= ni; ++i) {
    const bool end = i == ni;
    if (particle_start) particle_start[i] = end ? h->n : h->inst[i].poff;
    if (vertex_start) vertex_start[i] = end ? h->dt.n_vert : h->inst[i].vert_off;
    if (bucket_start) bucket_start[i] = end ? h->dt.n_keys / stride : h->inst[i].key_off / stride;
  }
  return PIC_OK;
}

int pic_info(pic_t h, pic_info_t *o) {
  if (check_handle(h) || !o) return PIC_EINVAL;
  o->d = h->d;
  o->scheme = h->scheme;
  o->precision = h->split ? PIC_FP32_SPLIT : PIC_FP64;
  o->depth = h->ht0().depth;
  o->n_particles = h->n;
  o->n_leaves = h->dt.n_leaves;
  o->n_vertices = h->dt.n_vert;
  o->n_buckets = h->scheme == PIC_PIT ? h->dt.n_leaves : h->dt.n_pv;
  o->n_keys = h->dt.n_keys;
  o->uniform = h->dt.uniform;
  o->brick = h->brick ? 1 : 0;
  o->n_instances = h->dt.n_inst;
  o->device_bytes = h->device_bytes;
  return PIC_OK;
}

int pic_init_leapfrog(pic_t h, double dt, pic_solve_fn hook, void *user) {
  if (check_handle(h)) return PIC_EINVAL;
  int rc;
  if ((rc = ensure_leaf(h))) return rc;
  if ((rc = deposit(h))) return rc;
  if ((rc = field(h, hook, user))) return rc;
  launch_gather_only(h->dt, h->split, h->pos[0], h->leaf[0], h->n, h->E, h->Ep, h->stream);
  launch_half_kick(h->split, h->Ep, h->n * h->d, h->cfg.qm * (0.5 * dt), h->vel[0], h->stream);
  CK(cudaGetLastError());
  return PIC_OK;
}

// PIDT on an adaptive tree: the owner-vertex table (levels; indices per axis
// as int32) of the installed tree on the device, uploaded again after every
// re-tree.
static int lift_tables(pic_t h) {
  if (h->scheme != PIC_PIDT || h->lift_gen == h->tree_gen) return PIC_OK;
  free_bufs(h, h->lift_tab_bufs);
  h->lift_pvl = h->lift_pvj = nullptr;
  if (!h->dt.uniform && h->grid_dev) {  // tabulated on the device: already int32 device arrays
    h->lift_pvl = h->gdev.pv_level;
    h->lift_pvj = h->gdev.pv_j;
  } else if (!h->dt.uniform) {
    HostTree &t = h->ht0();
    t.build_pidt();
    std::vector<int32_t> pvl(t.pv_level.begin(), t.pv_level.end());
    std::vector<int32_t> pvj(t.pv_j.size());
    for (size_t i = 0; i < pvj.size(); ++i) pvj[i] = (int32_t)t.pv_j[i];
    const int32_t *a = nullptr, *b = nullptr;
    int rc = upload(h, h->lift_tab_bufs, &a, pvl);
    if (!rc) rc = upload(h, h->lift_tab_bufs, &b, pvj);
    if (rc) {
      free_bufs(h, h->lift_tab_bufs);
      return rc;
    }
    h->lift_pvl = const_cast<int32_t *>(a);
    h->lift_pvj = const_cast<int32_t *>(b);
  }
  h->lift_gen = h->tree_gen;
  return PIC_OK;
}

// Lift and drop counting around the push and re-bin of a step: the leaf of
// every particle by id before, the per-particle counts after.
static int lift_before(pic_t h) {
  int rc;
  if ((rc = ensure_leaf(h)) || (rc = lift_tables(h))) return rc;
  launch_scatter_by_id(h->ids[0], h->leaf[0], h->n, h->lift_old, h->stream);
  if (h->scheme == PIC_PIDT) launch_scatter_by_id(h->ids[0], h->key[0], h->n, h->lift_oldkey, h->stream);
  CK(cudaGetLastError());
  return PIC_OK;
}

static int lift_after(pic_t h) {
  int rc;
  if ((rc = ensure_leaf(h))) return rc;
  if (h->scheme == PIC_PIDT)
    launch_lift_drop_pidt(h->dt, h->lift_pvl, h->lift_pvj, h->ids[0], h->leaf[0], h->key[0], h->lift_old,
                          h->lift_oldkey, h->n, h->lift_counts, h->stream);
  else
    launch_lift_drop(h->dt, h->ids[0], h->leaf[0], h->lift_old, h->n, h->lift_counts, h->stream);
  CK(cudaGetLastError());
  h->lift_steps++;
  return PIC_OK;
}

static int counted_push_and_rebin(pic_t h, double dt, MoveKind mk = MoveKind{}) {
  int rc;
  if (h->count_lifts && (rc = lift_before(h))) return rc;
  if ((rc = push_and_rebin(h, dt, mk))) return rc;
  if (h->count_lifts && (rc = lift_after(h))) return rc;
  return PIC_OK;
}

int pic_step(pic_t h, double dt, pic_solve_fn hook, void *user) {
  if (check_handle(h)) return PIC_EINVAL;
  int rc;
  if ((rc = deposit(h))) return rc;
  if ((rc = field(h, hook, user))) return rc;
  if ((rc = counted_push_and_rebin(h, dt))) return rc;
  h->step++;
  return PIC_OK;
}

int pic_step_fixed_field(pic_t h, double dt) {
  if (check_handle(h)) return PIC_EINVAL;
  int rc;
  if ((rc = deposit(h))) return rc;
  if ((rc = counted_push_and_rebin(h, dt))) return rc;
  h->step++;
  return PIC_OK;
}

static void lift_bufs_forget(pic_t h) {
  free_bufs(h, h->lift_tab_bufs);
  h->lift_gen = ~0ull;
  h->lift_old = nullptr;
  h->lift_oldkey = nullptr;
  h->lift_pvl = nullptr;
  h->lift_pvj = nullptr;
  h->lift_counts = nullptr;
}

int pic_step_particles(pic_t h, double dt, int32_t boundary, int32_t flops) {
  if (check_handle(h)) return PIC_EINVAL;
  if (boundary != PIC_PERIODIC && boundary != PIC_REFLECT)
    return fail(h, PIC_EINVAL, "boundary is PIC_PERIODIC or PIC_REFLECT");
  if (flops < 0 || flops > (1 << 16)) return fail(h, PIC_EINVAL, "flops outside [0, 65536]");
  if (!std::isfinite(dt)) return fail(h, PIC_EINVAL, "dt is not finite");
  MoveKind mk;
  mk.field = false;
  mk.reflect = boundary == PIC_REFLECT ? 1 : 0;
  mk.flops = flops;
  int rc;
  if ((rc = ensure_leaf(h))) return rc;
  drop_graphs(h);
  if ((rc = counted_push_and_rebin(h, dt, mk))) return rc;
  h->step++;
  return PIC_OK;
}

int pic_count_lifts(pic_t h, int32_t enable) {
  if (check_handle(h)) return PIC_EINVAL;
  if (!enable) {
    h->count_lifts = false;
    free_bufs(h, h->diag_bufs);
    lift_bufs_forget(h);
    return PIC_OK;
  }
  if (!h->cfg.track_ids) return fail(h, PIC_ESTATE, "lift and drop counts need track_ids = 1");
  if (h->scheme == PIC_PIDT && h->dt.n_inst > 1)
    return fail(h, PIC_ESTATE, "PIDT lift and drop counts are kept for single-instance handles");
  drop_graphs(h);
  int rc = PIC_OK;
  if (!h->count_lifts) {
    rc = dalloc(h, h->diag_bufs, &h->lift_old, h->n);
    if (!rc) rc = dalloc(h, h->diag_bufs, &h->lift_counts, 3);
    if (!rc && h->scheme == PIC_PIDT) rc = dalloc(h, h->diag_bufs, &h->lift_oldkey, h->n);
    if (!rc) rc = lift_tables(h);
    if (rc) {
      free_bufs(h, h->diag_bufs);
      lift_bufs_forget(h);
      return rc;
    }
  }
  CK(cudaMemsetAsync(h->lift_counts, 0, 3 * sizeof(unsigned long long), h->stream));
  h->lift_steps = 0;
  h->count_lifts = true;
  return PIC_OK;
}

int pic_lift_counts(pic_t h, int64_t *lifts, int64_t *drops, int64_t *tunnellers, int64_t *steps) {
  if (check_handle(h)) return PIC_EINVAL;
  if (!h->count_lifts) return fail(h, PIC_ESTATE, "lift counting is off (pic_count_lifts)");
  unsigned long long c[3] = {0, 0, 0};
  CK(cudaMemcpyAsync(c, h->lift_counts, sizeof(c), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (lifts) *lifts = (int64_t)c[0];
  if (drops) *drops = (int64_t)c[1];
  if (tunnellers) *tunnellers = (int64_t)c[2];
  if (steps) *steps = h->lift_steps;
  return PIC_OK;
}

pic_s::HostView host_view(pic_t h) {
  return {h->start_cur, h->start_new, h->ids[0], h->ids[1], h->leaf_stale, h->q_valid};
}

void set_host_view(pic_t h, const pic_s::HostView &v) {
  h->start_cur = v.start_cur;
  h->start_new = v.start_new;
  h->ids[0] = v.ids0;
  h->ids[1] = v.ids1;
  h->leaf_stale = v.leaf_stale;
  h->q_valid = v.q_valid;
}

// The captured step: deposit when due, the built-in solve if with_solve,
// gather + push + key, re-bin.
static int captured_step(pic_t h, double dt, bool with_solve) {
  int rc;
  if ((rc = deposit(h))) return rc;
  if (with_solve && (rc = field(h, nullptr, nullptr))) return rc;
  return push_and_rebin(h, dt);
}

static int graph_capture(pic_t h, double dt, bool with_solve) {
  if (check_handle(h)) return PIC_EINVAL;
  if (!h->stream) return fail(h, PIC_ESTATE, "graph capture needs a non-default stream");
  if (h->count_lifts) return fail(h, PIC_ESTATE, "lift counting is on; captured steps would not count");
  if (h->prof) return fail(h, PIC_ESTATE, "stop profiling before capturing");
  drop_graphs(h);
  int rc;
  // one ordinary step first, so that the captured steps start from the state
  // every later step starts from (brick path: charges already deposited)
  if ((rc = captured_step(h, dt, with_solve))) return rc;
  h->step++;
  if ((rc = ensure_leaf(h))) return rc;  // generic path: no expansion inside the graph
  CK(cudaStreamSynchronize(h->stream));
  const pic_s::HostView start = host_view(h);
  const int64_t k0 = launches();
  for (int g = 0; g < 2; ++g) {
    h->graph_pre[g] = host_view(h);
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    rc = captured_step(h, dt, with_solve);
    cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    h->graph_post[g] = host_view(h);
    if (!rc && e == cudaSuccess) e = cudaGraphInstantiate(&h->graph[g], graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (rc || e != cudaSuccess) {
      drop_graphs(h);
      set_host_view(h, start);  // nothing captured ran
      return rc ? rc : cuda_fail(h, e, "graph capture");
    }
  }
  set_host_view(h, start);
  h->graph_kernels = (launches() - k0) / 2;
  return PIC_OK;
}

int pic_graph_capture(pic_t h, double dt) { return graph_capture(h, dt, false); }

int pic_graph_capture_step(pic_t h, double dt) { return graph_capture(h, dt, true); }

int pic_graph_launch(pic_t h, int32_t steps) {
  if (check_handle(h) || steps < 0) return PIC_EINVAL;
  if (!h->graph[0]) return fail(h, PIC_ESTATE, "no captured step (pic_graph_capture)");
  for (int32_t i = 0; i < steps; ++i) {
    int rc;
    if (!h->graph_pre[0].leaf_stale && (rc = ensure_leaf(h))) return rc;
    const auto cur = host_view(h);
    int g = -1;
    for (int k = 0; k < 2; ++k) {
      const auto &p = h->graph_pre[k];
      if (p.start_cur == cur.start_cur && p.ids0 == cur.ids0 && (p.q_valid || !cur.q_valid)) g = k;
    }
    if (g < 0) return fail(h, PIC_ESTATE, "the state no longer matches the captured step; capture again");
    PhaseScope ps(h, PIC_PHASE_PUSH);
    CK(cudaGraphLaunch(h->graph[g], h->stream));
    count_launches(h->graph_kernels);
    set_host_view(h, h->graph_post[g]);
    h->step++;
  }
  return PIC_OK;
}

// ---------------------------------------------------------------------------
// autotuning: path (brick or generic) and threads per block
// ---------------------------------------------------------------------------

struct Snapshot {
  std::vector<DevBuf> bufs;
  void *pos = nullptr, *vel = nullptr;
  int32_t *leaf = nullptr, *key = nullptr, *ids = nullptr, *start = nullptr;
};

int snapshot_take(pic_t h, Snapshot &sn) {
  const size_t fs = h->split ? sizeof(float) : sizeof(double);
  const int64_t n = h->n, m = n * h->d, nk = h->dt.n_keys;
  char *p, *q;
  int rc;
  if ((rc = dalloc(h, sn.bufs, &p, fs * m)) || (rc = dalloc(h, sn.bufs, &q, fs * m)) ||
      (rc = dalloc(h, sn.bufs, &sn.leaf, n)) || (rc = dalloc(h, sn.bufs, &sn.key, n)) ||
      (rc = dalloc(h, sn.bufs, &sn.ids, n)) || (rc = dalloc(h, sn.bufs, &sn.start, nk + 1)))
    return rc;
  sn.pos = p;
  sn.vel = q;
  cudaStream_t s = h->stream;
  CK(cudaMemcpyAsync(sn.pos, h->pos[0], fs * m, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(sn.vel, h->vel[0], fs * m, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(sn.leaf, h->leaf[0], sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(sn.key, h->key[0], sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(sn.ids, h->ids[0], sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(sn.start, h->start_cur, sizeof(int32_t) * (nk + 1), cudaMemcpyDeviceToDevice, s));
  return PIC_OK;
}

int snapshot_restore(pic_t h, const Snapshot &sn) {
  const size_t fs = h->split ? sizeof(float) : sizeof(double);
  const int64_t n = h->n, m = n * h->d, nk = h->dt.n_keys;
  cudaStream_t s = h->stream;
  CK(cudaMemcpyAsync(h->pos[0], sn.pos, fs * m, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(h->vel[0], sn.vel, fs * m, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(h->leaf[0], sn.leaf, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(h->key[0], sn.key, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(h->ids[0], sn.ids, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(h->start_cur, sn.start, sizeof(int32_t) * (nk + 1), cudaMemcpyDeviceToDevice, s));
  h->leaf_stale = false;
  h->q_valid = false;
  return PIC_OK;
}

int apply_tuning(pic_t h, const int32_t *t) {
  if (t[0] != 0 && t[0] != 1) return fail(h, PIC_EINVAL, "path is 0 (generic) or 1 (brick)");
  if (t[0] == 1 && !h->brick_ok) return fail(h, PIC_EINVAL, "the brick path does not apply to this handle");
  for (int i = 1; i < 4; ++i)
    if (t[i] != 128 && t[i] != 256 && t[i] != 512) return fail(h, PIC_EINVAL, "block sizes are 128, 256 or 512");
  int rc;
  if ((rc = ensure_leaf(h))) return rc;
  drop_graphs(h);
  h->brick = t[0] == 1;
  h->dt.block_push = t[1];
  h->dt.block_leaf = t[2];
  h->dt.block_vert = t[3];
  return PIC_OK;
}

int pic_set_tuning(pic_t h, const int32_t *tuned) {
  if (check_handle(h) || !tuned) return PIC_EINVAL;
  return apply_tuning(h, tuned);
}

int pic_get_tuning(pic_t h, int32_t *tuned) {
  if (check_handle(h) || !tuned) return PIC_EINVAL;
  tuned[0] = h->brick ? 1 : 0;
  tuned[1] = h->dt.block_push > 0 ? h->dt.block_push : 256;
  tuned[2] = h->dt.block_leaf > 0 ? h->dt.block_leaf : 256;
  tuned[3] = h->dt.block_vert > 0 ? h->dt.block_vert : 256;
  return PIC_OK;
}

int pic_autotune(pic_t h, double dt, int32_t trials, int32_t *tuned) {
  if (check_handle(h)) return PIC_EINVAL;
  if (trials < 1) trials = 1;
  int rc;
  if ((rc = ensure_leaf(h))) return rc;
  const bool prof = h->prof;
  h->prof = false;
  Snapshot sn;
  if ((rc = snapshot_take(h, sn))) {
    free_bufs(h, sn.bufs);
    h->prof = prof;
    return rc;
  }
  std::vector<std::array<int32_t, 4>> cands;
  if (h->brick_ok) cands.push_back({1, 256, 256, 256});
  for (int32_t bp : {128, 256, 512})
    for (int32_t bl : {128, 256})
      cands.push_back({0, bp, bl, 256});
  cudaEvent_t e0 = take_event(h), e1 = take_event(h);
  float best = 1e30f;
  std::array<int32_t, 4> pick = cands[0];
  for (const auto &c : cands) {
    if ((rc = apply_tuning(h, c.data())) || (rc = snapshot_restore(h, sn))) break;
    if ((rc = deposit(h)) || (rc = push_and_rebin(h, dt))) break;  // warm-up
    CK(cudaEventRecord(e0, h->stream));
    for (int32_t i = 0; i < trials && !rc; ++i) {
      rc = deposit(h);
      if (!rc) rc = push_and_rebin(h, dt);
    }
    if (rc) break;
    CK(cudaEventRecord(e1, h->stream));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) {
      best = ms;
      pick = c;
    }
  }
  h->event_pool.push_back(e0);
  h->event_pool.push_back(e1);
  int rc2 = apply_tuning(h, pick.data());
  if (!rc2) rc2 = snapshot_restore(h, sn);
  if (!rc2) rc2 = cudaStreamSynchronize(h->stream) == cudaSuccess ? PIC_OK : PIC_ECUDA;
  free_bufs(h, sn.bufs);
  h->prof = prof;
  if (rc) return rc;
  if (rc2) return rc2;
  if (tuned) std::copy(pick.begin(), pick.end(), tuned);
  return PIC_OK;
}

int pic_set_wait_limit(pic_t h, int64_t cycles) {
  if (check_handle(h)) return PIC_EINVAL;
  if (cycles < 1000 || cycles > (int64_t)1 << 40) return fail(h, PIC_EINVAL, "wait limit outside [1e3, 2^40] cycles");
  h->wait_cycles = (long long)cycles;
  drop_graphs(h);  // captured launches carry the old limit
  return PIC_OK;
}

int pic_wait_selftest(int64_t cycles, void *stream) {
  if (cycles < 1 || cycles > (int64_t)1 << 40) return PIC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int32_t *flag = nullptr;
  if (cudaMalloc(&flag, sizeof(int32_t)) != cudaSuccess) return PIC_ENOMEM;
  int32_t got = 0;
  int rc = PIC_OK;
  if (cudaMemsetAsync(flag, 0, sizeof(int32_t), s) != cudaSuccess) rc = PIC_ECUDA;
  if (!rc) {
    launch_wait_selftest((long long)cycles, flag, s);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&got, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      rc = PIC_ECUDA;
  }
  cudaFree(flag);
  if (rc) return rc;
  return got == 1 ? PIC_ETIMEOUT : (got == 2 ? PIC_OK : PIC_ECUDA);
}

int pic_sync(pic_t h) {
  if (check_handle(h)) return PIC_EINVAL;
  int32_t err = 0;
  int rc = read_err(h, &err);
  if (rc) return rc;
  if (err & 1) return fail(h, PIC_ERANGE, "non-finite position or velocity");
  if (err & 8) return fail(h, PIC_ETIMEOUT, "a bounded device wait gave up");
  if (err) return fail(h, PIC_ESTATE, "device-side capacity exceeded (error bits " + std::to_string(err) + ")");
  return PIC_OK;
}

int pic_deposit(pic_t h, double *Q_out, int32_t where) {
  if (check_handle(h) || !Q_out) return PIC_EINVAL;
  int rc;
  if ((rc = deposit(h))) return rc;
  const int64_t nv = h->dt.n_vert;
  if (h->split) {
    launch_widen((const float *)h->Q, nv, (double *)h->Ep, h->stream);
    return copy_out(h, Q_out, h->Ep, sizeof(double) * nv, where);
  }
  return copy_out(h, Q_out, h->Q, sizeof(double) * nv, where);
}

int pic_field(pic_t h, double *E_out, int32_t where) {
  if (check_handle(h) || !E_out) return PIC_EINVAL;
  const int64_t m = h->dt.n_vert * h->d;
  if (h->split) {
    launch_widen((const float *)h->E, m, (double *)h->Ep, h->stream);
    return copy_out(h, E_out, h->Ep, sizeof(double) * m, where);
  }
  return copy_out(h, E_out, h->E, sizeof(double) * m, where);
}

int pic_potential(pic_t h, double *V_out, int32_t where) {
  if (check_handle(h) || !V_out) return PIC_EINVAL;
  const int64_t m = h->dt.n_vert;
  if (h->split) {
    launch_widen((const float *)h->V, m, (double *)h->Ep, h->stream);
    return copy_out(h, V_out, h->Ep, sizeof(double) * m, where);
  }
  return copy_out(h, V_out, h->V, sizeof(double) * m, where);
}

int pic_bins(pic_t h, int64_t *bucket_start, int32_t *perm, int32_t where) {
  if (check_handle(h)) return PIC_EINVAL;
  const int64_t nk = h->dt.n_keys;
  if (bucket_start) {
    std::vector<int32_t> st(nk + 1);
    CK(cudaMemcpyAsync(st.data(), h->start_cur, sizeof(int32_t) * (nk + 1), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    const int stride = h->scheme == PIC_PIT ? 1 : h->dt.nc;
    const int64_t nb = nk / stride;
    std::vector<int64_t> out(nb + 1);
    for (int64_t b = 0; b <= nb; ++b) out[b] = st[b * stride];
    if (where == PIC_HOST)
      std::memcpy(bucket_start, out.data(), sizeof(int64_t) * (nb + 1));
    else
      CK(cudaMemcpy(bucket_start, out.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice));
  }
  if (perm) {
    if (!h->cfg.track_ids) return fail(h, PIC_ESTATE, "particle ids are not tracked (track_ids = 0)");
    return copy_out(h, perm, h->ids[0], sizeof(int32_t) * h->n, where);
  }
  return PIC_OK;
}

int pic_keys(pic_t h, int32_t *keys, int32_t where) {
  if (check_handle(h) || !keys) return PIC_EINVAL;
  int rc = ensure_leaf(h);
  if (rc) return rc;
  return copy_out(h, keys, h->key[0], sizeof(int32_t) * h->n, where);
}

int pic_get_particles(pic_t h, double *x, double *v, int32_t where) {
  if (check_handle(h)) return PIC_EINVAL;
  const int64_t m = h->n * h->d;
  int rc;
  if ((rc = ensure_leaf(h))) return rc;
  if (h->split) {
    if (x) {
      launch_absolute_split(h->dt, h->leaf[0], (const float *)h->pos[0], h->n, (double *)h->Ep, h->stream);
      if ((rc = copy_out(h, x, h->Ep, sizeof(double) * m, where))) return rc;
    }
    if (v) {
      launch_widen((const float *)h->vel[0], m, (double *)h->Ep, h->stream);
      if ((rc = copy_out(h, v, h->Ep, sizeof(double) * m, where))) return rc;
    }
    return PIC_OK;
  }
  if ((rc = copy_out(h, x, h->pos[0], sizeof(double) * m, where))) return rc;
  return copy_out(h, v, h->vel[0], sizeof(double) * m, where);
}

int pic_get_state(pic_t h, int32_t *leaf, void *x_or_o, void *v, int32_t where) {
  if (check_handle(h)) return PIC_EINVAL;
  int rc0 = ensure_leaf(h);
  if (rc0) return rc0;
  const size_t fs = h->split ? sizeof(float) : sizeof(double);
  const size_t m = (size_t)h->n * h->d;
  cudaMemcpyKind kind = where == PIC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (leaf) CK(cudaMemcpyAsync(leaf, h->leaf[0], sizeof(int32_t) * h->n, kind, h->stream));
  if (x_or_o) CK(cudaMemcpyAsync(x_or_o, h->pos[0], fs * m, kind, h->stream));
  if (v) CK(cudaMemcpyAsync(v, h->vel[0], fs * m, kind, h->stream));
  if (where == PIC_HOST) CK(cudaStreamSynchronize(h->stream));
  return PIC_OK;
}

int pic_set_state(pic_t h, const int32_t *leaf, const void *x_or_o, const void *v, int32_t where) {
  if (check_handle(h) || !x_or_o || !v) return PIC_EINVAL;
  drop_graphs(h);
  if (h->split && !leaf) return fail(h, PIC_EINVAL, "split state needs the leaf array");
  const size_t fs = h->split ? sizeof(float) : sizeof(double);
  const size_t m = (size_t)h->n * h->d;
  int rc;
  if ((rc = copy_in(h, h->pos[1], x_or_o, fs * m, where))) return rc;
  if ((rc = copy_in(h, h->vel[1], v, fs * m, where))) return rc;
  if (h->split) {
    if ((rc = copy_in(h, h->leaf[1], leaf, sizeof(int32_t) * h->n, where))) return rc;
    launch_rekey32(h->dt, h->leaf[1], (const float *)h->pos[1], h->n, h->key[1], h->err, h->stream);
    CK(cudaGetLastError());
    return bin_fresh(h);
  }
  launch_init64(h->dt, (double *)h->pos[1], h->n, h->leaf[1], h->key[1], h->err, h->stream);
  CK(cudaGetLastError());
  return bin_fresh(h);
}

int pic_stats(pic_t h, pic_stats_t *o) {
  if (check_handle(h) || !o) return PIC_EINVAL;
  int32_t sc[8];
  double tot, r2;
  int32_t err;
  CK(cudaMemcpyAsync(sc, h->scalars, sizeof(sc), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(&tot, h->total, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(&r2, h->resid2, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(&err, h->err, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  o->step = h->step;
  o->movers = sc[1];
  o->max_bucket = sc[2];
  o->total_charge = tot;
  o->residual = std::sqrt(r2);
  o->error = (err & 1) ? PIC_ERANGE : (err & 8) ? PIC_ETIMEOUT : (err ? PIC_ESTATE : PIC_OK);
  o->tunnellers = -1;
  if (h->count_lifts) {
    unsigned long long c[3] = {0, 0, 0};
    CK(cudaMemcpyAsync(c, h->lift_counts, sizeof(c), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    o->tunnellers = (int64_t)c[2];
  }
  return PIC_OK;
}

int pic_profile(pic_t h, int32_t enable) {
  if (check_handle(h)) return PIC_EINVAL;
  int rc = drain_profile(h);
  if (rc) return rc;
  for (int i = 0; i < PIC_NPHASES; ++i) {
    h->phase_ms[i] = 0.0;
    h->phase_kernels[i] = 0;
  }
  h->prof = enable != 0;
  return PIC_OK;
}

int pic_phase_times(pic_t h, double *ms, int64_t *kernels) {
  if (check_handle(h)) return PIC_EINVAL;
  int rc = drain_profile(h);
  if (rc) return rc;
  for (int i = 0; i < PIC_NPHASES; ++i) {
    if (ms) ms[i] = h->phase_ms[i];
    if (kernels) kernels[i] = h->phase_kernels[i];
  }
  return PIC_OK;
}

int pic_leaf_table(pic_t h, int32_t *level, int64_t *coords) {
  if (check_handle(h)) return PIC_EINVAL;
  int64_t base = 0;
  for (const auto &t : h->hts) {
    for (int64_t l = 0; l < t.n_leaves; ++l) {
      if (level) level[base + l] = t.leaf_level[l];
      if (coords)
        for (int a = 0; a < t.d; ++a) coords[(base + l) * t.d + a] = t.leaf_coords[l * t.d + a];
    }
    base += t.n_leaves;
  }
  return PIC_OK;
}

int pic_vertex_table(pic_t h, int64_t *pos) {
  if (check_handle(h) || !pos) return PIC_EINVAL;
  const int64_t nv = h->dt.n_vert;
  std::vector<int64_t> dkeys;  // vertex keys of device-tabulated tables
  if (h->grid_dev) {
    dkeys.resize(nv);
    CK(cudaMemcpy(dkeys.data(), h->gdev.vert_key, sizeof(int64_t) * nv, cudaMemcpyDeviceToHost));
  }
  int64_t base = 0;
  for (const auto &t : h->hts) {
    for (int64_t v = 0; v < t.n_vert; ++v) {
      int64_t k = t.uniform ? v : (h->grid_dev ? dkeys[v] : t.vert_key[v]);
      for (int a = 0; a < t.d; ++a) {
        pos[a * nv + base + v] = k % t.M;
        k /= t.M;
      }
    }
    base += t.n_vert;
  }
  return PIC_OK;
}

int pic_tree_tabulate(int32_t d, const uint8_t *flags, int64_t n_flags, pic_tree_sizes_t *sizes,
                      int64_t *vertex_pos, double *ion_load, double *diag, int32_t *cexp_ptr, int32_t *cexp_vid,
                      double *cexp_w, int32_t *pidt_level, int64_t *pidt_j) {
  if (!sizes || !flags || n_flags < 1) return PIC_EINVAL;
  HostTree t;
  std::string err;
  if (t.build(d, n_flags, flags, &err)) return PIC_EINVAL;
  if (t.depth > 12 && !t.uniform) return PIC_EINVAL;  // as pic_create
  t.build_grid();
  t.build_pidt();
  sizes->d = t.d;
  sizes->depth = t.depth;
  sizes->uniform = t.uniform ? 1 : 0;
  sizes->reserved = 0;
  sizes->n_leaves = t.n_leaves;
  sizes->n_vertices = t.n_vert;
  sizes->n_corner_entries = t.uniform ? 0 : (int64_t)t.cexp_vid.size();
  sizes->n_pidt_vertices = t.n_pv;
  const int64_t nv = t.n_vert;
  if (vertex_pos)
    for (int64_t v = 0; v < nv; ++v) {
      int64_t k = t.uniform ? v : t.vert_key[v];
      for (int a = 0; a < t.d; ++a) {
        vertex_pos[a * nv + v] = k % t.M;
        k /= t.M;
      }
    }
  for (int64_t v = 0; v < t.n_pv; ++v) {
    int64_t k = v;
    if (pidt_level) pidt_level[v] = t.uniform ? t.depth : t.pv_level[v];
    if (pidt_j)
      for (int a = 0; a < t.d; ++a) {
        pidt_j[v * t.d + a] = t.uniform ? k % t.M : t.pv_j[v * t.d + a];
        k /= t.M;
      }
  }
  if (!t.uniform) {
    if (ion_load) std::copy(t.ion_load.begin(), t.ion_load.end(), ion_load);
    if (diag) std::copy(t.diag.begin(), t.diag.end(), diag);
    if (cexp_ptr) std::copy(t.cexp_ptr.begin(), t.cexp_ptr.end(), cexp_ptr);
    if (cexp_vid) std::copy(t.cexp_vid.begin(), t.cexp_vid.end(), cexp_vid);
    if (cexp_w) std::copy(t.cexp_w.begin(), t.cexp_w.end(), cexp_w);
  }
  return PIC_OK;
}

int pic_grid_tables(pic_t h, int64_t *n_entries, int32_t *cexp_ptr, int32_t *cexp_vid, double *cexp_w,
                    double *ion_load, double *diag) {
  if (check_handle(h)) return PIC_EINVAL;
  if (h->dt.n_inst != 1 || h->dt.uniform)
    return fail(h, PIC_ESTATE, "grid tables belong to single-instance handles with an adaptive tree");
  const int64_t nlc = h->dt.n_leaves * h->dt.nc, nv = h->dt.n_vert;
  int32_t nnz = 0;
  CK(cudaMemcpy(&nnz, h->dt.cexp_ptr + nlc, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (n_entries) *n_entries = nnz;
  if (cexp_ptr) CK(cudaMemcpy(cexp_ptr, h->dt.cexp_ptr, sizeof(int32_t) * (nlc + 1), cudaMemcpyDeviceToHost));
  if (cexp_vid) CK(cudaMemcpy(cexp_vid, h->dt.cexp_vid, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost));
  if (cexp_w) CK(cudaMemcpy(cexp_w, h->dt.cexp_w64, sizeof(double) * nnz, cudaMemcpyDeviceToHost));
  if (ion_load) CK(cudaMemcpy(ion_load, h->dt.ion64, sizeof(double) * nv, cudaMemcpyDeviceToHost));
  if (diag) CK(cudaMemcpy(diag, h->dt.diag64, sizeof(double) * nv, cudaMemcpyDeviceToHost));
  return PIC_OK;
}

int pic_pidt_table(pic_t h, int32_t *level, int64_t *j) {
  if (check_handle(h)) return PIC_EINVAL;
  if (h->scheme != PIC_PIDT) return fail(h, PIC_ESTATE, "owner-vertex tables belong to PIDT handles");
  if (h->grid_dev) {  // one adaptive instance, tabulated on the device
    const HostTree &t = h->ht0();
    std::vector<int32_t> pl(t.n_pv), pj(t.n_pv * t.d);
    CK(cudaMemcpy(pl.data(), h->gdev.pv_level, sizeof(int32_t) * pl.size(), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(pj.data(), h->gdev.pv_j, sizeof(int32_t) * pj.size(), cudaMemcpyDeviceToHost));
    for (int64_t v = 0; v < t.n_pv; ++v) {
      if (level) level[v] = pl[v];
      if (j)
        for (int a = 0; a < t.d; ++a) j[v * t.d + a] = pj[v * t.d + a];
    }
    return PIC_OK;
  }
  int64_t base = 0;
  for (auto &t : h->hts) {
    t.build_pidt();
    for (int64_t v = 0; v < t.n_pv; ++v) {
      if (t.uniform) {
        if (level) level[base + v] = t.depth;
        int64_t k = v;
        for (int a = 0; a < t.d; ++a) {
          if (j) j[(base + v) * t.d + a] = k % t.M;
          k /= t.M;
        }
      } else {
        if (level) level[base + v] = t.pv_level[v];
        if (j)
          for (int a = 0; a < t.d; ++a) j[(base + v) * t.d + a] = t.pv_j[v * t.d + a];
      }
    }
    base += t.n_pv;
  }
  return PIC_OK;
}

int pic_retree(pic_t h, const pic_tree_desc *tree) {
  if (check_handle(h) || !tree) return PIC_EINVAL;
  if (h->dt.n_inst > 1) return fail(h, PIC_ESTATE, "re-tree of batched handles is not supported");
  drop_graphs(h);
  if (tree->d != h->d) return fail(h, PIC_EINVAL, "tree dimension differs from the handle");
  int rc;
  if ((rc = ensure_leaf(h))) return rc;
  cudaStream_t s = h->stream;
  const int64_t n = h->n;
  // the particles stay in state [0] (storage order) while the tree and the
  // tree-sized buffers are rebuilt; the particle-sized buffers are kept and
  // the re-located state lands in [1]
  const DevTree old_dt = h->dt;
  std::vector<DevBuf> old_tree;
  if ((rc = install_tree(h, tree, &old_tree))) return rc;
  if ((rc = alloc_grid(h))) {
    free_bufs(h, old_tree);
    return rc;
  }
  CK(cudaMemsetAsync(h->err, 0, sizeof(int32_t), s));
  CK(cudaMemsetAsync(h->scalars, 0, sizeof(int32_t) * 8, s));
  if (h->split) {
    launch_relocate32(old_dt, h->dt, h->leaf[0], (const float *)h->pos[0], (const float *)h->vel[0], n,
                      h->leaf[1], (float *)h->pos[1], (float *)h->vel[1], s);
    launch_rekey32(h->dt, h->leaf[1], (const float *)h->pos[1], n, h->key[1], h->err, s);
  } else {
    std::swap(h->pos[0], h->pos[1]);  // FP64 positions do not change
    std::swap(h->vel[0], h->vel[1]);
    launch_init64(h->dt, (double *)h->pos[1], n, h->leaf[1], h->key[1], h->err, s);
  }
  CK(cudaGetLastError());
  if ((rc = bin_fresh(h))) {
    free_bufs(h, old_tree);
    return rc;
  }
  CK(cudaStreamSynchronize(s));  // the re-location read the old tables
  drop_spares(h, h->tree_gen);    // spares of earlier re-trees that this one did not take
  retire(h, old_tree);
  h->leaf_stale = false;
  h->q_valid = false;
  return setup_brick(h);
}

int pic_adapt(pic_t h, int64_t ppc, int32_t dmin, int32_t dmax) {
  if (check_handle(h)) return PIC_EINVAL;
  if (h->dt.n_inst > 1) return fail(h, PIC_ESTATE, "re-refinement of batched handles is not supported");
  const int d = h->d;
  if (ppc < 0 || dmin < 0 || dmin > dmax || dmax > (d == 3 ? 6 : 10))
    return fail(h, PIC_EINVAL, "adapt needs 0 <= dmin <= dmax <= 6 (3D) or 10 (2D)");
  int rc;
  if ((rc = ensure_leaf(h))) return rc;
  cudaStream_t s = h->stream;
  const int64_t n = h->n;
  const int nch = (int)pow3(d);
  // particles per cell on every decision level dmin .. dmax-1: one count on
  // level dmax-1, summed child by child up to dmin; one bit per cell (count
  // above ppc), every level's bits in one array read back at once
  std::vector<int64_t> coff(dmax + 1, 0), boff(dmax + 1, 0);
  int64_t cells = 0, words = 0;
  for (int m = dmin; m < dmax; ++m) {
    coff[m] = cells;
    boff[m] = words;
    cells += pow3(d * m);
    words += (pow3(d * m) + 31) / 32;
  }
  std::vector<uint32_t> bits(std::max<int64_t>(words, 1));
  if (dmax > dmin) {
    if (cells > h->adapt_cells || words > h->adapt_words) {
      free_bufs(h, h->adapt_bufs);
      h->adapt_cells = h->adapt_words = 0;
      if ((rc = dalloc(h, h->adapt_bufs, &h->adapt_count, cells)) ||
          (rc = dalloc(h, h->adapt_bufs, &h->adapt_bits, words)))
        return rc;
      h->adapt_cells = cells;
      h->adapt_words = words;
    }
    uint32_t *key = (uint32_t *)h->perm;  // scratch until the next re-bin
    launch_fine_keys(h->dt, h->split, h->pos[0], h->leaf[0], n, dmax, key, s);
    launch_adapt_bits(key, n, nch, dmin, dmax, ppc, h->adapt_count, coff.data(), h->adapt_bits, boff.data(), s);
  }
  // the criterion on the installed tree's leaves first: when it keeps the
  // tree, no flags are built
  {
    int32_t *changed = h->scalars + 7;  // free between re-bins
    CK(cudaMemsetAsync(changed, 0, sizeof(int32_t), s));
    launch_adapt_check(h->dt, h->adapt_count, coff.data(), dmin, dmax, ppc, changed, s);
    int32_t ch = 1;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&ch, changed, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (!ch) return reset_grid_state(h);
  }
  if (dmax > dmin) {
    CK(cudaMemcpyAsync(bits.data(), h->adapt_bits, sizeof(uint32_t) * words, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  // level-order flags: refined iff level < dmin, or level < dmax and the
  // cell holds more than ppc particles.  A cell is named by its index on its
  // level, base-3^d digits from the root (child ch of cell L: L 3^d + ch).
  std::vector<uint8_t> flags;
  flags.reserve(h->ht0().n_nodes + 64);
  std::vector<int64_t> cur(1, 0), nxt;
  for (int m = 0; m <= dmax && !cur.empty(); ++m) {
    nxt.clear();
    const uint32_t *bm = bits.data() + boff[m];
    for (int64_t L : cur) {
      bool refine = m < dmin;
      if (!refine && m < dmax) refine = (bm[L >> 5] >> (L & 31)) & 1u;
      flags.push_back(refine ? 1 : 0);
      if (refine)
        for (int ch = 0; ch < nch; ++ch) nxt.push_back(L * nch + ch);
    }
    cur.swap(nxt);
  }
  // the same tree: every particle keeps its bucket, and its storage order is
  // already the stable order by key that a re-tree produces
  const HostTree &t = h->ht0();
  bool same = (int64_t)flags.size() == t.n_nodes;
  for (int64_t i = 0; same && i < t.n_nodes; ++i) same = (t.child0[i] >= 0) == (flags[i] != 0);
  if (same) return reset_grid_state(h);
  pic_tree_desc td{d, (int64_t)flags.size(), flags.data()};
  return pic_retree(h, &td);
}

int pic_vmax(pic_t h, double *node_vmax, double dt, int64_t *n_closed) {
  if (check_handle(h)) return PIC_EINVAL;
  if (h->dt.n_inst > 1) return fail(h, PIC_ESTATE, "v_max is kept for single-instance handles");
  int rc;
  if ((rc = ensure_leaf(h))) return rc;
  const auto &t = h->ht0();
  std::vector<int64_t> lb(t.depth + 2, t.n_nodes);
  for (int64_t i = t.n_nodes - 1; i >= 0; --i) lb[t.level[i]] = i;  // level order: first node of each level
  for (int l = t.depth; l >= 0; --l) lb[l] = std::min(lb[l], lb[l + 1]);
  std::vector<DevBuf> tmp;
  const int32_t *c0 = nullptr, *lon = nullptr;
  double *leaf_v = nullptr, *node_v = nullptr;
  if ((rc = upload(h, tmp, &c0, t.child0)) || (rc = upload(h, tmp, &lon, t.leaf_of_node)) ||
      (rc = dalloc(h, tmp, &leaf_v, std::max<int64_t>(t.n_leaves, 1))) ||
      (rc = dalloc(h, tmp, &node_v, std::max<int64_t>(t.n_nodes, 1)))) {
    free_bufs(h, tmp);
    return rc;
  }
  launch_vmax(h->dt, h->split, h->start_cur, h->vel[0], h->n, c0, lon, lb.data(), t.depth, leaf_v, node_v,
              h->stream);
  std::vector<double> out(t.n_nodes);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out.data(), node_v, sizeof(double) * t.n_nodes, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  free_bufs(h, tmp);
  if (e != cudaSuccess) return cuda_fail(h, e, "v_max");
  if (node_vmax) std::copy(out.begin(), out.end(), node_vmax);
  if (n_closed) {
    // cells no particle can leave by a lift within dt: v_max dt < h = 3^-level
    int64_t c = 0;
    for (int64_t i = 0; i < t.n_nodes; ++i)
      if (out[i] * dt < 1.0 / (double)pow3(t.level[i])) ++c;
    *n_closed = c;
  }
  return PIC_OK;
}

int pic_tree_flags(pic_t h, uint8_t *flags, int64_t *n_nodes) {
  if (check_handle(h)) return PIC_EINVAL;
  int64_t total = 0;
  for (const auto &t : h->hts) {
    if (flags)
      for (int64_t i = 0; i < t.n_nodes; ++i) flags[total + i] = t.child0[i] >= 0 ? 1 : 0;
    total += t.n_nodes;
  }
  if (n_nodes) *n_nodes = total;
  return PIC_OK;
}

int pic_set_allocator(pic_alloc_fn alloc, pic_free_fn free_fn, void *user) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return PIC_EINVAL;
  std::lock_guard<std::mutex> lock(g_alloc_mu);
  g_alloc_fn = alloc;
  g_free_fn = free_fn;
  g_alloc_user = alloc ? user : nullptr;
  return PIC_OK;
}

int pic_save(pic_t h, const char *path) {
  if (check_handle(h) || !path) return PIC_EINVAL;
  int rc;
  int32_t err = 0;
  if ((rc = read_err(h, &err))) return rc;
  if (err) return fail(h, PIC_ESTATE, "the handle holds a sticky device error; nothing was saved");
  SnapshotMeta m;
  m.d = h->d;
  m.scheme = h->scheme;
  m.precision = h->split ? PIC_FP32_SPLIT : PIC_FP64;
  m.sweeps = h->cfg.sweeps;
  m.track_ids = h->cfg.track_ids ? 1 : 0;
  m.path = h->cfg.path == PIC_PATH_GENERIC ? PIC_PATH_GENERIC : PIC_PATH_AUTO;
  m.n_inst = (int32_t)h->hts.size();
  m.q = h->cfg.q;
  m.qm = h->cfg.qm;
  m.ion = h->cfg.ion;
  m.omega = h->cfg.omega;
  m.step = h->step;
  m.n = h->n;
  m.n_vert = h->dt.n_vert;
  if ((rc = pic_get_tuning(h, m.tuned))) return rc;
  for (int32_t i = 0; i < m.n_inst; ++i) {
    m.inst_flags.push_back(h->hts[i].n_nodes);
    const int64_t end = i + 1 < m.n_inst ? h->inst[i + 1].poff : h->n;
    m.inst_n.push_back(end - h->inst[i].poff);
    m.inst_q.push_back(h->inst[i].q);
  }
  SnapshotArrays a;
  int64_t n_nodes = 0;
  if ((rc = pic_tree_flags(h, nullptr, &n_nodes))) return rc;
  a.flags.resize(n_nodes);
  if ((rc = pic_tree_flags(h, a.flags.data(), nullptr))) return rc;
  const size_t fs = h->split ? sizeof(float) : sizeof(double);
  const size_t n = (size_t)h->n, d = (size_t)h->d, nv = (size_t)h->dt.n_vert;
  a.pos.resize(fs * d * n);
  a.vel.resize(fs * d * n);
  if (h->split) a.leaf.resize(n);
  if ((rc = pic_get_state(h, h->split ? a.leaf.data() : nullptr, a.pos.data(), a.vel.data(), PIC_HOST))) return rc;
  if (m.track_ids) {
    a.ids.resize(n);
    if ((rc = copy_out(h, a.ids.data(), h->ids[0], sizeof(int32_t) * n, PIC_HOST))) return rc;
  }
  a.V.resize(fs * nv);
  a.E.resize(fs * d * nv);
  if ((rc = copy_out(h, a.V.data(), h->V, a.V.size(), PIC_HOST)) ||
      (rc = copy_out(h, a.E.data(), h->E, a.E.size(), PIC_HOST)))
    return rc;
  std::string msg;
  if ((rc = snapshot_write(path, m, a, &msg))) return fail(h, rc, msg);
  return PIC_OK;
}

static int load_fail(int rc, const std::string &msg) {
  t_last_error = msg;
  return rc;
}

int pic_load(pic_t *out, const char *path, void *stream) {
  if (!out) return PIC_EINVAL;
  *out = nullptr;
  t_last_error.clear();
  SnapshotMeta m;
  SnapshotArrays a;
  std::string msg;
  int rc = snapshot_read(path, m, a, &msg);
  if (rc) return load_fail(rc, msg);
  const bool split = m.precision == PIC_FP32_SPLIT;
  const int d = m.d;
  const int64_t n = m.n;
  // Trees, and a creation position for every particle.  The creation
  // positions only size and order the new handle: the saved state replaces
  // them below.  FP64: the saved positions themselves.  Split: the centre of
  // the particle's leaf.  Velocities at creation are zero, likewise replaced.
  std::vector<pic_tree_desc> trees(m.n_inst);
  std::vector<pic_particles_desc> parts(m.n_inst);
  std::vector<int64_t> leaf_off(m.n_inst + 1, 0);
  std::vector<double> x0((size_t)d * n), v0((size_t)d * n, 0.0);
  int64_t foff = 0, poff = 0;
  for (int32_t i = 0; i < m.n_inst; ++i) {
    const int64_t ni = m.inst_n[i];
    trees[i] = {d, m.inst_flags[i], a.flags.data() + foff};
    double *xi = x0.data() + (size_t)d * poff;
    parts[i] = {ni, xi, v0.data() + (size_t)d * poff, PIC_HOST};
    if (split) {
      HostTree t;
      std::string terr;
      if (t.build(d, m.inst_flags[i], a.flags.data() + foff, &terr))
        return load_fail(PIC_EINVAL, "instance " + std::to_string(i) + ": " + terr);
      leaf_off[i + 1] = leaf_off[i] + t.n_leaves;
      for (int64_t k = 0; k < ni; ++k) {
        const int64_t L = a.leaf[poff + k] - leaf_off[i];
        if (L < 0 || L >= t.n_leaves)
          return load_fail(PIC_EINVAL, "particle " + std::to_string(poff + k) + " names a leaf outside its instance");
        const double w = std::pow(3.0, -(double)t.leaf_level[L]);
        for (int ax = 0; ax < d; ++ax) xi[ax * ni + k] = ((double)t.leaf_coords[L * d + ax] + 0.5) * w;
      }
    } else {
      const double *x = (const double *)a.pos.data();
      for (int ax = 0; ax < d; ++ax)
        for (int64_t k = 0; k < ni; ++k) xi[ax * ni + k] = x[ax * n + poff + k];
    }
    foff += m.inst_flags[i];
    poff += ni;
  }
  if (split && (rc = snapshot_check_leaves(m, a, leaf_off, &msg))) return load_fail(rc, msg);
  pic_config cfg{};
  cfg.scheme = m.scheme;
  cfg.precision = m.precision;
  cfg.q = m.q;
  cfg.qm = m.qm;
  cfg.ion = m.ion;
  cfg.sweeps = m.sweeps;
  cfg.omega = m.omega;
  cfg.track_ids = m.track_ids;
  cfg.stream = stream;
  cfg.path = m.path;
  pic_t h = nullptr;
  rc = create_forest(&h, m.n_inst, trees.data(), parts.data(), m.inst_q.data(), &cfg);
  std::vector<double>().swap(x0);
  std::vector<double>().swap(v0);
  if (rc) return load_fail(rc, "creating the handle from the checkpoint failed");
  auto bail = [&](int code, const std::string &why) {
    t_last_error = why.empty() ? h->last_error : why;
    pic_destroy(h);
    return code;
  };
  if (h->n != n || h->dt.n_vert != m.n_vert) return bail(PIC_EIO, "the checkpoint does not match its own tree");
  // ids first: pic_set_state permutes them along with the particles if the
  // saved order is not already bucket order
  if (m.track_ids && n > 0 && (rc = copy_in(h, h->ids[0], a.ids.data(), sizeof(int32_t) * n, PIC_HOST)))
    return bail(rc, "");
  if (n > 0 && (rc = pic_set_state(h, split ? a.leaf.data() : nullptr, a.pos.data(), a.vel.data(), PIC_HOST)))
    return bail(rc, "");
  if ((rc = copy_in(h, h->V, a.V.data(), a.V.size(), PIC_HOST)) ||
      (rc = copy_in(h, h->E, a.E.data(), a.E.size(), PIC_HOST)))
    return bail(rc, "");
  h->ecorner_valid = false;
  h->ebrick_valid = false;
  if ((rc = apply_tuning(h, m.tuned))) return bail(rc, "");
  h->step = m.step;
  int32_t err = 0;
  if ((rc = read_err(h, &err))) return bail(rc, "");
  if (err) return bail(PIC_EINVAL, "the saved particle state is out of range for its tree");
  *out = h;
  return PIC_OK;
}

}  // extern "C"
