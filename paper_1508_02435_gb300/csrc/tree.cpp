// Host-side spacetree tabulation; see tree.hpp.
#include "tree.hpp"

#include <algorithm>
#include <condition_variable>
#include <cstdlib>
#include <functional>
#include <memory>
#include <mutex>
#include <thread>

namespace pic {

int HostTree::build(int d_, int64_t n_flags, const uint8_t *flags, std::string *err) {
  if (d_ != 2 && d_ != 3) { *err = "d must be 2 or 3"; return -1; }
  if (n_flags < 1 || !flags) { *err = "empty tree"; return -1; }
  if (n_flags > INT32_MAX - 64) { *err = "tree too large"; return -1; }
  d = d_;
  pidt_built = false;
  nch = (int)pow3(d);
  nc = 1 << d;
  n_nodes = n_flags;
  level.assign(n_nodes, 0);
  child0.assign(n_nodes, -1);
  coords.assign(n_nodes * 3, 0);
  int64_t next = 1;
  depth = 0;
  n_leaves = 0;
  for (int64_t i = 0; i < n_nodes; ++i) {
    if (i >= next) { *err = "more flags than tree nodes"; return -1; }
    if (flags[i]) {
      if (level[i] >= kMaxLevel) { *err = "tree deeper than level 18"; return -1; }
      if (next + nch > n_nodes) { *err = "refined node without 3^d children"; return -1; }
      child0[i] = (int32_t)next;
      for (int c = 0; c < nch; ++c) {
        int64_t k = next + c;
        level[k] = level[i] + 1;
        int64_t dig = c;
        for (int a = 0; a < d; ++a) {
          coords[k * 3 + a] = 3 * coords[i * 3 + a] + dig % 3;
          dig /= 3;
        }
      }
      depth = std::max(depth, level[i] + 1);
      next += nch;
    } else {
      ++n_leaves;
    }
  }
  if (next != n_nodes) { *err = "flag count does not match the tree"; return -1; }
  if (n_leaves > INT32_MAX / 8) { *err = "too many leaves"; return -1; }

  // depth-first leaf numbering
  leaf_of_node.assign(n_nodes, -1);
  leaf_node.assign(n_leaves, 0);
  {
    std::vector<int32_t> stack;
    stack.reserve(1024);
    stack.push_back(0);
    int32_t nl = 0;
    while (!stack.empty()) {
      int32_t nd = stack.back();
      stack.pop_back();
      if (child0[nd] < 0) {
        leaf_of_node[nd] = nl;
        leaf_node[nl++] = nd;
      } else {
        for (int c = nch - 1; c >= 0; --c) stack.push_back(child0[nd] + c);
      }
    }
  }
  // complete-subtree depth per node (children have larger indices)
  std::vector<int8_t> cd(n_nodes, 0);
  for (int64_t i = n_nodes - 1; i >= 0; --i) {
    if (child0[i] < 0) { cd[i] = 0; continue; }
    int k = cd[child0[i]];
    for (int c = 1; c < nch && k >= 0; ++c)
      if (cd[child0[i] + c] != k) k = -1;
    cd[i] = (int8_t)(k < 0 ? -1 : k + 1);
  }
  uniform = cd[0] == depth;
  // leftmost leaf of every subtree
  auto leftmost = [&](int32_t nd) {
    while (child0[nd] >= 0) nd = child0[nd];
    return leaf_of_node[nd];
  };
  // breadth-first descent table
  tab.clear();
  tab.push_back({0, 0});
  std::vector<std::pair<int32_t, int32_t>> queue;  // (node, entry)
  queue.push_back({0, 0});
  for (size_t qi = 0; qi < queue.size(); ++qi) {
    int32_t nd = queue[qi].first, ent = queue[qi].second;
    if (cd[nd] >= 0) {
      tab[ent] = {-(int32_t)cd[nd] - 1, leftmost(nd)};
    } else {
      int32_t base = (int32_t)tab.size();
      tab[ent] = {base, 0};
      for (int c = 0; c < nch; ++c) {
        tab.push_back({0, 0});
        queue.push_back({child0[nd] + c, base + c});
      }
    }
  }
  leaf_level.resize(n_leaves);
  leaf_coords.resize(n_leaves * d);
  for (int64_t l = 0; l < n_leaves; ++l) {
    int32_t nd = leaf_node[l];
    leaf_level[l] = (uint8_t)level[nd];
    for (int a = 0; a < d; ++a) leaf_coords[l * d + a] = (int32_t)coords[nd * 3 + a];
  }
  M = pow3(depth);
  return 0;
}

namespace {

// Reference stiffness of -Laplace on the unit cell, d-linear elements, by the
// number of axes in which the two corners differ.
double kref(int d, int e, int f) {
  int diff = __builtin_popcount((unsigned)(e ^ f));
  if (d == 2) {
    const double k2[3] = {4.0 / 6.0, -1.0 / 6.0, -2.0 / 6.0};
    return k2[diff];
  }
  const double k3[4] = {4.0 / 12.0, 0.0, -1.0 / 12.0, -1.0 / 12.0};
  return k3[diff];
}

// Host threads for the tabulation: PIC_HOST_THREADS if set (1..64), else the
// hardware concurrency (at most 32).  The tables do not depend on it.
unsigned host_threads() {
  if (const char *env = std::getenv("PIC_HOST_THREADS")) {
    const long v = std::strtol(env, nullptr, 10);
    if (v >= 1 && v <= 64) return (unsigned)v;
  }
  const unsigned hw = std::thread::hardware_concurrency();
  return std::max(1u, std::min(hw == 0 ? 1u : hw, 32u));
}

// Worker threads started once per process; one job at a time (jobs from
// several handles queue on job_mu_).  The calling thread takes tasks as
// well, so a job completes with any number of workers, none included.
class Pool {
 public:
  explicit Pool(unsigned workers) {
    for (unsigned i = 0; i < workers; ++i) std::thread([this] { loop(); }).detach();
  }
  void run(unsigned tasks, const std::function<void(unsigned)> &fn) {
    std::lock_guard<std::mutex> job(job_mu_);
    std::unique_lock<std::mutex> lk(mu_);
    fn_ = &fn;
    tasks_ = tasks;
    next_ = done_ = 0;
    ++gen_;
    cv_.notify_all();
    work(lk);
    done_cv_.wait(lk, [&] { return done_ == tasks_; });
    fn_ = nullptr;
  }

 private:
  void work(std::unique_lock<std::mutex> &lk) {
    while (next_ < tasks_) {
      const unsigned t = next_++;
      const std::function<void(unsigned)> *fn = fn_;
      lk.unlock();
      (*fn)(t);
      lk.lock();
      if (++done_ == tasks_) done_cv_.notify_all();
    }
  }
  void loop() {
    std::unique_lock<std::mutex> lk(mu_);
    uint64_t seen = 0;
    for (;;) {
      cv_.wait(lk, [&] { return gen_ != seen; });
      seen = gen_;
      work(lk);
    }
  }
  std::mutex job_mu_, mu_;
  std::condition_variable cv_, done_cv_;
  const std::function<void(unsigned)> *fn_ = nullptr;
  unsigned tasks_ = 0, next_ = 0, done_ = 0;
  uint64_t gen_ = 0;
};

Pool &pool() {
  static Pool *p = new Pool(host_threads() - 1);  // lives as long as the process
  return *p;
}

// Runs fn(t, lo, hi) for t < nt over [0, n) split into nt equal chunks.
template <typename F>
void parallel_chunks(int64_t n, unsigned nt, F fn) {
  if (nt <= 1) {
    fn(0u, (int64_t)0, n);
    return;
  }
  pool().run(nt, [&](unsigned t) { fn(t, n * t / nt, n * (t + 1) / nt); });
}

// Chunks for a loop of n items: one per 16 Ki items, at most one per thread.
unsigned chunks_for(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(host_threads(), n >> 14));
}

// Stable LSD radix sort of records by the 64-bit value key(rec), 11 bits a
// pass, passes on host threads over contiguous chunks (counts per chunk, then
// bucket-major offsets, so equal keys keep their order).
template <typename Rec, typename Key>
void radix_sort(std::unique_ptr<Rec[]> &r, int64_t n, uint64_t key_max, Key key) {
  constexpr int kBits = 11;
  constexpr size_t kBuckets = size_t(1) << kBits;
  const unsigned nt = chunks_for(n);
  std::unique_ptr<Rec[]> tmp(new Rec[n > 0 ? n : 1]);
  std::vector<int64_t> cnt((size_t)nt * kBuckets);
  for (int shift = 0; shift < 64 && (shift == 0 || (key_max >> shift) != 0); shift += kBits) {
    auto digit = [&](const Rec &x) { return (size_t)((key(x) >> shift) & (kBuckets - 1)); };
    parallel_chunks(n, nt, [&](unsigned t, int64_t lo, int64_t hi) {
      int64_t *c = cnt.data() + (size_t)t * kBuckets;
      std::fill(c, c + kBuckets, 0);
      for (int64_t i = lo; i < hi; ++i) c[digit(r[i])]++;
    });
    int64_t run = 0;
    for (size_t k = 0; k < kBuckets; ++k)
      for (unsigned t = 0; t < nt; ++t) {
        const int64_t v = cnt[(size_t)t * kBuckets + k];
        cnt[(size_t)t * kBuckets + k] = run;
        run += v;
      }
    parallel_chunks(n, nt, [&](unsigned t, int64_t lo, int64_t hi) {
      int64_t *c = cnt.data() + (size_t)t * kBuckets;
      for (int64_t i = lo; i < hi; ++i) tmp[c[digit(r[i])]++] = r[i];
    });
    r.swap(tmp);
  }
}

}  // namespace

void HostTree::build_grid() {
  if (uniform) {
    n_vert = 1;
    for (int a = 0; a < d; ++a) n_vert *= M;
    double h = 1.0 / (double)M, vol = 1.0;
    for (int a = 0; a < d; ++a) vol *= h;
    ion_load.assign(1, vol);
    double hs = d == 2 ? 1.0 : h;
    diag.assign(1, (double)nc * kref(d, 0, 0) * hs);
    return;
  }
  auto key_of = [&](const int64_t p[3]) {
    int64_t k = 0, m = 1;
    for (int a = 0; a < d; ++a) { k += p[a] * m; m *= M; }
    return k;
  };
  const unsigned nt = chunks_for(n_leaves * nc);
  const int64_t nlc = n_leaves * nc;
  // grid points: the distinct leaf corners, by row-major key on the finest
  // level (sorted keys; a corner's point is its key's rank)
  struct KC {
    uint64_t key;
    int64_t lc;
  };
  std::unique_ptr<KC[]> kc(new KC[nlc > 0 ? nlc : 1]);
  parallel_chunks(n_leaves, nt, [&](unsigned, int64_t lo, int64_t hi) {
    for (int64_t l = lo; l < hi; ++l) {
      const int32_t nd = leaf_node[l];
      const int64_t s = pow3(depth - level[nd]);
      for (int e = 0; e < nc; ++e) {
        int64_t q[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) {
          q[a] = (coords[nd * 3 + a] + ((e >> a) & 1)) * s;
          if (q[a] >= M) q[a] -= M;
        }
        kc[l * nc + e] = {(uint64_t)key_of(q), l * nc + e};
      }
    }
  });
  uint64_t key_max = 1;
  for (int a = 0; a < d; ++a) key_max *= (uint64_t)M;
  radix_sort(kc, nlc, key_max, [](const KC &x) { return x.key; });
  table<int32_t> corner_pt;
  corner_pt.resize(nlc);  // every corner written below
  table<int64_t> pkey;
  {
    // ranks of the distinct keys: new keys counted per chunk, then offsets
    std::vector<int64_t> first(nt + 1, 0);
    parallel_chunks(nlc, nt, [&](unsigned t, int64_t lo, int64_t hi) {
      int64_t c = 0;
      for (int64_t i = lo; i < hi; ++i) c += (i == 0 || kc[i].key != kc[i - 1].key);
      first[t + 1] = c;
    });
    for (unsigned t = 0; t < nt; ++t) first[t + 1] += first[t];
    pkey.resize(first[nt]);
    parallel_chunks(nlc, nt, [&](unsigned t, int64_t lo, int64_t hi) {
      int64_t r = first[t] - 1;
      for (int64_t i = lo; i < hi; ++i) {
        if (i == 0 || kc[i].key != kc[i - 1].key) pkey[++r] = (int64_t)kc[i].key;
        corner_pt[kc[i].lc] = (int32_t)r;
      }
    });
  }
  kc.reset();
  const int64_t np = (int64_t)pkey.size();
  auto point = [&](const int64_t q[3]) -> int32_t {  // an existing point (a leaf corner)
    const int64_t k = key_of(q);
    return (int32_t)(std::lower_bound(pkey.begin(), pkey.end(), k) - pkey.begin());
  };
  // every point: the coarsest leaf whose closure holds it; non-hanging iff it
  // is a corner of that leaf, else (hanging) the d-linear interpolant of the
  // leaf's corners (weights by the point's place in the leaf)
  table<uint8_t> hanging;
  table<int32_t> best_of;
  hanging.resize(np);  // both written for every point below
  best_of.resize(np);
  parallel_chunks(np, nt, [&](unsigned, int64_t lo, int64_t hi) {
    for (int64_t id = lo; id < hi; ++id) {
      int64_t p[3] = {0, 0, 0}, k = pkey[id];
      for (int a = 0; a < d; ++a) { p[a] = k % M; k /= M; }
      // the leaf holding the finest cell just below (corner bit 0) or at
      // (bit 1) the point on every axis, by the base-3 digits of those cells
      // (most significant first): the descent of the quantised positions
      // p qs - 1 and p qs without their divisions
      uint8_t dig[2][3][kMaxLevel];
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < 2; ++b) {
          int64_t c = b ? p[a] : (p[a] == 0 ? M - 1 : p[a] - 1);
          for (int l = depth - 1; l >= 0; --l) {
            dig[b][a][l] = (uint8_t)(c % 3);
            c /= 3;
          }
        }
      int32_t best = -1;
      for (int e = 0; e < nc; ++e) {
        int32_t nd = 0;
        while (child0[nd] >= 0) {
          const int lv = level[nd];
          int digit = 0, mul = 1;
          for (int a = 0; a < d; ++a) { digit += dig[(e >> a) & 1][a][lv] * mul; mul *= 3; }
          nd = child0[nd] + digit;
        }
        if (best < 0 || level[nd] < level[best]) best = nd;
      }
      const int64_t s = pow3(depth - level[best]);
      bool corner = true;
      for (int a = 0; a < d; ++a) {
        int64_t rr = p[a] - coords[best * 3 + a] * s;
        if (rr < 0) rr += M;
        if (rr != 0 && rr != s) corner = false;
      }
      hanging[id] = corner ? 0 : 1;
      best_of[id] = best;
    }
  });
  // expansions of hanging points onto non-hanging ones, masters first
  // (memoised; the masters of a hanging point are corners of a coarser leaf)
  std::vector<int32_t> hslot(np, -1);
  std::vector<std::vector<std::pair<int32_t, double>>> hex;
  std::vector<int32_t> work;
  auto resolve = [&](int32_t root_id) {
    work.push_back(root_id);
    while (!work.empty()) {
      const int32_t id = work.back();
      if (!hanging[id] || hslot[id] >= 0) { work.pop_back(); continue; }
      int64_t p[3] = {0, 0, 0}, k = pkey[id];
      for (int a = 0; a < d; ++a) { p[a] = k % M; k /= M; }
      const int32_t best = best_of[id];
      const int64_t s = pow3(depth - level[best]);
      int64_t r[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) {
        int64_t rr = p[a] - coords[best * 3 + a] * s;
        if (rr < 0) rr += M;
        r[a] = rr;
      }
      bool ready = true;
      int32_t cid[8];
      double cw[8];
      for (int e = 0; e < nc; ++e) {
        double w = 1.0;
        int64_t q[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) {
          int ea = (e >> a) & 1;
          w *= ea ? (double)r[a] / (double)s : (double)(s - r[a]) / (double)s;
          q[a] = ((coords[best * 3 + a] + ea) * s) % M;
        }
        cw[e] = w;
        cid[e] = w == 0.0 ? -1 : point(q);
        if (cid[e] >= 0 && hanging[cid[e]] && hslot[cid[e]] < 0) {
          ready = false;
          work.push_back(cid[e]);
        }
      }
      if (!ready) continue;
      std::vector<std::pair<int32_t, double>> ex;
      for (int e = 0; e < nc; ++e) {
        if (cid[e] < 0) continue;
        auto merge = [&](int32_t pid, double wt) {
          for (auto &q : ex)
            if (q.first == pid) { q.second += cw[e] * wt; return; }
          ex.push_back({pid, cw[e] * wt});
        };
        if (!hanging[cid[e]]) merge(cid[e], 1.0);
        else for (auto &pr : hex[hslot[cid[e]]]) merge(pr.first, pr.second);
      }
      hslot[id] = (int32_t)hex.size();
      hex.push_back(std::move(ex));
      work.pop_back();
    }
  };
  for (int64_t id = 0; id < np; ++id)
    if (hanging[id]) resolve((int32_t)id);
  // vertex ids: the non-hanging points in key order
  std::vector<int32_t> vid_of_point(np, -1);
  {
    std::vector<int64_t> first(nt + 1, 0);  // non-hanging points per chunk, then offsets
    parallel_chunks(np, nt, [&](unsigned t, int64_t lo, int64_t hi) {
      int64_t c = 0;
      for (int64_t id = lo; id < hi; ++id) c += !hanging[id];
      first[t + 1] = c;
    });
    for (unsigned t = 0; t < nt; ++t) first[t + 1] += first[t];
    vert_key.resize(first[nt]);
    parallel_chunks(np, nt, [&](unsigned t, int64_t lo, int64_t hi) {
      int64_t r = first[t];
      for (int64_t id = lo; id < hi; ++id)
        if (!hanging[id]) {
          vid_of_point[id] = (int32_t)r;
          vert_key[r++] = pkey[id];
        }
    });
  }
  n_vert = (int64_t)vert_key.size();
  // leaf corner -> (vertex, weight), ascending vertex
  cexp_ptr.resize(nlc + 1);  // entries 1..nlc written below
  cexp_ptr[0] = 0;
  {
    // entries per corner, offsets by chunk sums
    std::vector<int64_t> part(nt + 1, 0);
    parallel_chunks(nlc, nt, [&](unsigned t, int64_t lo, int64_t hi) {
      int64_t run = 0;
      for (int64_t i = lo; i < hi; ++i) {
        const int32_t pt = corner_pt[i];
        run += hanging[pt] ? (int64_t)hex[hslot[pt]].size() : 1;
        cexp_ptr[i + 1] = (int32_t)run;
      }
      part[t + 1] = run;
    });
    for (unsigned t = 0; t < nt; ++t) part[t + 1] += part[t];
    parallel_chunks(nlc, nt, [&](unsigned t, int64_t lo, int64_t hi) {
      for (int64_t i = lo; i < hi; ++i) cexp_ptr[i + 1] += (int32_t)part[t];
    });
  }
  cexp_vid.resize(cexp_ptr[nlc]);  // every entry written below
  cexp_w.resize(cexp_ptr[nlc]);
  parallel_chunks(nlc, nt, [&](unsigned, int64_t lo, int64_t hi) {
    std::vector<std::pair<int32_t, double>> ex;
    for (int64_t i = lo; i < hi; ++i) {
      const int32_t pt = corner_pt[i];
      const int32_t o = cexp_ptr[i];
      if (!hanging[pt]) {
        cexp_vid[o] = vid_of_point[pt];
        cexp_w[o] = 1.0;
        continue;
      }
      ex.clear();
      for (auto &pr : hex[hslot[pt]]) ex.push_back({vid_of_point[pr.first], pr.second});
      std::sort(ex.begin(), ex.end(),
                [](const std::pair<int32_t, double> &a, const std::pair<int32_t, double> &b) {
                  return a.first < b.first;
                });
      for (size_t j = 0; j < ex.size(); ++j) {
        cexp_vid[o + j] = ex[j].first;
        cexp_w[o + j] = ex[j].second;
      }
    }
  });
  // transpose, stable in leaf-corner order (stable radix sort by vertex)
  const int64_t nnz = (int64_t)cexp_vid.size();
  struct VE {
    int32_t v, lc;
    double w;
  };
  std::unique_ptr<VE[]> ve(new VE[nnz > 0 ? nnz : 1]);
  parallel_chunks(nlc, nt, [&](unsigned, int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i)
      for (int32_t j = cexp_ptr[i]; j < cexp_ptr[i + 1]; ++j) ve[j] = {cexp_vid[j], (int32_t)i, cexp_w[j]};
  });
  radix_sort(ve, nnz, (uint64_t)std::max<int64_t>(n_vert, 1), [](const VE &x) { return (uint64_t)x.v; });
  inc_ptr.resize(n_vert + 1);  // every entry written below
  inc_lc.resize(nnz);
  inc_w.resize(nnz);
  parallel_chunks(nnz, nt, [&](unsigned, int64_t lo, int64_t hi) {
    for (int64_t j = lo; j < hi; ++j) {
      inc_lc[j] = ve[j].lc;
      inc_w[j] = ve[j].w;
      if (j == 0 || ve[j].v != ve[j - 1].v)
        for (int32_t v = j == 0 ? 0 : ve[j - 1].v + 1; v <= ve[j].v; ++v) inc_ptr[v] = (int32_t)j;
    }
  });
  for (int32_t v = nnz == 0 ? 0 : ve[nnz - 1].v + 1; v <= n_vert; ++v) inc_ptr[v] = (int32_t)nnz;
  ve.reset();
  // per vertex: the ion load, the number of corners that are the vertex
  // itself, and the diagonal of the stiffness matrix -- summed over the
  // vertex's incident leaf corners in leaf-corner order, pairs of corners of
  // one leaf in (e, f) order: the order of a loop over leaves and corners
  ion_load.resize(n_vert);  // every vertex written below
  diag.resize(n_vert);
  direct_cnt.resize(n_vert);
  parallel_chunks(n_vert, nt, [&](unsigned, int64_t lo, int64_t hi) {
    for (int64_t v = lo; v < hi; ++v) {
      double ion = 0.0, dg = 0.0;
      int32_t dc = 0;
      for (int32_t j = inc_ptr[v]; j < inc_ptr[v + 1];) {
        const int64_t leaf = inc_lc[j] / nc;
        int32_t k = j;
        while (k < inc_ptr[v + 1] && inc_lc[k] / nc == leaf) ++k;  // this leaf's corners at v
        const double h = 1.0 / (double)pow3(level[leaf_node[leaf]]);
        double vol = 1.0;
        for (int a = 0; a < d; ++a) vol *= h;
        const double cint = vol / (double)nc, hs = d == 2 ? 1.0 : h;
        for (int32_t a1 = j; a1 < k; ++a1) {
          const int64_t i = inc_lc[a1];
          ion += inc_w[a1] * cint;
          if (cexp_ptr[i + 1] - cexp_ptr[i] == 1 && !hanging[corner_pt[i]]) ++dc;
          const int e = (int)(i % nc);
          for (int32_t a2 = j; a2 < k; ++a2) {
            const int f = (int)(inc_lc[a2] % nc);
            dg += kref(d, e, f) * hs * inc_w[a1] * inc_w[a2];
          }
        }
        j = k;
      }
      ion_load[v] = ion;
      diag[v] = dg;
      direct_cnt[v] = dc;
    }
  });
}


void HostTree::build_pidt() {
  if (pidt_built) return;
  pidt_built = true;
  if (uniform) {
    n_pv = 1;
    for (int a = 0; a < d; ++a) n_pv *= M;
    return;
  }
  // every leaf corner as (level, row-major index on that level, leaf corner);
  // owner vertices are the distinct (level, index) pairs in that order, and a
  // corner's owner is its pair's rank.  A stable LSD radix sort by the index,
  // then by the level, keeps equal pairs in leaf-corner order; its passes run
  // on host threads over contiguous chunks (counts per chunk, then offsets).
  struct Rec {
    uint64_t rm;
    int32_t lc;
    int32_t lev;
  };
  const int64_t nlc = n_leaves * nc;
  std::unique_ptr<Rec[]> r(new Rec[nlc > 0 ? nlc : 1]);
  const unsigned nt = chunks_for(nlc);
  std::vector<uint64_t> rm_max_t(nt, 0);
  parallel_chunks(n_leaves, nt, [&](unsigned t, int64_t lo, int64_t hi) {
    uint64_t mx = 0;
    for (int64_t l = lo; l < hi; ++l) {
      const int32_t nd = leaf_node[l];
      const int lev = level[nd];
      const int64_t per = pow3(lev);
      for (int e = 0; e < nc; ++e) {
        int64_t rm = 0, m = 1;
        for (int a = 0; a < d; ++a) {
          int64_t c = coords[nd * 3 + a] + ((e >> a) & 1);  // below per, or per itself (periodic wrap)
          if (c == per) c = 0;
          rm += c * m;
          m *= per;
        }
        r[l * nc + e] = {(uint64_t)rm, (int32_t)(l * nc + e), lev};
        mx = std::max(mx, (uint64_t)rm);
      }
    }
    rm_max_t[t] = mx;
  });
  // one stable sort by level * (rm_max + 1) + rm: the order of a sort by rm
  // followed by a stable sort by level, in fewer passes (adaptive trees have
  // at most 12 levels, so rm < 3^36 and the key stays below 2^61)
  const uint64_t rm_max = *std::max_element(rm_max_t.begin(), rm_max_t.end());
  const uint64_t span = rm_max + 1;
  int lev_max = 0;
  for (int64_t l = 0; l < n_leaves; ++l) lev_max = std::max(lev_max, (int)level[leaf_node[l]]);
  radix_sort(r, nlc, (uint64_t)lev_max * span + rm_max,
             [span](const Rec &x) { return (uint64_t)x.lev * span + x.rm; });
  // distinct pairs in order: new pairs counted per chunk, then offsets
  auto is_new = [&](int64_t i) { return i == 0 || r[i].lev != r[i - 1].lev || r[i].rm != r[i - 1].rm; };
  std::vector<int64_t> first(nt + 1, 0);
  parallel_chunks(nlc, nt, [&](unsigned t, int64_t lo, int64_t hi) {
    int64_t c = 0;
    for (int64_t i = lo; i < hi; ++i) c += is_new(i);
    first[t + 1] = c;
  });
  for (unsigned t = 0; t < nt; ++t) first[t + 1] += first[t];
  const int64_t nv = first[nt];
  corner_pv.resize(nlc);  // every corner and owner written below
  pv_level.resize(nv);
  pv_j.resize(nv * d);
  parallel_chunks(nlc, nt, [&](unsigned t, int64_t lo, int64_t hi) {
    int64_t id = first[t] - 1;
    for (int64_t i = lo; i < hi; ++i) {
      if (is_new(i)) {
        ++id;
        pv_level[id] = r[i].lev;
        int64_t per = pow3(r[i].lev), rm = (int64_t)r[i].rm;
        for (int a = 0; a < d; ++a) { pv_j[id * d + a] = rm % per; rm /= per; }
      }
      corner_pv[r[i].lc] = (int32_t)id;
    }
  });
  n_pv = nv;
}

}  // namespace pic
