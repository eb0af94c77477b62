// Host-side spacetree tabulation; see tree.hpp.
#include "tree.hpp"

#include <algorithm>
#include <unordered_map>

namespace pic {

int HostTree::build(int d_, int64_t n_flags, const uint8_t *flags, std::string *err) {
  if (d_ != 2 && d_ != 3) { *err = "d must be 2 or 3"; return -1; }
  if (n_flags < 1 || !flags) { *err = "empty tree"; return -1; }
  if (n_flags > INT32_MAX - 64) { *err = "tree too large"; return -1; }
  d = d_;
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

struct GridPoint {
  int state = 0;  // 0 new, 2 resolved
  bool hanging = false;
  std::vector<std::pair<int32_t, double>> ex;  // (point index, weight)
};

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
  const int64_t qs = 2 * pow3(kMaxLevel - depth);
  auto leaf_at = [&](const int64_t Q[3]) {
    int32_t nd = 0;
    while (child0[nd] >= 0) {
      int64_t step = 2 * pow3(kMaxLevel - (level[nd] + 1));
      int digit = 0, mul = 1;
      for (int a = 0; a < d; ++a) { digit += (int)((Q[a] / step) % 3) * mul; mul *= 3; }
      nd = child0[nd] + digit;
    }
    return nd;
  };
  auto key_of = [&](const int64_t p[3]) {
    int64_t k = 0, m = 1;
    for (int a = 0; a < d; ++a) { k += p[a] * m; m *= M; }
    return k;
  };
  std::unordered_map<int64_t, int32_t> index;
  index.reserve((size_t)n_leaves * 2);
  std::vector<GridPoint> pts;
  std::vector<int64_t> pkey;
  auto point = [&](const int64_t p[3]) -> int32_t {
    int64_t k = key_of(p);
    auto it = index.find(k);
    if (it != index.end()) return it->second;
    int32_t id = (int32_t)pts.size();
    index.emplace(k, id);
    pts.emplace_back();
    pkey.push_back(k);
    return id;
  };
  // resolve: non-hanging iff it is a corner of the coarsest leaf whose closure
  // holds it; else the d-linear interpolant of that leaf's corners
  std::vector<int32_t> work;
  auto resolve = [&](int32_t root_id) {
    work.push_back(root_id);
    while (!work.empty()) {
      int32_t id = work.back();
      if (pts[id].state == 2) { work.pop_back(); continue; }
      int64_t p[3] = {0, 0, 0}, k = pkey[id];
      for (int a = 0; a < d; ++a) { p[a] = k % M; k /= M; }
      int32_t best = -1;
      for (int e = 0; e < nc; ++e) {
        int64_t Q[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) {
          int64_t q = p[a] * qs - (((e >> a) & 1) ? 0 : 1);
          Q[a] = q < 0 ? q + (int64_t)kQSteps : q;
        }
        int32_t nd = leaf_at(Q);
        if (best < 0 || level[nd] < level[best]) best = nd;
      }
      int64_t s = pow3(depth - level[best]);
      int64_t r[3] = {0, 0, 0};
      bool corner = true;
      for (int a = 0; a < d; ++a) {
        int64_t rr = p[a] - coords[best * 3 + a] * s;
        if (rr < 0) rr += M;
        r[a] = rr;
        if (rr != 0 && rr != s) corner = false;
      }
      if (corner) {
        pts[id].hanging = false;
        pts[id].ex = {{id, 1.0}};
        pts[id].state = 2;
        work.pop_back();
        continue;
      }
      // the masters first
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
        if (cid[e] >= 0 && pts[cid[e]].state != 2) {
          ready = false;
          work.push_back(cid[e]);
        }
      }
      if (!ready) continue;
      std::vector<std::pair<int32_t, double>> ex;
      for (int e = 0; e < nc; ++e) {
        if (cid[e] < 0) continue;
        for (auto &pr : pts[cid[e]].ex) {
          bool merged = false;
          for (auto &q : ex)
            if (q.first == pr.first) { q.second += cw[e] * pr.second; merged = true; break; }
          if (!merged) ex.push_back({pr.first, cw[e] * pr.second});
        }
      }
      pts[id].hanging = true;
      pts[id].ex = std::move(ex);
      pts[id].state = 2;
      work.pop_back();
    }
  };
  const int64_t nlc = n_leaves * nc;
  std::vector<int32_t> corner_pt(nlc);
  for (int64_t l = 0; l < n_leaves; ++l) {
    int32_t nd = leaf_node[l];
    int64_t s = pow3(depth - level[nd]);
    for (int e = 0; e < nc; ++e) {
      int64_t q[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) q[a] = ((coords[nd * 3 + a] + ((e >> a) & 1)) * s) % M;
      corner_pt[l * nc + e] = point(q);
    }
  }
  for (int64_t i = 0; i < nlc; ++i) resolve(corner_pt[i]);
  // vertex ids by row-major key
  vert_key.clear();
  for (size_t i = 0; i < pts.size(); ++i)
    if (!pts[i].hanging) vert_key.push_back(pkey[i]);
  std::sort(vert_key.begin(), vert_key.end());
  n_vert = (int64_t)vert_key.size();
  std::vector<int32_t> vid_of_point(pts.size(), -1);
  for (size_t i = 0; i < pts.size(); ++i)
    if (!pts[i].hanging)
      vid_of_point[i] = (int32_t)(std::lower_bound(vert_key.begin(), vert_key.end(), pkey[i]) -
                                  vert_key.begin());
  cexp_ptr.assign(nlc + 1, 0);
  cexp_vid.clear();
  cexp_w.clear();
  for (int64_t i = 0; i < nlc; ++i) {
    cexp_ptr[i] = (int32_t)cexp_vid.size();
    std::vector<std::pair<int32_t, double>> ex;
    for (auto &pr : pts[corner_pt[i]].ex) ex.push_back({vid_of_point[pr.first], pr.second});
    std::sort(ex.begin(), ex.end(),
              [](const std::pair<int32_t, double> &a, const std::pair<int32_t, double> &b) {
                return a.first < b.first;
              });
    for (auto &pr : ex) { cexp_vid.push_back(pr.first); cexp_w.push_back(pr.second); }
  }
  cexp_ptr[nlc] = (int32_t)cexp_vid.size();
  // transpose, stable in leaf-corner order
  inc_ptr.assign(n_vert + 1, 0);
  for (int32_t v : cexp_vid) inc_ptr[v + 1]++;
  for (int64_t v = 0; v < n_vert; ++v) inc_ptr[v + 1] += inc_ptr[v];
  inc_lc.assign(cexp_vid.size(), 0);
  inc_w.assign(cexp_vid.size(), 0.0);
  {
    std::vector<int32_t> cur(inc_ptr.begin(), inc_ptr.end() - 1);
    for (int64_t i = 0; i < nlc; ++i)
      for (int32_t j = cexp_ptr[i]; j < cexp_ptr[i + 1]; ++j) {
        int32_t v = cexp_vid[j];
        inc_lc[cur[v]] = (int32_t)i;
        inc_w[cur[v]] = cexp_w[j];
        cur[v]++;
      }
  }
  ion_load.assign(n_vert, 0.0);
  diag.assign(n_vert, 0.0);
  direct_cnt.assign(n_vert, 0);
  for (int64_t l = 0; l < n_leaves; ++l) {
    double h = 1.0 / (double)pow3(level[leaf_node[l]]);
    double vol = 1.0;
    for (int a = 0; a < d; ++a) vol *= h;
    double cint = vol / (double)nc, hs = d == 2 ? 1.0 : h;
    for (int e = 0; e < nc; ++e) {
      int64_t i = l * nc + e;
      for (int32_t j = cexp_ptr[i]; j < cexp_ptr[i + 1]; ++j) ion_load[cexp_vid[j]] += cexp_w[j] * cint;
      if (cexp_ptr[i + 1] - cexp_ptr[i] == 1 && !pts[corner_pt[i]].hanging) direct_cnt[cexp_vid[cexp_ptr[i]]]++;
      for (int f = 0; f < nc; ++f) {
        int64_t jf = l * nc + f;
        double kef = kref(d, e, f) * hs;
        for (int32_t a1 = cexp_ptr[i]; a1 < cexp_ptr[i + 1]; ++a1)
          for (int32_t a2 = cexp_ptr[jf]; a2 < cexp_ptr[jf + 1]; ++a2)
            if (cexp_vid[a1] == cexp_vid[a2]) diag[cexp_vid[a1]] += kef * cexp_w[a1] * cexp_w[a2];
      }
    }
  }
}

void HostTree::build_pidt() {
  if (uniform) {
    n_pv = 1;
    for (int a = 0; a < d; ++a) n_pv *= M;
    return;
  }
  struct Rec {
    int64_t lev, rm, lc;
  };
  const int64_t nlc = n_leaves * nc;
  std::vector<Rec> r(nlc);
  for (int64_t l = 0; l < n_leaves; ++l) {
    int32_t nd = leaf_node[l];
    int lev = level[nd];
    int64_t per = pow3(lev);
    for (int e = 0; e < nc; ++e) {
      int64_t rm = 0, m = 1;
      for (int a = 0; a < d; ++a) {
        rm += ((coords[nd * 3 + a] + ((e >> a) & 1)) % per) * m;
        m *= per;
      }
      r[l * nc + e] = {lev, rm, l * nc + e};
    }
  }
  std::sort(r.begin(), r.end(), [](const Rec &a, const Rec &b) {
    if (a.lev != b.lev) return a.lev < b.lev;
    if (a.rm != b.rm) return a.rm < b.rm;
    return a.lc < b.lc;
  });
  corner_pv.assign(nlc, 0);
  pv_level.clear();
  pv_j.clear();
  int64_t nv = 0;
  for (int64_t i = 0; i < nlc; ++i) {
    if (i == 0 || r[i].lev != r[i - 1].lev || r[i].rm != r[i - 1].rm) {
      pv_level.push_back((int32_t)r[i].lev);
      int64_t per = pow3((int)r[i].lev), rm = r[i].rm;
      for (int a = 0; a < d; ++a) { pv_j.push_back(rm % per); rm /= per; }
      ++nv;
    }
    corner_pv[r[i].lc] = (int32_t)(nv - 1);
  }
  n_pv = nv;
}

}  // namespace pic
