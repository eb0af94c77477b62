// Host-side tabulation of a k = 3 spacetree (Section 4 of arXiv:1508.02435):
// node list from level-order flags, depth-first leaf numbering, the flattened
// descent table the kernels walk, leaf tables, the d-linear finite-element
// grid (non-hanging vertices, hanging-vertex constraints) and the PIDT owner
// vertices.
#pragma once
#include <cstdint>
#include <memory>
#include <new>
#include <string>
#include <utility>
#include <vector>

namespace pic {

// Allocator whose value-less construct leaves plain values uninitialised, so
// that resize(n) of a large table costs no serial zero fill: the threads that
// fill the table touch its pages first, in parallel.
template <typename T>
struct NoInitAllocator : std::allocator<T> {
  using value_type = T;
  template <typename U>
  struct rebind {
    using other = NoInitAllocator<U>;
  };
  NoInitAllocator() = default;
  template <typename U>
  NoInitAllocator(const NoInitAllocator<U> &) noexcept {}
  template <typename U>
  void construct(U *p) noexcept {
    ::new ((void *)p) U;
  }
  template <typename U, typename... Args>
  void construct(U *p, Args &&...args) {
    ::new ((void *)p) U(std::forward<Args>(args)...);
  }
};
template <typename T>
using table = std::vector<T, NoInitAllocator<T>>;

constexpr int kMaxLevel = 18;
constexpr uint32_t kQSteps = 774840978u;  // 2 * 3^18 integer steps per axis

inline int64_t pow3(int e) {
  int64_t r = 1;
  for (int i = 0; i < e; ++i) r *= 3;
  return r;
}

// Descent-table entry.  a >= 0: refined cell whose 3^d children are the
// entries a .. a + 3^d - 1 (digit order).  a < 0: the whole subtree below is
// complete with depth k = -a - 1 (k = 0: a leaf); its leaves are b, b + 1, ...
// in depth-first order, i.e. base-3^d digits of the local coordinates, most
// significant level first.
struct TabEntry {
  int32_t a, b;
};

struct HostTree {
  int d = 0, nch = 0, nc = 0, depth = 0;
  bool uniform = false;
  int64_t n_nodes = 0, n_leaves = 0;
  std::vector<int32_t> level, child0, leaf_node;
  std::vector<int64_t> coords;  // 3 per node
  std::vector<int32_t> leaf_of_node;

  std::vector<TabEntry> tab;
  std::vector<uint8_t> leaf_level;
  std::vector<int32_t> leaf_coords;  // d per leaf

  // finite-element grid
  int64_t M = 1;       // 3^depth
  int64_t n_vert = 0;  // non-hanging grid points
  table<int64_t> vert_key;  // row-major key on the finest level (adaptive only)
  // adaptive only: leaf corner -> (vertex, weight); vertex -> (leaf corner, weight)
  table<int32_t> cexp_ptr, cexp_vid, inc_ptr, inc_lc;
  table<double> cexp_w, inc_w;
  table<double> ion_load, diag;  // per vertex (adaptive), or one value (uniform)
  table<int32_t> direct_cnt;     // adaptive only

  // PIDT owner vertices (adaptive only; uniform trees use the FE vertices)
  int64_t n_pv = 0;
  bool pidt_built = false;  // build_pidt ran (PIT handles run it on demand)
  table<int32_t> corner_pv, pv_level;
  table<int64_t> pv_j;  // d per vertex

  int build(int d_, int64_t n_flags, const uint8_t *flags, std::string *err);
  void build_grid();
  void build_pidt();
};

}  // namespace pic
