// Device tabulation of an adaptive spacetree's finite-element grid and PIDT
// owner vertices (csrc/tree_dev.cu): the tables the kernels read, built on
// the GPU from the host's node list, descent table and leaf tables.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "tree.hpp"

namespace pic {

// Device memory for the tabulation: alloc(ctx, &p, bytes, keep) returns 0 or
// an error; keep = a table of the tree (freed with the tree), otherwise
// scratch, returned by release(ctx, p) before tabulate_on_device returns.
struct GridAlloc {
  void *ctx;
  int (*alloc)(void *ctx, void **out, size_t bytes, bool keep);
  void (*release)(void *ctx, void *p);
};

// The device tables (all kept allocations), in the layout of DevTree.
struct DeviceGrid {
  int64_t n_vert = 0, n_pv = 0, n_entries = 0;
  int32_t *cexp_ptr = nullptr, *cexp_vid = nullptr, *inc_ptr = nullptr, *inc_lc = nullptr, *dcnt = nullptr;
  int32_t *corner_pv = nullptr;
  double *cexp_w64 = nullptr, *inc_w64 = nullptr, *ion64 = nullptr, *diag64 = nullptr;
  float *cexp_w32 = nullptr, *inc_w32 = nullptr, *ion32 = nullptr, *diag32 = nullptr;
  int64_t *vert_key = nullptr;                      // row-major finest-lattice key per vertex
  int32_t *pv_level = nullptr, *pv_j = nullptr;     // PIDT owners: level, j[d] (int32)
};

constexpr int kTabUnsupported = 1;  // a hanging expansion too long for the device path: tabulate on the host
constexpr int kTabNoMemory = 2;
constexpr int kTabCuda = 3;

// Whether the device path applies: an adaptive tree of depth <= 12 whose
// finest lattice has at most 2^33 points (one bitmap bit each).
bool grid_on_device_fits(const HostTree &ht);

// Builds the tables of `ht` (HostTree::build done; grid and PIDT tables not
// needed) from the device copies of its descent table and leaf tables; the
// PIDT owners only when `pidt`.  Synchronous on `s`.  Returns 0, or one of
// the codes above (kept allocations made so far stay with the caller).
int tabulate_on_device(const HostTree &ht, const TabEntry *tab, const uint8_t *leaf_level, const int32_t *leaf_coords,
                       bool pidt, cudaStream_t s, const GridAlloc &A, DeviceGrid *out);

}  // namespace pic
