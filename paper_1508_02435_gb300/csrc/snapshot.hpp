// Checkpoint files of a handle (pic_save / pic_load): host-only format code.
//
// A checkpoint holds what the next step reads and nothing it recomputes:
// the refinement flags of every instance, the particle state in storage order
// and native precision (split: leaf ids, FP32 offsets and velocities; FP64:
// positions and velocities), the particle ids, the potential V (the starting
// guess of the next Jacobi solve) and the field E (read by a fixed-field step),
// the step counter, the configuration and the launch tuning.  Sort keys,
// bucket offsets, vertex charges and every scratch buffer follow from these.
//
// Layout (little-endian, every section padded with zeros to 8 bytes):
//   [0,8)   magic "PICSNAP" + NUL
//   [8,12)  u32 format version (1)
//   [12,16) u32 bytes of the meta block
//   [16,24) u64 checksum of every byte from offset 24 to the end
//   meta:   i32 d, scheme, precision, sweeps, track_ids, path, n_inst, 0
//           f64 q, qm, ion, omega
//           i64 step, n, n_vert
//           i32 tuned[4]
//           per instance: i64 n_flags, i64 n_particles, f64 q
//   flags   u8[sum n_flags]
//   leaf    i32[n]                 (split precision only)
//   pos     f[d][n]                (f = f32 split, f64 otherwise)
//   vel     f[d][n]
//   ids     i32[n]                 (track_ids only)
//   V       f[n_vert]
//   E       f[d][n_vert]
//
// The checksum folds the bytes as little-endian 64-bit words w_k in order:
// c_0 = 0x243f6a8885a308d3 (the leading hexadecimal digits of pi), then
// c_{k+1} = ((c_k xor w_k) * 0x9e3779b97f4a7c15) xor (that product >> 29),
// the multiplier being the odd integer nearest 2^64 / golden ratio.  It
// detects truncation and stray writes; it is not a cryptographic hash.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace pic {

struct SnapshotMeta {
  int32_t d = 0, scheme = 0, precision = 0, sweeps = 0, track_ids = 0, path = 0, n_inst = 0;
  double q = 0, qm = 0, ion = 0, omega = 0;
  int64_t step = 0, n = 0, n_vert = 0;
  int32_t tuned[4] = {0, 0, 0, 0};
  std::vector<int64_t> inst_flags, inst_n;  // per instance: flag count, particles
  std::vector<double> inst_q;               // per instance: charge per particle
};

// Host copies of the device arrays, native precision, storage order.
struct SnapshotArrays {
  std::vector<uint8_t> flags;
  std::vector<int32_t> leaf, ids;
  std::vector<uint8_t> pos, vel, V, E;
};

// Bytes of one floating-point value in the checkpoint's precision.
size_t snapshot_fsize(const SnapshotMeta &m);

// Checksum of `bytes` bytes (a multiple of 8) continuing from `c`.
uint64_t snapshot_fold(uint64_t c, const void *data, size_t bytes);
constexpr uint64_t kSnapshotSeed = 0x243f6a8885a308d3ull;

// Write a checkpoint; PIC_EIO if the file cannot be written completely.
int snapshot_write(const char *path, const SnapshotMeta &m, const SnapshotArrays &a, std::string *err);

// Read and check a checkpoint: the file must exist, carry the magic and the
// version, hold meta data that describe a valid configuration, have exactly
// the size those imply and match its checksum (PIC_EIO otherwise).  Every
// particle value must then be finite, split offsets and FP64 positions must
// lie in [0, 1) and the ids must be a permutation of [0, n) (PIC_EINVAL
// otherwise).  Leaf ids are checked by snapshot_check_leaves once the trees
// are known.
int snapshot_read(const char *path, SnapshotMeta &m, SnapshotArrays &a, std::string *err);

// Split precision: particle p of instance i must name a leaf in
// [leaf_off[i], leaf_off[i + 1]).  PIC_EINVAL otherwise.
int snapshot_check_leaves(const SnapshotMeta &m, const SnapshotArrays &a, const std::vector<int64_t> &leaf_off,
                          std::string *err);

}  // namespace pic
