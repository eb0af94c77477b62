// Checkpoint files (pic_save / pic_load): writing, reading and checking.
// Host code only; the layout is documented in snapshot.hpp and include/pic.h.
#include "snapshot.hpp"

#include <cmath>
#include <cstdio>
#include <cstring>

#include "../../include/pic.h"

#if !defined(__BYTE_ORDER__) || __BYTE_ORDER__ != __ORDER_LITTLE_ENDIAN__
#error "checkpoint files are written in the host byte order, which must be little-endian"
#endif

namespace pic {

namespace {

constexpr char kMagic[8] = {'P', 'I', 'C', 'S', 'N', 'A', 'P', 0};
constexpr uint32_t kVersion = 1;
constexpr size_t kPrefix = 24;        // magic, version, meta bytes, checksum
constexpr size_t kMetaFixed = 104;    // meta block without the instance table
constexpr size_t kMetaPerInst = 24;
constexpr int64_t kMaxInstances = int64_t(1) << 24;

size_t pad8(size_t b) { return (b + 7) & ~size_t(7); }

// Checksum of `bytes` bytes followed by zeros up to the next multiple of 8.
uint64_t fold_padded(uint64_t c, const void *data, size_t bytes) {
  const size_t full = bytes & ~size_t(7);
  c = snapshot_fold(c, data, full);
  if (full < bytes) {
    uint8_t w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    std::memcpy(w, (const uint8_t *)data + full, bytes - full);
    c = snapshot_fold(c, w, 8);
  }
  return c;
}

// Little-endian append of plain values (meta block).
struct Out {
  std::vector<uint8_t> b;
  template <typename T>
  void put(T v) {
    const size_t o = b.size();
    b.resize(o + sizeof(T));
    std::memcpy(b.data() + o, &v, sizeof(T));
  }
};

struct In {
  const uint8_t *p;
  size_t left;
  template <typename T>
  T get() {
    T v{};
    if (left >= sizeof(T)) {
      std::memcpy(&v, p, sizeof(T));
      p += sizeof(T);
      left -= sizeof(T);
    }
    return v;
  }
};

class File {
 public:
  File(const char *path, const char *mode) : f_(std::fopen(path, mode)) {}
  ~File() {
    if (f_) std::fclose(f_);
  }
  File(const File &) = delete;
  File &operator=(const File &) = delete;
  FILE *get() const { return f_; }
  bool close() {
    const bool ok = f_ && std::fclose(f_) == 0;
    f_ = nullptr;
    return ok;
  }

 private:
  FILE *f_;
};

int io_fail(std::string *err, const std::string &msg) {
  if (err) *err = msg;
  return PIC_EIO;
}

int inval(std::string *err, const std::string &msg) {
  if (err) *err = msg;
  return PIC_EINVAL;
}

// One section: data, zero padding to 8 bytes; folded into the checksum.
bool write_section(FILE *f, const void *data, size_t bytes, uint64_t &c) {
  static const uint8_t zeros[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (bytes && std::fwrite(data, 1, bytes, f) != bytes) return false;
  const size_t pad = pad8(bytes) - bytes;
  if (pad && std::fwrite(zeros, 1, pad, f) != pad) return false;
  c = fold_padded(c, data, bytes);
  return true;
}

bool read_section(FILE *f, void *data, size_t bytes, uint64_t &c) {
  if (bytes && std::fread(data, 1, bytes, f) != bytes) return false;
  const size_t pad = pad8(bytes) - bytes;
  uint8_t tail[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (pad && std::fread(tail, 1, pad, f) != pad) return false;
  for (size_t i = 0; i < pad; ++i)
    if (tail[i]) return false;
  c = fold_padded(c, data, bytes);
  return true;
}

size_t fsize_of(int32_t precision) { return precision == PIC_FP32_SPLIT ? sizeof(float) : sizeof(double); }

}  // namespace

size_t snapshot_fsize(const SnapshotMeta &m) { return fsize_of(m.precision); }

uint64_t snapshot_fold(uint64_t c, const void *data, size_t bytes) {
  const uint8_t *p = (const uint8_t *)data;
  for (size_t i = 0; i + 8 <= bytes; i += 8) {
    uint64_t w;
    std::memcpy(&w, p + i, 8);
    c = (c ^ w) * 0x9e3779b97f4a7c15ull;
    c ^= c >> 29;
  }
  return c;
}

int snapshot_write(const char *path, const SnapshotMeta &m, const SnapshotArrays &a, std::string *err) {
  if (!path) return inval(err, "no checkpoint path");
  const size_t fs = fsize_of(m.precision);
  const size_t n = (size_t)m.n, nv = (size_t)m.n_vert, d = (size_t)m.d;
  Out meta;
  for (int32_t v : {m.d, m.scheme, m.precision, m.sweeps, m.track_ids, m.path, m.n_inst, 0}) meta.put(v);
  for (double v : {m.q, m.qm, m.ion, m.omega}) meta.put(v);
  for (int64_t v : {m.step, m.n, m.n_vert}) meta.put(v);
  for (int32_t v : m.tuned) meta.put(v);
  for (int32_t i = 0; i < m.n_inst; ++i) {
    meta.put(m.inst_flags[i]);
    meta.put(m.inst_n[i]);
    meta.put(m.inst_q[i]);
  }
  const bool split = m.precision == PIC_FP32_SPLIT;
  if (a.pos.size() != fs * d * n || a.vel.size() != fs * d * n || (split && a.leaf.size() != n) ||
      (m.track_ids && a.ids.size() != n) || a.V.size() != fs * nv || a.E.size() != fs * d * nv)
    return inval(err, "checkpoint arrays do not match their sizes");
  File f(path, "wb");
  if (!f.get()) return io_fail(err, std::string("cannot open ") + path + " for writing");
  uint64_t c = kSnapshotSeed;
  uint8_t prefix[kPrefix];
  std::memcpy(prefix, kMagic, 8);
  const uint32_t mb = (uint32_t)meta.b.size();
  std::memcpy(prefix + 8, &kVersion, 4);
  std::memcpy(prefix + 12, &mb, 4);
  std::memset(prefix + 16, 0, 8);  // checksum, written last
  bool ok = std::fwrite(prefix, 1, kPrefix, f.get()) == kPrefix && write_section(f.get(), meta.b.data(), mb, c) &&
            write_section(f.get(), a.flags.data(), a.flags.size(), c) &&
            (!split || write_section(f.get(), a.leaf.data(), 4 * n, c)) &&
            write_section(f.get(), a.pos.data(), a.pos.size(), c) &&
            write_section(f.get(), a.vel.data(), a.vel.size(), c) &&
            (!m.track_ids || write_section(f.get(), a.ids.data(), 4 * n, c)) &&
            write_section(f.get(), a.V.data(), a.V.size(), c) && write_section(f.get(), a.E.data(), a.E.size(), c);
  ok = ok && std::fseek(f.get(), 16, SEEK_SET) == 0 && std::fwrite(&c, 1, 8, f.get()) == 8;
  ok = f.close() && ok;
  if (!ok) return io_fail(err, std::string("writing ") + path + " failed");
  return PIC_OK;
}

int snapshot_read(const char *path, SnapshotMeta &m, SnapshotArrays &a, std::string *err) {
  if (!path) return inval(err, "no checkpoint path");
  File f(path, "rb");
  if (!f.get()) return io_fail(err, std::string("cannot open ") + path);
  const std::string name(path);
  if (fseeko(f.get(), 0, SEEK_END) != 0) return io_fail(err, name + ": not seekable");
  const int64_t fsz = (int64_t)ftello(f.get());
  if (fsz < 0 || fseeko(f.get(), 0, SEEK_SET) != 0) return io_fail(err, name + ": not seekable");
  uint8_t prefix[kPrefix];
  if ((size_t)fsz < kPrefix || std::fread(prefix, 1, kPrefix, f.get()) != kPrefix)
    return io_fail(err, name + ": too short for a checkpoint");
  if (std::memcmp(prefix, kMagic, 8) != 0) return io_fail(err, name + ": not a checkpoint (bad magic)");
  uint32_t version, mb;
  uint64_t stored;
  std::memcpy(&version, prefix + 8, 4);
  std::memcpy(&mb, prefix + 12, 4);
  std::memcpy(&stored, prefix + 16, 8);
  if (version != kVersion) return io_fail(err, name + ": unsupported format version " + std::to_string(version));
  if (mb < kMetaFixed || (mb - kMetaFixed) % kMetaPerInst != 0 || (int64_t)(kPrefix + mb) > fsz)
    return io_fail(err, name + ": malformed meta block");
  std::vector<uint8_t> meta(mb);
  uint64_t c = kSnapshotSeed;
  if (!read_section(f.get(), meta.data(), mb, c)) return io_fail(err, name + ": truncated meta block");
  In in{meta.data(), meta.size()};
  m.d = in.get<int32_t>();
  m.scheme = in.get<int32_t>();
  m.precision = in.get<int32_t>();
  m.sweeps = in.get<int32_t>();
  m.track_ids = in.get<int32_t>();
  m.path = in.get<int32_t>();
  m.n_inst = in.get<int32_t>();
  const int32_t reserved = in.get<int32_t>();
  m.q = in.get<double>();
  m.qm = in.get<double>();
  m.ion = in.get<double>();
  m.omega = in.get<double>();
  m.step = in.get<int64_t>();
  m.n = in.get<int64_t>();
  m.n_vert = in.get<int64_t>();
  for (int32_t &t : m.tuned) t = in.get<int32_t>();
  const bool split = m.precision == PIC_FP32_SPLIT;
  if ((m.d != 2 && m.d != 3) || (m.scheme != PIC_PIT && m.scheme != PIC_PIDT) ||
      (m.precision != PIC_FP64 && !split) || m.sweeps < 0 || (m.track_ids != 0 && m.track_ids != 1) ||
      (m.path != PIC_PATH_AUTO && m.path != PIC_PATH_GENERIC) || reserved != 0 || m.step < 0 || m.n < 0 ||
      m.n >= INT32_MAX || m.n_vert < 1 || m.n_inst < 1 || m.n_inst > kMaxInstances ||
      (int64_t)(mb - kMetaFixed) / (int64_t)kMetaPerInst != m.n_inst || (m.tuned[0] != 0 && m.tuned[0] != 1))
    return io_fail(err, name + ": meta data describe no valid configuration");
  for (int i = 1; i < 4; ++i)
    if (m.tuned[i] != 128 && m.tuned[i] != 256 && m.tuned[i] != 512)
      return io_fail(err, name + ": meta data describe no valid configuration");
  const size_t fs = fsize_of(m.precision), d = (size_t)m.d;
  if (m.n_vert > fsz / (int64_t)(fs * (d + 1))) return io_fail(err, name + ": size does not match its meta data");
  m.inst_flags.resize(m.n_inst);
  m.inst_n.resize(m.n_inst);
  m.inst_q.resize(m.n_inst);
  int64_t n_flags = 0, n_sum = 0;
  for (int32_t i = 0; i < m.n_inst; ++i) {
    m.inst_flags[i] = in.get<int64_t>();
    m.inst_n[i] = in.get<int64_t>();
    m.inst_q[i] = in.get<double>();
    if (m.inst_flags[i] < 1 || m.inst_flags[i] > fsz || m.inst_n[i] < 0 || m.inst_n[i] > m.n ||
        !std::isfinite(m.inst_q[i]))
      return io_fail(err, name + ": meta data describe no valid configuration");
    n_flags += m.inst_flags[i];
    n_sum += m.inst_n[i];
    if (n_flags > fsz || n_sum > m.n) return io_fail(err, name + ": size does not match its meta data");
  }
  if (n_sum != m.n) return io_fail(err, name + ": instance particle counts do not add up");
  const size_t n = (size_t)m.n, nv = (size_t)m.n_vert;
  const size_t expect = kPrefix + pad8(mb) + pad8((size_t)n_flags) + (split ? pad8(4 * n) : 0) + 2 * pad8(fs * d * n) +
                        (m.track_ids ? pad8(4 * n) : 0) + pad8(fs * nv) + pad8(fs * d * nv);
  if ((size_t)fsz != expect) return io_fail(err, name + ": size does not match its meta data (truncated?)");
  a.flags.assign((size_t)n_flags, 0);
  a.leaf.assign(split ? n : 0, 0);
  a.ids.assign(m.track_ids ? n : 0, 0);
  a.pos.assign(fs * d * n, 0);
  a.vel.assign(fs * d * n, 0);
  a.V.assign(fs * nv, 0);
  a.E.assign(fs * d * nv, 0);
  const bool ok = read_section(f.get(), a.flags.data(), a.flags.size(), c) &&
                  (!split || read_section(f.get(), a.leaf.data(), 4 * n, c)) &&
                  read_section(f.get(), a.pos.data(), a.pos.size(), c) &&
                  read_section(f.get(), a.vel.data(), a.vel.size(), c) &&
                  (!m.track_ids || read_section(f.get(), a.ids.data(), 4 * n, c)) &&
                  read_section(f.get(), a.V.data(), a.V.size(), c) && read_section(f.get(), a.E.data(), a.E.size(), c);
  if (!ok) return io_fail(err, name + ": truncated or corrupt section");
  if (c != stored) return io_fail(err, name + ": checksum mismatch");

  // particle values
  const size_t m_all = d * n;
  if (split) {
    const float *o = (const float *)a.pos.data();
    const float *v = (const float *)a.vel.data();
    for (size_t k = 0; k < m_all; ++k) {
      if (!(o[k] >= 0.0f && o[k] < 1.0f)) return inval(err, name + ": cell offset outside [0, 1)");
      if (!std::isfinite(v[k])) return inval(err, name + ": non-finite velocity");
    }
  } else {
    const double *x = (const double *)a.pos.data();
    const double *v = (const double *)a.vel.data();
    for (size_t k = 0; k < m_all; ++k) {
      if (!(x[k] >= 0.0 && x[k] < 1.0)) return inval(err, name + ": position outside [0, 1)");
      if (!std::isfinite(v[k])) return inval(err, name + ": non-finite velocity");
    }
  }
  if (m.track_ids) {
    std::vector<uint8_t> seen(n, 0);
    for (size_t p = 0; p < n; ++p) {
      const int32_t id = a.ids[p];
      if (id < 0 || (size_t)id >= n || seen[id]) return inval(err, name + ": particle ids are not a permutation");
      seen[id] = 1;
    }
  }
  return PIC_OK;
}

int snapshot_check_leaves(const SnapshotMeta &m, const SnapshotArrays &a, const std::vector<int64_t> &leaf_off,
                          std::string *err) {
  if (m.precision != PIC_FP32_SPLIT) return PIC_OK;
  if ((int64_t)leaf_off.size() != (int64_t)m.n_inst + 1) return inval(err, "leaf offsets do not match the instances");
  int64_t p = 0;
  for (int32_t i = 0; i < m.n_inst; ++i)
    for (int64_t k = 0; k < m.inst_n[i]; ++k, ++p) {
      const int64_t L = a.leaf[p];
      if (L < leaf_off[i] || L >= leaf_off[i + 1])
        return inval(err, "particle " + std::to_string(p) + " names a leaf outside its instance");
    }
  return PIC_OK;
}

}  // namespace pic
