// Saving and loading a built query index (the offline product of
// Algorithm 1, Section 3.2: partition, M11 block inverses, couplings, S and
// M22^{-1}, the rank-r correction W_r D^{1/2}, the warm-start network).
//
// File layout (little-endian, version 3):
//   magic "KATZIDX\0", u32 version, u32 endian mark 0x01020304,
//   then one record per field in the order of serialize() below:
//     u64 tag (FNV-1a of the field name), u32 element size, u64 count,
//     count * element-size payload bytes,
//   then u64 checksum of every record (header and payload).
// A field list that changes shape changes the tags or sizes, so an old file
// is rejected with KATZ_EINVAL instead of being misread.
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "index.h"

namespace katz {
namespace {

constexpr char kMagic[8] = {'K', 'A', 'T', 'Z', 'I', 'D', 'X', '\0'};
constexpr uint32_t kVersion = 3;
constexpr uint32_t kEndianMark = 0x01020304u;
constexpr size_t kChunk = size_t(64) << 20;  // staging chunk (a multiple of 8)

uint64_t fnv1a(const std::string& s) {
  uint64_t h = 14695981039346656037ull;
  for (unsigned char c : s) {
    h ^= c;
    h *= 1099511628211ull;
  }
  return h;
}

// Running checksum over 8-byte words (a trailing partial word is zero
// padded); chunks other than the last of a record are multiples of 8, so
// the value does not depend on how a record is chunked.
uint64_t mix(uint64_t h, const uint8_t* p, size_t n) {
  size_t i = 0;
  for (; i + 8 <= n; i += 8) {
    uint64_t w;
    std::memcpy(&w, p + i, 8);
    h = (h ^ w) * 0x9E3779B97F4A7C15ull;
    h ^= h >> 29;
  }
  if (i < n) {
    uint64_t w = 0;
    std::memcpy(&w, p + i, n - i);
    h = (h ^ w ^ (uint64_t(n - i) << 56)) * 0x9E3779B97F4A7C15ull;
    h ^= h >> 29;
  }
  return h;
}

class Archive {
 public:
  Archive(FILE* f, bool saving, int64_t file_bytes)
      : f_(f), saving_(saving), left_(file_bytes) {}

  bool saving() const { return saving_; }

  template <class T>
  void scalar(const std::string& name, T& v) {
    static_assert(std::is_trivially_copyable<T>::value, "scalar field");
    uint64_t count = 1;
    header(name, sizeof(T), count);
    KATZ_REQUIRE(count == 1, KATZ_EINVAL, "index file: field " + name + " is not a scalar");
    bytes(&v, sizeof(T));
  }

  void flag(const std::string& name, bool& v) {
    uint8_t u = v ? 1 : 0;
    scalar(name, u);
    KATZ_REQUIRE(u <= 1, KATZ_EINVAL, "index file: field " + name + " is not a flag");
    v = u != 0;
  }

  template <class T>
  void vec(const std::string& name, std::vector<T>& v) {
    static_assert(std::is_trivially_copyable<T>::value, "vector field");
    uint64_t count = v.size();
    header(name, sizeof(T), count);
    if (!saving_) v.resize(count);
    if (count) bytes(v.data(), count * sizeof(T));
  }

  // Device buffer: staged through host memory in chunks.
  template <class T>
  void dbuf(const std::string& name, DBuf<T>& b) {
    uint64_t count = b.n;
    header(name, sizeof(T), count);
    if (!saving_) b.alloc(count);
    const size_t total = count * sizeof(T);
    if (!total) return;
    stage_.resize(std::min(total, kChunk));
    uint8_t* dev = reinterpret_cast<uint8_t*>(b.p);
    for (size_t off = 0; off < total; off += kChunk) {
      const size_t len = std::min(kChunk, total - off);
      if (saving_) {
        KATZ_CUDA(cudaMemcpy(stage_.data(), dev + off, len, cudaMemcpyDeviceToHost));
        bytes(stage_.data(), len);
      } else {
        bytes(stage_.data(), len);
        KATZ_CUDA(cudaMemcpy(dev + off, stage_.data(), len, cudaMemcpyHostToDevice));
      }
    }
  }

  void begin() {
    char magic[8];
    uint32_t ver = kVersion, mark = kEndianMark;
    std::memcpy(magic, kMagic, 8);
    raw(magic, 8);
    raw(&ver, 4);
    raw(&mark, 4);
    if (!saving_) {
      KATZ_REQUIRE(std::memcmp(magic, kMagic, 8) == 0, KATZ_EINVAL,
                   "not a katz index file (bad magic)");
      KATZ_REQUIRE(mark == kEndianMark, KATZ_EINVAL, "index file has the other byte order");
      KATZ_REQUIRE(ver == kVersion, KATZ_EINVAL,
                   "index file version " + std::to_string(ver) + " (this library reads " +
                       std::to_string(kVersion) + ")");
    }
  }

  void end() {
    uint64_t sum = h_;
    raw(&sum, 8);
    if (!saving_) {
      KATZ_REQUIRE(sum == h_, KATZ_EINVAL, "index file checksum mismatch (corrupt file)");
      KATZ_REQUIRE(left_ == 0, KATZ_EINVAL, "index file has trailing bytes");
    }
  }

 private:
  void header(const std::string& name, uint32_t esize, uint64_t& count) {
    uint64_t tag = fnv1a(name);
    uint32_t es = esize;
    bytes(&tag, 8);
    bytes(&es, 4);
    bytes(&count, 8);
    if (!saving_) {
      KATZ_REQUIRE(tag == fnv1a(name), KATZ_EINVAL,
                   "index file: expected field " + name + " (layout mismatch)");
      KATZ_REQUIRE(es == esize, KATZ_EINVAL, "index file: element size of " + name);
      KATZ_REQUIRE(count <= uint64_t(left_) / esize, KATZ_EINVAL,
                   "index file truncated at field " + name);
    }
  }

  // Payload bytes: written or read, and checksummed.
  void bytes(void* p, size_t n) {
    if (saving_) {
      h_ = mix(h_, static_cast<const uint8_t*>(p), n);
      raw(p, n);
    } else {
      raw(p, n);
      h_ = mix(h_, static_cast<const uint8_t*>(p), n);
    }
  }

  void raw(void* p, size_t n) {
    if (saving_) {
      KATZ_REQUIRE(std::fwrite(p, 1, n, f_) == n, KATZ_EINVAL, "index file write failed");
    } else {
      KATZ_REQUIRE(int64_t(n) <= left_ && std::fread(p, 1, n, f_) == n, KATZ_EINVAL,
                   "index file truncated");
      left_ -= int64_t(n);
    }
  }

  FILE* f_;
  bool saving_;
  int64_t left_;
  uint64_t h_ = 0x243F6A8885A308D3ull;
  std::vector<uint8_t> stage_;
};

void io_part(Archive& a, const std::string& p, GraphPart& g) {
  a.scalar(p + ".nrows", g.csr.nrows);
  a.scalar(p + ".ncols", g.csr.ncols);
  a.scalar(p + ".nnz", g.csr.nnz);
  a.scalar(p + ".vdt", g.csr.vdt);
  a.dbuf(p + ".rowptr", g.csr.rowptr);
  a.dbuf(p + ".col", g.csr.col);
  a.dbuf(p + ".val", g.csr.val);
  a.dbuf(p + ".heavy", g.heavy);
  a.scalar(p + ".n_heavy", g.n_heavy);
  a.dbuf(p + ".hseg_ptr", g.hseg_ptr);
  a.dbuf(p + ".hseg_row", g.hseg_row);
  a.scalar(p + ".n_hseg", g.n_hseg);
  a.dbuf(p + ".ps.bstart", g.ps.bstart);
  a.dbuf(p + ".ps.bentry", g.ps.bentry);
  a.dbuf(p + ".ps.ctr", g.ps.ctr);
  a.scalar(p + ".ps.nblocks", g.ps.nblocks);
  // autotuned launch shapes: (b, warps, col_tile, ctas, pipe, pipe_first,
  // fused_cps, gather_depth, row_pipeline, row_chunk)
  constexpr size_t kF = 10;
  std::vector<int32_t> t;
  if (a.saving())
    for (auto& kv : g.tuned) {
      const SpmmCfg& c = kv.second;
      t.insert(t.end(), {kv.first, c.warps_per_cta, c.col_tile, c.ctas_per_sm, int(c.pipe),
                         int(c.pipe_first), c.fused_cps, c.gather_depth, int(c.row_pipeline),
                         c.row_chunk});
    }
  a.vec(p + ".tuned10", t);
  if (!a.saving()) {
    KATZ_REQUIRE(t.size() % kF == 0, KATZ_EINVAL, "index file: " + p + ".tuned10");
    g.tuned.clear();
    for (size_t i = 0; i < t.size(); i += kF) {
      SpmmCfg c;
      c.warps_per_cta = t[i + 1];
      c.col_tile = t[i + 2];
      c.ctas_per_sm = t[i + 3];
      c.pipe = t[i + 4] != 0;
      c.pipe_first = t[i + 5] != 0;
      c.fused_cps = t[i + 6];
      c.gather_depth = t[i + 7];
      c.row_pipeline = t[i + 8] != 0;
      c.row_chunk = t[i + 9];
      KATZ_REQUIRE(c.ctas_per_sm >= 0 && c.ctas_per_sm <= 1024 && c.fused_cps >= 0 &&
                       c.fused_cps <= 1024 && c.col_tile >= 0 && c.col_tile <= 1024 &&
                       (c.gather_depth == 0 || c.gather_depth == 4 || c.gather_depth == 8) &&
                       c.row_chunk >= 0 && c.row_chunk <= 65536 &&
                       (c.row_chunk == 0 || c.row_chunk >= 8),
                   KATZ_EINVAL, "index file: launch shape out of range in " + p);
      g.tuned[t[i]] = c;
    }
  }
}

// The one list of stored fields, used in both directions.  Every field of
// katz_index except the scratch workspace and the per-query kernel
// preference is listed here.
void serialize(Archive& a, katz_index& x) {
  a.begin();
  a.scalar("n", x.n);
  a.scalar("nnz", x.nnz);
  a.scalar("beta", x.beta);
  a.scalar("lambda", x.lambda);
  a.scalar("lambda_up", x.lambda_up);
  a.vec("deg_h", x.deg_h);
  a.scalar("maxdeg", x.maxdeg);
  a.flag("unit_weights", x.unit_weights);
  a.scalar("vdt", x.vdt);
  io_part(a, "W", x.W);

  a.flag("lrc", x.lrc);
  a.scalar("rank", x.rank);
  a.scalar("block_max", x.block_max);
  a.scalar("split", x.split);
  a.scalar("n1", x.n1);
  a.scalar("n2", x.n2);
  a.scalar("n1s", x.n1s);
  a.scalar("n_large", x.n_large);
  a.scalar("lam11", x.lam11);
  a.scalar("lam11_min", x.lam11_min);
  a.vec("part.perm", x.part.perm);
  a.vec("part.block_ptr", x.part.block_ptr);
  a.scalar("part.n1", x.part.n1);
  a.scalar("part.n2", x.part.n2);
  a.dbuf("perm", x.perm);
  a.dbuf("iperm", x.iperm);
  io_part(a, "Wp", x.Wp);
  io_part(a, "W12", x.W12);
  io_part(a, "W21", x.W21);
  io_part(a, "W11L", x.W11L);

  uint64_t ncls = x.classes.size();
  a.scalar("classes", ncls);
  if (!a.saving()) {
    KATZ_REQUIRE(ncls <= 64, KATZ_EINVAL, "index file: block class count");
    x.classes.resize(ncls);
  }
  for (uint64_t k = 0; k < ncls; ++k) {
    BlockClass& c = x.classes[k];
    const std::string p = "class" + std::to_string(k);
    a.scalar(p + ".S", c.S);
    a.scalar(p + ".count", c.count);
    a.dbuf(p + ".start", c.start);
    a.dbuf(p + ".size", c.size);
    a.dbuf(p + ".inv32", c.inv32);
    a.dbuf(p + ".inv64", c.inv64);
  }

  a.scalar("ld2", x.ld2);
  a.dbuf("S32", x.S32);
  a.dbuf("M22inv32", x.M22inv32);
  a.dbuf("Wr32", x.Wr32);
  a.dbuf("S64", x.S64);
  a.dbuf("M22inv64", x.M22inv64);
  a.dbuf("Wr64", x.Wr64);
  a.dbuf("Wb", x.Wb);
  a.dbuf("WbT", x.WbT);
  a.scalar("ldr", x.ldr);
  a.scalar("ldn2", x.ldn2);
  a.dbuf("Wr32u", x.Wr32u);
  a.scalar("ldr4", x.ldr4);
  io_part(a, "W22", x.W22);
  a.dbuf("Hh", x.Hh);
  a.dbuf("Hl", x.Hl);
  a.scalar("ldH", x.ldH);
  a.flag("has_h", x.has_h);
  a.dbuf("Zc", x.Zc);
  a.scalar("ldZ", x.ldZ);
  a.flag("has_z", x.has_z);
  a.dbuf("Sh", x.Sh);
  a.dbuf("Sl", x.Sl);
  a.dbuf("Mh", x.Mh);
  a.dbuf("Ml", x.Ml);
  a.flag("dense_tc", x.dense_tc);
  a.flag("s_implicit", x.s_implicit);

  // warm-start network with its optimiser state (training can resume)
  a.scalar("mlp.din", x.mlp.din);
  a.scalar("mlp.dh", x.mlp.dh);
  a.scalar("mlp.dout", x.mlp.dout);
  a.flag("mlp.ready", x.mlp.ready);
  a.scalar("mlp.step_count", x.mlp.step_count);
  a.dbuf("mlp.params", x.mlp.params);
  a.dbuf("mlp.grads", x.mlp.grads);
  a.dbuf("mlp.mom", x.mlp.mom);
  a.dbuf("mlp.var", x.mlp.var);
  a.dbuf("mlp.w1b", x.mlp.w1b);
  a.dbuf("mlp.w2b", x.mlp.w2b);
  a.dbuf("feat", x.feat);
  a.vec("sigma", x.sigma);
  a.scalar("lanczos_steps", x.lanczos_steps);
  a.vec("seg_rank", x.seg_rank);
  a.end();
}

// Consistency of a loaded index beyond what the records fix.
void check_part(const GraphPart& g, const char* name) {
  const DevCsr& c = g.csr;
  // (uploads give col at least one element; an operator never uploaded has
  // no arrays at all)
  const bool ok = c.nrows >= 0 && c.nnz >= 0 && c.col.n >= size_t(c.nnz) &&
                  (c.rowptr.n == 0 ? c.nrows == 0 && c.nnz == 0
                                   : c.rowptr.n == size_t(c.nrows + 1)) &&
                  c.val.n >= size_t(c.nnz) * vdt_size(c.vdt) && g.heavy.n >= size_t(g.n_heavy) &&
                  (g.n_hseg == 0 || (g.hseg_ptr.n == size_t(g.n_heavy + 1) &&
                                     g.hseg_row.n >= size_t(g.n_hseg)));
  if (!ok) throw Error(KATZ_EINVAL, std::string("index file: inconsistent operator ") + name);
}

void check_loaded(const katz_index& x) {
  auto fail = [](const char* what) {
    throw Error(KATZ_EINVAL, std::string("index file: inconsistent ") + what);
  };
  check_part(x.W, "W");
  check_part(x.Wp, "Wp");
  check_part(x.W12, "W12");
  check_part(x.W21, "W21");
  check_part(x.W11L, "W11L");
  check_part(x.W22, "W22");
  if (x.n < 0 || x.n >= (int64_t(1) << 31) || int64_t(x.deg_h.size()) != x.n) fail("n");
  if (x.W.csr.nrows != x.n || int64_t(x.W.csr.rowptr.n) != x.n + 1 || x.W.csr.nnz != x.nnz)
    fail("graph");
  if (!(x.beta > 0) || !(x.lambda_up >= x.lambda) || !(x.beta * x.lambda_up < 1)) fail("beta");
  if (x.lrc) {
    if (x.n1 + x.n2 != x.n || int64_t(x.part.perm.size()) != x.n ||
        int64_t(x.perm.n) != x.n || int64_t(x.iperm.n) != x.n)
      fail("partition");
    if (int64_t(x.sigma.size()) != x.rank) fail("rank");
    if (x.has_z && (x.ldZ < x.n2 || x.ldZ % 4 != 0 ||
                    int64_t(x.Zc.n) != x.n1 * x.ldZ))
      fail("stored coupling Z");
  }
  if (x.has_z && !x.lrc) fail("stored coupling Z");
}

}  // namespace

void save_index(const katz_index& idx, const char* path) {
  KATZ_REQUIRE(path && *path, KATZ_EINVAL, "empty path");
  FILE* f = std::fopen(path, "wb");
  KATZ_REQUIRE(f, KATZ_EINVAL, std::string("cannot open ") + path + " for writing");
  try {
    Archive a(f, true, 0);
    serialize(a, const_cast<katz_index&>(idx));
  } catch (...) {
    std::fclose(f);
    std::remove(path);
    throw;
  }
  const bool ok = std::fclose(f) == 0;
  if (!ok) std::remove(path);
  KATZ_REQUIRE(ok, KATZ_EINVAL, std::string("closing ") + path + " failed");
}

std::unique_ptr<katz_index> load_index(const char* path) {
  KATZ_REQUIRE(path && *path, KATZ_EINVAL, "empty path");
  FILE* f = std::fopen(path, "rb");
  KATZ_REQUIRE(f, KATZ_EINVAL, std::string("cannot open ") + path);
  std::unique_ptr<katz_index> idx(new katz_index());
  try {
    std::fseek(f, 0, SEEK_END);
    const int64_t size = std::ftell(f);
    std::fseek(f, 0, SEEK_SET);
    KATZ_REQUIRE(size >= 0, KATZ_EINVAL, std::string("cannot size ") + path);
    Archive a(f, false, size);
    serialize(a, *idx);
    check_loaded(*idx);
  } catch (...) {
    std::fclose(f);
    throw;
  }
  std::fclose(f);
  return idx;
}

}  // namespace katz
