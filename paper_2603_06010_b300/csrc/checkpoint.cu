// Factor checkpoint and resume: the evaluation state of a factored segment
// written to a file and read back into a new segment, so a segment that left
// the device (or a process that restarted) does not pay the factor again (an
// O(N'^3) FP64 Cholesky, Sec. II.A; 22 s at N' = 32256 on this GPU).
//
// File layout (little-endian, this library's own format):
//   header  (CkptHeader below: magic, version, sizes, flags, scalars, payload
//            size and an FNV-1a 64 checksum of the payload)
//   payload, in this order:
//     acf        float64[n]
//     kept index int32[N']
//     operator   bf16[op_blocks * 4 * 256 * 32]          (flag CK_OP)
//     L          float64[N'p * N'p], dinv float64[N'p/64 * 64 * 64]   (flag CK_FP64)
//     GSCE       float2[M] S1, float2[M] S2, float2[M / 4] twiddles    (flag CK_GS)
// The header is checked against the file size before any device work; the
// checksum after the payload has been read.  A save writes "<path>.tmp" and
// renames it over <path>, so an interrupted save leaves no partial file.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "td_internal.h"

namespace td {
namespace {

constexpr char CK_MAGIC[8] = {'T', 'D', 'S', 'E', 'G', 'C', 'K', '1'};
constexpr uint32_t CK_VERSION = 1;
enum : uint32_t { CK_OP = 1u, CK_FP64 = 2u, CK_GS = 4u };

struct CkptHeader {
  char magic[8];
  uint32_t version;
  uint32_t flags;
  int64_t n, nk, nkp, op_blocks;
  double logdet;
  int32_t gs_logm;
  int32_t factored;
  double gs_x0, gs_logdet;
  uint64_t payload_bytes;
  uint64_t checksum;
};
static_assert(sizeof(CkptHeader) == 96, "checkpoint header layout");

struct Fnv {
  uint64_t h = 1469598103934665603ull;
  void add(const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
      h ^= b[i];
      h *= 1099511628211ull;
    }
  }
};

struct Sizes {   // payload section sizes in bytes
  uint64_t acf, t, op, L, dinv, gs_s, gs_tw;
  uint64_t total() const { return acf + t + op + L + dinv + 2 * gs_s + gs_tw; }
};

Sizes sizes_of(const CkptHeader& h) {
  Sizes z{};
  z.acf = (uint64_t)h.n * 8;
  z.t = (uint64_t)h.nk * 4;
  z.op = (h.flags & CK_OP) ? (uint64_t)h.op_blocks * OP_SLICES * OP_ROWS * OP_KB * 2 : 0;
  z.L = (h.flags & CK_FP64) ? (uint64_t)h.nkp * h.nkp * 8 : 0;
  z.dinv = (h.flags & CK_FP64) ? (uint64_t)(h.nkp / FT) * FT * FT * 8 : 0;
  const uint64_t M = (h.flags & CK_GS) ? (1ull << h.gs_logm) : 0;
  z.gs_s = M * 8;
  z.gs_tw = (M / 4) * 8;
  return z;
}

constexpr size_t CK_CHUNK = 64u << 20;   // host staging per copy

// device -> file, through a host chunk, adding to the checksum
bool write_dev(FILE* f, const void* dev, uint64_t bytes, std::vector<unsigned char>& buf, Fnv& sum,
               cudaStream_t st, std::string& err) {
  const unsigned char* p = static_cast<const unsigned char*>(dev);
  for (uint64_t off = 0; off < bytes; off += CK_CHUNK) {
    const size_t n = (size_t)std::min<uint64_t>(CK_CHUNK, bytes - off);
    cudaError_t e = cudaMemcpyAsync(buf.data(), p + off, n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      err = std::string("device read: ") + cudaGetErrorString(e);
      return false;
    }
    sum.add(buf.data(), n);
    if (fwrite(buf.data(), 1, n, f) != n) {
      err = "file write failed";
      return false;
    }
  }
  return true;
}

// file -> device, through a host chunk, adding to the checksum
bool read_dev(FILE* f, void* dev, uint64_t bytes, std::vector<unsigned char>& buf, Fnv& sum, cudaStream_t st,
              std::string& err) {
  unsigned char* p = static_cast<unsigned char*>(dev);
  for (uint64_t off = 0; off < bytes; off += CK_CHUNK) {
    const size_t n = (size_t)std::min<uint64_t>(CK_CHUNK, bytes - off);
    if (fread(buf.data(), 1, n, f) != n) {
      err = "file shorter than its header states";
      return false;
    }
    sum.add(buf.data(), n);
    cudaError_t e = cudaMemcpyAsync(p + off, buf.data(), n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // buf is reused by the next chunk
    if (e != cudaSuccess) {
      err = std::string("device write: ") + cudaGetErrorString(e);
      return false;
    }
  }
  return true;
}

template <class T>
td_status alloc_dev(T** p, uint64_t bytes, const char* what) {
  *p = nullptr;
  if (bytes == 0) return TD_OK;
  if (cudaMalloc((void**)p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(TD_ERR_OOM, std::string("device allocation failed: ") + what);
  }
  return TD_OK;
}

}  // namespace
}  // namespace td

using namespace td;

extern "C" td_status td_segment_save(const td_segment* s, const char* path, void* stream) {
  if (!s || !path || !*path) return fail(TD_ERR_INVALID, "NULL argument");
  if (!s->factored && !s->gs.ready) return fail(TD_ERR_NOT_FACTORED, "nothing to save: segment not factored");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  CkptHeader h;
  memset(&h, 0, sizeof h);
  memcpy(h.magic, CK_MAGIC, 8);
  h.version = CK_VERSION;
  h.flags = (s->factored && s->op ? CK_OP : 0u) | (s->factored && s->L && s->dinv ? CK_FP64 : 0u) |
            (s->gs.ready ? CK_GS : 0u);
  h.n = s->n;
  h.nk = s->nk;
  h.nkp = s->nkp;
  h.op_blocks = s->op_blocks;
  h.logdet = s->logdet;
  h.factored = s->factored ? 1 : 0;
  h.gs_logm = s->gs.ready ? s->gs.logm : 0;
  h.gs_x0 = s->gs.x0;
  h.gs_logdet = s->gs.logdet;
  const Sizes z = sizes_of(h);
  h.payload_bytes = z.total();
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = fopen(tmp.c_str(), "wb");
  if (!f) return fail(TD_ERR_INVALID, "cannot open " + tmp + " for writing");
  std::vector<unsigned char> buf((size_t)std::min<uint64_t>(CK_CHUNK, std::max<uint64_t>(z.total(), 1)));
  Fnv sum;
  std::string err;
  bool ok = fwrite(&h, sizeof h, 1, f) == 1;   // checksum filled in at the end
  if (!ok) err = "file write failed";
  if (ok) ok = write_dev(f, s->acf, z.acf, buf, sum, st, err) && write_dev(f, s->t, z.t, buf, sum, st, err);
  if (ok && (h.flags & CK_OP)) ok = write_dev(f, s->op, z.op, buf, sum, st, err);
  if (ok && (h.flags & CK_FP64))
    ok = write_dev(f, s->L, z.L, buf, sum, st, err) && write_dev(f, s->dinv, z.dinv, buf, sum, st, err);
  if (ok && (h.flags & CK_GS))
    ok = write_dev(f, s->gs.S1, z.gs_s, buf, sum, st, err) && write_dev(f, s->gs.S2, z.gs_s, buf, sum, st, err) &&
         write_dev(f, s->gs.tw, z.gs_tw, buf, sum, st, err);
  if (ok) {
    h.checksum = sum.h;
    ok = fseek(f, 0, SEEK_SET) == 0 && fwrite(&h, sizeof h, 1, f) == 1;
    if (!ok) err = "file write failed";
  }
  if (fclose(f) != 0 && ok) {
    ok = false;
    err = "file close failed";
  }
  if (ok && rename(tmp.c_str(), path) != 0) {
    ok = false;
    err = std::string("cannot rename onto ") + path;
  }
  if (!ok) {
    remove(tmp.c_str());
    return fail(err.rfind("device", 0) == 0 ? TD_ERR_CUDA : TD_ERR_INVALID, "td_segment_save: " + err);
  }
  return TD_OK;
}

extern "C" td_status td_segment_load(const char* path, void* stream, td_segment** out) {
  if (!out) return fail(TD_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!path || !*path) return fail(TD_ERR_INVALID, "path is NULL");
  FILE* f = fopen(path, "rb");
  if (!f) return fail(TD_ERR_INVALID, std::string("cannot open ") + path);
  CkptHeader h;
  std::string err;
  // ---- everything below up to the first device call checks the file only
  if (fread(&h, sizeof h, 1, f) != 1) err = "file shorter than a checkpoint header";
  else if (memcmp(h.magic, CK_MAGIC, 8) != 0) err = "not a segment checkpoint (magic)";
  else if (h.version != CK_VERSION) err = "unsupported checkpoint version";
  else if ((h.flags & ~(CK_OP | CK_FP64 | CK_GS)) != 0 || h.flags == 0) err = "bad section flags";
  else if (h.n < 1 || h.n > (int64_t)INT32_MAX || h.nk < 1 || h.nk > h.n || h.nkp != round_up(h.nk, OP_ROWS))
    err = "inconsistent sizes";
  else if ((h.flags & CK_OP) && h.op_blocks != op_row_offset(h.nkp / OP_ROWS)) err = "inconsistent operator size";
  else if ((h.flags & (CK_OP | CK_FP64)) && !h.factored) err = "factor sections without a factored segment";
  else if (!(h.flags & CK_OP) && h.factored) err = "factored segment without its operator";
  else if ((h.flags & CK_GS) && (h.gs_logm < 11 || h.gs_logm > 16 || (1ll << h.gs_logm) < 2 * h.n))
    err = "inconsistent GSCE length";
  else if (h.payload_bytes != sizes_of(h).total()) err = "payload size does not match the sections";
  else {
    long long cur = ftell(f);
    if (fseek(f, 0, SEEK_END) != 0 || ftell(f) - cur != (long long)h.payload_bytes) err = "file size does not match its header";
    else if (fseek(f, cur, SEEK_SET) != 0) err = "file seek failed";
  }
  if (!err.empty()) {
    fclose(f);
    return fail(TD_ERR_INVALID, std::string("td_segment_load: ") + err);
  }
  const Sizes z = sizes_of(h);
  Fnv sum;
  std::vector<double> acf((size_t)h.n);
  std::vector<int32_t> t((size_t)h.nk);
  bool ok = fread(acf.data(), 1, z.acf, f) == z.acf && fread(t.data(), 1, z.t, f) == z.t;
  if (ok) {
    sum.add(acf.data(), z.acf);
    sum.add(t.data(), z.t);
    for (int64_t i = 0; ok && i < h.nk; ++i)
      ok = t[(size_t)i] >= 0 && t[(size_t)i] < h.n && (i == 0 || t[(size_t)i] > t[(size_t)i - 1]);
    if (!ok) err = "kept indices out of order or out of range";
  } else {
    err = "file read failed";
  }
  if (!ok) {
    fclose(f);
    return fail(TD_ERR_INVALID, std::string("td_segment_load: ") + err);
  }
  std::vector<uint8_t> mask((size_t)h.n, 0);
  for (int32_t i : t) mask[(size_t)i] = 1;
  // ---- device work from here on
  td_segment* s = nullptr;
  td_status r = td_segment_create(acf.data(), h.n, mask.data(), stream, &s);
  if (r != TD_OK) {
    fclose(f);
    return r;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  std::vector<unsigned char> buf((size_t)std::min<uint64_t>(CK_CHUNK, std::max<uint64_t>(h.payload_bytes, 1)));
  GsState& g = s->gs;
  if ((h.flags & CK_OP) && (r = alloc_dev(&s->op, z.op, "operator slices")) != TD_OK) goto fail_r;
  if ((h.flags & CK_FP64) && ((r = alloc_dev(&s->L, z.L, "FP64 factor")) != TD_OK ||
                              (r = alloc_dev(&s->dinv, z.dinv, "diagonal inverses")) != TD_OK))
    goto fail_r;
  if ((h.flags & CK_GS) && ((r = alloc_dev(&g.S1, z.gs_s, "GSCE spectra")) != TD_OK ||
                            (r = alloc_dev(&g.S2, z.gs_s, "GSCE spectra")) != TD_OK ||
                            (r = alloc_dev(&g.tw, z.gs_tw, "GSCE twiddles")) != TD_OK))
    goto fail_r;
  ok = true;
  if (h.flags & CK_OP) ok = read_dev(f, s->op, z.op, buf, sum, st, err);
  if (ok && (h.flags & CK_FP64))
    ok = read_dev(f, s->L, z.L, buf, sum, st, err) && read_dev(f, s->dinv, z.dinv, buf, sum, st, err);
  if (ok && (h.flags & CK_GS))
    ok = read_dev(f, g.S1, z.gs_s, buf, sum, st, err) && read_dev(f, g.S2, z.gs_s, buf, sum, st, err) &&
         read_dev(f, g.tw, z.gs_tw, buf, sum, st, err);
  if (ok && sum.h != h.checksum) {
    ok = false;
    err = "checksum mismatch (corrupted file)";
  }
  fclose(f);
  if (!ok) {
    td_segment_destroy(s);
    return fail(err.rfind("device", 0) == 0 ? TD_ERR_CUDA : TD_ERR_INVALID, "td_segment_load: " + err);
  }
  if (h.flags & CK_OP) s->op_blocks = h.op_blocks;
  s->logdet = h.logdet;
  s->factored = h.factored != 0;
  if (h.flags & CK_GS) {
    g.logm = h.gs_logm;
    g.x0 = h.gs_x0;
    g.logdet = h.gs_logdet;
    g.ready = true;
  }
  *out = s;
  return TD_OK;
fail_r:
  fclose(f);
  td_segment_destroy(s);
  return r;
}
