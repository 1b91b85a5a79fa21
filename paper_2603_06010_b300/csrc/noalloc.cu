// td_loglike_batch_noalloc: the tensor-core likelihood batch with its scratch
// in a fixed, file-scope device array instead of memory from cudaMalloc.
//
// Who needs it: callers that cannot enter the CUDA allocator once they are
// running -- a host application whose device memory is all reserved by its
// own caching pool (so a cudaMalloc from this library would fail or evict
// its cache), a process under a hard device-memory cap, or a latency-critical
// sampler loop that must not call cudaMalloc (which can synchronise the
// device).  Such a caller still passes its own inputs and outputs; the
// residual slices and chi2 partials live in g_noalloc_scratch, which every
// GPU that loads this library holds (TD_NOALLOC_SCRATCH_BYTES) until the
// process exits.
//
// Host code must not use the array's name as a device address: on the host it
// is only a stand-in symbol.  The device address is looked up once per device
// with cudaGetSymbolAddress (with that device current) on the first call made
// on the device and cached.  That first call should therefore happen before
// any stream capture.
//
// All calls share the one array, and each call overwrites the part it uses:
// calls whose kernels overlap on the GPU (different streams, or different
// segments at once) race on it.  Every scratch byte a call reads is written
// earlier in the same call, so nothing has to start at zero.
#include <cudaTypedefs.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "td_internal.h"

namespace td {

static __device__ __align__(256) unsigned char g_noalloc_scratch[TD_NOALLOC_SCRATCH_BYTES];

static std::mutex g_na_mu;
static void* g_na_ptr[128] = {nullptr};
static PFN_cuTensorMapEncodeTiled_v12000 g_na_encode = nullptr;

// device address of g_noalloc_scratch for the current device (set up once per device)
static td_status noalloc_scratch(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 128) return fail(TD_ERR_UNSUPPORTED, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    g_na_ptr[dev] = p;
  }
  if (!g_na_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return fail(TD_ERR_CUDA, "cuTensorMapEncodeTiled entry point not available");
    g_na_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  *out = g_na_ptr[dev];
  return TD_OK;
}

static td_status na_encode(CUtensorMap* map, const void* ptr, uint64_t d0, uint64_t d1, uint64_t d2,
                           uint64_t s1, uint64_t s2, uint32_t b0, uint32_t b1, uint32_t b2) {
  cuuint64_t dims[3] = {d0, d1, d2};
  cuuint64_t strides[2] = {s1, s2};
  cuuint32_t box[3] = {b0, b1, b2};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = g_na_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(ptr), dims, strides, box,
                           es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(TD_ERR_CUDA, "cuTensorMapEncodeTiled failed (no-alloc path)");
  return TD_OK;
}

}  // namespace td

using namespace td;

extern "C" td_status td_loglike_batch_noalloc(td_segment* s, const float* R, int64_t ldr, int64_t K,
                                              double* logL, double* chi2, void* stream) {
  if (!s) return fail(TD_ERR_INVALID, "segment is NULL");
  if (K < 0) return fail(TD_ERR_INVALID, "K < 0");
  if (K > TD_MAX_K) return fail(TD_ERR_INVALID, "K above 2^30 columns");
  if (K == 0) return TD_OK;
  if (!R || !logL) return fail(TD_ERR_INVALID, "R or logL is NULL");
  if (ldr < s->nk) return fail(TD_ERR_INVALID, "ldr < N'");
  if (!s->factored) return fail(TD_ERR_NOT_FACTORED, "segment not factored");
  if (!s->op) return fail(TD_ERR_NOT_FACTORED, "the operator of this segment is not resident");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != s->device) return fail(TD_ERR_INVALID, "segment belongs to another device; set it current first");
  // scratch layout: residual slices [4][K][nkp8] bf16, then chi2 partials [N'p/64][K] f64
  const int64_t nm = s->nkp / 64;
  const int64_t rs_bytes = (int64_t)OP_SLICES * K * s->nkp8 * 2;
  const int64_t part_off = round_up(rs_bytes, 256);
  const int64_t need = part_off + nm * K * 8;
  if (need > (int64_t)TD_NOALLOC_SCRATCH_BYTES) {
    char buf[200];
    snprintf(buf, sizeof buf,
             "batch needs %lld scratch bytes (about 8 K N' for residual slices plus 8 K N'/64 for chi2 "
             "partials), above the fixed %lld-byte no-alloc scratch; use a smaller K or td_loglike_batch",
             (long long)need, (long long)TD_NOALLOC_SCRATCH_BYTES);
    return fail(TD_ERR_INVALID, buf);
  }
  void* base = nullptr;
  td_status r = noalloc_scratch(&base);
  if (r != TD_OK) return r;
  __nv_bfloat16* rs = reinterpret_cast<__nv_bfloat16*>(base);
  double* partials = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(base) + part_off);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // the slice count td_loglike_batch takes with its default options (ten
  // products below 2048 and above 32768 kept samples, six between)
  const int nsl = nslices_for(TD_PREC_AUTO, s->nk);

  TcSegDev seg;
  memset(&seg, 0, sizeof seg);
  if ((r = na_encode(&seg.mapA, rs, (uint64_t)s->nk, (uint64_t)K, OP_SLICES, (uint64_t)s->nkp8 * 2,
                     (uint64_t)K * s->nkp8 * 2, OP_KB, TC_COLS, 1)) != TD_OK)
    return r;
  if ((r = na_encode(&seg.mapB, s->op, OP_KB, OP_ROWS, (uint64_t)s->op_blocks * OP_SLICES, OP_KB * 2,
                     (uint64_t)OP_ROWS * OP_KB * 2, OP_KB, 64, (uint32_t)nsl)) != TD_OK)
    return r;
  seg.partials = partials;
  seg.a_rows = TC_COLS;
  seg.nk = (int)s->nk;
  seg.K = (int)K;
  seg.ldp = (int)K;
  seg.nm = (int)nm;
  TD_CUDA(launch_r_slices(R, ldr, s->nk, K, s->nkp8, K, rs, nsl, st));
  TD_CUDA(launch_tc_single(seg, 64, (int)ceil_div(K, TC_COLS), (int)ceil_div(s->nk, OP_KB), nsl,
                           s->status, 1000000000LL, st));
  TD_CUDA(launch_finalize(partials, K, (int)nm, K, s->logdet, s->nk, logL, chi2, st));
  return TD_OK;
}
