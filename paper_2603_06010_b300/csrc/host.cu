// Evaluation with host buffers: the batch (Sec. II.A, W = L^{-1}; Sec. III.A,
// the batched evaluation of cached operators) arrives in CPU memory and the
// results go back to CPU memory.  Column chunks are double-buffered: chunk
// j+1 is copied host -> device on the segment's copy stream while chunk j is
// evaluated on the caller's stream, so the transfer, not the evaluation, sets
// the pace.  Each chunk goes through td_loglike_batch, so every column gets
// the same bits as on the device-buffer path with the same options.
#include <algorithm>
#include <string>
#include <utility>
#include <vector>

#include "td_internal.h"

namespace td {

void free_host_stage(HostStage& h) {
  for (int b = 0; b < 2; ++b) {
    if (h.buf[b]) cudaFree(h.buf[b]);
    h.buf[b] = nullptr;
    if (h.copied[b]) cudaEventDestroy(h.copied[b]);
    if (h.consumed[b]) cudaEventDestroy(h.consumed[b]);
    h.copied[b] = h.consumed[b] = nullptr;
  }
  if (h.logL) cudaFree(h.logL);
  if (h.chi2) cudaFree(h.chi2);
  h.logL = h.chi2 = nullptr;
  if (h.copy) cudaStreamDestroy(h.copy);
  h.copy = nullptr;
  h.cols = h.cap = 0;
}

static td_status ensure_stage(td_segment* s, int64_t cols, int64_t K) {
  HostStage& h = s->hst;
  if (!h.copy) {
    if (cudaStreamCreateWithFlags(&h.copy, cudaStreamNonBlocking) != cudaSuccess)
      return cuda_fail(cudaGetLastError(), "copy stream");
    for (int b = 0; b < 2; ++b)
      if (cudaEventCreateWithFlags(&h.copied[b], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&h.consumed[b], cudaEventDisableTiming) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "stage events");
  }
  if (cols > h.cols) {
    for (int b = 0; b < 2; ++b) {
      if (h.buf[b]) cudaFree(h.buf[b]);
      h.buf[b] = nullptr;
    }
    h.cols = 0;
    for (int b = 0; b < 2; ++b)
      if (cudaMalloc((void**)&h.buf[b], (size_t)cols * s->nk * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return fail(TD_ERR_OOM, "host-batch staging buffers");
      }
    h.cols = cols;
  }
  if (K > h.cap) {
    if (h.logL) cudaFree(h.logL);
    if (h.chi2) cudaFree(h.chi2);
    h.logL = h.chi2 = nullptr;
    h.cap = 0;
    if (cudaMalloc((void**)&h.logL, (size_t)K * 8) != cudaSuccess ||
        cudaMalloc((void**)&h.chi2, (size_t)K * 8) != cudaSuccess) {
      cudaGetLastError();
      return fail(TD_ERR_OOM, "host-batch result buffers");
    }
    h.cap = K;
  }
  return TD_OK;
}

}  // namespace td

using namespace td;

extern "C" td_status td_loglike_batch_host(td_segment* s, const float* R, int64_t ldr, int64_t K, double* logL,
                                           const td_options* opt, double* chi2, void* stream) {
  if (!s || (K > 0 && (!R || !logL)) || K < 0) return fail(TD_ERR_INVALID, "bad arguments");
  if (K == 0) return TD_OK;
  if (ldr < s->nk) return fail(TD_ERR_INVALID, "ldr < N'");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != s->device) return fail(TD_ERR_INVALID, "segment belongs to another device; set it current first");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // chunks of 512 columns: small enough that the first copy is short, large
  // enough that each evaluation still fills the GPU.  The copies set the pace
  // and the last evaluation is the only one nothing overlaps, so the last
  // chunk is at most 128 columns (N' = 8192, K = 4096: 2.6 against 2.7 ms)
  const int64_t cols = std::min<int64_t>(K, 512);
  std::vector<std::pair<int64_t, int64_t>> chunks;   // (first column, columns)
  for (int64_t c0 = 0; c0 < K;) {
    const int64_t left = K - c0;
    const int64_t kc = left > cols + 128 ? cols : (left > 128 ? left - 128 : left);
    chunks.emplace_back(c0, kc);
    c0 += kc;
  }
  td_status r = ensure_stage(s, cols, K);
  if (r != TD_OK) return r;
  if ((r = td_reserve(s, cols, opt)) != TD_OK) return r;
  HostStage& h = s->hst;
  const int64_t nk = s->nk;
  const int64_t nch = (int64_t)chunks.size();
  for (int64_t j = 0; j < nch; ++j) {
    const int b = (int)(j & 1);
    const int64_t c0 = chunks[(size_t)j].first, kc = chunks[(size_t)j].second;
    if (j >= 2) TD_CUDA(cudaStreamWaitEvent(h.copy, h.consumed[b], 0));   // buffer free again
    TD_CUDA(cudaMemcpy2DAsync(h.buf[b], (size_t)nk * sizeof(float), R + c0 * ldr, (size_t)ldr * sizeof(float),
                              (size_t)nk * sizeof(float), (size_t)kc, cudaMemcpyHostToDevice, h.copy));
    TD_CUDA(cudaEventRecord(h.copied[b], h.copy));
    TD_CUDA(cudaStreamWaitEvent(st, h.copied[b], 0));
    if ((r = td_loglike_batch(s, h.buf[b], nk, kc, h.logL + c0, opt, chi2 ? h.chi2 + c0 : nullptr, stream)) != TD_OK)
      return r;
    TD_CUDA(cudaEventRecord(h.consumed[b], st));
  }
  TD_CUDA(cudaMemcpyAsync(logL, h.logL, (size_t)K * 8, cudaMemcpyDeviceToHost, st));
  if (chi2) TD_CUDA(cudaMemcpyAsync(chi2, h.chi2, (size_t)K * 8, cudaMemcpyDeviceToHost, st));
  TD_CUDA(cudaStreamSynchronize(st));
  return TD_OK;
}
