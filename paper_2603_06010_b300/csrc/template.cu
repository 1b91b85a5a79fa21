// Template-input evaluation (Sec. III.A, the production CDO form: the data
// vector is fixed, every evaluation brings a template h), with the SNRs of
// Sec. II.B item 7:
//   <a, b> = a^T C^{-1} b = (L^{-1} a) . (L^{-1} b)      (Eq. eqn:ip)
//   chi2   = <d - h, d - h>,   logL = -chi2/2 - logdet/2 - (N'/2) log 2 pi
//   rho_mf = <d, h> / sqrt(<h, h>),   rho_eff^2 = <d, d> - <d - h, d - h>
// <d, d> is computed once by td_set_data.  A batch forms r_k = d - h_k (the
// FP64 difference rounded once to FP32) and, when <h, h> is asked for,
// appends the templates themselves; both go through td_loglike_batch, and
// <d, h> = (<d, d> + <h, h> - chi2) / 2.  td_project_batch forms the templates
// on the device from polarizations, antenna factors and sample offsets
// (detector projection and placement, fused ahead of the same path).
#include <algorithm>
#include <string>

#include "td_internal.h"

namespace td {

// R[:, k] = fl32(d - H[:, k]) for k < K; R[:, K + k] = H[:, k] when with_h;
// with K = 0 and H = nullptr: R[:, 0] = fl32(d)
__global__ void k_form_residuals(const double* __restrict__ d, const float* __restrict__ H, int64_t ldh,
                                 int64_t nk, int64_t K, int with_h, float* __restrict__ R) {
  const int64_t k = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nk; i += (int64_t)gridDim.x * blockDim.x) {
    if (!H) {
      R[i] = (float)d[i];
      continue;
    }
    const float hv = H[k * ldh + i];
    R[k * nk + i] = (float)(d[i] - (double)hv);
    if (with_h) R[(K + k) * nk + i] = hv;
  }
}

// Detector projection and placement (Sec. II.B waveform conditioning; Sec.
// III.A data projection and conditioning), gathered to the kept samples:
//   h_k(t) = fp[k] hp[k][t - off[k]] + fc[k] hc[k][t - off[k]]  for 0 <= t - off[k] < lw, else 0
//   R[:, k] = fl32(d - h_k(t_j)),  R[:, K + k] = h_k(t_j) when with_h.
// h is formed in FP32 (antenna factors rounded to FP32, products and sum
// rounded one operation at a time, no contraction) and subtracted from d in
// FP64 as in td_template_batch: the batch equals td_template_batch on the
// templates fl32(fl32(fp hp) + fl32(fc hc)) built anywhere, bit for bit.  The
// FP32 sum adds one rounding of h, the size of the FP32 rounding of r itself;
// FP64 products here would cost more than the whole residual pass (FP64 runs
// at about 1.2 TFLOP/s on this GPU).
__global__ void k_project_residuals(const double* __restrict__ d, const int32_t* __restrict__ t,
                                    const float* __restrict__ hp, const float* __restrict__ hc, int64_t ldw,
                                    int64_t lw, const double* __restrict__ fp, const double* __restrict__ fc,
                                    const int64_t* __restrict__ off, int64_t nk, int64_t K, int with_h,
                                    float* __restrict__ R) {
  const int64_t k = blockIdx.y;
  const float a = (float)fp[k], b = hc ? (float)fc[k] : 0.f;
  const int64_t o = off[k];
  const float* wp = hp + k * ldw;
  const float* wc = hc ? hc + k * ldw : nullptr;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nk; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = (int64_t)t[i] - o;
    float h = 0.f;
    if (u >= 0 && u < lw) {
      h = __fmul_rn(a, wp[u]);
      if (wc) h = __fadd_rn(h, __fmul_rn(b, wc[u]));
    }
    R[k * nk + i] = (float)(d[i] - (double)h);
    if (with_h) R[(K + k) * nk + i] = h;
  }
}

// G[:, k] = R[t_j, k]: the kept rows of a full-length column-major batch
__global__ void k_gather_kept(const float* __restrict__ R, int64_t ldr, const int32_t* __restrict__ t, int64_t nk,
                              float* __restrict__ G) {
  const int64_t k = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nk; i += (int64_t)gridDim.x * blockDim.x)
    G[k * nk + i] = R[k * ldr + t[i]];
}

__global__ void k_template_finalize(const double* __restrict__ ll, const double* __restrict__ c2, int64_t K,
                                    int with_h, double dd, td_template_out out) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= K) return;
  const double chi2 = c2[k];
  out.logL[k] = ll[k];
  if (out.chi2) out.chi2[k] = chi2;
  if (out.rho_eff2) out.rho_eff2[k] = dd - chi2;
  if (with_h) {
    const double hh = c2[K + k];
    const double dh = 0.5 * (dd + hh - chi2);
    if (out.hh) out.hh[k] = hh;
    if (out.dh) out.dh[k] = dh;
    if (out.rho_mf) out.rho_mf[k] = hh > 0.0 ? dh / sqrt(hh) : 0.0;
  }
}

void free_template_state(TemplateState& T) {
  if (T.d) cudaFree(T.d);
  if (T.R) cudaFree(T.R);
  if (T.res) cudaFree(T.res);
  T = TemplateState{};
}

static td_status grow(void** p, size_t& cap, size_t bytes, const char* what) {
  if (bytes <= cap) return TD_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  cap = 0;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(TD_ERR_OOM, what);
  }
  cap = bytes;
  return TD_OK;
}

static unsigned row_blocks(int64_t nk) { return (unsigned)std::min<int64_t>(ceil_div(nk, 256), 512); }

}  // namespace td

using namespace td;

extern "C" td_status td_set_data(td_segment* s, const double* d, const td_options* opt, void* stream) {
  if (!s || !d) return fail(TD_ERR_INVALID, "NULL argument");
  if (!s->factored) return fail(TD_ERR_NOT_FACTORED, "segment not factored");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  TemplateState& T = s->tpl;
  T.has_data = false;
  td_status r;
  if ((r = grow((void**)&T.d, T.d_cap, (size_t)s->nk * 8, "data vector")) != TD_OK) return r;
  if ((r = grow((void**)&T.R, T.R_cap, (size_t)s->nk * 4, "template residuals")) != TD_OK) return r;
  if ((r = grow((void**)&T.res, T.res_cap, 2 * 8, "template results")) != TD_OK) return r;
  TD_CUDA(cudaMemcpyAsync(T.d, d, (size_t)s->nk * 8, cudaMemcpyDefault, st));
  // <d, d> = |L^{-1} d|^2: d rounded once to FP32, whitened by the batch path
  k_form_residuals<<<dim3(row_blocks(s->nk), 1), 256, 0, st>>>(T.d, nullptr, 0, s->nk, 0, 0, T.R);
  TD_CUDA(cudaGetLastError());
  if ((r = td_loglike_batch(s, T.R, s->nk, 1, T.res, opt, T.res + 1, stream)) != TD_OK) return r;
  double dd = 0.0;
  TD_CUDA(cudaMemcpyAsync(&dd, T.res + 1, 8, cudaMemcpyDeviceToHost, st));
  TD_CUDA(cudaStreamSynchronize(st));
  T.dd = dd;
  T.has_data = true;
  return TD_OK;
}

extern "C" td_status td_data_inner(const td_segment* s, double* dd) {
  if (!s || !dd) return fail(TD_ERR_INVALID, "NULL argument");
  if (!s->tpl.has_data) return fail(TD_ERR_INVALID, "no data vector set (td_set_data)");
  *dd = s->tpl.dd;
  return TD_OK;
}

// the batch of residuals (and templates) already in T.R through the dense path
static td_status template_tail(td_segment* s, int64_t K, int with_h, const td_template_out* out,
                               const td_options* opt, void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  TemplateState& T = s->tpl;
  const int64_t Kt = with_h ? 2 * K : K;
  double* ll = T.res;
  double* c2 = T.res + Kt;
  td_status r;
  if ((r = td_loglike_batch(s, T.R, s->nk, Kt, ll, opt, c2, stream)) != TD_OK) return r;
  k_template_finalize<<<(unsigned)ceil_div(K, 256), 256, 0, st>>>(ll, c2, K, with_h, T.dd, *out);
  TD_CUDA(cudaGetLastError());
  return TD_OK;
}

static td_status template_buffers(td_segment* s, int64_t K, int with_h) {
  TemplateState& T = s->tpl;
  const int64_t Kt = with_h ? 2 * K : K;
  td_status r;
  if ((r = grow((void**)&T.R, T.R_cap, (size_t)Kt * s->nk * 4, "template residuals")) != TD_OK) return r;
  return grow((void**)&T.res, T.res_cap, (size_t)2 * Kt * 8, "template results");
}

extern "C" td_status td_template_batch(td_segment* s, const float* H, int64_t ldh, int64_t K,
                                       const td_template_out* out, const td_options* opt, void* stream) {
  if (!s || !out || K < 0 || (K > 0 && (!H || !out->logL))) return fail(TD_ERR_INVALID, "bad arguments");
  if (!s->tpl.has_data) return fail(TD_ERR_INVALID, "no data vector set (td_set_data)");
  if (K == 0) return TD_OK;
  if (ldh < s->nk) return fail(TD_ERR_INVALID, "ldh < N'");
  if (K > 65535) return fail(TD_ERR_INVALID, "at most 65535 templates per call");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  TemplateState& T = s->tpl;
  const int with_h = (out->hh || out->dh || out->rho_mf) ? 1 : 0;
  td_status r;
  if ((r = template_buffers(s, K, with_h)) != TD_OK) return r;
  k_form_residuals<<<dim3(row_blocks(s->nk), (unsigned)K), 256, 0, st>>>(T.d, H, ldh, s->nk, K, with_h, T.R);
  TD_CUDA(cudaGetLastError());
  return template_tail(s, K, with_h, out, opt, stream);
}

extern "C" td_status td_project_batch(td_segment* s, const float* hp, const float* hc, int64_t ldw, int64_t lw,
                                      int64_t K, const double* fp, const double* fc, const int64_t* offset,
                                      const td_template_out* out, const td_options* opt, void* stream) {
  if (!s || !out || K < 0 || lw < 0) return fail(TD_ERR_INVALID, "bad arguments");
  if (K > 0 && (!out->logL || !hp || !fp || !offset || (hc && !fc)))
    return fail(TD_ERR_INVALID, "NULL argument (hp, fp, offset, logL; fc with hc)");
  if (!s->tpl.has_data) return fail(TD_ERR_INVALID, "no data vector set (td_set_data)");
  if (K == 0) return TD_OK;
  if (ldw < lw || ldw < 1) return fail(TD_ERR_INVALID, "ldw < lw");
  if (K > 65535) return fail(TD_ERR_INVALID, "at most 65535 templates per call");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  TemplateState& T = s->tpl;
  const int with_h = (out->hh || out->dh || out->rho_mf) ? 1 : 0;
  td_status r;
  if ((r = template_buffers(s, K, with_h)) != TD_OK) return r;
  k_project_residuals<<<dim3(row_blocks(s->nk), (unsigned)K), 256, 0, st>>>(T.d, s->t, hp, hc, ldw, lw, fp, fc,
                                                                           offset, s->nk, K, with_h, T.R);
  TD_CUDA(cudaGetLastError());
  return template_tail(s, K, with_h, out, opt, stream);
}

extern "C" td_status td_loglike_batch_gather(td_segment* s, const float* R, int64_t ldr, int64_t K, double* logL,
                                             const td_options* opt, double* chi2, void* stream) {
  if (!s || K < 0 || (K > 0 && (!R || !logL))) return fail(TD_ERR_INVALID, "bad arguments");
  if (K == 0) return TD_OK;
  if (ldr < s->n) return fail(TD_ERR_INVALID, "ldr < n (full-length columns)");
  if (K > 65535) return fail(TD_ERR_INVALID, "at most 65535 columns per call");
  if (!s->factored && !s->gs.ready) return fail(TD_ERR_NOT_FACTORED, "segment not factored");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (K > s->gat_cap) {
    cudaStreamSynchronize(st);   // the old buffer may still be read on this stream
    if (s->gat) cudaFree(s->gat);
    s->gat = nullptr;
    s->gat_cap = 0;
    if (cudaMalloc((void**)&s->gat, (size_t)K * s->nk * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return fail(TD_ERR_OOM, "gather buffer");
    }
    s->gat_cap = K;
  }
  k_gather_kept<<<dim3(row_blocks(s->nk), (unsigned)K), 256, 0, st>>>(R, ldr, s->t, s->nk, s->gat);
  TD_CUDA(cudaGetLastError());
  return td_loglike_batch(s, s->gat, s->nk, K, logL, opt, chi2, stream);
}
