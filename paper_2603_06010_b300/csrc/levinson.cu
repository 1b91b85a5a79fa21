// Whitening operator of a gap-free segment in O(N^2) by the Levinson-Durbin
// recursion (Sec. II.B item 6 cites Levinson and Durbin for re-truncating the
// ACF of a segment).
//
// For a stationary (Toeplitz) covariance the Cholesky whitening L^{-1} is the
// causal prediction-error filter: with a_t the order-t forward predictor of
// x_t from x_{t-1} .. x_0 and v_t its error variance,
//   (L^{-1} r)_t = (r_t - sum_j a_{t,j} r_{t-j}) / sqrt(v_t),
// so row t of L^{-1} is (-a_{t,t} .. -a_{t,1}, 1) / sqrt(v_t), and
// log det C = sum_t log v_t.  The recursion (reflection coefficient k_t,
// a_t = [a_{t-1} - k_t rev(a_{t-1}), k_t], v_t = v_{t-1}(1 - k_t^2)) costs
// O(t) per order, O(N^2) in all, instead of the O(N^3) Cholesky plus
// inverse.  It runs in FP64.
//
// k_levinson_rows: one CTA per segment (1024 threads).  The orders form a
// chain; the O(t) work of an order (one dot product, one predictor update,
// one row of L^{-1}) is spread over the threads, the predictor lives in
// global memory (L2-resident), and each row is stored in FP64, row-major.
// FP64 is a slow pipe on this part, so the chain does only these three
// multiply-adds per element; the per-row quantum and the bf16 slicing then
// run over all SMs in the same kernels the Cholesky route uses.  Segments
// are independent: one launch runs many chains at once.
#include <algorithm>
#include <climits>
#include <string>
#include <vector>

#include "td_internal.h"

namespace td {

struct LevJob {
  const double* acf;       // device, n lags
  int64_t n;               // samples (gap-free: N' = n)
  double* a0;              // device scratch, n doubles
  double* a1;              // device scratch, n doubles
  double* linv;            // device, row t at linv + t ld, columns 0..t written
  int64_t ld;
  double* logdet;          // device, one double
  DevStatus* status;       // NOT_PD pivot
};

constexpr int LEV_THREADS = 1024;
constexpr int64_t LEV_MAX_N = 1 << 20;

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < LEV_THREADS / 32; ++i) s += red[i];   // fixed order
    red[32] = s;
  }
  __syncthreads();
  return red[32];
}

__global__ void __launch_bounds__(LEV_THREADS, 1) k_levinson_rows(const LevJob* __restrict__ jobs) {
  __shared__ double red[40];
  __shared__ double sh_v;
  __shared__ int sh_bad;
  const LevJob jb = jobs[blockIdx.x];
  const int64_t n = jb.n;
  const int tid = threadIdx.x;
  double* a = jb.a0;      // a_{t-1}[1..t-1]
  double* an = jb.a1;     // a_t
  double logdet = 0.0;
  if (tid == 0) {
    sh_v = jb.acf[0];
    sh_bad = !(sh_v > 0.0) || !isfinite(sh_v);
    if (sh_bad) {
      atomicMin((unsigned long long*)&jb.status->pivot, 0ull);
      atomicCAS(&jb.status->code, 0, ST_NOT_PD);
    }
  }
  __syncthreads();
  for (int64_t t = 0; t < n && !sh_bad; ++t) {
    if (t > 0) {
      // k_t = (acf[t] - sum_{j=1}^{t-1} a_{t-1,j} acf[t-j]) / v_{t-1}
      double part = 0.0;
      for (int64_t j = 1 + tid; j < t; j += LEV_THREADS) part = fma(a[j], jb.acf[t - j], part);
      const double dot = block_sum(part, red);   // ends in a barrier: sh_v is settled
      const double vprev = sh_v;
      const double k = (jb.acf[t] - dot) / vprev;
      const double v = vprev * (1.0 - k * k);
      if (!(v > 0.0) || !isfinite(v)) {
        if (tid == 0) {
          atomicMin((unsigned long long*)&jb.status->pivot, (unsigned long long)t);
          atomicCAS(&jb.status->code, 0, ST_NOT_PD);
        }
        break;   // every thread computed the same v
      }
      for (int64_t j = 1 + tid; j < t; j += LEV_THREADS) an[j] = fma(-k, a[t - j], a[j]);
      if (tid == 0) an[t] = k;
      __syncthreads();   // a_t complete; everyone has read v_{t-1}
      if (tid == 0) sh_v = v;
      double* tmp = a;   // a <- a_t
      a = an;
      an = tmp;
    }
    __syncthreads();
    const double vt = sh_v;
    if (tid == 0) logdet += log(vt);
    // row t of L^{-1}: column c < t holds -a_{t, t-c} / sqrt(v_t), column t holds 1 / sqrt(v_t)
    const double inv = 1.0 / sqrt(vt);
    double* row = jb.linv + t * jb.ld;
    for (int64_t c = tid; c < t; c += LEV_THREADS) row[c] = -a[t - c] * inv;
    if (tid == 0) row[t] = inv;
  }
  if (tid == 0) *jb.logdet = logdet;
}

cudaError_t launch_levinson_rows(const LevJob* jobs, int njobs, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  k_levinson_rows<<<njobs, LEV_THREADS, 0, st>>>(jobs);
  return cudaGetLastError();
}

}  // namespace td

using namespace td;

namespace {

struct LevSeg {
  td_segment* s;
  double* linv = nullptr;
  double* qrow = nullptr;
  double* a0 = nullptr;
  double* a1 = nullptr;
  double* ld = nullptr;
};

void free_lev(LevSeg& x) {
  for (double** p : {&x.linv, &x.qrow, &x.a0, &x.a1, &x.ld}) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
}

// One batch: the chains in one launch, then per segment the row quanta and slices.
td_status run_lev_batch(std::vector<LevSeg>& b, cudaStream_t st) {
  std::vector<LevJob> jobs;
  td_status r = TD_OK;
  for (LevSeg& x : b) {
    td_segment* s = x.s;
    const size_t op_bytes = (size_t)s->op_blocks * OP_SLICES * OP_ROWS * OP_KB * 2;
    if (!s->op && cudaMalloc((void**)&s->op, op_bytes) != cudaSuccess) {
      cudaGetLastError();
      s->op = nullptr;
      r = fail(TD_ERR_OOM, "operator slices");
      break;
    }
    if (cudaMalloc((void**)&x.linv, (size_t)s->nkp * s->nkp * 8) != cudaSuccess ||
        cudaMalloc((void**)&x.qrow, (size_t)s->nkp * 8) != cudaSuccess ||
        cudaMalloc((void**)&x.a0, (size_t)s->n * 8) != cudaSuccess ||
        cudaMalloc((void**)&x.a1, (size_t)s->n * 8) != cudaSuccess || cudaMalloc((void**)&x.ld, 8) != cudaSuccess) {
      cudaGetLastError();
      r = fail(TD_ERR_OOM, "Levinson scratch");
      break;
    }
    DevStatus h{0, 0, LLONG_MAX};
    cudaMemcpyAsync(s->status, &h, sizeof h, cudaMemcpyHostToDevice, st);
    jobs.push_back(LevJob{s->acf, s->n, x.a0, x.a1, x.linv, s->nkp, x.ld, s->status});
  }
  LevJob* dj = nullptr;
  if (r == TD_OK) {
    cudaError_t e = cudaMalloc((void**)&dj, jobs.size() * sizeof(LevJob));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dj, jobs.data(), jobs.size() * sizeof(LevJob), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_levinson_rows(dj, (int)jobs.size(), st);
    // the rows of a chain that stopped (not positive definite) are sliced too but never used
    for (size_t i = 0; i < b.size() && e == cudaSuccess; ++i) {
      td_segment* s = b[i].s;
      e = launch_row_quantum(b[i].linv, s->nkp, s->nk, s->nkp, b[i].qrow, st, true);
      if (e == cudaSuccess) e = launch_op_slices(b[i].linv, s->nkp, s->nk, s->nkp, b[i].qrow, s->op, st, true);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) r = fail(TD_ERR_CUDA, std::string("Levinson operator build: ") + cudaGetErrorString(e));
  }
  if (r == TD_OK) {
    for (size_t i = 0; i < b.size(); ++i) {
      td_segment* s = b[i].s;
      DevStatus hs;
      double ldv = 0.0;
      cudaMemcpy(&hs, s->status, sizeof hs, cudaMemcpyDeviceToHost);
      cudaMemcpy(&ldv, b[i].ld, 8, cudaMemcpyDeviceToHost);
      if (hs.code == ST_NOT_PD) {
        s->pivot = hs.pivot;
        if (r == TD_OK) {
          char buf[128];
          snprintf(buf, sizeof buf, "covariance not positive definite at kept sample %lld", (long long)hs.pivot);
          r = fail(TD_ERR_NOT_PD, buf);
        }
        continue;
      }
      s->logdet = ldv;
      s->factored = true;
    }
  }
  if (dj) cudaFree(dj);
  for (LevSeg& x : b) free_lev(x);
  return r;
}

}  // namespace

// Gap-free segments get their operator from the recursion, in batches whose
// FP64 row buffers (N'^2 doubles each) fit a bounded share of free memory;
// segments with gaps are factored by the blocked Cholesky.  The FP64 factor L
// is not formed on the recursion route, so those segments' FP64 path is
// unavailable (TD_ERR_UNSUPPORTED); the tensor-core paths are.
extern "C" td_status td_factor_many(td_segment* const* segs, int nseg, int flags, void* stream) {
  if (nseg < 0 || (nseg > 0 && !segs)) return fail(TD_ERR_INVALID, "bad arguments");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = -1;
  cudaGetDevice(&dev);
  for (int i = 0; i < nseg; ++i) {
    if (!segs[i]) return fail(TD_ERR_INVALID, "NULL segment");
    if (dev != segs[i]->device) return fail(TD_ERR_INVALID, "segment belongs to another device; set it current first");
  }
  std::vector<td_segment*> lev;
  td_status first_err = TD_OK;
  for (int i = 0; i < nseg; ++i) {
    td_segment* s = segs[i];
    const bool gapfree = (s->nk == s->n);
    if (!(flags & TD_FACTOR_NO_FP64) || !gapfree || s->nk > LEV_MAX_N) {
      const td_status r = td_factor(s, stream);
      if (r == TD_OK && (flags & TD_FACTOR_NO_FP64)) td_segment_release_fp64(s);
      if (r == TD_OK) continue;
      if (r != TD_ERR_NOT_PD) return r;
      if (first_err == TD_OK) first_err = r;
      continue;
    }
    s->factored = false;
    s->pivot = -1;
    td_segment_release_fp64(s);   // a factor from an earlier td_factor would be stale
    s->op_blocks = op_row_offset(s->nkp / OP_ROWS);
    lev.push_back(s);
  }
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  const size_t budget = std::max<size_t>((size_t)1 << 30, std::min<size_t>(free_b / 3, (size_t)32 << 30));
  std::vector<LevSeg> batch;
  size_t used = 0;
  for (size_t i = 0; i <= lev.size(); ++i) {
    const size_t need = i < lev.size() ? (size_t)lev[i]->nkp * lev[i]->nkp * 8 : 0;
    if (!batch.empty() && (i == lev.size() || used + need > budget)) {
      const td_status rb = run_lev_batch(batch, st);
      if (rb != TD_OK && rb != TD_ERR_NOT_PD) return rb;
      if (rb != TD_OK && first_err == TD_OK) first_err = rb;
      batch.clear();
      used = 0;
    }
    if (i < lev.size()) {
      batch.push_back(LevSeg{lev[i]});
      used += need;
    }
  }
  return first_err;
}
