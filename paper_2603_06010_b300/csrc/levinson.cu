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
// k_levinson_rows: one cluster of up to 8 CTAs x 1024 threads per segment.  The
// orders form a chain; the O(t) work of an order (one dot product, one
// predictor update, one row of L^{-1}) is spread over the cluster, the
// predictor lives in global memory (L2-resident), and each row is stored in
// FP64, row-major.  The order's scalars are formed by one thread per CTA.
// FP64 is a slow pipe on this part, so the chain does only these three
// multiply-adds per element; the per-row quantum and the bf16 slicing then
// run over all SMs in the same kernels the Cholesky route uses.  Segments
// are independent: one launch runs many chains at once.
#include <algorithm>
#include <climits>
#include <string>
#include <vector>

#include <cooperative_groups.h>

#include "td_internal.h"

namespace cg = cooperative_groups;

namespace td {


constexpr int LEV_THREADS = 1024;
constexpr int64_t LEV_MAX_N = 1 << 20;

// Sum of the block's values in a fixed order, into lane 0 of warp 0: the
// values go through shared memory to one warp (each lane adds 32 of them in
// order, then a fixed shuffle tree).  FP64 is a slow pipe on this part, so the
// reduction keeps FP64 adds to one warp rather than a shuffle tree in every warp.
__device__ __forceinline__ double block_sum_to_lead(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    for (int i = threadIdx.x; i < LEV_THREADS; i += 32) s += red[i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  }
  return s;   // valid in thread 0
}

// One thread-block cluster of CL CTAs per segment (CL = 1: one CTA): the
// O(t) work of an order is spread over CL x 1024 threads (element j to
// cluster thread (j - 1) mod CL*1024, so warps stay coalesced, the mirrored
// index too).  Per order: each CTA's dot-product partial; one cluster barrier
// (order t's dot product reads only the predictor elements this thread itself
// wrote at order t-1, the newest one, k_{t-1}, from a register, so it needs
// no barrier before it); thread 0 of every CTA then adds the CL partials in
// rank order and forms k_t, v_t and 1/sqrt(v_{t-1}) (the same bits in every
// CTA), which one CTA barrier hands to its threads; every thread writes its
// share of row t-1 of L^{-1} (a_{t-1} is complete everywhere now) and updates
// its share of the predictor.  The FP64 division, square root and log stay
// off the other 1023 threads of a CTA (they would saturate the FP64 pipe);
// the log det is summed once at the end from the v_t history.  The cluster
// size is a launch attribute, chosen per batch.
template <int CL>
__global__ void __launch_bounds__(LEV_THREADS, 1) k_levinson_rows(const LevJob* __restrict__ jobs) {
  __shared__ double red[LEV_THREADS];
  // partials double-buffered by order parity: with one cluster barrier per
  // order a CTA may publish order t+1's partial while a peer still reads order t's
  __shared__ double sh_part[2];
  __shared__ double sh_bc[3];   // k_t, v_t, 1/sqrt(v_{t-1}) of the current order
  const int rank = CL > 1 ? (int)cg::this_cluster().block_rank() : 0;
  const LevJob jb = jobs[blockIdx.x / CL];
  const int64_t n = jb.n;
  const int tid = threadIdx.x;
  const int64_t g = (int64_t)rank * LEV_THREADS + tid;   // this thread's place in the cluster
  constexpr int64_t STRIDE = (int64_t)CL * LEV_THREADS;
  const bool lead = (g == 0);
  double* a = jb.a0;      // a_{t-1}[1..t-1]
  double* an = jb.a1;     // a_t
  double v = jb.acf[0];   // v_{t-1}, the same in every thread
  double kp = 0.0;        // k_{t-1} = a_{t-1}[t-1]
  bool bad = !(v > 0.0) || !isfinite(v);
  if (bad && lead) {
    atomicMin((unsigned long long*)&jb.status->pivot, 0ull);
    atomicCAS(&jb.status->code, 0, ST_NOT_PD);
  }
  for (int64_t t = 1; t <= n && !bad; ++t) {
    if (t < n) {
      // k_t = (acf[t] - sum_{j=1}^{t-1} a_{t-1,j} acf[t-j]) / v_{t-1}
      double part = 0.0;
      for (int64_t j = 1 + g; j < t; j += STRIDE) part = fma(j == t - 1 ? kp : a[j], jb.acf[t - j], part);
      part = block_sum_to_lead(part, red);
      if (tid == 0) sh_part[t & 1] = part;
    }
    if constexpr (CL > 1)
      cg::this_cluster().sync();   // partials published; a_{t-1} complete in every share
    else
      __syncthreads();
    if (tid == 0) {
      double k = 0.0, vn = v;
      if (t < n) {
        double dot = 0.0;
        if constexpr (CL > 1) {
#pragma unroll
          for (int r = 0; r < CL; ++r) dot += *cg::this_cluster().map_shared_rank(&sh_part[t & 1], r);
        } else {
          dot = sh_part[t & 1];
        }
        k = (jb.acf[t] - dot) / v;
        vn = v * (1.0 - k * k);
      }
      sh_bc[0] = k;
      sh_bc[1] = vn;
      sh_bc[2] = 1.0 / sqrt(v);
    }
    __syncthreads();
    const double k = sh_bc[0], vn = sh_bc[1], inv = sh_bc[2];
    if (lead) jb.vhist[t - 1] = v;   // log det = sum_t log v_t, added at the end
    // row t-1 of L^{-1}: column c < t-1 holds -a_{t-1, t-1-c} / sqrt(v_{t-1}), column t-1 holds 1 / sqrt(v_{t-1})
    if (jb.linv) {
      double* row = jb.linv + (t - 1) * jb.ld;
      for (int64_t c = g; c < t - 1; c += STRIDE) row[c] = -a[t - 1 - c] * inv;
      if (lead) row[t - 1] = inv;
    }
    if (t == n) {
      // C^{-1} e_1 = (1, -a_{n-1,1}, ..., -a_{n-1,n-1}) / v_{n-1} (persymmetry of the
      // Toeplitz inverse; its last column is the last row of L^{-1} over sqrt(v_{n-1}))
      if (jb.x) {
        const double iv = 1.0 / v;
        for (int64_t j = 1 + g; j < n; j += STRIDE) jb.x[j] = -a[j] * iv;
        if (lead) jb.x[0] = iv;
      }
      break;
    }
    if (!(vn > 0.0) || !isfinite(vn)) {
      if (lead) {
        atomicMin((unsigned long long*)&jb.status->pivot, (unsigned long long)t);
        atomicCAS(&jb.status->code, 0, ST_NOT_PD);
      }
      bad = true;   // every thread of the cluster holds the same vn
      break;
    }
    for (int64_t j = 1 + g; j < t; j += STRIDE) an[j] = fma(-k, a[t - j], a[j]);
    if (lead) an[t] = k;
    v = vn;
    kp = k;
    double* tmp = a;   // a <- a_t
    a = an;
    an = tmp;
  }
  if (rank == 0 && !bad) {
    // log det C = sum_{t=0}^{n-1} log v_t: the logs spread over the CTA, added in a fixed order
    __syncthreads();   // the lead's v_t stores are visible to the CTA
    double sl = 0.0;
    for (int64_t i = tid; i < n; i += LEV_THREADS) sl += log(jb.vhist[i]);
    sl = block_sum_to_lead(sl, red);
    if (tid == 0) *jb.logdet = sl;
  }
  if constexpr (CL > 1) cg::this_cluster().sync();   // no CTA leaves while a peer may still read its partial
}

template <int CL>
cudaLaunchConfig_t lev_config(int njobs, cudaStream_t st, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)njobs * CL);
  cfg.blockDim = dim3(LEV_THREADS);
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// Clusters of CL CTAs that can be resident at once (0 if the query fails).
template <int CL>
int lev_max_clusters(int njobs, cudaStream_t st) {
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = lev_config<CL>(njobs, st, attr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_levinson_rows<CL>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <int CL>
cudaError_t lev_launch(const LevJob* jobs, int njobs, cudaStream_t st) {
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = lev_config<CL>(njobs, st, attr);
  return cudaLaunchKernelEx(&cfg, k_levinson_rows<CL>, jobs);
}

// The chains of a batch run side by side, each on the largest cluster that
// still lets every chain be resident at once (a chain's time is set by its
// order count, so a second wave would double the batch's time): 8 CTAs for
// a few long segments, one CTA each for many.
cudaError_t launch_levinson_rows(const LevJob* jobs, int njobs, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  if (njobs <= lev_max_clusters<8>(njobs, st)) return lev_launch<8>(jobs, njobs, st);
  if (njobs <= lev_max_clusters<4>(njobs, st)) return lev_launch<4>(jobs, njobs, st);
  if (njobs <= lev_max_clusters<2>(njobs, st)) return lev_launch<2>(jobs, njobs, st);
  k_levinson_rows<1><<<(unsigned)njobs, LEV_THREADS, 0, st>>>(jobs);
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
  double* vh = nullptr;
  double* ld = nullptr;
};

void free_lev(LevSeg& x) {
  for (double** p : {&x.linv, &x.qrow, &x.a0, &x.a1, &x.vh, &x.ld}) {
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
        cudaMalloc((void**)&x.a1, (size_t)s->n * 8) != cudaSuccess ||
        cudaMalloc((void**)&x.vh, (size_t)s->n * 8) != cudaSuccess || cudaMalloc((void**)&x.ld, 8) != cudaSuccess) {
      cudaGetLastError();
      r = fail(TD_ERR_OOM, "Levinson scratch");
      break;
    }
    DevStatus h{0, 0, LLONG_MAX};
    cudaMemcpyAsync(s->status, &h, sizeof h, cudaMemcpyHostToDevice, st);
    jobs.push_back(LevJob{s->acf, s->n, x.a0, x.a1, x.linv, s->nkp, x.ld, s->status, nullptr, x.vh});
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
static td_status check_device_of(const td_segment* s) {
  int dev = -1;
  cudaGetDevice(&dev);
  return dev == s->device ? TD_OK : fail(TD_ERR_INVALID, "segment belongs to another device; set it current first");
}

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
      td_status r = TD_OK;
      if (flags & TD_FACTOR_FP64_CORES) {
        r = check_device_of(s);
        if (r == TD_OK) r = factor_fp64_cores(s, st);
      } else {
        r = td_factor(s, stream);
      }
      if (r == TD_OK && (flags & TD_FACTOR_NO_FP64)) td_segment_release_fp64(s);
      if (r == TD_OK) continue;
      if (r != TD_ERR_NOT_PD) return r;
      if (first_err == TD_OK) first_err = r;
      continue;
    }
    s->factored = false;
    s->pivot = -1;
    td_segment_release_fp64(s);   // a factor from an earlier td_factor would be stale
    free_refine_state(s);
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
