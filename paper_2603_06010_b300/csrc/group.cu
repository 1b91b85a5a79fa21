// Grouped evaluation: many segments (uneven N', each its own K) in one
// persistent tensor-core launch.  The joint covariance of disjoint segments
// and detectors is block-diagonal (Sec. II.B items 1 and 3), so each
// segment's whitening is independent and the work items of all segments share
// one launch.  The main kernel takes them from a work counter as its CTAs
// become free (segment by segment, most work first); the small-batch
// orientation deals them in snake order, longest first.
//
// Each segment takes the slice count td_loglike_batch would take for it; a
// group whose segments need different counts runs one product launch (and
// one chunk reduction) per count.
//
// A td_group is a plan: it owns the device work lists, segment descriptors
// and scratch, so td_group_launch only launches kernels (and zeroes the
// product kernel's work counter before each product launch), whatever the
// number of segments, and can be captured in a CUDA graph;
// td_group_graph_launch captures it once and replays the graph.  The
// autotuner (td_group_tune) times the candidate tile shapes and chunk sizes
// on the real inputs and keeps the fastest.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "td_internal.h"

namespace td {

constexpr int GROUP_NC = 256;   // default residual columns per tile of the small-batch orientation

static td_status group_alloc(void** p, size_t bytes, const char* what) {
  *p = nullptr;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(TD_ERR_OOM, std::string("device allocation failed: ") + what);
  }
  return TD_OK;
}

struct RsJob {          // one segment's residual slicing for the grouped slicing kernel
  const float* R;
  int64_t ldr;
  int64_t nk;
  int64_t K;
  int64_t nkp8;
  int64_t capK;
  __nv_bfloat16* rs;
  int64_t col0;         // first global column of this segment
  int nsl;              // slices this segment's product reads
  int pad;
};

// per-column quantum and slices for every segment of the group (the same
// r_quantum / r_slice_value arithmetic as k_r_slices, so a column's slices
// do not depend on the group).  One CTA per column at a time; each thread
// takes row pairs (2t, 2t + 1) + 512 i.  The maximum pass keeps 16 loads in
// flight per thread; the slicing pass loads 8 values before any store and
// writes bf16 pairs (4-byte stores: a slice column starts 16-byte aligned).
// Rows at or beyond N' are never written.
constexpr int RSG_THREADS = 256;
__global__ void __launch_bounds__(RSG_THREADS) k_r_slices_grouped(const RsJob* __restrict__ jobs, int njobs,
                                                                  int64_t total_cols) {
  __shared__ float red[RSG_THREADS / 32];
  constexpr int64_t STEP = 2 * RSG_THREADS;   // rows per pass of the CTA
  for (int64_t gc = blockIdx.x; gc < total_cols; gc += gridDim.x) {
    int lo = 0, hi = njobs - 1;   // last job with col0 <= gc
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (jobs[mid].col0 <= gc) lo = mid; else hi = mid - 1;
    }
    const RsJob& jb = jobs[lo];
    const int64_t k = gc - jb.col0;
    const int64_t nk = jb.nk;
    const float* col = jb.R + k * jb.ldr;
    float mx = 0.f;
    for (int64_t j0 = 2 * threadIdx.x; j0 < nk; j0 += 8 * STEP) {
      float x[16];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t j = j0 + u * STEP;
        x[2 * u] = j < nk ? col[j] : 0.f;
        x[2 * u + 1] = j + 1 < nk ? col[j + 1] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) mx = fmaxf(mx, fabsf(x[u]));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = red[0];
#pragma unroll
    for (int w = 1; w < RSG_THREADS / 32; ++w) mx = fmaxf(mx, red[w]);
    __syncthreads();   // red is reused by the next column
    const float p = r_quantum(mx);
    const int64_t ss = jb.capK * jb.nkp8;
    const int nslices = jb.nsl;
    __nv_bfloat16* dst = jb.rs + k * jb.nkp8;
    for (int64_t j0 = 2 * threadIdx.x; j0 < nk; j0 += 4 * STEP) {
      float x[8];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t j = j0 + u * STEP;
        x[2 * u] = j < nk ? col[j] : 0.f;
        x[2 * u + 1] = j + 1 < nk ? col[j + 1] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t j = j0 + u * STEP;
        if (j >= nk) break;
        __nv_bfloat16 a[4], b[4];
        r_slice_value(x[2 * u], p, a);
        r_slice_value(x[2 * u + 1], p, b);
        if (j + 1 < nk) {
#pragma unroll
          for (int sl = 0; sl < 4; ++sl)
            if (sl < nslices) {
              __nv_bfloat162 v;
              v.x = a[sl];
              v.y = b[sl];
              *reinterpret_cast<__nv_bfloat162*>(dst + sl * ss + j) = v;
            }
        } else {
#pragma unroll
          for (int sl = 0; sl < 4; ++sl)
            if (sl < nslices) dst[sl * ss + j] = a[sl];
        }
      }
    }
  }
}

}  // namespace td

using namespace td;

// The work of one slice count: a grouped launch runs each segment with the
// slice count td_loglike_batch would take for it (under TD_PREC_AUTO ten
// products below 2048 and above 32768 kept samples, six between), one
// product launch per count present.
struct GroupClass {
  int nsl = 3;
  TcItem* d_items = nullptr;
  SplitUnit* d_units = nullptr;
  int n_items = 0, n_units = 0;
  float2* wpart = nullptr;
};

struct td_group {
  int device = 0;
  int nseg = 0;
  int nsl = 3;                // the largest slice count of the group
  std::vector<int> seg_nsl;   // each segment's slice count
  int bn = 256;
  int s_factor = 1;           // chunk size multiplier chosen by the autotuner
  int small_nc = GROUP_NC;    // small-batch orientation: residual columns per tile (128 or 256)
  int64_t wait_limit_ns = 1000000000LL;
  int64_t total_cols = 0;
  int64_t maxK = 0;
  std::vector<td_segment*> segs;
  std::vector<const void*> ops;   // each segment's operator when the tensor maps were encoded
  std::vector<TcSegDev> host_seg;
  std::vector<RsJob> host_jobs;
  // device
  TcSegDev* d_seg = nullptr;
  RsJob* d_jobs = nullptr;
  std::vector<GroupClass> cls;   // one per slice count present
  __nv_bfloat16* rs = nullptr;
  double* partials = nullptr;
  DevStatus* status = nullptr;
  cudaGraphExec_t graph = nullptr;
  cudaStream_t graph_stream = nullptr;
  int* sched = nullptr;       // work counter of the product kernel's dynamic schedule
  double* joint = nullptr;    // optional: sum over the segments of logL (all with joint_K columns)
  int64_t joint_K = 0;
};

namespace td {

static void group_free_lists(td_group* g) {
  for (GroupClass& c : g->cls) {
    if (c.d_items) cudaFree(c.d_items);
    if (c.d_units) cudaFree(c.d_units);
    if (c.wpart) cudaFree(c.wpart);
  }
  g->cls.clear();
  if (g->graph) {
    cudaGraphExecDestroy(g->graph);
    g->graph = nullptr;
  }
}

// build work lists and maps for a tile shape and chunk multiplier.  bn > 0:
// the main kernel (128 residual columns as the MMA M, bn operator rows as
// N); bn == 0: the small-batch kernel's orientation (128 operator rows as M,
// up to nc = 128 or 256 residual columns as N, each segment's last column tile
// only as wide as its columns rounded up to 16), every item a chunk whose
// accumulator pairs the grouped chunk reduction adds.  At 128 columns TMEM
// holds two accumulator pairs, so an item's epilogue overlaps the next
// item's MMAs; at 256 one.
static td_status group_build(td_group* g, int bn, int s_factor, int nc = GROUP_NC) {
  group_free_lists(g);
  g->bn = bn;
  g->s_factor = s_factor;
  g->small_nc = nc;
  const bool small = bn == 0;
  const int rows = small ? 128 : bn, cols = small ? nc : TC_COLS;
  td_status r;
  // one work list per slice count present, each balanced over the SMs on its own
  for (int nsl = 2; nsl <= 4; ++nsl) {
    bool any = false;
    for (int i = 0; i < g->nseg; ++i) any = any || g->seg_nsl[(size_t)i] == nsl;
    if (!any) continue;
    // work per residual-column tile summed over the class's segments; chunk so
    // that the longest item is about 1/(2 s_factor) of an SM's even share
    int64_t tiles_work = 0;
    for (int i = 0; i < g->nseg; ++i) {
      if (g->seg_nsl[(size_t)i] != nsl) continue;
      td_segment* s = g->segs[(size_t)i];
      const int64_t nm = s->nkp / rows, per = rows / OP_KB, nkb_max = ceil_div(s->nk, OP_KB);
      int64_t w = 0;
      for (int64_t m = 0; m < nm; ++m) w += std::min<int64_t>(per * (m + 1), nkb_max);
      tiles_work += w * ceil_div(g->host_seg[(size_t)i].K, cols);
    }
    int S = (int)ceil_div(tiles_work, 2LL * s_factor * tc_num_sms());
    if (S < 4) S = 4;
    std::vector<TcItem> items;
    std::vector<SplitUnit> units;
    int n_slots = 0;
    for (int i = 0; i < g->nseg; ++i) {
      if (g->seg_nsl[(size_t)i] != nsl) continue;
      td_segment* s = g->segs[(size_t)i];
      plan_split_segment(i, s->nk, s->nkp, g->host_seg[(size_t)i].K, rows, S, items, units, n_slots, small, cols);
    }
    // the small-batch kernel deals its items round by round, longest first;
    // the main kernel takes them dynamically, segment by segment
    if (small)
      sort_items(items);
    else
      sort_items_by_segment(items, g->nseg);
    g->cls.push_back(GroupClass());
    GroupClass& c = g->cls.back();
    c.nsl = nsl;
    const size_t wbytes = (size_t)n_slots * (small ? nc * 128 : TC_COLS * bn) * sizeof(float2);
    if ((r = group_alloc((void**)&c.d_items, std::max<size_t>(1, items.size()) * sizeof(TcItem), "items")) !=
            TD_OK ||
        (r = group_alloc((void**)&c.d_units, std::max<size_t>(1, units.size()) * sizeof(SplitUnit), "units")) !=
            TD_OK ||
        (r = group_alloc((void**)&c.wpart, std::max<size_t>(8, wbytes), "split accumulators")) != TD_OK)
      return r;
    if ((!items.empty() &&
         cudaMemcpy(c.d_items, items.data(), items.size() * sizeof(TcItem), cudaMemcpyHostToDevice) != cudaSuccess) ||
        (!units.empty() && cudaMemcpy(c.d_units, units.data(), units.size() * sizeof(SplitUnit),
                                      cudaMemcpyHostToDevice) != cudaSuccess))
      return fail(TD_ERR_CUDA, "upload of group work lists failed");
    c.n_items = (int)items.size();
    c.n_units = (int)units.size();
  }
  for (int i = 0; i < g->nseg; ++i) {
    TcSegDev& sd = g->host_seg[(size_t)i];
    td_segment* s = g->segs[(size_t)i];
    const int nsl = g->seg_nsl[(size_t)i];
    sd.a_rows = small ? nc : TC_COLS;
    for (const GroupClass& c : g->cls)
      if (c.nsl == nsl) sd.wpart = c.wpart;
    sd.nm = (int)(s->nkp / (small ? 128 : 64));   // chi2 partials per 128-row tile or per 64 rows
    if (sd.K == 0) continue;   // no work item refers to an empty segment
    // residual map over this segment's slice region of the group buffer
    const int64_t cap = sd.ldp;
    td_segment tmp_view;   // only the fields encode_seg_maps reads
    tmp_view.nk = s->nk;
    tmp_view.nkp8 = s->nkp8;
    tmp_view.op = s->op;
    tmp_view.op_blocks = s->op_blocks;
    tmp_view.scr.rs = g->host_jobs[(size_t)i].rs;
    tmp_view.scr.capK = cap;
    TcSegDev enc;
    memset(&enc, 0, sizeof enc);
    if ((r = encode_seg_maps(&tmp_view, sd.K, nsl, rows, &enc, small ? nc : TC_COLS)) != TD_OK) {
      tmp_view.scr.rs = nullptr;
      tmp_view.op = nullptr;
      return r;
    }
    tmp_view.scr.rs = nullptr;   // not owned
    tmp_view.op = nullptr;
    sd.mapA = enc.mapA;
    sd.mapB = enc.mapB;
  }
  if (cudaMemcpy(g->d_seg, g->host_seg.data(), g->host_seg.size() * sizeof(TcSegDev), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return fail(TD_ERR_CUDA, "upload of group work lists failed");
  g->ops.clear();
  for (td_segment* sp : g->segs) g->ops.push_back(sp->op);
  return TD_OK;
}

// The tensor maps hold operator addresses: a segment re-factored (or its
// operator freed and rebuilt) after the group was built makes the group stale.
static td_status group_check_current(const td_group* g) {
  for (size_t i = 0; i < g->segs.size(); ++i)
    if (i >= g->ops.size() || g->segs[i]->op != g->ops[i] || !g->segs[i]->factored)
      return fail(TD_ERR_INVALID, "a segment of the group was re-factored since the group was built");
  return TD_OK;
}

// joint logL over the segments of a group (Sec. II.B item 3: detectors'
// log-likelihoods add), segment order fixed
__global__ void k_joint_sum(const TcSegDev* __restrict__ segs, int nseg, int64_t K, double* __restrict__ out) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= K) return;
  double s = 0.0;
  for (int i = 0; i < nseg; ++i) s += segs[i].logL[k];
  out[k] = s;
}

static td_status group_launch_impl(td_group* g, cudaStream_t st) {
  int gx = (int)std::min<int64_t>(g->total_cols, 8192);
  if (gx > 0) {
    k_r_slices_grouped<<<gx, RSG_THREADS, 0, st>>>(g->d_jobs, g->nseg, g->total_cols);
    TD_CUDA(cudaGetLastError());
  }
  for (const GroupClass& c : g->cls) {
    if (g->bn == 0) {
      TD_CUDA(launch_tc_small(c.d_items, c.n_items, g->d_seg, c.nsl, g->small_nc, g->status, g->wait_limit_ns, st));
      TD_CUDA(launch_small_reduce_grouped(c.d_units, c.n_units, g->d_seg, g->small_nc, st));
    } else {
      TD_CUDA(cudaMemsetAsync(g->sched, 0, sizeof(int), st));
      TD_CUDA(launch_tc_cdo(c.d_items, c.n_items, g->d_seg, c.nsl, g->bn, true, g->status, g->wait_limit_ns, st,
                            false, g->sched));
      TD_CUDA(launch_split_reduce(c.d_units, c.n_units, g->d_seg, g->bn, st, g->maxK));
    }
  }
  TD_CUDA(launch_tc_finalize(g->d_seg, g->nseg, g->maxK, st));
  if (g->joint && g->joint_K > 0) {
    k_joint_sum<<<(unsigned)ceil_div(g->joint_K, 256), 256, 0, st>>>(g->d_seg, g->nseg, g->joint_K, g->joint);
    TD_CUDA(cudaGetLastError());
  }
  return TD_OK;
}

// process-wide autotuner decisions: signature -> (bn, s_factor, small_nc)
struct TuneEntry {
  std::string key;
  int bn;
  int s_factor;
  int nc;
  double ms;
};
static std::mutex g_tune_mu;
static std::vector<TuneEntry> g_tune;

static std::string group_signature(const td_group* g) {
  // device name + bucketed shape of the work: log2 of total N'^2 K and of the segment count
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, g->device);
  double work = 0.0;
  for (int i = 0; i < g->nseg; ++i) {
    const double n = (double)g->segs[(size_t)i]->nk;
    work += n * n * (double)g->host_seg[(size_t)i].K;
  }
  std::string classes;   // the slice counts present
  for (int ns = 2; ns <= 4; ++ns)
    if (std::find(g->seg_nsl.begin(), g->seg_nsl.end(), ns) != g->seg_nsl.end()) classes += std::to_string(ns);
  return std::string(prop.name) + "|nsl" + std::to_string(g->nsl) + classes + "|w" +
         std::to_string((int)std::log2(std::max(1.0, work))) + "|s" +
         std::to_string((int)std::log2((double)std::max(1, g->nseg)));
}

}  // namespace td

extern "C" {

td_status td_group_create(td_segment* const* segs, const float* const* R, const int64_t* ldr, const int64_t* K,
                          double* const* logL, double* const* chi2, int nseg, const td_options* opt, void* stream,
                          td_group** out) {
  if (!out) return fail(TD_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (nseg <= 0 || !segs || !R || !ldr || !K || !logL) return fail(TD_ERR_INVALID, "bad arguments");
  td_options o;
  td_options_default(&o);
  if (opt) o = *opt;
  if (o.precision == TD_PREC_FP64) return fail(TD_ERR_UNSUPPORTED, "grouped launches use the tensor-core path");
  if (o.refine) return fail(TD_ERR_UNSUPPORTED, "refinement runs on single-segment batches");
  td_group* g = new td_group();
  cudaGetDevice(&g->device);
  g->nseg = nseg;
  // each segment with the slice count td_loglike_batch takes for it
  g->nsl = 2;
  for (int i = 0; i < nseg; ++i) {
    const int ns = nslices_for(o.precision, segs[i] ? segs[i]->nk : 0);
    g->seg_nsl.push_back(ns);
    g->nsl = std::max(g->nsl, ns);
  }
  g->wait_limit_ns = o.wait_limit_ns > 0 ? o.wait_limit_ns : 1000000000LL;
  int64_t rs_elems = 0, part_elems = 0;
  for (int i = 0; i < nseg; ++i) {
    td_segment* s = segs[i];
    if (!s || !s->factored) {
      delete g;
      return fail(!s ? TD_ERR_INVALID : TD_ERR_NOT_FACTORED, "segment missing or not factored");
    }
    if (s->device != g->device || K[i] < 0 || K[i] > TD_MAX_K || (K[i] > 0 && (!R[i] || !logL[i])) ||
        ldr[i] < s->nk) {
      delete g;
      return fail(TD_ERR_INVALID, "bad segment arguments");
    }
    g->segs.push_back(s);
    const int64_t cap = round_up(std::max<int64_t>(K[i], 1), TC_COLS);
    rs_elems += OP_SLICES * cap * s->nkp8;
    part_elems += (s->nkp / 64) * cap;
  }
  td_status r;
  if ((r = group_alloc((void**)&g->rs, (size_t)rs_elems * 2, "group residual slices")) != TD_OK ||
      (r = group_alloc((void**)&g->partials, (size_t)part_elems * 8, "group partials")) != TD_OK ||
      (r = group_alloc((void**)&g->d_seg, (size_t)nseg * sizeof(TcSegDev), "segment descriptors")) != TD_OK ||
      (r = group_alloc((void**)&g->d_jobs, (size_t)nseg * sizeof(RsJob), "slicing jobs")) != TD_OK ||
      (r = group_alloc((void**)&g->status, sizeof(DevStatus), "status")) != TD_OK ||
      (r = group_alloc((void**)&g->sched, sizeof(int), "work counter")) != TD_OK) {
    td_group_destroy(g);
    return r;
  }
  int64_t rs_off = 0, part_off = 0, col0 = 0;
  for (int i = 0; i < nseg; ++i) {
    td_segment* s = segs[i];
    const int64_t cap = round_up(std::max<int64_t>(K[i], 1), TC_COLS);
    TcSegDev sd;
    memset(&sd, 0, sizeof sd);
    sd.partials = g->partials + part_off;
    sd.nk = (int)s->nk;
    sd.K = (int)K[i];
    sd.ldp = (int)cap;
    sd.nm = (int)(s->nkp / 64);
    sd.logdet = s->logdet;
    sd.logL = logL[i];
    sd.chi2 = chi2 ? chi2[i] : nullptr;
    g->host_seg.push_back(sd);
    RsJob jb{R[i], ldr[i], s->nk, K[i], s->nkp8, cap, g->rs + rs_off, col0, g->seg_nsl[(size_t)i], 0};
    g->host_jobs.push_back(jb);
    rs_off += OP_SLICES * cap * s->nkp8;
    part_off += (s->nkp / 64) * cap;
    col0 += K[i];
    g->maxK = std::max(g->maxK, K[i]);
  }
  g->total_cols = col0;
  DevStatus hs{0, 0, 0};
  if (cudaMemcpy(g->d_jobs, g->host_jobs.data(), (size_t)nseg * sizeof(RsJob), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(g->status, &hs, sizeof hs, cudaMemcpyHostToDevice) != cudaSuccess) {
    td_group_destroy(g);
    return fail(TD_ERR_CUDA, "group upload failed");
  }
  // tile shape: a decision the autotuner made for this kind of group, else 256-row tiles
  int bn = 256, sf = 1, nc = GROUP_NC;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const std::string key = group_signature(g);
    for (const TuneEntry& e : g_tune)
      if (e.key == key) {
        bn = e.bn;
        sf = e.s_factor;
        nc = e.nc;
      }
  }
  if (o.path == TD_PATH_STREAM64) bn = 64;
  if (o.path == TD_PATH_STREAM) bn = 256;
  if (o.path == TD_PATH_SMALLK) bn = 0;
  if ((r = group_build(g, bn, sf, nc)) != TD_OK) {
    td_group_destroy(g);
    return r;
  }
  (void)stream;
  *out = g;
  return TD_OK;
}

td_status td_group_set_joint(td_group* g, double* joint) {
  if (!g) return fail(TD_ERR_INVALID, "group is NULL");
  int64_t K = -1;
  for (const TcSegDev& sd : g->host_seg) {
    if (K >= 0 && sd.K != K) return fail(TD_ERR_INVALID, "a joint logL needs the same K in every segment");
    K = sd.K;
  }
  if (joint && !g->host_seg.empty() && !g->host_seg[0].logL)
    return fail(TD_ERR_INVALID, "segment outputs are missing");
  if (g->graph) {   // the captured launch does not contain the sum (or contains a stale one)
    cudaGraphExecDestroy(g->graph);
    g->graph = nullptr;
  }
  g->joint = joint;
  g->joint_K = joint ? std::max<int64_t>(K, 0) : 0;
  return TD_OK;
}

td_status td_group_launch(td_group* g, void* stream) {
  if (!g) return fail(TD_ERR_INVALID, "group is NULL");
  td_status r = group_check_current(g);
  if (r != TD_OK) return r;
  return group_launch_impl(g, reinterpret_cast<cudaStream_t>(stream));
}

td_status td_group_graph_launch(td_group* g, void* stream) {
  if (!g) return fail(TD_ERR_INVALID, "group is NULL");
  if (td_status rc = group_check_current(g); rc != TD_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (!g->graph) {
    cudaStream_t cap;
    TD_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    td_status r = TD_OK;
    if (e == cudaSuccess) r = group_launch_impl(g, cap);
    cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess || e2 != cudaSuccess || r != TD_OK) {
      if (graph) cudaGraphDestroy(graph);
      return r != TD_OK ? r : cuda_fail(e != cudaSuccess ? e : e2, "graph capture of the grouped launch");
    }
    e = cudaGraphInstantiate(&g->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  }
  TD_CUDA(cudaGraphLaunch(g->graph, st));
  return TD_OK;
}

td_status td_group_tune(td_group* g, void* stream, double* best_ms) {
  if (!g) return fail(TD_ERR_INVALID, "group is NULL");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // tile rows (0: the small-batch orientation), chunk multiplier, and the
  // small orientation's residual columns per tile
  const int cand[][3] = {{256, 1, 0},   {256, 2, 0},   {128, 1, 0},   {128, 2, 0},   {128, 4, 0},
                         {64, 1, 0},    {64, 2, 0},    {0, 1, 256},   {0, 2, 256},   {0, 4, 256},
                         {0, 1, 128},   {0, 2, 128},   {0, 4, 128}};
  double best = 1e300;
  int bb = g->bn, bs = g->s_factor, bc = g->small_nc;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  for (const auto& c : cand) {
    td_status r = group_build(g, c[0], c[1], c[2] ? c[2] : GROUP_NC);
    if (r != TD_OK) continue;
    for (int w = 0; w < 2; ++w) group_launch_impl(g, st);
    cudaEventRecord(a, st);
    for (int it = 0; it < 5; ++it) group_launch_impl(g, st);
    cudaEventRecord(b, st);
    if (cudaEventSynchronize(b) != cudaSuccess) continue;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    const double per = ms / 5.0;
    if (per < best) {
      best = per;
      bb = c[0];
      bs = c[1];
      bc = c[2] ? c[2] : GROUP_NC;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  td_status r = group_build(g, bb, bs, bc);
  if (r != TD_OK) return r;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const std::string key = group_signature(g);
    bool found = false;
    for (TuneEntry& e : g_tune)
      if (e.key == key) {
        e.bn = bb;
        e.s_factor = bs;
        e.nc = bc;
        e.ms = best;
        found = true;
      }
    if (!found) g_tune.push_back(TuneEntry{key, bb, bs, bc, best});
  }
  if (best_ms) *best_ms = best;
  return TD_OK;
}

td_status td_group_check(td_group* g, void* stream) {
  if (!g) return fail(TD_ERR_INVALID, "group is NULL");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  DevStatus hs;
  TD_CUDA(cudaMemcpyAsync(&hs, g->status, sizeof hs, cudaMemcpyDeviceToHost, st));
  TD_CUDA(cudaStreamSynchronize(st));
  if (hs.code != 0) {
    DevStatus z{0, 0, 0};
    cudaMemcpy(g->status, &z, sizeof z, cudaMemcpyHostToDevice);
    return fail(hs.code == ST_TIMEOUT ? TD_ERR_TIMEOUT : (td_status)hs.code, "device reported an error");
  }
  return TD_OK;
}

td_status td_group_clock(td_group* g, void* stream, double* mhz) {
  if (!g) return fail(TD_ERR_INVALID, "group is NULL");
  return read_clock(g->status, reinterpret_cast<cudaStream_t>(stream), mhz);
}

int td_group_shape(const td_group* g, int* bn, int* s_factor, int* n_items) {
  if (!g) return -1;
  if (bn) *bn = g->bn;
  if (s_factor) *s_factor = g->s_factor;
  if (n_items) {
    *n_items = 0;
    for (const GroupClass& c : g->cls) *n_items += c.n_items;
  }
  return 0;
}

void td_group_destroy(td_group* g) {
  if (!g) return;
  cudaDeviceSynchronize();
  group_free_lists(g);
  if (g->rs) cudaFree(g->rs);
  if (g->partials) cudaFree(g->partials);
  if (g->d_seg) cudaFree(g->d_seg);
  if (g->d_jobs) cudaFree(g->d_jobs);
  if (g->status) cudaFree(g->status);
  if (g->sched) cudaFree(g->sched);
  delete g;
}

td_status td_loglike_grouped(td_segment* const* segs, const float* const* R, const int64_t* ldr, const int64_t* K,
                             double* const* logL, int nseg, const td_options* opt, void* stream) {
  td_group* g = nullptr;
  td_status r = td_group_create(segs, R, ldr, K, logL, nullptr, nseg, opt, stream, &g);
  if (r != TD_OK) return r;
  r = td_group_launch(g, stream);
  if (r == TD_OK) r = td_group_check(g, stream);
  td_group_destroy(g);
  return r;
}

}  // extern "C"
