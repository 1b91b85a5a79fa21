// C ABI of libtd: segment lifetime, factor, per-evaluation batches.
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "td_internal.h"

namespace td {

static thread_local std::string g_last_error;

td_status fail(td_status code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

td_status cuda_fail(cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  g_last_error = m;
  if (e == cudaErrorMemoryAllocation) return TD_ERR_OOM;
  return TD_ERR_CUDA;
}

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::mutex g_encode_mu;

static td_status get_encode(PFN_cuTensorMapEncodeTiled_v12000* out) {
  std::lock_guard<std::mutex> lk(g_encode_mu);
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return fail(TD_ERR_CUDA, "cuTensorMapEncodeTiled entry point not available");
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  *out = g_encode;
  return TD_OK;
}

td_status encode_3d(CUtensorMap* map, const void* ptr, uint64_t d0, uint64_t d1, uint64_t d2,
                           uint64_t s1_bytes, uint64_t s2_bytes, uint32_t b0, uint32_t b1, uint32_t b2) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  td_status st = get_encode(&enc);
  if (st != TD_OK) return st;
  cuuint64_t dims[3] = {d0, d1, d2};
  cuuint64_t strides[2] = {s1_bytes, s2_bytes};
  cuuint32_t box[3] = {b0, b1, b2};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(ptr), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    char buf[160];
    snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled failed (%d): dims %llu %llu %llu", (int)r,
             (unsigned long long)d0, (unsigned long long)d1, (unsigned long long)d2);
    return fail(TD_ERR_CUDA, buf);
  }
  return TD_OK;
}

// residual-slice map (A operand: a box of a_rows residual columns) and operator
// map (B operand, tiles of bn rows) of one segment
td_status encode_seg_maps(td_segment* s, int64_t K, int nsl, int bn, TcSegDev* out, int a_rows,
                          const __nv_bfloat16* op, const Scratch* sc) {
  if (!sc) sc = &s->scr;
  out->a_rows = a_rows;
  td_status st = encode_3d(&out->mapA, sc->rs, (uint64_t)s->nk, (uint64_t)K, OP_SLICES,
                           (uint64_t)s->nkp8 * 2, (uint64_t)sc->capK * s->nkp8 * 2, OP_KB, (uint32_t)a_rows,
                           1);
  if (st != TD_OK) return st;
  return encode_3d(&out->mapB, op ? op : s->op, OP_KB, OP_ROWS, (uint64_t)s->op_blocks * OP_SLICES, OP_KB * 2,
                   (uint64_t)OP_ROWS * OP_KB * 2, OP_KB, (uint32_t)bn, (uint32_t)nsl);
}

// Tile shape and split for a batch: the small-batch kernel (bn = 0) for few
// and mid-size batches, 128-row chunks between them; for wide batches 256- or
// 128-row tiles over whole rows, chosen by how many work items they give, else
// 128-row chunks.  td_options.path can force any shape.
struct Shape {
  int bn;
  bool split;
  int S = 0;   // split: chunk length in k-blocks (0: split_chunk's, which depends on N' alone)
};

// Whole rows of bn rows over nc column tiles: when the longest row alone is
// longer than twice an SM's mean share of the work, it holds the launch back;
// the chunk length that splits only the rows above the mean share (else 0:
// keep whole rows).  Measured on B300, one call after an L2 flush: N' = 4096,
// K = 300 / 384 / 512 (longest row 2.2 to 3 mean shares): 67 / 66 / 74 us
// against 83 / 82 / 88 us whole; at 1.5 mean shares it is a toss-up
// (N' = 8192, K = 384: 141 against 153 us; N' = 4096, K = 768: 92 against 86)
static int balanced_chunk(const td_segment* s, int bn, int64_t nc) {
  const int64_t per = bn / OP_KB, nm = s->nkp / bn, nkb_max = ceil_div(s->nk, OP_KB);
  int64_t total = 0;
  for (int64_t m = 0; m < nm; ++m) total += std::min<int64_t>(per * (m + 1), nkb_max);
  total *= nc;
  const int64_t mean = ceil_div(total, (int64_t)tc_num_sms());
  const int64_t longest = std::min<int64_t>(per * nm, nkb_max);
  return longest > 2 * mean ? (int)std::max<int64_t>(mean, 4) : 0;
}
static Shape choose_shape(const td_segment* s, int64_t K, int path) {
  if (path == TD_PATH_TENSOR) return {256, false};
  if (path == TD_PATH_STREAM) return {256, true};
  if (path == TD_PATH_STREAM64) return {64, true};
  if (path == TD_PATH_TENSOR128) return {128, false};
  if (path == TD_PATH_STREAM128) return {128, true};
  // measured on B300 (one call after an L2 flush, N' = 2048 ... 32768):
  // K <= 32 and 64 < K <= 256 take the small-batch kernel (N' = 8192, K = 256:
  // 108 us against 135 us as 128-row chunks and 152 us as 128-row whole rows;
  // N' = 16384, K = 256: 284 / 329 / 291 us) up to N' = 16384; at N' = 32768
  // 256-row whole rows win (923 against 992 us).  32 < K <= 64 takes 128-row
  // chunks (N' = 16384: 178 us; whole rows 286 us, held back by the longest row)
  if (path == TD_PATH_SMALLK) return {0, true};
  if (path == TD_PATH_AUTO && (K <= 32 || (K > 64 && K <= 256 && s->nk < 24576))) return {0, true};
  if (path == TD_PATH_AUTO && K <= 64) return {128, true};
  // measured on B300 (N' = 8192, one call after an L2 flush): 256-row whole
  // rows win from K = 1024 (250 us vs 275 us for 128-row); 128-row whole rows
  // (two TMEM accumulator pairs, so epilogues overlap MMAs) at K = 384..512
  // (155 us vs 238 us for 256-row); 128-row tiles with k-chunks below that
  // (K = 128: 91 us vs 149 us whole rows; K = 256: a tie at 155 us).  Whole
  // 128-row tiles from half an item per SM: N' = 4096, K = 384 (96 items)
  // 83 us against 109 us in k-chunks
  const int64_t nc = ceil_div(K, TC_COLS);
  const int64_t items256 = (s->nkp / OP_ROWS) * nc;
  const int64_t items128 = (s->nkp / 128) * nc;
  if (2 * items256 >= 3 * (int64_t)tc_num_sms()) {
    const int S = balanced_chunk(s, 256, nc);
    return S > 0 ? Shape{256, true, S} : Shape{256, false};
  }
  if (2 * items128 >= (int64_t)tc_num_sms()) {
    const int S = balanced_chunk(s, 128, nc);
    return S > 0 ? Shape{128, true, S} : Shape{128, false};
  }
  return {128, true};
}

template <class T>
static td_status dev_alloc(T** p, size_t count, const char* what) {
  *p = nullptr;
  if (count == 0) return TD_OK;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(TD_ERR_OOM, std::string("device allocation failed: ") + what);
  }
  return TD_OK;
}

template <class T>
static void dev_free(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

static td_status check_device(const td_segment* s) {
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != s->device) return fail(TD_ERR_INVALID, "segment belongs to another device; set it current first");
  return TD_OK;
}

// TD_PREC_AUTO: six products while the expected |dlogL| (about N' x 1e-8 from
// chi2 ~ N' at ~2e-8 relative, measured) stays under a third of the 1e-3 bar,
// ten products beyond N' = 32768.  Ten products also below N' = 512: with few
// rows one column's chi2 can rest on a single row, whose six-product value is
// good to ~6e-8 relative, so chi2 can miss 1e-7 (1.15e-7 measured at N' = 47);
// many rows average that away.  Small segments cost little either way.
int nslices_for(int precision, int64_t nk) {
  if (precision == TD_PREC_AUTO) return (nk > 32768 || nk < AUTO_SIX_MIN) ? 4 : 3;
  return precision == TD_PREC_BF16X3 ? 2 : (precision == TD_PREC_BF16X10 ? 4 : 3);
}

static void free_plan(SplitPlan& p) {
  dev_free(p.items);
  dev_free(p.units);
  dev_free(p.segdev);
  dev_free(p.counters);
}

static void free_plans(Scratch& sc) {
  for (SplitPlan& p : sc.plans) free_plan(p);
  sc.plans.clear();
}

void scratch_free(Scratch& sc) {
  free_plans(sc);
  dev_free(sc.rs);
  dev_free(sc.partials);
  dev_free(sc.w64);
  dev_free(sc.wpart);
  for (float2*& w : sc.wpart_old) dev_free(w);
  sc.wpart_old.clear();
  sc.capK = sc.wpart_slots = sc.rs_elems = sc.part_elems = 0;
}

// A scratch for any segment of up to max_kept samples and batches of up to
// maxK columns, allocated once (a server stream's).
td_status scratch_init_shared(Scratch& sc, int64_t max_kept, int64_t maxK) {
  const int64_t cap = round_up(std::max<int64_t>(maxK, 1), TC_COLS);
  const int64_t nkp = round_up(max_kept, OP_ROWS), nkp8 = round_up(max_kept, 8);
  sc.shared = true;
  sc.max_plans = 1u << 14;
  sc.capK = cap;
  sc.rs_elems = OP_SLICES * cap * nkp8;
  sc.part_elems = (nkp / FT) * cap;
  td_status r = dev_alloc(&sc.rs, (size_t)sc.rs_elems, "residual slices");
  if (r == TD_OK) r = dev_alloc(&sc.partials, (size_t)sc.part_elems, "chi2 partials");
  return r;
}

// Grow the scratch so batches of K columns of segment s fit (a shared scratch
// only checks: it was sized for every segment it may serve).
static td_status ensure_scratch(td_segment* s, Scratch& sc, int64_t K, bool fp64_path, cudaStream_t st) {
  if (sc.shared) {
    if (fp64_path) return fail(TD_ERR_UNSUPPORTED, "the FP64 path runs on the segment's own scratch");
    if (K > sc.capK || OP_SLICES * sc.capK * s->nkp8 > sc.rs_elems || (s->nkp / FT) * sc.capK > sc.part_elems)
      return fail(TD_ERR_INVALID, "batch wider or segment longer than the shared scratch was sized for");
    return TD_OK;
  }
  if (K > sc.capK) {
    cudaStreamSynchronize(st);   // old buffers may still be in use on this stream
    free_plans(sc);              // their tensor maps point at the old residual slices
    dev_free(sc.rs);
    dev_free(sc.partials);
    dev_free(sc.w64);
    const int64_t cap = round_up(K, TC_COLS);
    td_status r = dev_alloc(&sc.rs, (size_t)(OP_SLICES * cap * s->nkp8), "residual slices");
    if (r != TD_OK) return r;
    r = dev_alloc(&sc.partials, (size_t)((s->nkp / FT) * cap), "chi2 partials");
    if (r != TD_OK) return r;
    sc.capK = cap;
  }
  if (fp64_path && !sc.w64) {
    td_status r = dev_alloc(&sc.w64, (size_t)(s->nkp * sc.capK), "FP64 whitened residuals");
    if (r != TD_OK) return r;
  }
  return TD_OK;
}

// Width of the cached plan that serves a batch of K columns: plans are keyed
// by width, not by K, so a server whose batch sizes vary does not rebuild
// them.  Columns in [K, width) are computed on stale slice rows and dropped
// (the residual slices and partials hold capK >= width columns); a column's
// own arithmetic does not depend on the width.
// TD_PATH_AUTO on a gap-free segment prepared by td_gs_prepare takes GSCE where
// it measured faster than the dense product (N = 8192: 29 vs 54 us at K <= 8,
// 39 vs 68 us at K = 64, 175 vs ~155 us at K = 512; N = 32768: 0.09 vs 0.57 ms
// at K = 1, 1.15 vs 1.64 ms at K = 512), and whenever the dense operator is
// absent; not with refinement or FP64, which it does not provide.
bool gs_preferred(const td_segment* s, int64_t K) { return K <= 256 || s->nk >= 24576; }

static bool gs_auto(const td_segment* s, int64_t K, const td_options& o) {
  if (o.path != TD_PATH_AUTO || !s->gs.ready || o.refine || o.precision == TD_PREC_FP64) return false;
  if (!s->factored || !s->op) return true;
  return gs_preferred(s, K);
}

static int64_t plan_width(int64_t K) {
  if (K > TC_COLS) return round_up(K, TC_COLS);
  int64_t w = 8;
  while (w < K) w <<= 1;
  return w;
}

// device work lists for a 64-row-tile batch of K columns (cached per width)
// nc > 0: plan for the small-batch kernel (128-row operator tiles as the MMA
// M dimension, nc residual columns per tile, chi2 partials per 32 rows).
static td_status get_split_plan(td_segment* s, Scratch& sc, int64_t K, int nsl, int bn, cudaStream_t st,
                                SplitPlan** out, int nc = 0, int S_force = 0) {
  ++sc.use_clock;
  const int S = S_force > 0 ? S_force : split_chunk(s->nk, s->nkp, bn);
  const int key_bn = nc > 0 ? -nc : bn;
  // a re-factored segment (new log det) drops its plans; an operator that only
  // moved (evicted and reloaded by a server) keeps them: their operator maps
  // are re-encoded and the descriptors re-uploaded on `st`, with no device
  // synchronisation (no kernel of this segment runs while its operator moves)
  for (size_t i = 0; i < sc.plans.size();)
    if (sc.plans[i].seg == (const void*)s && sc.plans[i].logdet != s->logdet) {
      cudaStreamSynchronize(st);
      free_plan(sc.plans[i]);
      sc.plans.erase(sc.plans.begin() + (long)i);
    } else {
      ++i;
    }
  for (SplitPlan& p : sc.plans)
    if (p.seg == (const void*)s && p.op != (const void*)s->op) {
      td_status rr = encode_3d(&p.host_seg.mapB, s->op, OP_KB, OP_ROWS, (uint64_t)s->op_blocks * OP_SLICES,
                               OP_KB * 2, (uint64_t)OP_ROWS * OP_KB * 2, OP_KB, (uint32_t)p.map_bn,
                               (uint32_t)p.nsl);
      if (rr != TD_OK) return rr;
      if (st)
        TD_CUDA(cudaMemcpyAsync(p.segdev, &p.host_seg, sizeof(TcSegDev), cudaMemcpyHostToDevice, st));
      else   // the legacy stream: copy synchronously, so streams created non-blocking see it too
        TD_CUDA(cudaMemcpy(p.segdev, &p.host_seg, sizeof(TcSegDev), cudaMemcpyHostToDevice));
      p.op = s->op;
    }
  for (SplitPlan& p : sc.plans)
    if (p.seg == (const void*)s && p.K == K && p.nsl == nsl && p.bn == key_bn && p.S == S) {
      p.last_use = sc.use_clock;
      *out = &p;
      return TD_OK;
    }
  std::vector<TcItem> items;
  std::vector<SplitUnit> units;
  int n_slots = 0;
  // from 128 columns on every row tile of the small-batch kernel goes through
  // the chunk reduction: its in-kernel chi2 epilogue (a shuffle tree per
  // column) would hold back the CTAs that take whole rows
  plan_split_segment(0, s->nk, s->nkp, K, bn, S, items, units, n_slots, nc >= 128, nc > 0 ? nc : TC_COLS);
  const int64_t slot_elems = (int64_t)std::max(TC_COLS, nc) * bn;   // float2 per slot
  sort_items(items);
  td_status r;
  if (n_slots * slot_elems > sc.wpart_slots) {   // wpart_slots counts float2 elements
    // a larger buffer for this and later plans; the older plans keep naming
    // the old one, which stays allocated with the scratch (their batches run
    // in stream order on the scratch's stream, so the two are never in use at once)
    float2* w = nullptr;
    if ((r = dev_alloc(&w, (size_t)(n_slots * slot_elems), "split accumulators")) != TD_OK) return r;
    if (sc.wpart) sc.wpart_old.push_back(sc.wpart);
    sc.wpart = w;
    sc.wpart_slots = n_slots * slot_elems;
  }
  if (sc.plans.size() >= sc.max_plans) {   // evict the least recently used plan
    size_t lru = 0;
    for (size_t i = 1; i < sc.plans.size(); ++i)
      if (sc.plans[i].last_use < sc.plans[lru].last_use) lru = i;
    cudaStreamSynchronize(st);
    dev_free(sc.plans[lru].items);
    dev_free(sc.plans[lru].units);
    dev_free(sc.plans[lru].segdev);
    dev_free(sc.plans[lru].counters);
    sc.plans.erase(sc.plans.begin() + (long)lru);
  }
  SplitPlan p;
  p.seg = s;
  p.K = K;
  p.nsl = nsl;
  p.bn = key_bn;
  p.S = S;
  p.n_items = (int)items.size();
  p.n_units = (int)units.size();
  p.n_slots = n_slots;
  p.op = s->op;
  p.logdet = s->logdet;
  TcSegDev seg;
  memset(&seg, 0, sizeof seg);
  const int a_rows = nc > 0 ? nc : (int)std::min<int64_t>(TC_COLS, round_up(K, 8));
  if ((r = encode_seg_maps(s, K, nsl, bn, &seg, a_rows, nullptr, &sc)) != TD_OK) return r;
  seg.partials = sc.partials;
  seg.wpart = sc.wpart;
  seg.nk = (int)s->nk;
  seg.K = (int)K;
  seg.ldp = (int)sc.capK;                                   // small: the buffer as [N'p/128][capK]
  seg.nm = nc > 0 ? (int)(s->nkp / 128) : (int)(s->nkp / 64);   // partials: per 128-row tile (small) or 64 rows
  seg.logdet = s->logdet;
  if ((r = dev_alloc(&p.items, items.size(), "work items")) != TD_OK ||
      (r = dev_alloc(&p.units, std::max<size_t>(1, units.size()), "split units")) != TD_OK ||
      (r = dev_alloc(&p.segdev, 1, "segment descriptor")) != TD_OK ||
      (nc > 0 && (r = dev_alloc(&p.counters, (size_t)std::max<int>(SMALL_GROUPS, (int)units.size() + 1),
                                 "completion counters")) != TD_OK)) {
    dev_free(p.items);
    dev_free(p.units);
    dev_free(p.segdev);
    dev_free(p.counters);
    return r;
  }
  p.n_counters = p.counters ? std::max<int>(SMALL_GROUPS, (int)units.size() + 1) : 0;
  if (p.counters) TD_CUDA(cudaMemset(p.counters, 0, (size_t)p.n_counters * sizeof(int)));
  TD_CUDA(cudaMemcpy(p.items, items.data(), items.size() * sizeof(TcItem), cudaMemcpyHostToDevice));
  if (!units.empty())
    TD_CUDA(cudaMemcpy(p.units, units.data(), units.size() * sizeof(SplitUnit), cudaMemcpyHostToDevice));
  TD_CUDA(cudaMemcpy(p.segdev, &seg, sizeof seg, cudaMemcpyHostToDevice));
  p.host_seg = seg;
  p.map_bn = bn;
  p.last_use = sc.use_clock;
  sc.plans.push_back(p);
  *out = &sc.plans.back();
  return TD_OK;
}

td_status read_status(td_segment* s, cudaStream_t st, DevStatus* out) {
  TD_CUDA(cudaMemcpyAsync(out, s->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
  TD_CUDA(cudaStreamSynchronize(st));
  return TD_OK;
}

// the clock sums of a device status word: read, convert, clear
td_status read_clock(DevStatus* dst, cudaStream_t st, double* mhz) {
  if (!mhz) return fail(TD_ERR_INVALID, "mhz is NULL");
  unsigned long long v[2] = {0, 0};
  TD_CUDA(cudaMemcpyAsync(v, &dst->mma_cycles, sizeof v, cudaMemcpyDeviceToHost, st));
  TD_CUDA(cudaStreamSynchronize(st));
  TD_CUDA(cudaMemsetAsync(&dst->mma_cycles, 0, sizeof v, st));
  TD_CUDA(cudaStreamSynchronize(st));
  if (v[1] == 0) return fail(TD_ERR_INVALID, "no split-product kernel ran since the last clock read");
  *mhz = 1000.0 * (double)v[0] / (double)v[1];
  return TD_OK;
}

td_status reset_status(td_segment* s, cudaStream_t st) {
  DevStatus h{0, 0, LLONG_MAX};
  TD_CUDA(cudaMemcpyAsync(s->status, &h, sizeof h, cudaMemcpyHostToDevice, st));
  TD_CUDA(cudaStreamSynchronize(st));
  return TD_OK;
}

// bracket the dominant kernel with events when profiling is on
static void prof_mark(td_segment* s, cudaStream_t st, bool start) {
  if (!s->prof) return;
  if (start && s->ev_used + 2 > s->ev.size()) {
    if (s->ev.size() >= 8192) return;
    for (int i = 0; i < 64; ++i) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      s->ev.push_back(e);
    }
  }
  if (start) {
    cudaEventRecord(s->ev[s->ev_used], st);
  } else {
    cudaEventRecord(s->ev[s->ev_used + 1], st);
    s->ev_used += 2;
  }
}

}  // namespace td

using namespace td;

extern "C" {

void td_options_default(td_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof *opt);
  opt->precision = TD_PREC_AUTO;
  opt->path = TD_PATH_AUTO;
  opt->refine = 0;
  opt->wait_limit_ns = 1000000000LL;
}

const char* td_last_error(void) { return g_last_error.c_str(); }

td_status td_segment_create(const double* acf, int64_t n, const uint8_t* mask, void* stream, td_segment** out) {
  if (!out) return fail(TD_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!acf) return fail(TD_ERR_INVALID, "acf is NULL");
  if (n < 1) return fail(TD_ERR_INVALID, "n must be >= 1");
  if (n > (int64_t)INT32_MAX) return fail(TD_ERR_INVALID, "n too large");
  if (!(acf[0] > 0.0) || !std::isfinite(acf[0])) return fail(TD_ERR_INVALID, "acf[0] must be positive and finite");
  for (int64_t k = 0; k < n; ++k)
    if (!std::isfinite(acf[k])) return fail(TD_ERR_INVALID, "acf has a non-finite entry");
  std::vector<int32_t> t;
  t.reserve((size_t)n);
  for (int64_t i = 0; i < n; ++i)
    if (!mask || mask[i]) t.push_back((int32_t)i);
  if (t.empty()) return fail(TD_ERR_INVALID, "mask keeps no sample");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  td_segment* s = new td_segment();
  cudaGetDevice(&s->device);
  s->n = n;
  s->nk = (int64_t)t.size();
  s->nkp = round_up(s->nk, OP_ROWS);
  s->nkp8 = round_up(s->nk, 8);
  td_status r;
  if ((r = dev_alloc(&s->acf, (size_t)n, "acf")) != TD_OK ||
      (r = dev_alloc(&s->t, t.size(), "kept index")) != TD_OK ||
      (r = dev_alloc(&s->status, 1, "status")) != TD_OK) {
    td_segment_destroy(s);
    return r;
  }
  cudaError_t e = cudaMemcpyAsync(s->acf, acf, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->t, t.data(), t.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    td_segment_destroy(s);
    return cuda_fail(e, "td_segment_create copies");
  }
  if ((r = reset_status(s, st)) != TD_OK) {
    td_segment_destroy(s);
    return r;
  }
  *out = s;
  return TD_OK;
}

int64_t td_kept(const td_segment* s) { return s ? s->nk : -1; }

int64_t td_last_pivot(const td_segment* s) { return s ? s->pivot : -1; }

td_status td_logdet(const td_segment* s, double* out) {
  if (!s || !out) return fail(TD_ERR_INVALID, "NULL argument");
  if (!s->factored && s->gs.ready) {
    *out = s->gs.logdet;
    return TD_OK;
  }
  if (!s->factored) return fail(TD_ERR_NOT_FACTORED, "segment not factored");
  *out = s->logdet;
  return TD_OK;
}

int64_t td_resident_bytes(const td_segment* s) {
  if (!s) return 0;
  int64_t b = s->n * 8 + s->nk * 4;
  if (s->L) b += s->nkp * s->nkp * 8;
  if (s->dinv) b += (s->nkp / FT) * FT * FT * 8;
  if (s->op) b += s->op_blocks * OP_SLICES * OP_ROWS * OP_KB * 2;
  return b;
}

td_status td_factor(td_segment* s, void* stream) {
  if (!s) return fail(TD_ERR_INVALID, "segment is NULL");
  td_status r = check_device(s);
  if (r != TD_OK) return r;
  return factor_tensor(s, reinterpret_cast<cudaStream_t>(stream), EMU_SLICES);
}

}  // extern "C"

namespace td {

td_status reserve_with(td_segment* s, Scratch& sc, int64_t K, const td_options* opt) {
  if (!s || K < 0) return fail(TD_ERR_INVALID, "bad argument");
  td_options o;
  td_options_default(&o);
  if (opt) o = *opt;
  const bool fp64 = o.path == TD_PATH_FP64 || o.precision == TD_PREC_FP64;
  td_status r = ensure_scratch(s, sc, K, fp64, 0);
  if (r != TD_OK || fp64 || !s->factored || !s->op) return r;
  // the work lists the batch path will use for widths up to K, built now so
  // that later calls allocate nothing
  const int nsl = nslices_for(o.precision, s->nk);
  SplitPlan* plan = nullptr;
  for (int ncs = 16; ncs <= 256; ncs *= 2)
    if ((o.path == TD_PATH_AUTO || o.path == TD_PATH_SMALLK) &&
        (r = get_split_plan(s, sc, ncs, nsl, 128, 0, &plan, ncs)) != TD_OK)
      return r;
  for (int64_t k = 8; k <= K; k = (k < TC_COLS) ? 2 * k : k + TC_COLS) {
    const Shape sh = choose_shape(s, k, o.path);
    if (sh.bn != 0 && sh.split && (r = get_split_plan(s, sc, plan_width(k), nsl, sh.bn, 0, &plan, 0, sh.S)) != TD_OK)
      return r;
  }
  return TD_OK;
}

}  // namespace td

extern "C" {

td_status td_reserve(td_segment* s, int64_t K, const td_options* opt) {
  if (!s) return fail(TD_ERR_INVALID, "bad argument");
  return reserve_with(s, s->scr, K, opt);
}

td_status td_loglike_batch(td_segment* s, const float* R, int64_t ldr, int64_t K, double* logL,
                           const td_options* opt, double* chi2, void* stream) {
  if (!s) return fail(TD_ERR_INVALID, "segment is NULL");
  return loglike_batch_with(s, s->scr, R, ldr, K, logL, opt, chi2, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace td {

td_status loglike_batch_with(td_segment* s, Scratch& sc, const float* R, int64_t ldr, int64_t K, double* logL,
                             const td_options* opt, double* chi2, cudaStream_t stream) {
  if (!s) return fail(TD_ERR_INVALID, "segment is NULL");
  if (K < 0) return fail(TD_ERR_INVALID, "K < 0");
  if (K > TD_MAX_K) return fail(TD_ERR_INVALID, "K above 2^30 columns");
  if (K == 0) return TD_OK;
  if (!R || !logL) return fail(TD_ERR_INVALID, "R or logL is NULL");
  if (ldr < s->nk) return fail(TD_ERR_INVALID, "ldr < N'");
  td_options o;
  td_options_default(&o);
  if (opt) o = *opt;
  if (o.path == TD_PATH_GSCE || gs_auto(s, K, o)) {
    td_status rg = check_device(s);
    if (rg != TD_OK) return rg;
    if (o.refine) return fail(TD_ERR_INVALID, "refinement applies to the split-product paths, not to GSCE");
    if (!s->gs.ready) return fail(TD_ERR_NOT_FACTORED, "GSCE path: call td_gs_prepare first");
    return gs_batch(s, R, ldr, K, logL, chi2, reinterpret_cast<cudaStream_t>(stream));
  }
  if (!s->factored) return fail(TD_ERR_NOT_FACTORED, "segment not factored");
  td_status r = check_device(s);
  if (r != TD_OK) return r;
  if (o.wait_limit_ns <= 0) o.wait_limit_ns = 1000000000LL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const bool fp64 = (o.precision == TD_PREC_FP64) || (o.path == TD_PATH_FP64);
  if (fp64 && o.refine) return fail(TD_ERR_INVALID, "refinement applies to the split-product paths, not to FP64");
  if (fp64 && !s->L) return fail(TD_ERR_UNSUPPORTED, "the FP64 factor of this segment was released");
  if (!fp64 && !s->op) return fail(TD_ERR_NOT_FACTORED, "the operator of this segment is not resident");
  if ((r = ensure_scratch(s, sc, K, fp64, st)) != TD_OK) return r;
  const int64_t ldp = sc.capK;
  if (fp64) {
    const int nt = (int)(s->nkp / FT);
    const bool pm = s->prof && s->ev_used + 2 <= 8192;
    if (pm) prof_mark(s, st, true);
    TD_CUDA(launch_fp64_solve(s->L, s->nkp, s->dinv, R, ldr, s->nk, s->nkp, K, sc.w64, s->nkp, sc.partials, ldp,
                              st));
    if (pm) prof_mark(s, st, false);
    TD_CUDA(launch_finalize(sc.partials, ldp, nt, K, s->logdet, s->nk, logL, chi2, st));
    s->prof_kernels += 2 * nt + 1;
    return TD_OK;
  }
  const int nsl = nslices_for(o.precision, s->nk);
  if (o.refine) {
    if (&sc != &s->scr) return fail(TD_ERR_UNSUPPORTED, "refinement runs on the segment's own scratch");
    return refine_batch(s, R, ldr, K, logL, chi2, nsl, o.refine == 2 ? 2 : 1, o.path, o.wait_limit_ns, st);
  }
  const Shape shape = choose_shape(s, K, o.path);
  const int bn = shape.bn;
  const int ngroups = (int)(s->nkp / 64);
  const int nc = (int)ceil_div(K, TC_COLS);
  const int nkb_max = (int)ceil_div(s->nk, OP_KB);
  const bool pm = s->prof && s->ev_used + 2 <= 8192;
  if (bn == 0) {   // small batch: operator rows as the MMA M dimension
    if (K > 256) return fail(TD_ERR_UNSUPPORTED, "the small-batch path takes K <= 256");
    const int ncs = K <= 16 ? 16 : (K <= 32 ? 32 : (K <= 64 ? 64 : (K <= 128 ? 128 : 256)));
    SplitPlan* plan = nullptr;
    if ((r = get_split_plan(s, sc, ncs, nsl, 128, st, &plan, ncs)) != TD_OK) return r;
    // launches chained as programmatic dependents: the slicing (which also
    // clears the plan's completion counters), the product, the chunk
    // reduction with chi2 and logL.  Up to SMALL_FUSED_K columns the product
    // kernel reduces in-kernel instead (one launch less; its arrival-count tail
    // grows with the columns, the separate kernel's does not).  Up to 64
    // columns the slicing is itself a programmatic dependent of the preceding
    // launch (it waits for it before touching memory), so the next call's
    // launches are resident while this one finishes.
    const bool fused = K <= SMALL_FUSED_K;
    TD_CUDA(launch_r_slices(R, ldr, s->nk, K, s->nkp8, sc.capK, sc.rs, nsl, st, plan->counters,
                            plan->n_counters, ncs <= 64));
    const SmallFinal fin{plan->units, plan->counters, plan->n_units, (int)K, logL, chi2, std::max(TC_COLS, ncs)};
    if (pm) prof_mark(s, st, true);   // the events bracket the product kernel alone
    TD_CUDA(launch_tc_small(plan->items, plan->n_items, plan->segdev, nsl, ncs, s->status, o.wait_limit_ns, st,
                            fused ? &fin : nullptr));
    if (pm) prof_mark(s, st, false);
    if (!fused) TD_CUDA(launch_small_reduce(plan->segdev, fin, st));
    s->prof_kernels += fused ? 2 : 3;
    return TD_OK;
  }
  TD_CUDA(launch_r_slices(R, ldr, s->nk, K, s->nkp8, sc.capK, sc.rs, nsl, st));
  if (shape.split) {
    SplitPlan* plan = nullptr;
    if ((r = get_split_plan(s, sc, plan_width(K), nsl, bn, st, &plan, 0, shape.S)) != TD_OK) return r;
    if (pm) prof_mark(s, st, true);   // the events bracket the product kernel alone
    TD_CUDA(launch_tc_cdo(plan->items, plan->n_items, plan->segdev, nsl, bn, true, s->status, o.wait_limit_ns,
                          st));
    if (pm) prof_mark(s, st, false);
    TD_CUDA(launch_split_reduce(plan->units, plan->n_units, plan->segdev, bn, st, plan->K));
    TD_CUDA(launch_finalize(sc.partials, ldp, ngroups, K, s->logdet, s->nk, logL, chi2, st));
    s->prof_kernels += plan->n_units > 0 ? 4 : 3;
    return TD_OK;
  }
  TcSegDev seg;   // whole rows: one segment, implicit item list
  memset(&seg, 0, sizeof seg);
  if ((r = encode_seg_maps(s, K, nsl, bn, &seg, TC_COLS, nullptr, &sc)) != TD_OK) return r;
  seg.partials = sc.partials;
  seg.nk = (int)s->nk;
  seg.K = (int)K;
  seg.ldp = (int)ldp;
  seg.nm = ngroups;
  if (pm) prof_mark(s, st, true);
  TD_CUDA(launch_tc_single(seg, bn, nc, nkb_max, nsl, s->status, o.wait_limit_ns, st));
  if (pm) prof_mark(s, st, false);
  TD_CUDA(launch_finalize(sc.partials, ldp, ngroups, K, s->logdet, s->nk, logL, chi2, st));
  s->prof_kernels += 3;
  return TD_OK;
}

}  // namespace td

extern "C" {

td_status td_segment_release_fp64(td_segment* s) {
  if (!s) return fail(TD_ERR_INVALID, "segment is NULL");
  cudaDeviceSynchronize();
  dev_free(s->L);
  dev_free(s->dinv);
  dev_free(s->scr.w64);
  free_refine_state(s);   // the slices of L go with L: refinement then returns TD_ERR_UNSUPPORTED
  return TD_OK;
}

td_status td_check(td_segment* s, void* stream) {
  if (!s) return fail(TD_ERR_INVALID, "segment is NULL");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  DevStatus hs;
  td_status r = read_status(s, st, &hs);
  if (r != TD_OK) return r;
  if (hs.code != 0) {
    reset_status(s, st);
    if (hs.code == ST_TIMEOUT) {
      char buf[96];
      snprintf(buf, sizeof buf, "a bounded in-kernel wait ran out (site %d)", hs.where);
      return fail(TD_ERR_TIMEOUT, buf);
    }
    return fail((td_status)hs.code, "device reported an error");
  }
  return TD_OK;
}

td_status td_profile_enable(td_segment* s, int enable) {
  if (!s) return fail(TD_ERR_INVALID, "segment is NULL");
  s->prof = enable != 0;
  s->ev_used = 0;
  s->prof_kernels = 0;
  TD_CUDA(cudaDeviceSynchronize());   // no kernel of this segment still adds to the clock sums
  TD_CUDA(cudaMemset(&s->status->mma_cycles, 0, 2 * sizeof(unsigned long long)));
  TD_CUDA(cudaDeviceSynchronize());
  return TD_OK;
}


td_status td_profile_clock(td_segment* s, void* stream, double* mhz) {
  if (!s) return fail(TD_ERR_INVALID, "segment is NULL");
  return read_clock(s->status, reinterpret_cast<cudaStream_t>(stream), mhz);
}

td_status td_profile_read(td_segment* s, double* ms_total, int64_t* dominant_launches, int64_t* kernels_launched) {
  if (!s) return fail(TD_ERR_INVALID, "segment is NULL");
  double tot = 0.0;
  for (size_t i = 0; i + 1 < s->ev_used; i += 2) {
    TD_CUDA(cudaEventSynchronize(s->ev[i + 1]));
    float ms = 0.f;
    TD_CUDA(cudaEventElapsedTime(&ms, s->ev[i], s->ev[i + 1]));
    tot += ms;
  }
  if (ms_total) *ms_total = tot;
  if (dominant_launches) *dominant_launches = (int64_t)(s->ev_used / 2);
  if (kernels_launched) *kernels_launched = s->prof_kernels;
  s->ev_used = 0;
  s->prof_kernels = 0;
  return TD_OK;
}

void td_segment_destroy(td_segment* s) {
  if (!s) return;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != s->device) cudaSetDevice(s->device);
  cudaDeviceSynchronize();
  dev_free(s->acf);
  dev_free(s->t);
  dev_free(s->L);
  dev_free(s->dinv);
  dev_free(s->ldpart);
  dev_free(s->op);
  dev_free(s->status);
  scratch_free(s->scr);
  free_host_stage(s->hst);
  free_template_state(s->tpl);
  if (s->gat) cudaFree(s->gat);
  free_refine_state(s);
  free_gs_state(s);
  for (cudaEvent_t e : s->ev) cudaEventDestroy(e);
  if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
  delete s;
}

td_status td_debug_bounded_wait(int64_t limit_ns, void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  DevStatus* d = nullptr;
  td_status r = dev_alloc(&d, 1, "probe status");
  if (r != TD_OK) return r;
  DevStatus h{0, 0, 0};
  cudaError_t e = cudaMemcpyAsync(d, &h, sizeof h, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_bounded_wait_probe(d, limit_ns, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "bounded wait probe");
  if (h.code == ST_TIMEOUT) return fail(TD_ERR_TIMEOUT, "bounded wait ran out as expected");
  return TD_OK;
}

}  // extern "C"
