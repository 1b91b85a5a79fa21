// Serving runtime: many concurrent likelihood requests on many resident
// segments, continuously batched.
//
// The paper parallelises a sampler by a pool of processes that each evaluate
// proposals (Sec. III.B, "CPU acceleration"); here those proposals are
// requests -- (segment, K residual columns) -- from any number of host
// threads.  A scheduler thread packs the pending columns of one segment into
// one batch whenever a stream is free (continuous batching: requests that
// arrive while other batches run join the next batch of their segment), so
// batches of different segments run concurrently on separate streams.  The
// whitening operators stay resident in HBM under a byte budget with LRU
// eviction; an evicted operator is kept in pinned host memory and copied back
// on its next use.  Admission is bounded by a pending-column capacity
// (TD_ERR_BUSY beyond it).  A completion thread timestamps finished batches;
// p50/p99 latency is measured from submission to completion.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "td_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t ticket;
  int64_t seg;
  const float* R;
  int64_t ldr;
  int64_t K;
  double* logL;
  Clock::time_point t_submit;
  int state;   // 0 pending, 1 in flight, 2 done, 3 cancelled, 4 failed
  double lat_us = -1.0;   // submission to completion, once done
};

struct SegEntry {
  td_segment* s = nullptr;
  bool resident = false;      // operator slices on the device
  bool pooled = false;        // the device copy came from the server's memory pool
  void* host_op = nullptr;    // pinned host copy of the operator slices
  bool host_op_pooled = false;  // carved from the server's spill pool (not freed on its own)
  cudaEvent_t spilled = nullptr;  // recorded after the spill copy: a reload on any stream waits for it
  size_t op_bytes = 0;
  int inflight = 0;           // batches of this segment on the GPU
  uint64_t last_use = 0;
  std::deque<int64_t> queue;  // pending tickets
};

struct ColRef {               // one column of a batch: where it comes from, where its logL goes
  const float* src;
  double* dst;
};

struct Slot {                 // one stream and its batch buffers
  td::Scratch scr;            // residual slices, partials and work lists of this stream's batches
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  float* Rb = nullptr;        // N'max x max_cols batch residuals
  double* Lb = nullptr;       // max_cols batch logL
  ColRef* refs_h = nullptr;   // pinned host, max_cols: the batch's column map
  ColRef* refs_d = nullptr;   // device copy of it
  bool busy = false;
  int64_t seg = -1;
  std::vector<int64_t> tickets;
};

}  // namespace

struct td_server {
  td_server_config cfg;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::thread sched, compl_thr;
  std::atomic<bool> stop{false};
  bool paused = false;
  std::vector<SegEntry> segs;
  std::unordered_map<int64_t, Request> reqs;
  int64_t next_ticket = 1;
  int64_t pending_cols = 0;
  std::vector<Slot> slots;
  std::deque<int> inflight_order;   // slot indices in launch order
  int64_t max_nk = 0;
  uint64_t clock = 0;
  size_t resident_bytes = 0;
  // statistics
  cudaMemPool_t pool = nullptr;     // stream-ordered pool for reloaded operators
  void* spill = nullptr;            // pinned host spill pool
  size_t spill_cap = 0, spill_used = 0;
  std::vector<double> lat_us;
  int64_t evals = 0, batches = 0, hits = 0, misses = 0, evictions = 0, refused = 0, failed = 0, reloads = 0;
  Clock::time_point t_first, t_last;
  bool any_done = false;
  td_status last_err = TD_OK;
};

namespace td {

// a batch's columns, gathered from the requests' buffers into one N' x cols
// block (one CTA per column) and its logL scattered back: two launches per
// batch instead of two copies per request
__global__ void k_gather_cols(const ColRef* __restrict__ refs, int64_t nk, float* __restrict__ Rb) {
  const float* src = refs[blockIdx.x].src;
  float* dst = Rb + (int64_t)blockIdx.x * nk;
  for (int64_t j = threadIdx.x; j < nk; j += blockDim.x) dst[j] = src[j];
}

__global__ void k_scatter_logl(const ColRef* __restrict__ refs, int64_t cols, const double* __restrict__ Lb) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < cols) *refs[k].dst = Lb[k];
}

// The pinned host copy of a segment's operator, made once, at its first
// eviction, by an asynchronous copy on `st` (the operator does not change
// afterwards).  It is carved from the server's pinned spill pool
// (host_spill_bytes, pinned once at creation) while that has room, else
// allocated on its own (cudaMallocHost, which blocks).
static td_status seg_spill_copy(td_server* srv, SegEntry& e, cudaStream_t st) {
  if (e.host_op) return TD_OK;
  const size_t need = (e.op_bytes + 255) & ~(size_t)255;
  if (srv->spill && srv->spill_used + need <= srv->spill_cap) {
    e.host_op = static_cast<unsigned char*>(srv->spill) + srv->spill_used;
    e.host_op_pooled = true;
    srv->spill_used += need;
  } else if (cudaMallocHost(&e.host_op, e.op_bytes) != cudaSuccess) {
    cudaGetLastError();
    e.host_op = nullptr;
    return fail(TD_ERR_OOM, "pinned host copy of an operator");
  }
  TD_CUDA(cudaMemcpyAsync(e.host_op, e.s->op, e.op_bytes, cudaMemcpyDeviceToHost, st));
  if (!e.spilled) TD_CUDA(cudaEventCreateWithFlags(&e.spilled, cudaEventDisableTiming));
  TD_CUDA(cudaEventRecord(e.spilled, st));
  return TD_OK;
}

// Evict on `st` (the segment has no batch in flight): the spill copy (first
// time only) and the release of the device copy to the pool are both queued
// in stream order, with no host or device synchronisation.
static td_status seg_evict(td_server* srv, SegEntry& e, cudaStream_t st) {
  if (!e.resident) return TD_OK;
  td_status r = seg_spill_copy(srv, e, st);
  if (r != TD_OK) return r;
  if (e.pooled)
    TD_CUDA(cudaFreeAsync(e.s->op, st));
  else
    TD_CUDA(cudaFree(e.s->op));
  e.s->op = nullptr;
  e.pooled = false;
  e.resident = false;
  srv->resident_bytes -= e.op_bytes;
  srv->evictions++;
  return TD_OK;
}

// Move a freshly built operator into the server's device pool (set-up time):
// later evictions and reloads of the segment then stay stream-ordered.
static td_status seg_rehome(td_server* srv, SegEntry& e, cudaStream_t st) {
  void* p = nullptr;
  TD_CUDA(cudaMallocFromPoolAsync(&p, e.op_bytes, srv->pool, st));
  TD_CUDA(cudaMemcpyAsync(p, e.s->op, e.op_bytes, cudaMemcpyDeviceToDevice, st));
  TD_CUDA(cudaStreamSynchronize(st));
  TD_CUDA(cudaFree(e.s->op));
  e.s->op = reinterpret_cast<__nv_bfloat16*>(p);
  e.pooled = true;
  return TD_OK;
}

// make the segment's operator resident (evicting least recently used idle
// segments while over budget); called with the lock held
// cols > 0: the width of the batch about to run; a batch that TD_PATH_AUTO
// sends to GSCE needs only the segment's Gohberg-Semencul data (made here on
// first use when the server is configured for it), not the dense operator
static td_status seg_make_resident(td_server* srv, int64_t id, cudaStream_t st, int64_t cols = 0) {
  SegEntry& e = srv->segs[(size_t)id];
  e.last_use = ++srv->clock;
  const bool use_gs = srv->cfg.gs_gapfree && !srv->cfg.deterministic;
  if (use_gs && !e.s->gs.ready && gs_supported(e.s)) {
    const td_status rg = td_gs_prepare(e.s, st);
    if (rg != TD_OK) return rg;
  }
  if (cols > 0 && use_gs && e.s->gs.ready && srv->cfg.precision != TD_PREC_FP64 && gs_preferred(e.s, cols)) {
    srv->hits++;   // the batch runs on the (resident) GS data whether or not the operator is
    return TD_OK;
  }
  if (e.resident) {
    srv->hits++;
    return TD_OK;
  }
  srv->misses++;
  const int64_t budget = srv->cfg.resident_bytes_budget;
  // e.op_bytes is known from N' before the first factor
  while (budget > 0 && (int64_t)(srv->resident_bytes + e.op_bytes) > budget) {
    int64_t victim = -1;
    for (size_t i = 0; i < srv->segs.size(); ++i) {
      SegEntry& c = srv->segs[i];
      if ((int64_t)i == id || !c.resident || c.inflight > 0) continue;
      // while serving, a victim needs a spill copy already or room for one in
      // the pinned pool: pinning new host memory (cudaMallocHost) would block
      // the scheduler for about a second per GB-scale operator
      if (srv->spill && !c.host_op && srv->spill_used + ((c.op_bytes + 255) & ~(size_t)255) > srv->spill_cap)
        continue;
      if (victim < 0 || c.last_use < srv->segs[(size_t)victim].last_use) victim = (int64_t)i;
    }
    if (victim < 0) break;   // everything else is busy or cannot spill: exceed the budget for now
    const td_status re = seg_evict(srv, srv->segs[(size_t)victim], st);
    if (re != TD_OK) return re;
  }
  if (!e.s->factored) {
    // gap-free: O(N^2) Levinson-Durbin operator; gapped: Cholesky, FP64 factor then released
    td_segment* one = e.s;
    td_status r = td_factor_many(&one, 1, TD_FACTOR_NO_FP64, st);
    if (r != TD_OK) return r;
    if ((r = seg_rehome(srv, e, st)) != TD_OK) return r;   // pooled, so eviction never synchronises
    // work lists for every batch width on every stream's scratch up front: no
    // allocation while serving
    td_options o;
    td_options_default(&o);
    o.precision = srv->cfg.precision;
    if (srv->cfg.deterministic) o.path = TD_PATH_SMALLK;
    for (Slot& sl : srv->slots)
      if ((r = reserve_with(e.s, sl.scr, srv->cfg.max_batch_cols, &o)) != TD_OK) return r;
  } else {
    void* p = nullptr;
    TD_CUDA(cudaMallocFromPoolAsync(&p, e.op_bytes, srv->pool, st));
    e.s->op = reinterpret_cast<__nv_bfloat16*>(p);
    e.pooled = true;
    if (e.spilled) TD_CUDA(cudaStreamWaitEvent(st, e.spilled, 0));   // the spill copy may be on another stream
    TD_CUDA(cudaMemcpyAsync(e.s->op, e.host_op, e.op_bytes, cudaMemcpyHostToDevice, st));
    srv->reloads++;
  }
  e.resident = true;
  srv->resident_bytes += e.op_bytes;
  return TD_OK;
}

static void scheduler_loop(td_server* srv) {
  cudaSetDevice(srv->device);
  td_options opt;
  td_options_default(&opt);
  opt.precision = srv->cfg.precision;
  if (srv->cfg.deterministic) opt.path = TD_PATH_SMALLK;
  std::unique_lock<std::mutex> lk(srv->mu);
  Clock::time_point last_batch = Clock::now();
  while (!srv->stop) {
    // a free slot and a segment with pending columns that has no batch in flight
    int slot = -1;
    for (size_t i = 0; i < srv->slots.size(); ++i)
      if (!srv->slots[i].busy) {
        slot = (int)i;
        break;
      }
    int64_t pick = -1;
    Clock::time_point oldest = Clock::time_point::max();
    if (slot >= 0 && !srv->paused) {
      for (size_t i = 0; i < srv->segs.size(); ++i) {
        SegEntry& e = srv->segs[i];
        // batches of one segment may run on several streams at once (each
        // stream has its own scratch); the Gohberg-Semencul form keeps one
        // product buffer per segment, so such segments take one at a time
        if (e.queue.empty() || (e.inflight > 0 && (e.s->gs.ready || !e.resident))) continue;
        const Request& r = srv->reqs[e.queue.front()];
        if (r.t_submit < oldest) {
          oldest = r.t_submit;
          pick = (int64_t)i;
        }
      }
    }
    if (slot < 0 || pick < 0) {
      // idle: spin for up to a millisecond after the last batch (a condition
      // variable wake-up costs tens of microseconds per request), then sleep
      if (Clock::now() - last_batch < std::chrono::milliseconds(1)) {
        lk.unlock();
        std::this_thread::yield();
        lk.lock();
      } else {
        srv->cv_sched.wait_for(lk, std::chrono::milliseconds(5));
      }
      continue;
    }
    last_batch = Clock::now();
    Slot& sl = srv->slots[(size_t)slot];
    SegEntry& e = srv->segs[(size_t)pick];
    // gather whole requests up to the batch width (oldest first)
    sl.tickets.clear();
    int64_t cols = 0;
    while (!e.queue.empty()) {
      Request& r = srv->reqs[e.queue.front()];
      if (cols > 0 && cols + r.K > srv->cfg.max_batch_cols) break;
      e.queue.pop_front();
      if (r.state != 0) continue;   // cancelled
      r.state = 1;
      sl.tickets.push_back(r.ticket);
      cols += r.K;
    }
    if (sl.tickets.empty()) continue;
    td_status st = seg_make_resident(srv, pick, sl.st, cols);
    const int64_t nk = e.s->nk;
    // deterministic: the small-batch path in chunks of at most 256 columns, whose
    // per-column arithmetic does not depend on the other columns of the call
    auto run = [&](const float* R, int64_t ldr, int64_t K, double* L) -> td_status {
      if (!srv->cfg.deterministic) return loglike_batch_with(e.s, sl.scr, R, ldr, K, L, &opt, nullptr, sl.st);
      for (int64_t c0 = 0; c0 < K; c0 += 256) {
        const td_status rc = loglike_batch_with(e.s, sl.scr, R + c0 * ldr, ldr, std::min<int64_t>(256, K - c0),
                                                L + c0, &opt, nullptr, sl.st);
        if (rc != TD_OK) return rc;
      }
      return TD_OK;
    };
    if (st == TD_OK && sl.tickets.size() == 1) {
      // one request: evaluate it in place (its R and logL are device buffers)
      const Request& r = srv->reqs[sl.tickets[0]];
      st = run(r.R, r.ldr, r.K, r.logL);
    } else if (st == TD_OK) {
      // the batch's column map (the slot's previous batch has completed, so the
      // pinned map is free), gather, evaluate, scatter logL
      int64_t off = 0;
      for (int64_t t : sl.tickets) {
        const Request& r = srv->reqs[t];
        for (int64_t k = 0; k < r.K; ++k) sl.refs_h[off + k] = ColRef{r.R + k * r.ldr, r.logL + k};
        off += r.K;
      }
      cudaError_t ce = cudaMemcpyAsync(sl.refs_d, sl.refs_h, (size_t)cols * sizeof(ColRef), cudaMemcpyHostToDevice,
                                       sl.st);
      if (ce == cudaSuccess) {
        k_gather_cols<<<(unsigned)cols, 256, 0, sl.st>>>(sl.refs_d, nk, sl.Rb);
        ce = cudaGetLastError();
      }
      st = ce == cudaSuccess ? run(sl.Rb, nk, cols, sl.Lb) : cuda_fail(ce, "server batch gather");
      if (st == TD_OK) {
        k_scatter_logl<<<(unsigned)ceil_div(cols, 256), 256, 0, sl.st>>>(sl.refs_d, cols, sl.Lb);
        if ((ce = cudaGetLastError()) != cudaSuccess) st = cuda_fail(ce, "server batch scatter");
      }
    }
    if (st != TD_OK) {
      for (int64_t t : sl.tickets) srv->reqs[t].state = 4;
      srv->failed += (int64_t)sl.tickets.size();
      srv->pending_cols -= cols;
      srv->last_err = st;
      srv->cv_done.notify_all();
      continue;
    }
    cudaEventRecord(sl.done, sl.st);
    sl.busy = true;
    sl.seg = pick;
    e.inflight++;
    srv->batches++;
    srv->inflight_order.push_back(slot);
    srv->cv_done.notify_all();
  }
}

static void completion_loop(td_server* srv) {
  cudaSetDevice(srv->device);
  std::unique_lock<std::mutex> lk(srv->mu);
  while (!srv->stop || !srv->inflight_order.empty()) {
    if (srv->inflight_order.empty()) {
      srv->cv_done.wait_for(lk, std::chrono::milliseconds(5));
      continue;
    }
    // poll every in-flight batch (they may finish out of order on different streams)
    bool progressed = false;
    for (size_t k = 0; k < srv->inflight_order.size();) {
      const int slot = srv->inflight_order[k];
      Slot& sl = srv->slots[(size_t)slot];
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) {
        ++k;
        continue;
      }
      // any other error: the batch is lost and its requests fail (no waiter is left hanging)
      const bool ok = (q == cudaSuccess);
      if (!ok) {
        srv->failed += (int64_t)sl.tickets.size();
        srv->last_err = cuda_fail(q, "server batch");
      }
      const Clock::time_point now = Clock::now();
      int64_t cols = 0;
      for (int64_t t : sl.tickets) {
        Request& r = srv->reqs[t];
        if (!ok) {
          r.state = 4;
          cols += r.K;
          continue;
        }
        r.state = 2;
        cols += r.K;
        r.lat_us = std::chrono::duration<double, std::micro>(now - r.t_submit).count();
        srv->lat_us.push_back(r.lat_us);
        if (!srv->any_done) {
          srv->t_first = r.t_submit;
          srv->any_done = true;
        }
      }
      if (ok) {
        srv->t_last = now;
        srv->evals += cols;
      }
      srv->pending_cols -= cols;
      srv->segs[(size_t)sl.seg].inflight--;
      sl.busy = false;
      sl.tickets.clear();
      srv->inflight_order.erase(srv->inflight_order.begin() + (long)k);
      progressed = true;
    }
    if (progressed) {
      srv->cv_done.notify_all();
      srv->cv_sched.notify_all();
    } else {
      // batches in flight: poll again at once (a sleep here costs tens of
      // microseconds of latency per request); this thread spins a core
      lk.unlock();
      std::this_thread::yield();
      lk.lock();
    }
  }
}

}  // namespace td

using namespace td;

extern "C" {

void td_server_config_default(td_server_config* c) {
  if (!c) return;
  memset(c, 0, sizeof *c);
  c->max_batch_cols = 4096;
  c->max_pending_cols = 1 << 20;
  c->resident_bytes_budget = 0;
  c->n_streams = 4;
  c->precision = TD_PREC_AUTO;
  c->max_kept = 32768;
}

td_status td_server_create(const td_server_config* cfg, td_server** out) {
  if (!out) return fail(TD_ERR_INVALID, "out is NULL");
  *out = nullptr;
  td_server* srv = new td_server();
  td_server_config_default(&srv->cfg);
  if (cfg) srv->cfg = *cfg;
  if (srv->cfg.n_streams < 1 || srv->cfg.n_streams > 16 || srv->cfg.max_batch_cols < 1 || srv->cfg.max_kept < 1) {
    delete srv;
    return fail(TD_ERR_INVALID, "bad server configuration");
  }
  cudaGetDevice(&srv->device);
  {
    cudaMemPoolProps pp;
    memset(&pp, 0, sizeof pp);
    pp.allocType = cudaMemAllocationTypePinned;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = srv->device;
    uint64_t keep = UINT64_MAX;   // freed operator memory stays in the pool for the next reload
    if (cudaMemPoolCreate(&srv->pool, &pp) != cudaSuccess ||
        cudaMemPoolSetAttribute(srv->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
      cudaGetLastError();
      if (srv->pool) cudaMemPoolDestroy(srv->pool);
      delete srv;
      return fail(TD_ERR_CUDA, "server memory pool");
    }
  }
  if (srv->cfg.host_spill_bytes > 0) {
    if (cudaMallocHost(&srv->spill, (size_t)srv->cfg.host_spill_bytes) != cudaSuccess) {
      cudaGetLastError();
      srv->spill = nullptr;
      cudaMemPoolDestroy(srv->pool);
      delete srv;
      return fail(TD_ERR_OOM, "pinned host spill pool");
    }
    srv->spill_cap = (size_t)srv->cfg.host_spill_bytes;
  }
  srv->slots.resize((size_t)srv->cfg.n_streams);
  for (Slot& sl : srv->slots) {
    if (scratch_init_shared(sl.scr, srv->cfg.max_kept, srv->cfg.max_batch_cols) != TD_OK ||
        cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&sl.Rb, (size_t)srv->cfg.max_kept * srv->cfg.max_batch_cols * 4) != cudaSuccess ||
        cudaMalloc(&sl.Lb, (size_t)srv->cfg.max_batch_cols * 8) != cudaSuccess ||
        cudaMallocHost(&sl.refs_h, (size_t)srv->cfg.max_batch_cols * sizeof(ColRef)) != cudaSuccess ||
        cudaMalloc(&sl.refs_d, (size_t)srv->cfg.max_batch_cols * sizeof(ColRef)) != cudaSuccess) {
      cudaGetLastError();
      td_server_destroy(srv);
      return fail(TD_ERR_OOM, "server stream buffers");
    }
  }
  srv->sched = std::thread(scheduler_loop, srv);
  srv->compl_thr = std::thread(completion_loop, srv);
  *out = srv;
  return TD_OK;
}

td_status td_server_add_segment(td_server* srv, const double* acf, int64_t n, const uint8_t* mask, int64_t* seg_id) {
  if (!srv || !seg_id) return fail(TD_ERR_INVALID, "NULL argument");
  td_segment* s = nullptr;
  td_status r = td_segment_create(acf, n, mask, nullptr, &s);
  if (r != TD_OK) return r;
  if (s->nk > srv->cfg.max_kept) {
    td_segment_destroy(s);
    return fail(TD_ERR_INVALID, "segment longer than the server's max_kept");
  }
  std::lock_guard<std::mutex> lk(srv->mu);
  SegEntry e;
  e.s = s;
  e.op_bytes = (size_t)op_row_offset(s->nkp / OP_ROWS) * OP_SLICES * OP_ROWS * OP_KB * 2;
  srv->segs.push_back(e);
  *seg_id = (int64_t)srv->segs.size() - 1;
  return TD_OK;
}

td_status td_server_set_budget(td_server* srv, int64_t resident_bytes_budget) {
  if (!srv || resident_bytes_budget < 0) return fail(TD_ERR_INVALID, "bad argument");
  std::lock_guard<std::mutex> lk(srv->mu);
  srv->cfg.resident_bytes_budget = resident_bytes_budget;
  // evict least recently used idle segments now until the new budget holds
  cudaStream_t st = srv->slots[0].st;
  while (resident_bytes_budget > 0 && (int64_t)srv->resident_bytes > resident_bytes_budget) {
    int64_t victim = -1;
    for (size_t i = 0; i < srv->segs.size(); ++i) {
      const SegEntry& c = srv->segs[i];
      if (!c.resident || c.inflight > 0) continue;
      if (victim < 0 || c.last_use < srv->segs[(size_t)victim].last_use) victim = (int64_t)i;
    }
    if (victim < 0) break;   // the rest is busy: later misses evict it
    const td_status r = seg_evict(srv, srv->segs[(size_t)victim], st);
    if (r != TD_OK) return r;
  }
  TD_CUDA(cudaStreamSynchronize(st));
  return TD_OK;
}

td_status td_server_prefetch(td_server* srv, int64_t seg_id) {
  if (!srv) return fail(TD_ERR_INVALID, "NULL server");
  std::lock_guard<std::mutex> lk(srv->mu);
  if (seg_id < 0 || seg_id >= (int64_t)srv->segs.size()) return fail(TD_ERR_INVALID, "bad segment id");
  cudaStream_t st = srv->slots[0].st;
  const int64_t hits = srv->hits, misses = srv->misses, reloads = srv->reloads;
  td_status r = seg_make_resident(srv, seg_id, st);
  srv->hits = hits;       // set-up is not a request: do not count it
  srv->misses = misses;
  srv->reloads = reloads;
  cudaStreamSynchronize(st);
  return r;
}

td_status td_server_submit(td_server* srv, int64_t seg_id, const float* R, int64_t ldr, int64_t K, double* logL,
                           int64_t* ticket) {
  if (!srv || !ticket) return fail(TD_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(srv->mu);
  if (seg_id < 0 || seg_id >= (int64_t)srv->segs.size()) return fail(TD_ERR_INVALID, "bad segment id");
  SegEntry& e = srv->segs[(size_t)seg_id];
  if (K < 1 || K > srv->cfg.max_batch_cols || !R || !logL || ldr < e.s->nk)
    return fail(TD_ERR_INVALID, "bad request");
  if (srv->pending_cols + K > srv->cfg.max_pending_cols) {
    srv->refused++;
    return fail(TD_ERR_BUSY, "admission refused: pending-column capacity reached");
  }
  Request r{srv->next_ticket++, seg_id, R, ldr, K, logL, Clock::now(), 0, -1.0};
  srv->reqs[r.ticket] = r;
  e.queue.push_back(r.ticket);
  srv->pending_cols += K;
  *ticket = r.ticket;
  srv->cv_sched.notify_one();
  return TD_OK;
}

td_status td_server_poll(td_server* srv, int64_t ticket, int* state) {
  if (!srv || !state) return fail(TD_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return fail(TD_ERR_INVALID, "unknown ticket");
  *state = it->second.state;
  return TD_OK;
}

td_status td_server_latency(td_server* srv, int64_t ticket, double* us) {
  if (!srv || !us) return fail(TD_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return fail(TD_ERR_INVALID, "unknown ticket");
  if (it->second.state != 2) return fail(TD_ERR_BUSY, "request not done");
  *us = it->second.lat_us;
  return TD_OK;
}

td_status td_server_wait(td_server* srv, int64_t ticket, int64_t timeout_us) {
  if (!srv) return fail(TD_ERR_INVALID, "NULL server");
  std::unique_lock<std::mutex> lk(srv->mu);
  const Clock::time_point end = Clock::now() + std::chrono::microseconds(timeout_us);
  while (true) {
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return fail(TD_ERR_INVALID, "unknown ticket");
    const int s = it->second.state;
    if (s == 2) return TD_OK;
    if (s == 3) return fail(TD_ERR_INVALID, "request was cancelled");
    if (s == 4) return fail(srv->last_err != TD_OK ? srv->last_err : TD_ERR_CUDA, "request failed");
    if (Clock::now() >= end) return fail(TD_ERR_TIMEOUT, "request not finished within the timeout");
    srv->cv_done.wait_until(lk, std::min(end, Clock::now() + std::chrono::milliseconds(5)));
  }
}

td_status td_server_cancel(td_server* srv, int64_t ticket) {
  if (!srv) return fail(TD_ERR_INVALID, "NULL server");
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return fail(TD_ERR_INVALID, "unknown ticket");
  if (it->second.state != 0) return fail(TD_ERR_BUSY, "request already running or finished");
  it->second.state = 3;
  srv->pending_cols -= it->second.K;
  srv->cv_done.notify_all();
  return TD_OK;
}

td_status td_server_pause(td_server* srv, int paused) {
  if (!srv) return fail(TD_ERR_INVALID, "NULL server");
  std::lock_guard<std::mutex> lk(srv->mu);
  srv->paused = paused != 0;
  srv->cv_sched.notify_all();
  return TD_OK;
}

td_status td_server_drain(td_server* srv, int64_t timeout_us) {
  if (!srv) return fail(TD_ERR_INVALID, "NULL server");
  std::unique_lock<std::mutex> lk(srv->mu);
  const Clock::time_point end = Clock::now() + std::chrono::microseconds(timeout_us);
  while (srv->pending_cols > 0 || !srv->inflight_order.empty()) {
    if (Clock::now() >= end) return fail(TD_ERR_TIMEOUT, "server did not drain within the timeout");
    srv->cv_done.wait_until(lk, std::min(end, Clock::now() + std::chrono::milliseconds(5)));
  }
  return TD_OK;
}

td_status td_server_get_stats(td_server* srv, td_server_stats* out, int reset) {
  if (!srv || !out) return fail(TD_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(srv->mu);
  memset(out, 0, sizeof *out);
  std::vector<double> v = srv->lat_us;
  if (!v.empty()) {
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) { return v[(size_t)std::min<double>((double)v.size() - 1, p * (double)(v.size() - 1) + 0.5)]; };
    out->p50_us = pct(0.50);
    out->p99_us = pct(0.99);
    out->max_us = v.back();
  }
  out->requests_done = (int64_t)srv->lat_us.size();
  out->evals = srv->evals;
  out->batches = srv->batches;
  out->hits = srv->hits;
  out->misses = srv->misses;
  out->evictions = srv->evictions;
  out->refused = srv->refused;
  out->failed = srv->failed;
  out->resident_bytes = (int64_t)srv->resident_bytes;
  out->reloads = srv->reloads;
  if (srv->any_done) {
    const double secs = std::chrono::duration<double>(srv->t_last - srv->t_first).count();
    out->evals_per_s = secs > 0 ? (double)srv->evals / secs : 0.0;
  }
  if (reset) {
    srv->lat_us.clear();
    srv->evals = srv->batches = srv->hits = srv->misses = srv->evictions = srv->refused = srv->failed = 0;
    srv->reloads = 0;
    srv->any_done = false;
  }
  return TD_OK;
}

td_status td_server_replay(td_server* srv, const double* t_submit_s, const int64_t* seg, const float* const* R,
                           const int64_t* ldr, const int64_t* K, double* const* logL, int64_t n, int64_t* tickets) {
  if (!srv || (n > 0 && (!t_submit_s || !seg || !R || !ldr || !K || !logL))) return fail(TD_ERR_INVALID, "NULL argument");
  const Clock::time_point t0 = Clock::now();
  for (int64_t i = 0; i < n; ++i) {
    const Clock::time_point due = t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(t_submit_s[i]));
    while (Clock::now() < due) {
      const auto left = due - Clock::now();
      if (left > std::chrono::microseconds(200)) std::this_thread::sleep_for(left - std::chrono::microseconds(100));
    }
    int64_t t = -1;
    if (td_server_submit(srv, seg[i], R[i], ldr[i], K[i], logL[i], &t) != TD_OK) t = -1;
    if (tickets) tickets[i] = t;
  }
  return TD_OK;
}

void td_server_destroy(td_server* srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv_sched.notify_all();
  srv->cv_done.notify_all();
  if (srv->sched.joinable()) srv->sched.join();
  if (srv->compl_thr.joinable()) srv->compl_thr.join();
  cudaDeviceSynchronize();
  for (Slot& sl : srv->slots) {
    scratch_free(sl.scr);
    if (sl.Rb) cudaFree(sl.Rb);
    if (sl.Lb) cudaFree(sl.Lb);
    if (sl.refs_h) cudaFreeHost(sl.refs_h);
    if (sl.refs_d) cudaFree(sl.refs_d);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.st) cudaStreamDestroy(sl.st);
  }
  for (SegEntry& e : srv->segs) {
    if (e.host_op && !e.host_op_pooled) cudaFreeHost(e.host_op);
    if (e.spilled) cudaEventDestroy(e.spilled);
    if (e.pooled && e.s->op) {   // pool memory goes back to the pool, not through cudaFree
      cudaFreeAsync(e.s->op, 0);
      e.s->op = nullptr;
    }
  }
  cudaDeviceSynchronize();
  for (SegEntry& e : srv->segs) td_segment_destroy(e.s);
  if (srv->pool) cudaMemPoolDestroy(srv->pool);
  if (srv->spill) cudaFreeHost(srv->spill);
  delete srv;
}

}  // extern "C"
