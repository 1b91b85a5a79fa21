// One step of iterative refinement of the whitening solve W = L^{-1} R
// (Sec. III.C: the operator is evaluated in reduced precision; the accuracy
// that loses is won back by a residual formed more accurately than the solve):
//   w~    = L^{-1} r          split product at the caller's precision
//   s     = r - L w~          split product with bf16 slices of L itself,
//                             ten products (exact hi*hi accumulator)
//   delta = L^{-1} s          caller's precision
//   w     = w~ + delta,  chi2 = |w|^2,  then logL as for one pass.
// w~ is rounded to FP32 before the residual is formed, so s is the exact
// residual of the iterate that gets corrected.  s is about as small as the
// first pass's error, and the residual product's own error (about 1e-9 of
// |L| |w~|) is what the corrected w keeps: the result lands near the
// ten-product accuracy whatever the first pass's precision was.
//
// With enough tiles to fill the GPU the three products cover whole rows
// (256- or 128-row tiles, by the one-pass rules) and do the element-wise part
// in their epilogue (write w~, form s from r, add w~ and square).  Otherwise
// they run split-k on 128-row tiles with every row tile leaving its
// accumulator pairs (chunks of at least 64 k-blocks, a length fixed by N'
// alone) and the chunk reduction's modes do it.  A fixed path (TD_PATH_TENSOR*/STREAM*) fixes the shape, so a
// column's result then does not depend on its batch.
//
// Mode 2 (td_options.refine = 2) forms s = r - L w~ to FP64 accuracy instead:
// split products of six exact bf16 slices of L and of w~ on the tensor cores
// (the factor's emulation, emu_gemm.cu), one 128-column chunk of L at a time,
// accumulated in FP64 and rounded to FP32 once (s is small, so its FP32
// rounding costs about 6e-8 of s); the correction delta = L^{-1} s runs with
// at least six products (BF16X3's own bias, ~1e-5 of delta, would otherwise
// remain at ~1e-10 of w).  The refined chi2 then carries the operator's error
// squared, far below FP64 chi2's own summation error of the first pass.
//
// Needs the FP64 factor L to slice (once per factor); segments whose L was
// released, or whose operator came from the Levinson-Durbin route, return
// TD_ERR_UNSUPPORTED.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "emu_gemm.h"

namespace td {

constexpr int REF_BN = 128;        // operator rows per tile
constexpr int REF_MIN_CHUNK = 64;  // k-blocks

template <class T>
static td_status ref_alloc(T** p, size_t count, const char* what) {
  *p = nullptr;
  if (count == 0) return TD_OK;
  if (cudaMalloc((void**)p, count * sizeof(T)) != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(TD_ERR_OOM, std::string("device allocation failed: ") + what);
  }
  return TD_OK;
}

template <class T>
static void ref_free(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

// Whole-row tile rows for the refined products, 0 for the split form: the
// one-pass rules (256-row tiles from two waves of them, 128-row tiles from
// three quarters of a wave with two TMEM accumulator pairs); a fixed path
// fixes the shape.
static int refine_whole_rows(const td_segment* s, int64_t K, int path) {
  if (path == TD_PATH_TENSOR) return 256;
  if (path == TD_PATH_TENSOR128) return 128;
  if (path != TD_PATH_AUTO) return 0;
  const int64_t nc = ceil_div(K, TC_COLS), sms = tc_num_sms();
  if (2 * (s->nkp / 256) * nc >= 3 * sms) return 256;
  if (4 * (s->nkp / 128) * nc >= 3 * sms) return 128;
  return 0;
}

// whole-row descriptors: [0] L^{-1} with nsl slices; [1] mode 1: L's slices
// (four), mode 2: L^{-1} with nsl1 slices (the correction's product)
static td_status refine_whole_maps(td_segment* s, int64_t K, int nsl, int bn, int mode, int nsl1) {
  RefineState& f = s->ref;
  const Scratch& sc = s->scr;
  if (f.whole_K == K && f.whole_nsl == nsl && f.whole_bn == bn && f.whole_rs == sc.rs && f.whole_op == s->op &&
      f.mode == mode && f.nsl1 == nsl1)
    return TD_OK;
  f.whole_K = -1;
  f.K = -1;   // the split lists hold the other mode's descriptors
  f.mode = mode;
  f.nsl1 = nsl1;
  for (int w = 0; w < 2; ++w) {
    TcSegDev& d = f.whole[w];
    memset(&d, 0, sizeof d);
    const int ns = w == 0 ? nsl : (mode == 2 ? nsl1 : OP_SLICES);
    const __nv_bfloat16* op = (w == 0 || mode == 2) ? s->op : f.lop;
    td_status r = encode_seg_maps(s, K, ns, bn, &d, TC_COLS, op);
    if (r != TD_OK) return r;
    d.partials = sc.partials;
    d.nk = (int)s->nk;
    d.K = (int)K;
    d.ldp = (int)sc.capK;
    d.nm = (int)(s->nkp / 64);
    d.logdet = s->logdet;
  }
  f.whole_K = K;
  f.whole_nsl = nsl;
  f.whole_bn = bn;
  f.whole_rs = sc.rs;
  f.whole_op = s->op;
  return TD_OK;
}

static void drop_plan(RefineState& f) {
  ref_free(f.items);
  ref_free(f.units);
  ref_free(f.seg_op);
  f.n_items = f.n_units = 0;
  f.K = -1;
  f.nsl = 0;
  f.rs = f.op = nullptr;
  f.whole_K = -1;
}

struct EmuRefine {          // mode 2: slices of one 128-column chunk of L and of w~
  SliceBuf a, b;
  int64_t cap = 0;
};

static void free_emu(RefineState& f) {
  if (!f.emu) return;
  EmuRefine* m = static_cast<EmuRefine*>(f.emu);
  free_slice_buf(m->a);
  free_slice_buf(m->b);
  delete m;
  f.emu = nullptr;
}

void free_refine_state(td_segment* s) {
  RefineState& f = s->ref;
  drop_plan(f);
  ref_free(f.lop);
  ref_free(f.w32);
  ref_free(f.s32);
  ref_free(f.s64);
  ref_free(f.wpart);
  free_emu(f);
  f.cap = 0;
  f.wpart_elems = 0;
}

// bf16 slices of L (same packing and per-row quanta as the whitening operator)
static td_status build_lop(td_segment* s, cudaStream_t st) {
  if (!s->L)
    return fail(TD_ERR_UNSUPPORTED,
                "refinement needs the FP64 factor L, which this segment released or never formed "
                "(Levinson-Durbin route)");
  RefineState& f = s->ref;
  td_status r = ref_alloc(&f.lop, (size_t)(s->op_blocks * OP_SLICES * OP_ROWS * OP_KB), "slices of L");
  if (r != TD_OK) return r;
  double* qrow = nullptr;
  if ((r = ref_alloc(&qrow, (size_t)s->nkp, "row quanta of L")) != TD_OK) {
    ref_free(f.lop);
    return r;
  }
  cudaError_t e = launch_row_quantum(s->L, s->nkp, s->nk, s->nkp, qrow, st);
  if (e == cudaSuccess) e = launch_op_slices(s->L, s->nkp, s->nk, s->nkp, qrow, f.lop, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(qrow);
  if (e != cudaSuccess) {
    ref_free(f.lop);
    return cuda_fail(e, "slicing L");
  }
  return TD_OK;
}

static td_status refine_plan(td_segment* s, int64_t K, int nsl, int mode, int nsl1, cudaStream_t st) {
  RefineState& f = s->ref;
  const Scratch& sc = s->scr;
  if (f.K == K && f.nsl == nsl && f.rs == sc.rs && f.op == s->op && f.mode == mode && f.nsl1 == nsl1) return TD_OK;
  cudaStreamSynchronize(st);   // the old lists may still be read on this stream
  drop_plan(f);
  const int S = std::max(split_chunk(s->nk, s->nkp, REF_BN), REF_MIN_CHUNK);
  std::vector<TcItem> items;
  std::vector<SplitUnit> units;
  int n_slots = 0;
  plan_split_segment(0, s->nk, s->nkp, K, REF_BN, S, items, units, n_slots, true);
  sort_items(items);
  td_status r;
  const int64_t need = (int64_t)n_slots * TC_COLS * REF_BN;
  if (need > f.wpart_elems) {
    ref_free(f.wpart);
    f.wpart_elems = 0;
    if ((r = ref_alloc(&f.wpart, (size_t)need, "refinement accumulators")) != TD_OK) return r;
    f.wpart_elems = need;
  }
  TcSegDev seg[2];
  memset(seg, 0, sizeof seg);
  const int a_rows = (int)std::min<int64_t>(TC_COLS, round_up(K, 8));
  for (int w = 0; w < 2; ++w) {
    const int ns = w == 0 ? nsl : (mode == 2 ? nsl1 : OP_SLICES);
    const __nv_bfloat16* op = (w == 0 || mode == 2) ? s->op : f.lop;
    if ((r = encode_seg_maps(s, K, ns, REF_BN, &seg[w], a_rows, op)) != TD_OK) return r;
    seg[w].partials = sc.partials;
    seg[w].wpart = f.wpart;
    seg[w].nk = (int)s->nk;
    seg[w].K = (int)K;
    seg[w].ldp = (int)sc.capK;
    seg[w].nm = (int)(s->nkp / 64);
    seg[w].logdet = s->logdet;
  }
  if ((r = ref_alloc(&f.items, items.size(), "refinement work items")) != TD_OK ||
      (r = ref_alloc(&f.units, units.size(), "refinement units")) != TD_OK ||
      (r = ref_alloc(&f.seg_op, 2, "refinement descriptors")) != TD_OK) {
    drop_plan(f);
    return r;
  }
  TD_CUDA(cudaMemcpy(f.items, items.data(), items.size() * sizeof(TcItem), cudaMemcpyHostToDevice));
  TD_CUDA(cudaMemcpy(f.units, units.data(), units.size() * sizeof(SplitUnit), cudaMemcpyHostToDevice));
  TD_CUDA(cudaMemcpy(f.seg_op, seg, sizeof seg, cudaMemcpyHostToDevice));
  f.n_items = (int)items.size();
  f.n_units = (int)units.size();
  f.K = K;
  f.nsl = nsl;
  f.whole_K = -1;   // the whole-row descriptors may hold the other mode's
  f.mode = mode;
  f.nsl1 = nsl1;
  f.rs = sc.rs;
  f.op = s->op;
  return TD_OK;
}

// s64 = r (kept rows, FP64), zero beyond K columns and N' rows
__global__ void k_s64_init(const float* __restrict__ R, int64_t ldr, int64_t nk, int64_t nkp, int64_t K, int64_t Kp,
                           double* __restrict__ s64) {
  const int64_t n = nkp * Kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % nkp, k = e / nkp;
    s64[e] = (i < nk && k < K) ? (double)R[i + k * ldr] : 0.0;
  }
}

// s32 = fl32(s64)
__global__ void k_s32_from_s64(const double* __restrict__ s64, int64_t n, float* __restrict__ s32) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    s32[e] = __double2float_rn(s64[e]);
}

// s = r - L w~ to FP64 accuracy (mode 2): for each 128-column chunk c of L,
// the rows of L at and below the chunk's diagonal block and the columns of w~
// over the chunk's 128 rows become six exact bf16 slices, and their split
// product is subtracted from s64 (FP64) on the tensor cores.
static td_status refine_residual_fp64(td_segment* s, const float* R, int64_t ldr, int64_t K, int64_t lim,
                                      cudaStream_t st) {
  RefineState& f = s->ref;
  const int64_t nkp = s->nkp, nk = s->nk, Kp = round_up(K, 64);
  td_status r;
  EmuRefine* m = static_cast<EmuRefine*>(f.emu);
  if (!m) {
    m = new EmuRefine();
    f.emu = m;
    if ((r = slice_buf(m->a, (int)nkp, EMU_SLICES)) != TD_OK) return r;
  }
  if (m->cap < f.cap) {
    cudaStreamSynchronize(st);
    free_slice_buf(m->b);
    ref_free(f.s64);
    m->cap = 0;
    if ((r = slice_buf(m->b, (int)f.cap, EMU_SLICES)) != TD_OK ||
        (r = ref_alloc(&f.s64, (size_t)(f.cap * nkp), "FP64 refinement residual")) != TD_OK)
      return r;
    m->cap = f.cap;
  }
  const unsigned grid = (unsigned)std::min<int64_t>(4096, ceil_div(nkp * Kp, 256));
  k_s64_init<<<grid, 256, 0, st>>>(R, ldr, nk, nkp, K, Kp, f.s64);
  TD_CUDA(cudaGetLastError());
  const int64_t ld = nkp;
  for (int64_t c = 0; c * EK < nk; ++c) {
    const int64_t c0 = c * EK, rows = nkp - c0;
    EmuSplitParams S{};
    add_split_job(S, s->L + c0 * (1 + ld), 1, ld, (int)rows, m->a, EMU_SLICES, false, -1, true, (int)(nk - c0));
    add_split_job(S, f.w32 + c0, ld, 1, (int)Kp, m->b, EMU_SLICES, true, (int)K, false, (int)(nk - c0));
    TD_CUDA(launch_emu_split(S, st));
    EmuParams G{};
    add_product(G, m->a, m->b, f.s64 + c0, ld, -1.0, 1.0, (int)(rows / EK), (int)(Kp / 64), false);
    TD_CUDA(launch_emu_gemm(G, EMU_SLICES, s->status, lim, st));
  }
  k_s32_from_s64<<<grid, 256, 0, st>>>(f.s64, nkp * K, f.s32);
  TD_CUDA(cudaGetLastError());
  return TD_OK;
}

td_status refine_batch(td_segment* s, const float* R, int64_t ldr, int64_t K, double* logL, double* chi2, int nsl,
                       int mode, int path, int64_t wait_limit_ns, cudaStream_t st) {
  RefineState& f = s->ref;
  Scratch& sc = s->scr;
  td_status r;
  if (!s->L)
    return fail(TD_ERR_UNSUPPORTED,
                "refinement needs the FP64 factor L, which this segment released or never formed "
                "(Levinson-Durbin route)");
  if (mode == 1 && !f.lop && (r = build_lop(s, st)) != TD_OK) return r;
  const int nsl1 = mode == 2 ? std::max(nsl, 3) : OP_SLICES;   // slices of the second product
  if (sc.capK > f.cap) {
    cudaStreamSynchronize(st);
    ref_free(f.w32);
    ref_free(f.s32);
    f.cap = 0;
    if ((r = ref_alloc(&f.w32, (size_t)(sc.capK * s->nkp), "first iterate")) != TD_OK ||
        (r = ref_alloc(&f.s32, (size_t)(sc.capK * s->nkp), "refinement residual")) != TD_OK)
      return r;
    f.cap = sc.capK;
  }
  const int64_t ld = s->nkp;
  const int ncorr = mode == 2 ? nsl1 : nsl;   // slices of the correction delta = L^{-1} s
  if (const int bn = refine_whole_rows(s, K, path)) {
    if ((r = refine_whole_maps(s, K, nsl, bn, mode, nsl1)) != TD_OK) return r;
    const int nc = (int)ceil_div(K, TC_COLS), nkb_max = (int)ceil_div(s->nk, OP_KB);
    RefineIO io;
    io.out = f.w32;
    io.ldo = ld;
    TD_CUDA(launch_r_slices(R, ldr, s->nk, K, s->nkp8, sc.capK, sc.rs, nsl, st));
    TD_CUDA(launch_tc_single_ew(f.whole[0], bn, 3, nc, nkb_max, nsl, io, s->status, wait_limit_ns, st));
    if (mode == 2) {
      if ((r = refine_residual_fp64(s, R, ldr, K, wait_limit_ns, st)) != TD_OK) return r;
    } else {
      io = RefineIO();
      io.in = R;
      io.ldi = ldr;
      io.out = f.s32;
      io.ldo = ld;
      TD_CUDA(launch_r_slices(f.w32, ld, s->nk, K, s->nkp8, sc.capK, sc.rs, OP_SLICES, st));
      TD_CUDA(launch_tc_single_ew(f.whole[1], bn, 4, nc, nkb_max, OP_SLICES, io, s->status, wait_limit_ns, st));
    }
    io = RefineIO();
    io.in = f.w32;
    io.ldi = ld;
    TD_CUDA(launch_r_slices(f.s32, ld, s->nk, K, s->nkp8, sc.capK, sc.rs, ncorr, st));
    TD_CUDA(launch_tc_single_ew(f.whole[mode == 2 ? 1 : 0], bn, 5, nc, nkb_max, ncorr, io, s->status, wait_limit_ns,
                                st));
    TD_CUDA(launch_finalize(sc.partials, sc.capK, (int)(s->nkp / 64), K, s->logdet, s->nk, logL, chi2, st));
    s->prof_kernels += 7;
    return TD_OK;
  }
  if ((r = refine_plan(s, K, nsl, mode, nsl1, st)) != TD_OK) return r;
  const TcSegDev* seg_linv = f.seg_op;
  const TcSegDev* seg_l = f.seg_op + 1;   // mode 2: L^{-1} with nsl1 slices
  // w~ = L^{-1} r, rounded to FP32
  TD_CUDA(launch_r_slices(R, ldr, s->nk, K, s->nkp8, sc.capK, sc.rs, nsl, st));
  TD_CUDA(launch_tc_cdo(f.items, f.n_items, seg_linv, nsl, REF_BN, true, s->status, wait_limit_ns, st));
  RefineIO io;
  io.out = f.w32;
  io.ldo = ld;
  TD_CUDA(launch_split_reduce(f.units, f.n_units, seg_linv, REF_BN, st, K, RED_WRITE, io));
  // s = r - L w~
  if (mode == 2) {
    if ((r = refine_residual_fp64(s, R, ldr, K, wait_limit_ns, st)) != TD_OK) return r;
  } else {
    TD_CUDA(launch_r_slices(f.w32, ld, s->nk, K, s->nkp8, sc.capK, sc.rs, OP_SLICES, st));
    TD_CUDA(launch_tc_cdo(f.items, f.n_items, seg_l, OP_SLICES, REF_BN, true, s->status, wait_limit_ns, st));
    io = RefineIO();
    io.in = R;
    io.ldi = ldr;
    io.out = f.s32;
    io.ldo = ld;
    TD_CUDA(launch_split_reduce(f.units, f.n_units, seg_l, REF_BN, st, K, RED_RESID, io));
  }
  // delta = L^{-1} s; chi2 of w~ + delta
  const TcSegDev* seg_corr = mode == 2 ? seg_l : seg_linv;
  TD_CUDA(launch_r_slices(f.s32, ld, s->nk, K, s->nkp8, sc.capK, sc.rs, ncorr, st));
  TD_CUDA(launch_tc_cdo(f.items, f.n_items, seg_corr, ncorr, REF_BN, true, s->status, wait_limit_ns, st));
  io = RefineIO();
  io.in = f.w32;
  io.ldi = ld;
  TD_CUDA(launch_split_reduce(f.units, f.n_units, seg_corr, REF_BN, st, K, RED_FINAL, io));
  TD_CUDA(launch_finalize(sc.partials, sc.capK, (int)(s->nkp / 64), K, s->logdet, s->nk, logL, chi2, st));
  s->prof_kernels += 10;
  return TD_OK;
}

}  // namespace td
