// Host-side internals of libtd: the segment object, scratch, kernel launchers.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/td.h"
#include "td_common.cuh"

namespace td {

constexpr int FT = 64;          // FP64 tile (factor, FP64 forward substitution)
constexpr int OP_ROWS = 256;    // operator row tile (tensor-core N)
constexpr int OP_KB = 32;       // operator k-block (64 B of bf16)
constexpr int TC_COLS = 128;    // residual columns per tensor-core tile (MMA M)
constexpr int OP_SLICES = 4;    // bf16 slices per operand element (fixed-point hi + 3 floating)
constexpr double LOG2PI = 1.8378770664093454836;   // log(2 pi), the constant of logL
constexpr int64_t TD_MAX_K = (int64_t)1 << 30;     // columns per batch (tile and column indices stay in int)

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
inline int64_t ceil_div(int64_t x, int64_t m) { return (x + m - 1) / m; }

// offset (in 256x32 blocks) of operator row tile m in the packed lower triangle
inline int64_t op_row_offset(int64_t m) { return (OP_ROWS / OP_KB) * m * (m + 1) / 2; }

struct TcItem {      // one tensor-core work item
  int seg;           // index into the launch's segment table
  int m;             // W row tile (BN rows)
  int c;             // residual column tile (128 columns)
  int nkb;           // k-blocks of 32 to accumulate
  int kb0;           // first k-block
  int slot;          // split mode: accumulator-pair slot this item writes
  int unit;          // split mode: index of the SplitUnit the chunk belongs to
};

struct SplitUnit {   // one (segment, row tile, column tile) whose chunks are reduced together
  int seg;
  int m;
  int c;
  int slot0;         // first slot; the unit's chunks are slot0 .. slot0 + nchunk - 1
  int nchunk;
  int pad;
};

struct TcSegDev {    // per-segment launch data (device-resident)
  CUtensorMap mapA;  // residual slices  (j: N', k: K, slice: 4)
  CUtensorMap mapB;  // operator slices  (32, 256, blocks*4)
  double* partials;  // [n_row_tiles][ldp]
  int nk;
  int K;
  int ldp;
  int nm;            // operator row tiles
  double logdet;
  double* logL;
  double* chi2;
  float2* wpart;     // split mode: accumulator pairs [slot][128 columns][BN rows]
  int a_rows;        // rows of the residual box (<= 128); the rest of each A stage stays zero
  int pad;
};
static_assert(sizeof(CUtensorMap) == 128, "tensor map size");

struct SplitPlan {           // device work lists for one batch width (split mode)
  const void* seg = nullptr;  // the segment it was built for (a scratch may serve several)
  int64_t K = -1;
  int nsl = 0;
  int bn = 0;
  int S = 0;
  TcItem* items = nullptr;
  int n_items = 0;
  SplitUnit* units = nullptr;
  int n_units = 0;
  int n_slots = 0;
  TcSegDev* segdev = nullptr;
  int* counters = nullptr;    // small-batch plans: arrival counts (n_counters, see SmallFinal)
  int n_counters = 0;
  const void* op = nullptr;   // operator the tensor maps in segdev were encoded for
  double logdet = 0.0;        // and the log det copied into it
  uint64_t last_use = 0;
  TcSegDev host_seg;          // host copy of *segdev
  int map_bn = 0;             // operator tile rows its operator map was encoded with
};

struct Scratch {
  int64_t capK = 0;          // columns the buffers hold
  __nv_bfloat16* rs = nullptr;  // residual slices [4][capK][nkp8]
  double* partials = nullptr;   // chi2 partials [row groups][capK] (layout per path)
  double* w64 = nullptr;        // FP64 W for the plain path [nkp][capK]
  float2* wpart = nullptr;      // split-mode accumulator pairs
  int64_t wpart_slots = 0;
  std::vector<float2*> wpart_old;   // outgrown accumulator buffers, still named by older plans
  std::vector<SplitPlan> plans;
  uint64_t use_clock = 0;
  // a scratch shared by several segments (a server stream's): buffers sized
  // once for max_kept samples and capK columns, never regrown
  bool shared = false;
  int64_t rs_elems = 0, part_elems = 0;
  size_t max_plans = 24;
};

// one Levinson-Durbin chain (gap-free segment of n samples)
struct LevJob {
  const double* acf;       // device, n lags
  int64_t n;               // samples (gap-free: N' = n)
  double* a0;              // device scratch, n doubles
  double* a1;              // device scratch, n doubles
  double* linv;            // device, row t at linv + t ld, columns 0..t written; nullptr: rows not stored
  int64_t ld;
  double* logdet;          // device, one double
  DevStatus* status;       // NOT_PD pivot
  double* x;               // nullptr, or device n doubles: receives C^{-1} e_1
  double* vhist;           // device scratch, n doubles: the prediction-error variances v_0 .. v_{n-1}
};
cudaError_t launch_levinson_rows(const LevJob* jobs, int njobs, cudaStream_t st);

// Kernel attributes (dynamic shared memory above 48 KB) are per device: true
// while the current device's bit in `done` is clear.  Set the attribute, then
// mark_device_done; setting it twice (two threads at once) is harmless.
inline bool device_needs_setup(const std::atomic<unsigned long long>& done) {
  int dev = 0;
  cudaGetDevice(&dev);
  return !(done.load(std::memory_order_acquire) & (1ull << (dev & 63)));
}
inline void mark_device_done(std::atomic<unsigned long long>& done) {
  int dev = 0;
  cudaGetDevice(&dev);
  done.fetch_or(1ull << (dev & 63), std::memory_order_release);
}

int split_chunk(int64_t nk, int64_t nkp, int bn);
// bf16 slices per operand element for a td_options precision on a segment of
// nk kept samples (TD_PREC_AUTO: 3, or 4 below 512 and above 32768 kept samples)
int nslices_for(int precision, int64_t nk);
void plan_split_segment(int seg, int64_t nk, int64_t nkp, int64_t K, int bn, int S, std::vector<TcItem>& items,
                        std::vector<SplitUnit>& units, int& n_slots, bool all_slots = false, int cols = TC_COLS);
void sort_items(std::vector<TcItem>& items);
void sort_items_by_segment(std::vector<TcItem>& items, int nseg);

}  // namespace td

struct HostStage {            // td_loglike_batch_host: device copies of host column chunks
  float* buf[2] = {nullptr, nullptr};   // double buffer, [cols][nk] each
  int64_t cols = 0;
  double* logL = nullptr;      // device results [cap]
  double* chi2 = nullptr;
  int64_t cap = 0;
  cudaStream_t copy = nullptr;  // host->device copies run here
  cudaEvent_t copied[2] = {nullptr, nullptr}, consumed[2] = {nullptr, nullptr};
};

struct TemplateState {        // td_set_data / td_template_batch
  double* d = nullptr;         // device data vector, N' kept samples
  size_t d_cap = 0;
  float* R = nullptr;          // device [d - h_k | h_k] columns of a batch
  size_t R_cap = 0;
  double* res = nullptr;       // device logL and chi2 of a batch
  size_t res_cap = 0;
  double dd = 0.0;             // <d, d>
  bool has_data = false;
};

struct RefineState {          // td_options.refine
  __nv_bfloat16* lop = nullptr;     // bf16 slices of L, packed like the operator
  float* w32 = nullptr;             // first iterate w~ rounded to FP32, [cap][N'p]
  float* s32 = nullptr;             // residual s = r - L w~ in FP32, [cap][N'p]
  int64_t cap = 0;
  float2* wpart = nullptr;          // accumulator pairs of every row tile
  int64_t wpart_elems = 0;
  // the cached work list (one batch width)
  int64_t K = -1;
  int nsl = 0;
  const void* rs = nullptr;         // residual slices and operator the maps were encoded for
  const void* op = nullptr;
  td::TcItem* items = nullptr;
  int n_items = 0;
  td::SplitUnit* units = nullptr;
  int n_units = 0;
  td::TcSegDev* seg_op = nullptr;   // [0]: L^{-1} slices (nsl), [1]: L slices (4), or L^{-1} (mode 2)
  int mode = 0;                     // refinement mode the cached lists were built for
  int nsl1 = 0;                     // slices of the second product's operator
  double* s64 = nullptr;            // mode 2: FP64 residual r - L w~, [cap][N'p]
  void* emu = nullptr;              // mode 2: operand slice buffers of the residual's split products
  // whole-row descriptors (host copies, passed by value to the kernel)
  td::TcSegDev whole[2];
  int64_t whole_K = -1;
  int whole_nsl = 0;
  int whole_bn = 0;
  const void* whole_rs = nullptr;
  const void* whole_op = nullptr;
};

struct GsState {              // td_gs_prepare / TD_PATH_GSCE (gap-free segments)
  int logm = 0;                 // circulant length M = 2^logm >= 2N
  float2* S1 = nullptr;         // spectra of the two circulant embeddings, bit-reversed order,
  float2* S2 = nullptr;         //   scaled by 1 / (M x_0); [M]
  double x0 = 0.0;              // (C^{-1})_00
  float2* tw = nullptr;         // twiddle shears (-tan(theta/2), sin(theta)), theta = -2 pi j / M, j < M/4
  float2* scr = nullptr;        // per-CTA product buffer of a batch
  int64_t scr_elems = 0;
  double logdet = 0.0;          // from the recursion's prediction-error variances
  bool ready = false;
};

struct td_segment {
  int device = 0;
  int64_t n = 0;          // samples
  int64_t nk = 0;         // kept samples N'
  int64_t nkp = 0;        // N' padded to 256
  int64_t nkp8 = 0;       // N' padded to 8 (row stride of residual slices)
  double* acf = nullptr;          // device [n]
  int32_t* t = nullptr;           // device kept indices [nk]
  double* L = nullptr;            // device FP64 [nkp x nkp] column-major, lower = factor
  double* dinv = nullptr;         // device FP64 [nkp/64][64*64] inverse diagonal tiles
  double* ldpart = nullptr;       // device [nkp/64]
  __nv_bfloat16* op = nullptr;    // device operator slices, packed 256x32 blocks x 4
  int64_t op_blocks = 0;
  td::DevStatus* status = nullptr;  // device
  bool factored = false;
  double logdet = 0.0;
  int64_t pivot = -1;
  td::Scratch scr;
  HostStage hst;
  TemplateState tpl;
  float* gat = nullptr;    // td_loglike_batch_gather: kept rows of a full-length batch [cap][N']
  int64_t gat_cap = 0;     // columns
  RefineState ref;
  GsState gs;
  // instrumentation
  bool prof = false;
  std::vector<cudaEvent_t> ev;   // start/stop pairs
  size_t ev_used = 0;
  int64_t prof_kernels = 0;
};

namespace td {
void free_host_stage(HostStage& h);
void free_template_state(TemplateState& T);
// error plumbing
td_status fail(td_status code, const std::string& msg);
td_status cuda_fail(cudaError_t e, const char* what);
#define TD_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return td::cuda_fail(e_, #call); \
  } while (0)

// kernel launchers (return cudaError_t of the launch)
cudaError_t launch_gather(const double* acf, const int32_t* t, int64_t nk, int64_t nkp, double* A,
                          cudaStream_t st);
cudaError_t launch_potrf_diag(double* A, int64_t ld, int64_t nk, int j, double* dinv, double* ldpart,
                              DevStatus* status, cudaStream_t st);
cudaError_t launch_panel(double* A, int64_t ld, int j, int nt, const double* dinv, cudaStream_t st);
cudaError_t launch_syrk(double* A, int64_t ld, int j, int nt, cudaStream_t st);

// FP64 forward substitution of block row I: W_I = Dinv_I (RHS_I - sum_J L_IJ W_J)
//   rhs32 != nullptr: RHS = float32 R (ldr); else identity (computes L^{-1}).
cudaError_t launch_trsm_f64_row(const double* L, int64_t ld, const double* dinv, int I, const float* rhs32,
                                int64_t ldr, int64_t nk, int64_t ncols, double* W, int64_t ldw,
                                double* partials, int64_t ldp, cudaStream_t st);
// the plain FP64 evaluation: W = L^{-1} R by right-looking 64-row blocks into
// T (N'p x K FP64, leading dimension ldw), chi2 partials per 64 rows
cudaError_t launch_fp64_solve(const double* L, int64_t ld, const double* dinv, const float* R, int64_t ldr,
                              int64_t nk, int64_t nkp, int64_t K, double* T, int64_t ldw, double* partials,
                              int64_t ldp, cudaStream_t st);
cudaError_t launch_finalize(const double* partials, int64_t ldp, int nparts, int64_t K, double logdet,
                            int64_t nk, double* logL, double* chi2, cudaStream_t st);

// Linv element (i, j) at Linv[i + j ld] (column-major) or Linv[i ld + j] (row_major)
cudaError_t launch_row_quantum(const double* Linv, int64_t ld, int64_t nk, int64_t nkp, double* qrow,
                               cudaStream_t st, bool row_major = false);
cudaError_t launch_op_slices(const double* Linv, int64_t ld, int64_t nk, int64_t nkp, const double* qrow,
                             __nv_bfloat16* op, cudaStream_t st, bool row_major = false);
// zero / nzero: ints the launch clears first (the next small-batch kernel's counters).
// The kernel lets a programmatic dependent launch start early.  pdl (K <= 64):
// launched as a programmatic dependent of the preceding kernel; it waits for
// that kernel before it reads R or writes anything.
cudaError_t launch_r_slices(const float* R, int64_t ldr, int64_t nk, int64_t K, int64_t nkp8,
                            int64_t capK, __nv_bfloat16* rs, int nslices, cudaStream_t st, int* zero = nullptr,
                            int nzero = 0, bool pdl = false);

// tensor-core CDO product + chi2 partials (one per 64-row group) over a work list
// pdl: launch as a programmatic dependent of the preceding kernel (which
// must trigger early); off for the grouped path, where it measured slower.
// sched: a device int that is zero when the kernel starts: items are then
// taken in list order as CTAs become free (the dynamic schedule), instead of
// dealt round by round
cudaError_t launch_tc_cdo(const TcItem* items, int n_items, const TcSegDev* segs, int nslices, int bn,
                          bool split, DevStatus* status, int64_t wait_limit_ns, cudaStream_t st, bool pdl = true,
                          int* sched = nullptr);
// partials per 64-row group; max_cols: the widest column tile of the units
// (one CTA per 64 rows and 16 columns).  mode: RED_CHI2, or one of the
// refinement modes (element-wise output or chi2 of in + w, through io).
enum { RED_CHI2 = 0, RED_WRITE = 1, RED_RESID = 2, RED_FINAL = 3 };
struct RefineIO {
  const float* in = nullptr;   // RED_RESID: r; RED_FINAL: w~   ([i + k ldi])
  int64_t ldi = 0;
  float* out = nullptr;        // RED_WRITE, RED_RESID           ([i + k ldo], rows < N'p)
  int64_t ldo = 0;
};
cudaError_t launch_split_reduce(const SplitUnit* units, int n_units, const TcSegDev* segs, int bn, cudaStream_t st,
                                int64_t max_cols = 128, int mode = RED_CHI2, const RefineIO& io = RefineIO());
// Small batches, one segment: the chunk reduction and the final chi2 / logL
// run inside the kernel (the last chunk of a row tile, then the last CTA);
// launched as a programmatic dependent of the residual slicing.
constexpr int SMALL_GROUPS = 64;   // 4-column groups of the widest small batch (256 columns)
// TD_PREC_AUTO: six split products from this many kept samples up to 32768,
// ten outside.  Six products give chi2 to about 2e-8 relative at N' = 8192,
// growing as the rows that carry a column's chi2 get fewer (1.03e-7 measured
// on a gapped N' = 739 segment, 1.15e-7 at N' = 47), so below 2048 the default
// takes ten
constexpr int64_t AUTO_SIX_MIN = 2048;
constexpr int SMALL_FUSED_K = 8;   // small batches up to this width reduce inside the product kernel
struct SmallFinal {
  const SplitUnit* units;
  // zero at launch.  Separate reduction kernel: [SMALL_GROUPS] arrivals per
  // 4-column group.  In-kernel reduction: [n_units] chunk arrivals per split
  // unit, then [1] completed 128-row tiles.
  int* counters;
  int n_units;
  int K;             // columns of this call (the plan may be wider)
  double* logL;
  double* chi2;      // optional
  int slot_cols;     // columns per split slot: max(128, the kernel's column tile)
};
// fin: a single-segment call whose chunk reduction, chi2 and logL the kernel
// does itself (NC <= 64); nullptr: chunk pairs and partials only (a separate
// reduction follows)
cudaError_t launch_tc_small(const TcItem* items, int n_items, const TcSegDev* segs, int nslices, int nc,
                            DevStatus* status, int64_t wait_limit_ns, cudaStream_t st,
                            const SmallFinal* fin = nullptr);
cudaError_t launch_small_reduce(const TcSegDev* segs, const SmallFinal& fin, cudaStream_t st);
// the chunk reduction of a grouped small-orientation launch (nc-column tiles,
// every item a chunk); writes each unit's chi2 partials for k_tc_finalize
cudaError_t launch_small_reduce_grouped(const SplitUnit* units, int n_units, const TcSegDev* segs, int nc,
                                        cudaStream_t st);
cudaError_t launch_tc_single(const TcSegDev& seg, int bn, int nc, int nkb_max, int nslices, DevStatus* status,
                             int64_t wait_limit_ns, cudaStream_t st);
// refinement products over whole bn-row tiles (256 or 128) with an element-wise
// epilogue: mode 3 out = fl32(w), 4 out = fl32(in - w), 5 chi2 partials of in + w
cudaError_t launch_tc_single_ew(const TcSegDev& seg, int bn, int mode, int nc, int nkb_max, int nslices,
                                const RefineIO& io, DevStatus* status, int64_t wait_limit_ns, cudaStream_t st);
int tc_num_sms();
cudaError_t launch_tc_finalize(const TcSegDev* segs, int nseg, int64_t maxK, cudaStream_t st);

cudaError_t launch_bounded_wait_probe(DevStatus* status, int64_t limit_ns, cudaStream_t st);

// 3-D bf16 tensor map with 64-byte swizzle: dims d0 (innermost) .. d2, byte
// strides of dims 1 and 2, box b0 x b1 x b2
td_status encode_3d(CUtensorMap* map, const void* ptr, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t s1_bytes,
                    uint64_t s2_bytes, uint32_t b0, uint32_t b1, uint32_t b2);
// the factor C = L L^T with L^{-1} and the operator slices: blocks of 128 on
// the tensor cores (split products of ns bf16 slices), or the FP64 CUDA-core
// route (64-wide tiles)
td_status factor_tensor(td_segment* s, cudaStream_t st, int ns);
td_status factor_fp64_cores(td_segment* s, cudaStream_t st);
constexpr int EMU_SLICES = 6;   // bf16 slices per FP64 operand value in the tensor-core factor
// shared steps of both routes: allocate L (and the diagonal-tile inverses and
// log det shares), clear the status and gather C_kept into L; afterwards
// check the pivots, sum log det and build the operator slices from the
// column-major L^{-1} (freed by the call)
td_status factor_begin(td_segment* s, cudaStream_t st);
td_status factor_end(td_segment* s, double* linv, cudaStream_t st);
td_status read_status(td_segment* s, cudaStream_t st, DevStatus* out);
td_status read_clock(DevStatus* dst, cudaStream_t st, double* mhz);
td_status reset_status(td_segment* s, cudaStream_t st);

// tensor maps of one segment: residual slices (A, boxes of a_rows columns)
// and an operator's packed slices (B, tiles of bn rows, nsl slices); op =
// nullptr takes the segment's whitening operator
td_status encode_seg_maps(td_segment* s, int64_t K, int nsl, int bn, TcSegDev* out, int a_rows = TC_COLS,
                          const __nv_bfloat16* op = nullptr, const Scratch* sc = nullptr);
// td_loglike_batch / td_reserve with an explicit scratch (a server stream's
// shared one); the segment's own scratch otherwise
td_status loglike_batch_with(td_segment* s, Scratch& sc, const float* R, int64_t ldr, int64_t K, double* logL,
                             const td_options* opt, double* chi2, cudaStream_t st);
td_status reserve_with(td_segment* s, Scratch& sc, int64_t K, const td_options* opt);
td_status scratch_init_shared(Scratch& sc, int64_t max_kept, int64_t maxK);
void scratch_free(Scratch& sc);
// one refinement step (td_options.refine), launched on st
td_status refine_batch(td_segment* s, const float* R, int64_t ldr, int64_t K, double* logL, double* chi2, int nsl, int mode,
                       int path, int64_t wait_limit_ns, cudaStream_t st);
void free_refine_state(td_segment* s);
// Gohberg-Semencul path (TD_PATH_GSCE)
td_status gs_batch(td_segment* s, const float* R, int64_t ldr, int64_t K, double* logL, double* chi2,
                   cudaStream_t st);
void free_gs_state(td_segment* s);
bool gs_supported(const td_segment* s);             // gap-free, 1024 <= N <= 32768
bool gs_preferred(const td_segment* s, int64_t K);  // TD_PATH_AUTO's choice when both forms are there

}  // namespace td
