// Tensor-core whitening W = L^{-1} R with split bf16 products and the fused
// chi2 epilogue (Sec. II.A, W = L^{-1} and Eq. eq:td_like_whitened; Sec.
// III.A, the cached-operator "CDO" evaluation; Sec. III.C, precision: the
// operator is precomputed in FP64 and evaluated in lower precision).
//
// The product is computed transposed, W^T = R^T (L^{-1})^T, so that each
// TMEM lane holds one residual column and the chi2 sum over rows happens in
// one thread's registers with no cross-thread reduction:
//   MMA M = 128 residual columns  (A = R^T slices, K-major),
//   MMA N = BN rows of W, BN = 256, 128 or 64
//                                 (B = L^{-1} slices, K-major),
//   reduction over the kept samples j in k-blocks of 32 (64-byte swizzle).
// Each operand is held as bf16 slices x = x0 + x1 + x2 (+ x3) with x0 a
// fixed-point hi slice (integer multiple, |.| <= 255, of a per-row /
// per-column power-of-two quantum) and x1.. floating slices of the remainder.
// The tensor core accumulates in FP32 with truncation, which biases every sum
// that is not exactly representable; so the hi*hi products, whose partial sums
// are exact integer multiples of one quantum, go to their own accumulator
// (exact), and the products x_a * y_b with 1 <= a + b <= NSL - 1 (five for
// three slices, nine for four) go, smallest first, to a second accumulator
// whose magnitude (and so its truncation error) is small.  The epilogue adds
// the two in double-float and emits one FP64 chi2 partial per 64-row group.
//
// A given (tile shape, k-range split) fixes every rounding, so a column's
// result does not depend on the other columns of its batch; chi2 partials
// are always per 64-row group.
//
// Work: one output tile = (segment, row tile m, column tile c); the row tile
// needs the k-blocks up to its diagonal (the lower triangle).  Tiles are
// dealt to the persistent CTAs in snake order (one segment: largest first),
// or, for a list with a work counter, taken in list order as CTAs become free
// (see the item-order note in the kernel).
//
// Warp roles (192 threads, one CTA per SM):
//   warp 0 lane 0 : TMA producer, STAGES-deep ring of (A, B) slice stages
//   warp 1        : TMEM allocator; lane 0 issues tcgen05.mma
//   warps 2..5    : epilogue; TMEM -> registers, exact squares, compensated
//                   sums, FP64 partials
// TMEM holds NBUF pairs of accumulators (one pair for BN = 256, two for
// BN = 128 and 64 so the epilogue of one tile overlaps the MMAs of the next).  Every
// wait is bounded (wait_limit_ns).
#include <algorithm>

#include "td_internal.h"

namespace td {
namespace tc {
constexpr int BM = TC_COLS;      // 128 residual columns
constexpr int BK = OP_KB;        // 32
constexpr int A_SLICE = BM * BK * 2;   // 8 KB
constexpr int BAR_BYTES = 512;
constexpr int NRING = 8;         // item-index ring of the dynamic schedule
constexpr int THREADS = 192;
template <int NSL, int BN> struct Cfg {
  static constexpr int B_SLICE = BN * BK * 2;
  static constexpr int A_STAGE = NSL * A_SLICE;
  static constexpr int B_STAGE = NSL * B_SLICE;
  static constexpr int STAGE = A_STAGE + B_STAGE;
  static constexpr int STAGES = (220 * 1024) / STAGE > 8 ? 8 : (220 * 1024) / STAGE;
  static constexpr int SMEM = STAGES * STAGE + BAR_BYTES + 1024;
  static constexpr int NBUF = (4 * BN <= 512) ? 2 : 1;           // accumulator pairs in TMEM
  static constexpr uint32_t TMEM_COLS = (NBUF * 2 * BN <= 256) ? 256 : 512;
  static constexpr int GROUPS = BN / 64;                          // 64-row chi2 groups per tile
};
}  // namespace tc

struct TcSingle {           // single-segment launch: item list is implicit
  TcSegDev seg;
  int nm;                   // row tiles of BN rows
  int nc;                   // column tiles
  int nkb_max;              // k-blocks available (ceil(N'/32))
  int* sched;               // list modes: work counter of the dynamic schedule (zero at launch), or null
  RefineIO io;              // element-wise modes 3..5: element (i, k) of in / out at [i + k ld]
};

template <int BN>
__device__ __forceinline__ TcItem single_item(const TcSingle& p, int idx) {
  TcItem it;
  it.seg = 0;
  it.m = p.nm - 1 - idx / p.nc;
  it.c = idx % p.nc;
  const int nkb = (BN / tc::BK) * (it.m + 1);
  it.nkb = nkb < p.nkb_max ? nkb : p.nkb_max;
  it.kb0 = 0;
  it.slot = -1;
  return it;
}

// MODE 0: one segment, implicit item list, chi2 partials in the epilogue
// MODE 1: explicit item list (many segments), chi2 partials in the epilogue
// MODE 2: explicit item list whose items may cover part of a row's k-range
//         (slot >= 0): the epilogue stores the accumulator pair and
//         k_split_reduce finishes; items with slot < 0 cover whole rows
// MODE 3..5: one segment, whole rows, the refinement step's element-wise
//         epilogues (w = hi + corrections of each element):
//         3 out = fl32(w);  4 out = fl32(in - w);  5 chi2 partials of in + w
template <int NSL, int BN, int MODE>
__global__ void __launch_bounds__(tc::THREADS, 1)
    k_tc_cdo(const __grid_constant__ TcSingle single, const TcItem* __restrict__ items, int n_items,
             const TcSegDev* __restrict__ segs, DevStatus* status, uint64_t limit_ns) {
  using namespace tc;
  using C = Cfg<NSL, BN>;
  constexpr int A_STAGE = C::A_STAGE;
  constexpr int B_SLICE = C::B_SLICE;
  constexpr int STAGE = C::STAGE;
  constexpr int STAGES = C::STAGES;
  constexpr int NBUF = C::NBUF;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + NBUF;
  uint64_t* fin = tempty + NBUF;
  uint64_t* ring_full = fin + 1;          // NRING: item index published
  uint64_t* ring_empty = ring_full + NRING;   // NRING: read by the MMA thread and the four epilogue warps
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(ring_empty + NRING);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* ring = abort_flag + 1;    // NRING item indices (-1: no more work)

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the kernels after this one may be scheduled now; they wait for this grid
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
    }
    mbar_init(fin, 1);
    for (int i = 0; i < NRING; ++i) {
      mbar_init(&ring_full[i], 1);
      mbar_init(&ring_empty[i], 5);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, C::TMEM_COLS);
    tmem_relinquish();
  }
  // residual rows the TMA box does not cover must read as zero in every stage
  // (a narrow box is only used when every item of the launch has it)
  constexpr bool GROUPED = MODE == 1 || MODE == 2;
  if ((GROUPED ? segs[0].a_rows : single.seg.a_rows) < BM) {
    for (int s = 0; s < STAGES; ++s) {
      uint4* a = reinterpret_cast<uint4*>(smem + s * STAGE);
      for (int i = threadIdx.x; i < A_STAGE / 16; i += blockDim.x) a[i] = make_uint4(0, 0, 0, 0);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the tensor core
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int G = gridDim.x, b = blockIdx.x;
  const int n_total = GROUPED ? n_items : single.nm * single.nc;
  // Item order.  Static: round r of CTA b takes item r G + b (G - 1 - b on odd
  // rounds).  Dynamic (list modes with a work counter): the producer takes the
  // next item from the counter when it starts one and publishes its index to
  // the MMA thread and the epilogue through a ring in shared memory.  Items
  // that read the same operator tile (the column tiles of one row tile) sit
  // next to each other in the list, so the dynamic order starts them within
  // microseconds of each other and all but the first read its k-blocks from
  // L2; dealt statically, CTAs reach the same round at different times and
  // each would stream the tile from HBM again.
  const bool dyn = GROUPED && single.sched != nullptr;
  // consumers: the next item index (-1: none), false when the wait ran out
  auto ring_take = [&](int& j, int& idx) -> bool {
    const int slot = j % NRING;
    if (!mbar_wait(&ring_full[slot], (uint32_t)(j / NRING) & 1u, limit_ns)) return false;
    idx = ring[slot];
    ++j;
    return true;
  };

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------ TMA producer
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued_mask = 0, issued_phase = 0;
      if (!GROUPED) {
        prefetch_tmap(&single.seg.mapA);
        prefetch_tmap(&single.seg.mapB);
      }
      // launched as a programmatic dependent of the residual slicing: the first
      // STAGES operator tiles are requested before the wait for the slices
      bool dep = false;
      int pend_n = 0;
      int pend_stage[STAGES], pend_kb[STAGES], pend_c[STAGES];
      const TcSegDev* pend_sd[STAGES];
      auto flush = [&]() {
        asm volatile("griddepcontrol.wait;" ::: "memory");
        dep = true;
        for (int i = 0; i < pend_n; ++i) {
          uint8_t* sa = smem + pend_stage[i] * STAGE;
#pragma unroll
          for (int sl = 0; sl < NSL; ++sl)
            tma_load_3d(sa + sl * A_SLICE, &pend_sd[i]->mapA, &full[pend_stage[i]], pend_kb[i] * BK,
                        pend_c[i] * BM, sl);
        }
        pend_n = 0;
      };
      int jpub = 0;
      bool ended = false;   // the end marker is in the ring
      auto publish = [&](int idx) -> bool {
        const int slot = jpub % NRING;
        if (!mbar_wait(&ring_empty[slot], ((uint32_t)(jpub / NRING) & 1u) ^ 1u, limit_ns)) return false;
        ring[slot] = idx;
        mbar_arrive(&ring_full[slot]);
        ++jpub;
        return true;
      };
      for (int r = 0;; ++r) {
        int idx;
        if (dyn) {
          idx = *abort_flag ? -1 : atomicAdd(single.sched, 1);
          if (idx >= n_total) idx = -1;
          if (!publish(idx)) {
            set_status(status, ST_TIMEOUT, 11);
            *abort_flag = 1;
            ended = true;   // the consumers' own bounded waits end them
            break;
          }
          if (idx < 0) {
            ended = true;
            break;
          }
        } else {
          if ((int64_t)r * G >= n_total || *abort_flag) break;
          idx = r * G + ((r & 1) ? (G - 1 - b) : b);
          if (idx >= n_total) continue;
        }
        const TcItem it = GROUPED ? items[idx] : single_item<BN>(single, idx);
        const TcSegDev* sd = GROUPED ? &segs[it.seg] : &single.seg;
        const int row0 = it.m * BN;                      // first W row of the tile
        const int M256 = row0 / OP_ROWS;                 // 256-row operator tile holding it
        const int yoff = row0 - M256 * OP_ROWS;          // row offset inside the 256-row block
        const int blk0 = (OP_ROWS / BK) * M256 * (M256 + 1) / 2;
        bool ok = true;
        for (int kb = it.kb0; kb < it.kb0 + it.nkb; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, limit_ns)) {
            set_status(status, ST_TIMEOUT, 10);
            *abort_flag = 1;
            ok = false;
            break;
          }
          uint8_t* sa = smem + stage * STAGE;
          uint8_t* sb = sa + A_STAGE;
          mbar_arrive_expect_tx(&full[stage], (uint32_t)(NSL * (sd->a_rows * BK * 2 + B_SLICE)));
          tma_load_3d(sb, &sd->mapB, &full[stage], 0, yoff, (blk0 + kb) * OP_SLICES);
          if (dep) {
#pragma unroll
            for (int sl = 0; sl < NSL; ++sl)   // one box per slice: each slice owns an 8 KB region
              tma_load_3d(sa + sl * A_SLICE, &sd->mapA, &full[stage], kb * BK, it.c * BM, sl);
          } else {
            pend_stage[pend_n] = stage;
            pend_kb[pend_n] = kb;
            pend_c[pend_n] = it.c;
            pend_sd[pend_n] = sd;
            if (++pend_n == STAGES) flush();   // every stage is in use: nothing more can be issued first
          }
          issued_mask |= 1u << stage;
          issued_phase = (issued_phase & ~(1u << stage)) | (phase << stage);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
      }
      if (dyn && !ended) publish(-1);   // after an abort: let the consumers stop
      if (!dep) flush();
      // every issued copy must land before the CTA may exit
      for (int s = 0; s < STAGES; ++s)
        if (issued_mask & (1u << s)) mbar_wait(&full[s], (issued_phase >> s) & 1u, limit_ns);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------ MMA issuer
      constexpr uint32_t idesc = idesc_bf16_f32(BM, BN);
      int stage = 0;
      uint32_t phase = 0;
      int tl = 0;
      const uint64_t g0 = globaltimer_ns();
      const long long c0 = clock64();
      int jtake = 0;
      for (int r = 0;; ++r) {
        int idx;
        if (dyn) {
          const int slot = jtake % NRING;
          if (!ring_take(jtake, idx)) {
            set_status(status, ST_TIMEOUT, 22);
            *abort_flag = 1;
            break;
          }
          mbar_arrive(&ring_empty[slot]);
          if (idx < 0) break;
        } else {
          if ((int64_t)r * G >= n_total || *abort_flag) break;
          idx = r * G + ((r & 1) ? (G - 1 - b) : b);
          if (idx >= n_total) continue;
        }
        const TcItem it = GROUPED ? items[idx] : single_item<BN>(single, idx);
        const int buf = tl % NBUF;
        const uint32_t use = (uint32_t)(tl / NBUF);
        if (!mbar_wait(&tempty[buf], (use & 1u) ^ 1u, limit_ns)) {
          set_status(status, ST_TIMEOUT, 20);
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t d_hi = tmem_base + (uint32_t)(buf * 2 * BN);   // hi*hi (exact)
        const uint32_t d_lo = d_hi + (uint32_t)BN;                      // corrections
        bool ok = true;
        for (int kb = it.kb0; kb < it.kb0 + it.nkb; ++kb) {
          if (!mbar_wait(&full[stage], phase, limit_ns)) {
            set_status(status, ST_TIMEOUT, 21);
            *abort_flag = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + stage * STAGE);
          const uint32_t sb = sa + A_STAGE;
          // residual slices (A) against operator slices (B), grouped by the
          // residual slice so the collector buffer reuses it
#pragma unroll
          for (int kk = 0; kk < 2; ++kk)
            split_products_step<NSL>(d_hi, d_lo, sa, A_SLICE, sb, B_SLICE, kk * 32, idesc,
                                     (kb > it.kb0 || kk > 0) ? 1u : 0u);
          tc_commit(&empty[stage]);   // frees this smem stage once these MMAs retire
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        tc_commit(&tfull[buf]);       // accumulators ready for the epilogue
        ++tl;
      }
      tc_commit(fin);                 // all MMAs issued by this thread retired
      mbar_wait(fin, 0, limit_ns);
      if (tl > 0) {   // the clock this SM ran at over its share of the work
        const long long c1 = clock64();
        const uint64_t g1 = globaltimer_ns();
        atomicAdd(&status->mma_cycles, (unsigned long long)(c1 - c0));
        atomicAdd(&status->mma_ns, (unsigned long long)(g1 - g0));
      }
    }
  } else {
    // -------------------------------------------------- epilogue (warps 2..5)
    const int q = warp & 3;   // TMEM lane quarter this warp may access
    int tl = 0;
    int jtake = 0;
    for (int r = 0;; ++r) {
      int idx;
      if (dyn) {
        const int slot = jtake % NRING;
        if (!ring_take(jtake, idx)) {
          if (lane == 0) set_status(status, ST_TIMEOUT, 32);
          *abort_flag = 1;
          break;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&ring_empty[slot]);
        if (idx < 0) break;
      } else {
        if ((int64_t)r * G >= n_total || *abort_flag) break;
        idx = r * G + ((r & 1) ? (G - 1 - b) : b);
        if (idx >= n_total) continue;
      }
      const TcItem it = GROUPED ? items[idx] : single_item<BN>(single, idx);
      const TcSegDev* sd = GROUPED ? &segs[it.seg] : &single.seg;
      const int buf = tl % NBUF;
      const uint32_t use = (uint32_t)(tl / NBUF);
      if (!mbar_wait(&tfull[buf], use & 1u, limit_ns)) {
        if (lane == 0) set_status(status, ST_TIMEOUT, 30);
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const uint32_t ta = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * 2 * BN);
      const int col = it.c * BM + q * 32 + lane;
      if (MODE == 2 && it.slot >= 0) {
        // accumulator pair of this chunk, for k_split_reduce: [slot][column][row]
        float2* dst = sd->wpart + ((int64_t)it.slot * BM + q * 32 + lane) * BN;
#pragma unroll 1
        for (int ch = 0; ch < BN / 32; ++ch) {
          float v0[32], v1[32];
          tmem_ld32(ta + (uint32_t)(ch * 32), v0);
          tmem_ld32(ta + (uint32_t)(BN + ch * 32), v1);
          if (col < sd->K) {
            float4* d4 = reinterpret_cast<float4*>(dst + ch * 32);
#pragma unroll
            for (int i = 0; i < 16; ++i) d4[i] = make_float4(v0[2 * i], v1[2 * i], v0[2 * i + 1], v1[2 * i + 1]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[buf]);
      } else if (MODE == 3 || MODE == 4) {
        // 32 consecutive rows of this thread's column per TMEM load
        const RefineIO& io = single.io;
#pragma unroll 1
        for (int ch = 0; ch < BN / 32; ++ch) {
          float v0[32], v1[32];
          tmem_ld32(ta + (uint32_t)(ch * 32), v0);
          tmem_ld32(ta + (uint32_t)(BN + ch * 32), v1);
          if (col < sd->K) {
            const int64_t row0 = (int64_t)it.m * BN + ch * 32;
            float4* d4 = reinterpret_cast<float4*>(io.out + (int64_t)col * io.ldo + row0);
            float o[32];
            if (MODE == 3) {
#pragma unroll
              for (int i = 0; i < 32; ++i) o[i] = v0[i] + v1[i];
            } else {
              const float* r = io.in + (int64_t)col * io.ldi;
#pragma unroll
              for (int i = 0; i < 32; ++i) {
                const float x = row0 + i < sd->nk ? r[row0 + i] : 0.f;
                o[i] = (x - v0[i]) - v1[i];   // x - v0 is exact while they are within a factor 2
              }
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) d4[i] = make_float4(o[4 * i], o[4 * i + 1], o[4 * i + 2], o[4 * i + 3]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[buf]);
      } else {
        double part[C::GROUPS];
#pragma unroll
        for (int g = 0; g < C::GROUPS; ++g) {
          float hi = 0.f, lo = 0.f;
#pragma unroll 1
          for (int ch = 2 * g; ch < 2 * g + 2; ++ch) {
            float v0[32], v1[32];
            tmem_ld32(ta + (uint32_t)(ch * 32), v0);
            tmem_ld32(ta + (uint32_t)(BN + ch * 32), v1);
            if (MODE == 5) {
              // w = w~ + delta: two-sum of w~ and the exact hi*hi part, the corrections
              // joining the tail; rows past N' and columns past K read w~ = 0
              const int64_t row0 = (int64_t)it.m * BN + ch * 32;
              const float* wt = single.io.in + (int64_t)(col < sd->K ? col : 0) * single.io.ldi;
#pragma unroll
              for (int i = 0; i < 32; ++i) {
                const float x = (col < sd->K && row0 + i < sd->nk) ? wt[row0 + i] : 0.f;
                const float t = x + v0[i], bp = t - x;
                const float et = (x - (t - bp)) + (v0[i] - bp);
                ff_add_square2(t, et + v1[i], hi, lo);
              }
            } else {
#pragma unroll
              for (int i = 0; i < 32; ++i) ff_add_square2(v0[i], v1[i], hi, lo);
            }
          }
          part[g] = (double)hi + (double)lo;
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[buf]);
        if (col < sd->K) {
          const int64_t g0 = (int64_t)it.m * C::GROUPS;
#pragma unroll
          for (int g = 0; g < C::GROUPS; ++g) sd->partials[(g0 + g) * sd->ldp + col] = part[g];
        }
      }
      ++tl;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem_base, C::TMEM_COLS);
  }
}

static int g_num_sms = 0;

int tc_num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 148;
  }
  return g_num_sms;
}

template <int NSL, int BN, int MODE>
static cudaError_t launch_impl(const TcSingle& single, const TcItem* items, int n_items, const TcSegDev* segs,
                               DevStatus* status, int64_t wait_limit_ns, cudaStream_t st, bool pdl) {
  using C = tc::Cfg<NSL, BN>;
  static std::atomic<unsigned long long> attr_done{0};
  if (device_needs_setup(attr_done)) {
    cudaError_t e =
        cudaFuncSetAttribute(k_tc_cdo<NSL, BN, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    mark_device_done(attr_done);
  }
  const int n_total = (MODE == 1 || MODE == 2) ? n_items : single.nm * single.nc;
  if (n_total <= 0) return cudaSuccess;
  int grid = tc_num_sms();
  if (grid > n_total) grid = n_total;
  // programmatic dependent of the residual slicing when pdl (see the producer)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(tc::THREADS);
  cfg.dynamicSmemBytes = C::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k_tc_cdo<NSL, BN, MODE>, single, items, n_items, segs, status,
                            (uint64_t)wait_limit_ns);
}

template <int MODE>
static cudaError_t dispatch(int nslices, int bn, const TcSingle& p, const TcItem* items, int n_items,
                            const TcSegDev* segs, DevStatus* status, int64_t lim, cudaStream_t st, bool pdl) {
  if (bn == 256) {
    if (nslices == 3) return launch_impl<3, 256, MODE>(p, items, n_items, segs, status, lim, st, pdl);
    if (nslices == 4) return launch_impl<4, 256, MODE>(p, items, n_items, segs, status, lim, st, pdl);
    if (nslices == 2) return launch_impl<2, 256, MODE>(p, items, n_items, segs, status, lim, st, pdl);
  } else if (bn == 128) {
    if (nslices == 3) return launch_impl<3, 128, MODE>(p, items, n_items, segs, status, lim, st, pdl);
    if (nslices == 4) return launch_impl<4, 128, MODE>(p, items, n_items, segs, status, lim, st, pdl);
    if (nslices == 2) return launch_impl<2, 128, MODE>(p, items, n_items, segs, status, lim, st, pdl);
  } else if (bn == 64) {
    if (nslices == 3) return launch_impl<3, 64, MODE>(p, items, n_items, segs, status, lim, st, pdl);
    if (nslices == 4) return launch_impl<4, 64, MODE>(p, items, n_items, segs, status, lim, st, pdl);
    if (nslices == 2) return launch_impl<2, 64, MODE>(p, items, n_items, segs, status, lim, st, pdl);
  }
  return cudaErrorInvalidValue;
}

// single segment: tiles of bn rows (256, 128 or 64); seg.partials holds one row per
// 64-row group, seg.ldp apart
cudaError_t launch_tc_single(const TcSegDev& seg, int bn, int nc, int nkb_max, int nslices, DevStatus* status,
                             int64_t wait_limit_ns, cudaStream_t st) {
  TcSingle p{};
  p.seg = seg;
  p.nm = (int)(ceil_div((int64_t)seg.nk, OP_ROWS) * OP_ROWS / bn);
  p.nc = nc;
  p.nkb_max = nkb_max;
  return dispatch<0>(nslices, bn, p, nullptr, 0, nullptr, status, wait_limit_ns, st, true);
}

// the refinement step's whole-row element-wise products (256- or 128-row tiles)
cudaError_t launch_tc_single_ew(const TcSegDev& seg, int bn, int mode, int nc, int nkb_max, int nslices,
                                const RefineIO& io, DevStatus* status, int64_t wait_limit_ns, cudaStream_t st) {
  TcSingle p{};
  p.seg = seg;
  p.nm = (int)(ceil_div((int64_t)seg.nk, OP_ROWS) * OP_ROWS / bn);
  p.nc = nc;
  p.nkb_max = nkb_max;
  p.io = io;
#define TD_EW_CASE(BN_, MODE_)                                                                                    \
  if (bn == BN_ && mode == MODE_) {                                                                               \
    if (nslices == 2) return launch_impl<2, BN_, MODE_>(p, nullptr, 0, nullptr, status, wait_limit_ns, st, true); \
    if (nslices == 3) return launch_impl<3, BN_, MODE_>(p, nullptr, 0, nullptr, status, wait_limit_ns, st, true); \
    if (nslices == 4) return launch_impl<4, BN_, MODE_>(p, nullptr, 0, nullptr, status, wait_limit_ns, st, true); \
  }
  TD_EW_CASE(128, 3) TD_EW_CASE(128, 4) TD_EW_CASE(128, 5)
  TD_EW_CASE(256, 3) TD_EW_CASE(256, 4) TD_EW_CASE(256, 5)
#undef TD_EW_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_tc_cdo(const TcItem* items, int n_items, const TcSegDev* segs, int nslices, int bn,
                          bool split, DevStatus* status, int64_t wait_limit_ns, cudaStream_t st, bool pdl,
                          int* sched) {
  TcSingle p{};
  p.sched = sched;
  if (split) return dispatch<2>(nslices, bn, p, items, n_items, segs, status, wait_limit_ns, st, pdl);
  return dispatch<1>(nslices, bn, p, items, n_items, segs, status, wait_limit_ns, st, pdl);
}

// Reduce the accumulator pairs of a split row tile (one block per 64 rows and
// 16 columns): for each row, w = sum over chunks of (hi*hi sum + correction
// sum), in double-float (the hi*hi sums are exact, their sum stays exact well
// past these lengths); then the chi2 share of the rows in double-float, as
// FP64 partials per 64-row group.  Thread (row, column group): rows are
// contiguous in the slot layout, so a warp's loads are coalesced; the four
// column groups take columns round-robin; the sum over a warp's 32 rows is a
// fixed shuffle tree, the two warps of a group are added in a fixed order.
//
// RM selects what is done with w (the refinement step of td_options.refine):
//   RED_CHI2   chi2 partials of w (above)
//   RED_WRITE  out = fl32(w)                        (the first iterate w~)
//   RED_RESID  out = fl32(in - w), in = r           (s = r - L w~)
//   RED_FINAL  chi2 partials of in + w, in = w~     (w = w~ + L^{-1} s)
// Element (row i, column k) of in / out sits at [i + k ld]; rows at or past
// N' read as zero.
template <int RM>
__global__ void __launch_bounds__(256) k_split_reduce(const SplitUnit* __restrict__ units,
                                                       const TcSegDev* __restrict__ segs, int bn, RefineIO io) {
  __shared__ float red_hi[16][2], red_lo[16][2];
  const SplitUnit u = units[blockIdx.x];
  const int g64 = blockIdx.y;                   // 64-row group of the bn-row tile
  const int c16 = blockIdx.z * 16;              // 16-column slice of the 128-column tile
  const TcSegDev& sd = segs[u.seg];
  const int row = threadIdx.x & 63, grp = threadIdx.x >> 6;   // 4 column groups of 2 warps
  const int wig = (threadIdx.x >> 5) & 1, lane = threadIdx.x & 31;
  const int ncol = min(128, sd.K - u.c * 128);
  if (c16 >= ncol) return;
  const float2* base = sd.wpart + (int64_t)u.slot0 * 128 * bn + g64 * 64 + row;
  // this thread's four columns c16 + grp + 4 c: the chunk pairs are loaded eight
  // chunks deep from clamped (in-range) addresses, then added in chunk order
  constexpr int CB = 4, CH = 8;
  float wh[CB], wl[CB];
#pragma unroll
  for (int c = 0; c < CB; ++c) wh[c] = wl[c] = 0.f;
  for (int ch0 = 0; ch0 < u.nchunk; ch0 += CH) {
    float2 v[CH][CB];
#pragma unroll
    for (int i = 0; i < CH; ++i)
#pragma unroll
      for (int c = 0; c < CB; ++c) {
        const int ch = min(ch0 + i, u.nchunk - 1), cl = min(c16 + grp + 4 * c, ncol - 1);
        v[i][c] = __ldcg(base + ((int64_t)ch * 128 + cl) * bn);
      }
#pragma unroll
    for (int i = 0; i < CH; ++i)
      if (ch0 + i < u.nchunk) {
#pragma unroll
        for (int c = 0; c < CB; ++c) {
          ff_add(v[i][c].x, wh[c], wl[c]);
          ff_add(v[i][c].y, wh[c], wl[c]);
        }
      }
  }
  const int64_t i = (int64_t)u.m * bn + g64 * 64 + row;   // row of W
  if constexpr (RM == RED_WRITE || RM == RED_RESID) {
#pragma unroll
    for (int c = 0; c < CB; ++c) {
      const int cl = c16 + grp + 4 * c;
      if (cl >= ncol) continue;
      const int64_t k = (int64_t)u.c * 128 + cl;
      if constexpr (RM == RED_WRITE) {
        io.out[i + k * io.ldo] = wh[c] + wl[c];
      } else {
        const float r = i < sd.nk ? io.in[i + k * io.ldi] : 0.f;
        io.out[i + k * io.ldo] = (r - wh[c]) - wl[c];   // r - wh is exact while they are within a factor 2
      }
    }
  } else {   // RED_CHI2, RED_FINAL
    if constexpr (RM == RED_FINAL) {
#pragma unroll
      for (int c = 0; c < CB; ++c) {
        const int cl = min(c16 + grp + 4 * c, ncol - 1);
        const float x = i < sd.nk ? io.in[i + ((int64_t)u.c * 128 + cl) * io.ldi] : 0.f;
        ff_add(x, wh[c], wl[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < CB; ++c) {
      const int cl = c16 + grp + 4 * c;
      float hi = 0.f, lo = 0.f;
      ff_add_square2(wh[c], wl[c], hi, lo);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const float oh = __shfl_down_sync(0xffffffffu, hi, off);
        const float ol = __shfl_down_sync(0xffffffffu, lo, off);
        ff_add(oh, hi, lo);
        lo += ol;
      }
      if (lane == 0 && cl < ncol) {
        red_hi[cl - c16][wig] = hi;
        red_lo[cl - c16][wig] = lo;
      }
    }
    __syncthreads();
    if (threadIdx.x < 16 && c16 + (int)threadIdx.x < ncol) {
      const int cl = threadIdx.x;
      const double s = ((double)red_hi[cl][0] + (double)red_lo[cl][0]) + ((double)red_hi[cl][1] + (double)red_lo[cl][1]);
      sd.partials[((int64_t)u.m * (bn / 64) + g64) * sd.ldp + u.c * 128 + c16 + cl] = s;
    }
  }
}

cudaError_t launch_split_reduce(const SplitUnit* units, int n_units, const TcSegDev* segs, int bn,
                                cudaStream_t st, int64_t max_cols, int mode, const RefineIO& io) {
  if (n_units <= 0) return cudaSuccess;
  const unsigned nz = (unsigned)ceil_div(std::min<int64_t>(std::max<int64_t>(max_cols, 1), 128), 16);
  const dim3 grid(n_units, bn / 64, nz);
  switch (mode) {
    case RED_CHI2: k_split_reduce<RED_CHI2><<<grid, 256, 0, st>>>(units, segs, bn, io); break;
    case RED_WRITE: k_split_reduce<RED_WRITE><<<grid, 256, 0, st>>>(units, segs, bn, io); break;
    case RED_RESID: k_split_reduce<RED_RESID><<<grid, 256, 0, st>>>(units, segs, bn, io); break;
    case RED_FINAL: k_split_reduce<RED_FINAL><<<grid, 256, 0, st>>>(units, segs, bn, io); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// chi2 and logL per column from the per-group partials, for every segment of
// a grouped launch (TcSegDev::nm = number of 64-row groups); same order as
// k_finalize: one warp per column, strided sums, fixed shuffle tree.
__global__ void k_tc_finalize(const TcSegDev* __restrict__ segs) {
  const TcSegDev& sd = segs[blockIdx.y];
  const int lane = threadIdx.x & 31;
  for (int64_t col = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); col < sd.K;
       col += (int64_t)gridDim.x * (blockDim.x >> 5)) {
    double s = 0.0;
    for (int m = lane; m < sd.nm; m += 32) s += sd.partials[(int64_t)m * sd.ldp + col];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) {
      if (sd.chi2) sd.chi2[col] = s;
      sd.logL[col] = -0.5 * s - 0.5 * sd.logdet - 0.5 * (double)sd.nk * LOG2PI;
    }
  }
}

cudaError_t launch_tc_finalize(const TcSegDev* segs, int nseg, int64_t maxK, cudaStream_t st) {
  if (nseg <= 0 || maxK <= 0) return cudaSuccess;
  int gx = (int)ceil_div(maxK, 8);
  if (gx > 64) gx = 64;
  k_tc_finalize<<<dim3(gx, nseg), 256, 0, st>>>(segs);
  return cudaGetLastError();
}

}  // namespace td
