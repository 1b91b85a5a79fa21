// Tensor-core whitening for small and mid-size batches (K <= 256 residual
// columns).
//
// Same method and slices as the main kernel (Sec. II.A, W = L^{-1}; Sec.
// III.A, the cached-operator evaluation), with the operand roles swapped so
// the MMA is not padded to 128 residual columns:
//   MMA M = 128 rows of W           (A = L^{-1} slices, K-major),
//   MMA N = NC residual columns, 16 ... 256 (B = R^T slices, K-major),
// so D[lane i][col n] = W[i][n].  Every operator tile is read once, whatever
// the batch width: at NC <= 64 the MMA work per 24 KB tile (three slices) is
// tiny and the kernel streams the packed operator from HBM; at NC = 256 a
// k-block moves 72 KB of operands for 12.6 MFLOP of products, the ratio of
// the 256-row main kernel, so mid-size batches stay on the tensor pipe
// (128-column residual tiles against 128-row operator tiles move a third
// more bytes per product).  Long rows are cut into balanced k-chunks;
// a chunk stores its accumulator pair (exact hi*hi sum, corrections) for
// k_small_reduce; a whole row reduces chi2 directly: w = hi + corrections in
// double-float, exact squares, a fixed shuffle tree over the 32 rows of a
// warp, then the four warps in a fixed order -> one FP64 partial per
// 128-row tile and column.
//
// Three launches per call, chained as programmatic dependents so no launch
// gap is exposed: the residual slicing; this kernel, whose producer streams
// the first operator stages before it waits for the slices; k_small_reduce,
// which adds the chunks of each split row tile (chunk order fixed) and whose
// last CTA sums each column's partials in a fixed order into chi2 and logL.
// Up to eight columns this kernel does the reduction's work itself (the last
// chunk of a split row tile to arrive reduces it, the CTA that completes the
// last tile forms chi2 and logL), with the same arithmetic: two launches.
//
// Warp roles as in the main kernel: warp 0 lane 0 TMA producer, warp 1
// TMEM owner and MMA issuer, warps 2..5 epilogue.  Every wait is bounded;
// the completion counter is an arrival count only (no thread waits on it).
#include <type_traits>

#include "td_internal.h"

namespace td {
namespace tsm {
constexpr int BM = 128;                 // operator rows per tile (MMA M)
constexpr int BK = OP_KB;               // 32
constexpr int A_SLICE = BM * BK * 2;    // 8 KB of operator per slice
constexpr int THREADS = 192;
template <int NSL, int NC> struct Cfg {
  static constexpr int B_SLICE = NC * BK * 2;
  static constexpr int A_STAGE = NSL * A_SLICE;
  static constexpr int STAGE = A_STAGE + NSL * B_SLICE;
  // four stages: measured at N' = 8192 (one call, K = 1): 44.0 us against 47.0 us
  // with eight and 55.5 us with two; deeper queues did not raise the rate
  static constexpr int STAGES = (216 * 1024) / STAGE > 4 ? 4 : (216 * 1024) / STAGE;
  // accumulator pairs in TMEM: four up to NC = 64, two at 128, one at 256
  static constexpr int NBUF = (512 / (2 * NC)) < 4 ? (512 / (2 * NC)) : 4;
  static constexpr uint32_t TMEM_COLS = (NBUF * 2 * NC <= 128) ? 128 : ((NBUF * 2 * NC <= 256) ? 256 : 512);
  // split slots hold 128 columns (NC <= 128) or NC
  static constexpr int SLOT_COLS = NC > 128 ? NC : 128;
  static constexpr int SMEM = STAGES * STAGE + 256 + 1024;   // stages + barriers + alignment
};
}  // namespace tsm

// 32 lanes x 16 consecutive 32-bit columns
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }   // warps 2..5

// Chunk pairs of one split row tile, CB columns n0 .. n0+CB-1, for the row of
// this thread (base = its row in the unit's first slot): double-float sums in
// chunk order (loads issued CH chunks x CB columns ahead), the exact square,
// then the fixed shuffle tree over the 32 rows of the warp; lane 0 returns
// the warp's partial of each column.  A column's arithmetic does not depend
// on CB.
template <int CH, int CB = 4>
__device__ __forceinline__ void unit_cols4(const float2* base, int nchunk, int slot_cols, int n0, int kcols,
                                           double (&part)[CB]) {
  float wh[CB], wl[CB];
#pragma unroll
  for (int c = 0; c < CB; ++c) wh[c] = wl[c] = 0.f;
  for (int ch0 = 0; ch0 < nchunk; ch0 += CH) {
    float2 v[CH][CB];
    // CH x CB predicated loads in flight at once, then the additions in chunk order
#pragma unroll
    for (int i = 0; i < CH; ++i)
#pragma unroll
      for (int c = 0; c < CB; ++c) {
        const int n = min(n0 + c, kcols - 1);
        v[i][c] = ch0 + i < nchunk ? __ldcg(base + ((int64_t)(ch0 + i) * slot_cols + n) * 128)
                                   : make_float2(0.f, 0.f);
      }
#pragma unroll
    for (int i = 0; i < CH; ++i)
      if (ch0 + i < nchunk) {
#pragma unroll
        for (int c = 0; c < CB; ++c) {
          ff_add(v[i][c].x, wh[c], wl[c]);
          ff_add(v[i][c].y, wh[c], wl[c]);
        }
      }
  }
#pragma unroll
  for (int c = 0; c < CB; ++c) {
    float hi = 0.f, lo = 0.f;
    ff_add_square2(wh[c], wl[c], hi, lo);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float oh = __shfl_down_sync(0xffffffffu, hi, off);
      const float ol = __shfl_down_sync(0xffffffffu, lo, off);
      ff_add(oh, hi, lo);
      lo += ol;
    }
    part[c] = (double)hi + (double)lo;
  }
}

// chi2 and logL of columns c0 .. c0+ncols-1 from the per-tile partials of a
// single-segment small-batch call: thread (q, lane) adds the tiles of quarter
// q in order, then the four quarters in order.  128 threads (q = row quarter)
// meeting at `bar`.
template <typename Bar>
__device__ __forceinline__ void small_final_cols(const TcSegDev* sd, const SmallFinal& fin, int c0, int ncols,
                                                 double (*sh)[32], int q, int lane, Bar bar) {
  const int nparts = sd->nm;
  const int per = (nparts + 3) / 4;
  const int p0 = q * per, p1 = min(nparts, p0 + per);
  const int col = min(c0 + lane, fin.K - 1);
  double s = 0.0;
  if (lane < ncols)
    for (int pb = p0; pb < p1; pb += 16) {
      double v[16];   // sixteen loads in flight (clamped addresses), then the additions in order
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = __ldcg(&sd->partials[(int64_t)min(pb + i, p1 - 1) * sd->ldp + col]);
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (pb + i < p1) s += v[i];
    }
  bar();   // sh is free
  sh[q][lane] = s;
  bar();
  if (q == 0 && lane < ncols && c0 + lane < fin.K) {
    const double t = ((sh[0][lane] + sh[1][lane]) + sh[2][lane]) + sh[3][lane];
    if (fin.chi2) fin.chi2[c0 + lane] = t;
    fin.logL[c0 + lane] = -0.5 * t - 0.5 * sd->logdet - 0.5 * (double)sd->nk * LOG2PI;
  }
}

// One 128-row tile's chi2 partials are complete (written and fenced by the
// epilogue warps): count it; the CTA that completes the last tile of the call
// sums every column's tile partials into chi2 and logL.  An arrival count
// only: no thread waits on another CTA.
__device__ __forceinline__ void small_tile_done(const TcSegDev* sd, const SmallFinal& fin, int q, int lane,
                                                double (*sh)[32], int& sh_last) {
  if (q == 0 && lane == 0) sh_last = atomicAdd(&fin.counters[fin.n_units], 1) == sd->nm - 1;
  epi_bar();
  if (sh_last) {
    __threadfence();
    for (int c0 = 0; c0 < fin.K; c0 += 32) small_final_cols(sd, fin, c0, 32, sh, q, lane, epi_bar);
  }
}

template <int NSL, int NC>
__global__ void __launch_bounds__(tsm::THREADS, 1)
    k_tc_small(const TcItem* __restrict__ items, int n_items, const TcSegDev* __restrict__ segs,
               DevStatus* status, uint64_t limit_ns, const SmallFinal red) {
  using namespace tsm;
  using C = Cfg<NSL, NC>;
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
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  __shared__ int sh_ok[4];
  __shared__ double sh_part[4][NC];
  // in-kernel reduction (single segment, NC <= 64): unit and final partials
  __shared__ double sh_fin[NC <= 64 ? 4 : 1][32];
  __shared__ int sh_last;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // The reduction kernel may be scheduled once every CTA has triggered (it
  // waits for this grid's completion in any case).  Small batches trigger at
  // once, so its few CTAs are resident before the product ends.  From 128
  // columns its grid is units x K/4 CTAs; resident early they would hold SM
  // slots that kernels of other streams (a server's other requests) need for
  // the whole product, so those CTAs trigger when their last item is done.
  // With the in-kernel reduction the dependent is the next call's slicing,
  // which measured faster launched late (K = 4: 50.1 against 51.2 us a call).
  if constexpr (NC < 128) {
    if (red.logL == nullptr) pdl_trigger();
  }
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
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, C::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int G = gridDim.x, b = blockIdx.x;

  if (warp == 0) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued_mask = 0, issued_phase = 0;
      // the operator does not depend on the preceding launch: the first stages
      // stream it while the residual slices are still being written
      bool dep = false;
      int pend_n = 0;
      int pend_stage[STAGES], pend_kb[STAGES], pend_c[STAGES];
      const TcSegDev* pend_sd[STAGES];
      auto flush = [&]() {
        pdl_wait();
        dep = true;
        for (int i = 0; i < pend_n; ++i) {
          uint8_t* sb = smem + pend_stage[i] * STAGE + A_STAGE;
#pragma unroll
          for (int sl = 0; sl < NSL; ++sl)
            tma_load_3d(sb + sl * B_SLICE, &pend_sd[i]->mapA, &full[pend_stage[i]], pend_kb[i] * BK,
                        pend_c[i] * NC, sl);
        }
        pend_n = 0;
      };
      for (int r = 0; (int64_t)r * G < n_items && !*abort_flag; ++r) {
        const int idx = r * G + ((r & 1) ? (G - 1 - b) : b);
        if (idx >= n_items) continue;
        const TcItem it = items[idx];
        const TcSegDev* sd = &segs[it.seg];
        const int row0 = it.m * BM;
        const int M256 = row0 / OP_ROWS;
        const int yoff = row0 - M256 * OP_ROWS;
        const int blk0 = (OP_ROWS / BK) * M256 * (M256 + 1) / 2;
        bool ok = true;
        for (int kb = it.kb0; kb < it.kb0 + it.nkb; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, limit_ns)) {
            set_status(status, ST_TIMEOUT, 40);
            *abort_flag = 1;
            ok = false;
            break;
          }
          uint8_t* sa = smem + stage * STAGE;    // operator slices (A)
          uint8_t* sb = sa + A_STAGE;            // residual slices (B)
          mbar_arrive_expect_tx(&full[stage], (uint32_t)(NSL * (A_SLICE + B_SLICE)));
          tma_load_3d(sa, &sd->mapB, &full[stage], 0, yoff, (blk0 + kb) * OP_SLICES);
          if (dep) {
#pragma unroll
            for (int sl = 0; sl < NSL; ++sl)
              tma_load_3d(sb + sl * B_SLICE, &sd->mapA, &full[stage], kb * BK, it.c * NC, sl);
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
      if (!dep) flush();
      for (int s = 0; s < STAGES; ++s)
        if (issued_mask & (1u << s)) mbar_wait(&full[s], (issued_phase >> s) & 1u, limit_ns);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int tl = 0;
      for (int r = 0; (int64_t)r * G < n_items && !*abort_flag; ++r) {
        const int idx = r * G + ((r & 1) ? (G - 1 - b) : b);
        if (idx >= n_items) continue;
        const TcItem it = items[idx];
        // the MMA covers the item's columns rounded up to 16, not the whole tile
        // (a segment's last column tile in a grouped launch): each column's
        // arithmetic is the same either way
        const int ncol_m = min(NC, segs[it.seg].K - it.c * NC);
        const uint32_t idesc = idesc_bf16_f32(BM, (ncol_m + 15) & ~15);
        const int buf = tl % NBUF;
        const uint32_t use = (uint32_t)(tl / NBUF);
        if (!mbar_wait(&tempty[buf], (use & 1u) ^ 1u, limit_ns)) {
          set_status(status, ST_TIMEOUT, 41);
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t d_hi = tmem_base + (uint32_t)(buf * 2 * NC);
        const uint32_t d_lo = d_hi + (uint32_t)NC;
        bool ok = true;
        for (int kb = it.kb0; kb < it.kb0 + it.nkb; ++kb) {
          if (!mbar_wait(&full[stage], phase, limit_ns)) {
            set_status(status, ST_TIMEOUT, 42);
            *abort_flag = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + stage * STAGE);
          const uint32_t sb = sa + A_STAGE;
          // operator slices (A) against residual slices (B), grouped by the
          // operator slice so the collector buffer reuses it
#pragma unroll
          for (int kk = 0; kk < 2; ++kk)
            split_products_step<NSL>(d_hi, d_lo, sa, A_SLICE, sb, B_SLICE, kk * 32, idesc,
                                     (kb > it.kb0 || kk > 0) ? 1u : 0u);
          tc_commit(&empty[stage]);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        tc_commit(&tfull[buf]);
        ++tl;
      }
      tc_commit(fin);
      mbar_wait(fin, 0, limit_ns);
    }
  } else {
    const int q = warp & 3;          // TMEM lane quarter = rows 32q .. 32q+31 of the tile
    // in-kernel reduction: these warps read and write buffers and counters that
    // the preceding launch may still use, so they wait for it (a no-op without
    // a programmatic dependency)
    const bool fused = NC <= 64 && red.logL != nullptr;
    if (fused) pdl_wait();
    int tl = 0;
    for (int r = 0; (int64_t)r * G < n_items; ++r) {
      const int idx = r * G + ((r & 1) ? (G - 1 - b) : b);
      if (idx >= n_items) continue;
      const TcItem it = items[idx];
      const TcSegDev* sd = &segs[it.seg];
      const int buf = tl % NBUF;
      const uint32_t use = (uint32_t)(tl / NBUF);
      // all four warps take the same decision (they meet at named barriers below)
      const bool got = mbar_wait(&tfull[buf], use & 1u, limit_ns);
      if (lane == 0) sh_ok[q] = got ? 1 : 0;
      epi_bar();
      const bool all_ok = sh_ok[0] && sh_ok[1] && sh_ok[2] && sh_ok[3];
      epi_bar();
      if (!all_ok) {
        if (lane == 0 && !got) set_status(status, ST_TIMEOUT, 43);
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const uint32_t ta = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * 2 * NC);
      const int ncol = min(NC, sd->K - it.c * NC);
      // 16 columns at a time: both accumulators of a column group, then its
      // stores or its chi2 terms (NC = 256 would not fit in registers at once)
      float2* dst = it.slot >= 0 ? sd->wpart + (int64_t)it.slot * C::SLOT_COLS * BM + q * 32 + lane : nullptr;
#pragma unroll 1
      for (int h = 0; h < (ncol + 15) / 16; ++h) {
        float t0[16], t1[16];
        tmem_ld16(ta + (uint32_t)(h * 16), t0);
        tmem_ld16(ta + (uint32_t)(NC + h * 16), t1);
        if (it.slot >= 0) {
          // accumulator pair of this chunk: [slot][SLOT_COLS columns][128 rows]
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (h * 16 + i < ncol) dst[(int64_t)(h * 16 + i) * BM] = make_float2(t0[i], t1[i]);
        } else {
          // chi2 of this warp's 32 rows per column: exact squares, fixed shuffle tree
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            float hi = 0.f, lo = 0.f;
            ff_add_square2(t0[i], t1[i], hi, lo);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
              const float oh = __shfl_down_sync(0xffffffffu, hi, off);
              const float ol = __shfl_down_sync(0xffffffffu, lo, off);
              ff_add(oh, hi, lo);
              lo += ol;
            }
            if (lane == 0) sh_part[q][h * 16 + i] = (double)hi + (double)lo;
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[buf]);
      if (it.slot < 0) {
        // the tile's four 32-row groups in a fixed order
        epi_bar();
        if (q == 0) {
          for (int n = lane; n < ncol; n += 32)
            sd->partials[(int64_t)it.m * sd->ldp + it.c * NC + n] =
                ((sh_part[0][n] + sh_part[1][n]) + sh_part[2][n]) + sh_part[3][n];
          if (fused) __threadfence();
        }
        epi_bar();
        if constexpr (NC <= 64)
          if (fused) small_tile_done(sd, red, q, lane, sh_fin, sh_last);
      } else if constexpr (NC <= 64) {
        if (fused) {
          // the last chunk of a split row tile to arrive reduces the unit: the
          // chunk pairs in chunk order, as the separate reduction kernel does
          const SplitUnit u = red.units[it.unit];   // loaded while the fence drains
          __threadfence();   // this thread's chunk pairs
          epi_bar();
          if (q == 0 && lane == 0) sh_last = atomicAdd(&red.counters[it.unit], 1) == u.nchunk - 1;
          epi_bar();
          if (sh_last) {
            __threadfence();
            const float2* base = sd->wpart + (int64_t)u.slot0 * red.slot_cols * BM + q * 32 + lane;
            // all of the call's columns in one pass (up to SMALL_FUSED_K = 8):
            // four columns eight chunks deep, or eight columns four chunks deep
            // (measured at N' = 8192: K <= 4 calls 49.5-50 against 51.5 us with
            // the eight-column form, K = 5 .. 8 51.5-52.3 against 53-56 us with
            // the separate reduction)
            auto pass = [&](auto cb) {
              constexpr int FCB = decltype(cb)::value;
              double part[FCB];
              unit_cols4<32 / FCB, FCB>(base, u.nchunk, red.slot_cols, 0, red.K, part);
              if (lane == 0)
#pragma unroll
                for (int c = 0; c < FCB; ++c) sh_fin[q][c] = part[c];
              epi_bar();
              // the tile's four 32-row groups in a fixed order
              if (q == 0 && lane < FCB && lane < red.K)
                sd->partials[(int64_t)u.m * sd->ldp + u.c * 128 + lane] =
                    ((sh_fin[0][lane] + sh_fin[1][lane]) + sh_fin[2][lane]) + sh_fin[3][lane];
              epi_bar();
            };
            if (red.K <= 4)
              pass(std::integral_constant<int, 4>());
            else
              pass(std::integral_constant<int, 8>());
            if (q == 0) __threadfence();
            epi_bar();
            small_tile_done(sd, red, q, lane, sh_fin, sh_last);
          }
        }
      }
      ++tl;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (NC >= 128 || red.logL != nullptr) pdl_trigger();   // after every role of this CTA is done
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem_base, C::TMEM_COLS);
  }
}

// Chunk reduction + chi2 / logL for the small-batch kernel when it does not
// reduce in-kernel (NC >= 128).  Grid: (split units, column groups of 4); 128
// threads, one per row of the 128-row tile: unit_cols4, then the four 32-row
// groups in order give the tile's partial.  The last CTA of each column group
// (one arrival counter per group) sums its four columns' tile partials in a
// fixed order into chi2 and logL (small_final_cols).  Without split units
// (short segments) one CTA does the same for all columns.
__global__ void __launch_bounds__(128) k_small_reduce(const TcSegDev* __restrict__ segs, const SmallFinal fin) {
  __shared__ int sh_last;
  __shared__ double sh[4][32];
  // no early trigger: the next call's slicing and product launched while this
  // grid runs measured slower (K = 8, N' = 8192: 57.5 against 54.3 us a call)
  pdl_wait();   // the product kernel's pairs and partials are complete and visible
  const TcSegDev* sd = &segs[0];
  const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
  auto sync = [] { __syncthreads(); };
  if (fin.n_units == 0) {
    for (int c0 = 0; c0 < fin.K; c0 += 32) small_final_cols(sd, fin, c0, 32, sh, q, lane, sync);
    return;
  }
  const SplitUnit u = fin.units[blockIdx.x];
  const int n0 = blockIdx.y * 4;
  const float2* base = sd->wpart + (int64_t)u.slot0 * fin.slot_cols * 128 + threadIdx.x;
  constexpr int CB = 4;
  double part[CB];
  unit_cols4<4>(base, u.nchunk, fin.slot_cols, n0, fin.K, part);
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < CB; ++c) sh[q][c] = part[c];
  __syncthreads();
  // the tile's four 32-row groups in a fixed order
  if (threadIdx.x < CB && n0 + threadIdx.x < fin.K) {
    const int c = threadIdx.x;
    sd->partials[(int64_t)u.m * sd->ldp + u.c * 128 + n0 + c] = ((sh[0][c] + sh[1][c]) + sh[2][c]) + sh[3][c];
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) sh_last = (atomicAdd(&fin.counters[blockIdx.y], 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!sh_last) return;
  __threadfence();
  small_final_cols(sd, fin, n0, CB, sh, q, lane, sync);
}

// Chunk reduction of a grouped small-orientation launch (many segments, every
// item a chunk): grid (units, nc / 4), 128 threads (rows of the 128-row
// tile).  As k_small_reduce for one unit's four columns (chunk order fixed,
// double-float, exact squares, fixed shuffle tree, the four 32-row groups in
// order), writing the tile's chi2 partial of each column; the per-segment
// sums over tiles are k_tc_finalize's.
__global__ void __launch_bounds__(128) k_small_reduce_grouped(const SplitUnit* __restrict__ units,
                                                              const TcSegDev* __restrict__ segs, int nc,
                                                              int slot_cols) {
  __shared__ double sh[4][4];
  const SplitUnit u = units[blockIdx.x];
  const TcSegDev* sd = &segs[u.seg];
  const int ncol = min(nc, sd->K - u.c * nc);
  const int n0 = blockIdx.y * 4;
  if (n0 >= ncol) return;
  const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
  const float2* base = sd->wpart + (int64_t)u.slot0 * slot_cols * 128 + threadIdx.x;
  constexpr int CB = 4, CH = 4;
  float wh[CB], wl[CB];
#pragma unroll
  for (int c = 0; c < CB; ++c) wh[c] = wl[c] = 0.f;
  for (int ch0 = 0; ch0 < u.nchunk; ch0 += CH) {
    float2 v[CH][CB];
#pragma unroll
    for (int i = 0; i < CH; ++i)
#pragma unroll
      for (int c = 0; c < CB; ++c) {
        const int n = min(n0 + c, ncol - 1);
        v[i][c] = ch0 + i < u.nchunk ? __ldcg(base + ((int64_t)(ch0 + i) * slot_cols + n) * 128)
                                     : make_float2(0.f, 0.f);
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
#pragma unroll
  for (int c = 0; c < CB; ++c) {
    float hi = 0.f, lo = 0.f;
    ff_add_square2(wh[c], wl[c], hi, lo);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float oh = __shfl_down_sync(0xffffffffu, hi, off);
      const float ol = __shfl_down_sync(0xffffffffu, lo, off);
      ff_add(oh, hi, lo);
      lo += ol;
    }
    if (lane == 0) sh[q][c] = (double)hi + (double)lo;
  }
  __syncthreads();
  if (threadIdx.x < CB && n0 + threadIdx.x < ncol) {
    const int c = threadIdx.x;
    sd->partials[(int64_t)u.m * sd->ldp + u.c * nc + n0 + c] = ((sh[0][c] + sh[1][c]) + sh[2][c]) + sh[3][c];
  }
}

cudaError_t launch_small_reduce_grouped(const SplitUnit* units, int n_units, const TcSegDev* segs, int nc,
                                        cudaStream_t st) {
  if (n_units <= 0) return cudaSuccess;
  k_small_reduce_grouped<<<dim3((unsigned)n_units, (unsigned)(nc / 4)), 128, 0, st>>>(units, segs, nc,
                                                                                    nc > 128 ? nc : 128);
  return cudaGetLastError();
}

static cudaError_t launch_pdl(const void* fn, dim3 grid, dim3 block, size_t smem, cudaStream_t st, void** args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

template <int NSL, int NC>
static cudaError_t launch_small_impl(const TcItem* items, int n_items, const TcSegDev* segs, DevStatus* status,
                                     int64_t lim, cudaStream_t st, const SmallFinal* fin) {
  using C = tsm::Cfg<NSL, NC>;
  static std::atomic<unsigned long long> attr_done{0};
  if (device_needs_setup(attr_done)) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_small<NSL, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    mark_device_done(attr_done);
  }
  if (n_items <= 0) return cudaSuccess;
  int grid = tc_num_sms();
  if (grid > n_items) grid = n_items;
  uint64_t lim64 = (uint64_t)lim;
  SmallFinal f{};
  if (fin) f = *fin;   // logL set: the kernel reduces in-kernel (NC <= 64)
  void* a1[] = {(void*)&items, (void*)&n_items, (void*)&segs, (void*)&status, (void*)&lim64, (void*)&f};
  return launch_pdl((const void*)k_tc_small<NSL, NC>, dim3((unsigned)grid), dim3(tsm::THREADS), C::SMEM, st, a1);
}

cudaError_t launch_tc_small(const TcItem* items, int n_items, const TcSegDev* segs, int nslices, int nc,
                            DevStatus* status, int64_t wait_limit_ns, cudaStream_t st, const SmallFinal* fin) {
  if (fin && nc > 64) return cudaErrorInvalidValue;   // the in-kernel reduction covers NC <= 64
#define TD_SMALL_CASE(NSL_, NC_) \
  if (nslices == NSL_ && nc == NC_)                   \
    return launch_small_impl<NSL_, NC_>(items, n_items, segs, status, wait_limit_ns, st, fin);
  TD_SMALL_CASE(3, 16) TD_SMALL_CASE(4, 16) TD_SMALL_CASE(2, 16)
  TD_SMALL_CASE(3, 32) TD_SMALL_CASE(4, 32) TD_SMALL_CASE(2, 32)
  TD_SMALL_CASE(3, 64) TD_SMALL_CASE(4, 64) TD_SMALL_CASE(2, 64)
  TD_SMALL_CASE(3, 128) TD_SMALL_CASE(4, 128) TD_SMALL_CASE(2, 128)
  TD_SMALL_CASE(3, 256) TD_SMALL_CASE(4, 256) TD_SMALL_CASE(2, 256)
#undef TD_SMALL_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_small_reduce(const TcSegDev* segs, const SmallFinal& fin, cudaStream_t st) {
  const dim3 rgrid(fin.n_units > 0 ? (unsigned)fin.n_units : 1u, fin.n_units > 0 ? (unsigned)((fin.K + 3) / 4) : 1u);
  SmallFinal f = fin;
  void* a2[] = {(void*)&segs, (void*)&f};
  return launch_pdl((const void*)k_small_reduce, rgrid, dim3(128), 0, st, a2);
}

}  // namespace td
