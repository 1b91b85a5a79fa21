// FP64-accurate matrix products on the bf16 tensor cores (tcgen05), for the
// covariance factor C = L L^T and its inverse (Sec. II.A, the Cholesky
// whitening; Sec. III.A, "Factorization of the covariance matrix": O(N^3),
// once per segment).  B300's FP64 rate (about 1.2 TF/s on the CUDA cores) is
// far below its bf16 tensor rate, so the O(N^3) part of the factor runs as
// split products on the tensor cores instead.
//
// Splitting (error-free transformation of the operands into exact bf16
// slices, after Ozaki, Ogita, Oishi and Rump): one operand row is a run of
// EK = 128 FP64 values sharing one power of two 2^e, with e chosen from the
// row's largest magnitude so that x = 2^e sum_{s < NS} a_s 2^{-8s} with
// integers |a_0| <= 256 and |a_s| <= 128 for s >= 1 (round to nearest at each
// step; the remainder after NS slices is below 2^{-8(NS-1)-1}).  Each
// a_s 2^{-8s} is exact in bf16 (8 significant bits).
//
// Products: D = alpha A B^T + beta D over K = EK, A and B given as slices.
// The product of slices s and t has weight 2^{-8(s+t)}; products of the same
// level l = s + t (l < NS) share an FP32 accumulator in tensor memory, one per
// level.  With K = 128, in units of the level's weight, the level sums are
// below 2^24 for every l <= 5 (level 0: 128 * 256^2 = 2^23; level l >= 1:
// 128 * (2 * 256 * 128 + (l - 1) * 128^2) <= 2^24), so each is an integer sum
// that FP32 holds exactly and its tensor-core accumulation is exact.  Levels
// >= NS are not formed (about 2^-47 of sum |a||b| for NS = 6, 2^-39 for
// NS = 5), and the operand remainders after NS slices are of the same order.
// The epilogue adds the accumulators smallest first as an FP32 pair with
// error-free additions and scales by 2^{ea+eb}.
//
// One MMA covers one A slice s against the B slices 0 .. NS-1-s, which sit
// next to each other in shared memory, so that N runs over the levels s ..
// NS-1 and the D columns of level l start at 64 l: B's stage is read as one
// operand of up to 256 rows (four levels) instead of once per pair: NS = 6
// takes 8 MMAs of N = 64 .. 256 per 16-deep step instead of 21 of N = 64, and
// reads 74 KB of shared memory instead of 126 KB for the same 672 cycles of
// tensor work (at 128 B per clock the pairwise form was bound by shared
// memory, this one by the tensor pipe).
//
// Tiles: 128 rows (TMEM lanes) x 64 columns, K = 128 in four k-blocks of 32
// (64-byte swizzle); a 3-stage TMA ring of (A, B) slice stages.  TMEM holds
// one set of NS accumulators (64 columns each); the epilogue copies them to
// registers and frees them before its global read-modify-write, so the MMAs
// of the next tile overlap that traffic.  One launch serves up to two
// problems (a tile list over both); a problem is rectangular or the lower
// triangle of a square output.
//
// Warp roles (320 threads, one CTA per SM):
//   warp 0 lane 0 : TMA producer
//   warp 1        : TMEM allocator; lane 0 issues tcgen05.mma
//   warps 2..9    : epilogue, warp w on TMEM lanes 32 (w & 3) .. + 31 and
//                   columns 32 ((w - 2) / 4) .. + 31 of the tile
// Every wait is bounded (the caller's limit); on expiry the kernel records
// TD_ERR_TIMEOUT, drains its own copies and MMAs, frees TMEM and returns.
#include <algorithm>
#include <cmath>

#include "emu_gemm.h"

namespace td {
namespace emu {
constexpr int BM = 128, BN = 64, BK = 32;
constexpr int THREADS = 320;
constexpr int EPI_WARPS = 8;
constexpr int A_SLICE = BM * BK * 2;   // 8 KB
constexpr int B_SLICE = BN * BK * 2;   // 4 KB
constexpr int NACC_MAX = 6;
template <int NS> struct Cfg {
  static constexpr int STAGE = NS * (A_SLICE + B_SLICE);
  static constexpr int STAGES = 3;
  static constexpr int SMEM = STAGES * STAGE + 256 + 1024;
};
static_assert(Cfg<6>::SMEM <= 227 * 1024, "shared memory");
static_assert(NACC_MAX * BN <= 512, "tensor memory");
}  // namespace emu

// The MMAs of one 16-deep step: A slice s against B slices t0 .. t0+n-1
// (levels s+t0 .. s+t0+n-1, N = 64 n <= 256).  The s = 0 MMAs come first and
// cover every level, so they alone start the accumulators of a tile.
template <int NS>
struct Mmas {
  int s[2 * NS], t0[2 * NS], n[2 * NS];
  int count;
  __host__ __device__ constexpr Mmas() : s(), t0(), n(), count(0) {
    for (int a = 0; a < NS; ++a)
      for (int t = 0; t < NS - a; t += 4) {
        s[count] = a;
        t0[count] = t;
        n[count] = (NS - a - t) < 4 ? (NS - a - t) : 4;
        ++count;
      }
  }
};

// f 2^sc as a double, assembled from f's bits with integer operations (no FP64
// instruction); f = 0 or subnormal gives 0, and sc keeps the result within
// the normal double range for every value the factor forms
__device__ __forceinline__ double f32_to_f64_scaled(float f, int sc) {
  const uint32_t u = __float_as_uint(f);
  const int ex = (int)((u >> 23) & 0xFFu);
  const int e64 = ex + (1023 - 127) + sc;
  if (ex == 0 || e64 <= 0) return 0.0;
  const uint64_t bits = ((uint64_t)(u >> 31) << 63) | ((uint64_t)(e64 < 2047 ? e64 : 2047) << 52) |
                        ((uint64_t)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ void emu_tile(const EmuParams& P, int tile, int& prob, int& mi, int& ni) {
  prob = (P.nprob > 1 && tile >= P.p[1].tile_begin) ? 1 : 0;
  const EmuProb& q = P.p[prob];
  const int u = tile - q.tile_begin;
  if (q.lower) {
    // row tile r holds column tiles 0 .. 2r+1 (64 columns against 128 rows):
    // u = r (r + 1) + c
    int r = (int)((sqrt(4.0 * (double)u + 1.0) - 1.0) * 0.5);
    while ((r + 1) * (r + 2) <= u) ++r;
    while (r * (r + 1) > u) --r;
    mi = r;
    ni = u - r * (r + 1);
  } else {
    mi = u / q.n_tiles;
    ni = u - mi * q.n_tiles;
  }
}

template <int NS>
__global__ void __launch_bounds__(emu::THREADS, 1)
    k_emu_gemm(const __grid_constant__ EmuParams P, DevStatus* status, uint64_t limit_ns) {
  using namespace emu;
  using C = Cfg<NS>;
  constexpr int STAGE = C::STAGE, STAGES = C::STAGES;
  constexpr int A_STAGE = NS * A_SLICE;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 1;
  uint64_t* fin = tempty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, EPI_WARPS);
    mbar_init(fin, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int G = gridDim.x, b = blockIdx.x;
  const int n_total = P.total_tiles;

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------ TMA producer
      for (int q = 0; q < P.nprob; ++q) {
        prefetch_tmap(&P.p[q].mapA);
        prefetch_tmap(&P.p[q].mapB);
      }
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued_mask = 0, issued_phase = 0;
      for (int tile = b; tile < n_total && !*abort_flag; tile += G) {
        int prob, mi, ni;
        emu_tile(P, tile, prob, mi, ni);
        const EmuProb& q = P.p[prob];
        bool ok = true;
        for (int kb = 0; kb < EK / BK; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, limit_ns)) {
            set_status(status, ST_TIMEOUT, 60);
            *abort_flag = 1;
            ok = false;
            break;
          }
          uint8_t* sa = smem + stage * STAGE;
          mbar_arrive_expect_tx(&full[stage], (uint32_t)STAGE);
          tma_load_3d(sa, &q.mapA, &full[stage], kb * BK, q.a_row0 + mi * BM, 0);
          tma_load_3d(sa + A_STAGE, &q.mapB, &full[stage], kb * BK, q.b_row0 + ni * BN, 0);
          issued_mask |= 1u << stage;
          issued_phase = (issued_phase & ~(1u << stage)) | (phase << stage);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
      }
      for (int s = 0; s < STAGES; ++s)   // every issued copy lands before the CTA exits
        if (issued_mask & (1u << s)) mbar_wait(&full[s], (issued_phase >> s) & 1u, limit_ns);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------ MMA issuer
      constexpr Mmas<NS> MM{};
      int stage = 0;
      uint32_t phase = 0;
      int tl = 0;
      for (int tile = b; tile < n_total && !*abort_flag; tile += G, ++tl) {
        if (!mbar_wait(tempty, ((uint32_t)tl & 1u) ^ 1u, limit_ns)) {
          set_status(status, ST_TIMEOUT, 61);
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        bool ok = true;
        for (int kb = 0; kb < EK / BK; ++kb) {
          if (!mbar_wait(&full[stage], phase, limit_ns)) {
            set_status(status, ST_TIMEOUT, 62);
            *abort_flag = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + stage * STAGE);
          // descriptors of every slice are the stage's plus the slice offset
          // (in 16-byte units, the start-address field)
          const uint64_t ad0 = smem_desc_sw64(sa), bd0 = smem_desc_sw64(sa + A_STAGE);
          const uint32_t fresh = kb == 0 ? 0u : 1u;   // 0: this tile's first k-block
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {
#pragma unroll
            for (int i = 0; i < MM.count; ++i) {
              const uint32_t accumulate = (kk > 0 || MM.s[i] > 0) ? 1u : fresh;
              tc_mma_f16(tmem_base + (uint32_t)((MM.s[i] + MM.t0[i]) * BN),
                         ad0 + (uint64_t)((MM.s[i] * A_SLICE + kk * 32) >> 4),
                         bd0 + (uint64_t)((MM.t0[i] * B_SLICE + kk * 32) >> 4), idesc_bf16_f32(BM, BN * MM.n[i]),
                         accumulate);
            }
          }
          tc_commit(&empty[stage]);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        tc_commit(tfull);
      }
      tc_commit(fin);
      mbar_wait(fin, 0, limit_ns);
    }
  } else {
    // -------------------------------------------------- epilogue (warps 2..9)
    const int qd = warp & 3, half = (warp - 2) >> 2;
    int tl = 0;
    for (int tile = b; tile < n_total && !*abort_flag; tile += G, ++tl) {
      int prob, mi, ni;
      emu_tile(P, tile, prob, mi, ni);
      const EmuProb& q = P.p[prob];
      if (!mbar_wait(tfull, (uint32_t)tl & 1u, limit_ns)) {
        if (lane == 0) set_status(status, ST_TIMEOUT, 63);
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const uint32_t ta = tmem_base + ((uint32_t)(qd * 32) << 16) + (uint32_t)(half * 32);
      // the five accumulators summed smallest first as an FP32 pair (hi, lo)
      // with error-free additions: B300's FP64 rate is a few operations per
      // clock per SM, so FP64 is kept to the final one or two additions
      float hi[32], lo[32];
      tmem_ld32(ta + (uint32_t)((NS - 1) * BN), hi);
#pragma unroll
      for (int j = 0; j < 32; ++j) lo[j] = 0.f;
#pragma unroll
      for (int ac = NS - 2; ac >= 0; --ac) {
        float v[32];
        tmem_ld32(ta + (uint32_t)(ac * BN), v);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float sm = hi[j] + v[j];
          const float bb = sm - hi[j];
          lo[j] += (hi[j] - (sm - bb)) + (v[j] - bb);
          hi[j] = sm;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty);   // the accumulators are free for the next tile
      const int row = mi * BM + qd * 32 + lane;
      const int ea = q.ea[q.a_row0 + row];
      const int col0 = ni * BN + half * 32;
      double* crow = q.C + row;
      // per half of the columns, every load first (the exponents, then the
      // old values: 16 loads in flight, one memory latency), then the
      // arithmetic, then the stores -- loads interleaved with stores to
      // possibly aliasing addresses would wait out one latency per column
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        int sc[16];
        double v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) sc[j] = ea + __ldg(q.eb + q.b_row0 + col0 + 16 * hh + j);
        if (q.beta != 0.0) {
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = crow[(int64_t)(col0 + 16 * hh + j) * q.ldc];
        }
        if (q.beta == 1.0 && q.alpha == -1.0) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            v[j] = (v[j] - f32_to_f64_scaled(hi[16 * hh + j], sc[j])) - f32_to_f64_scaled(lo[16 * hh + j], sc[j]);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const double w = f32_to_f64_scaled(hi[16 * hh + j], sc[j]) + f32_to_f64_scaled(lo[16 * hh + j], sc[j]);
            v[j] = q.beta == 0.0 ? (q.alpha == 1.0 ? w : q.alpha * w) : fma(q.alpha, w, q.beta * v[j]);
          }
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) crow[(int64_t)(col0 + 16 * hh + j) * q.ldc] = v[j];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 512);
  }
}

// ---------------------------------------------------------------- splitting
// One CTA: 32 operand rows x EK values of one job, staged through shared
// memory so that both source layouts read coalesced; warp w splits rows
// 4w .. 4w+3, lane l values 4l .. 4l+3.  The digits come from the doubles'
// bits by integer arithmetic (no FP64 instruction): |x| 2^{8-E+8(NS-1)} is
// rounded to an integer X < 2^{8 NS} (E the exponent of the row's largest
// |x|), then split into balanced base-256 digits from the bottom
// (a_s in [-127, 128] for s >= 1, a_0 <= 256), each exact in bf16.
template <int NS>
__device__ __forceinline__ void split_value(uint64_t bits, int ex_max, __nv_bfloat16 (&h)[NS]) {
  const int ex = (int)((bits >> 52) & 0x7FF);
  uint64_t X = 0;
  const int sh = ex_max - ex + 53 - 8 * NS;   // |x| 2^{8 - E + 8(NS-1)} = M 2^{-sh}
  if (ex != 0 && sh < 63) {
    const uint64_t M = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    X = sh > 0 ? (M + (1ull << (sh - 1))) >> sh : M << (-sh);
  }
  int a[NS];
#pragma unroll
  for (int t = NS - 1; t >= 1; --t) {
    int d = (int)(X & 0xFFu);
    X >>= 8;
    if (d > 128) {
      d -= 256;
      X += 1;
    }
    a[t] = d;
  }
  a[0] = (int)X;
  const bool neg = (bits >> 63) != 0;
#pragma unroll
  for (int t = 0; t < NS; ++t) {
    const float v = (float)(neg ? -a[t] : a[t]) * __int_as_float((127 - 8 * t) << 23);   // a_t 2^{-8t}, exact
    h[t] = __float2bfloat16_rn(v);
  }
}

template <int NS>
__global__ void __launch_bounds__(256) k_emu_split(const EmuSplitParams P) {
  __shared__ uint64_t tile[32][EK + 1];
  int j = 0;
  while (j + 1 < P.njobs && (int)blockIdx.x >= P.job[j + 1].block0) ++j;
  const EmuSplitJob& J = P.job[j];
  const int r0 = ((int)blockIdx.x - J.block0) * 32;
  const int tid = threadIdx.x;
  const int nvalid = J.rows_valid < J.rows ? J.rows_valid : J.rows;
  // the value's double bits (an FP32 value converts exactly), zero outside
  auto value = [&](int r, int k) -> uint64_t {
    if (r >= nvalid || k >= J.k_valid || (J.lower && k > r)) return 0ull;
    const int64_t off = (int64_t)r * J.rs + (int64_t)k * J.ks;
    if (J.src_f32) {   // FP32 bits -> FP64 bits with integer operations (subnormal FP32 as zero)
      const uint32_t u = __float_as_uint(reinterpret_cast<const float*>(J.src)[off]);
      const uint32_t ex = (u >> 23) & 0xFFu;
      if (ex == 0) return 0ull;
      return ((uint64_t)(u >> 31) << 63) | ((uint64_t)(ex + 896u) << 52) | ((uint64_t)(u & 0x7FFFFFu) << 29);
    }
    return reinterpret_cast<const uint64_t*>(J.src)[off];
  };
  if (J.rs == 1) {            // rows contiguous: 32 rows per k
    for (int idx = tid; idx < 32 * EK; idx += 256) {
      const int r = idx & 31, k = idx >> 5;
      tile[r][k] = value(r0 + r, k);
    }
  } else {                    // values of a row contiguous
    for (int idx = tid; idx < 32 * EK; idx += 256) {
      const int k = idx % EK, r = idx / EK;
      tile[r][k] = value(r0 + r, k);
    }
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  for (int rr = 0; rr < 4; ++rr) {
    const int r = warp * 4 + rr;
    const int grow = r0 + r;
    if (grow >= J.rows) break;
    uint64_t b[4];
    uint64_t mx = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      b[i] = tile[r][4 * lane + i];
      const uint64_t m = b[i] & 0x7FFFFFFFFFFFFFFFull;   // |x| orders like its bits
      mx = m > mx ? m : mx;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const uint64_t o = __shfl_xor_sync(0xffffffffu, mx, off);
      mx = o > mx ? o : mx;
    }
    const int ex_max = (int)(mx >> 52);
    __nv_bfloat16 h[4][NS];
#pragma unroll
    for (int i = 0; i < 4; ++i) split_value<NS>(ex_max ? b[i] : 0ull, ex_max, h[i]);
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      uint2 pk;
      pk.x = (uint32_t)__bfloat16_as_ushort(h[0][t]) | ((uint32_t)__bfloat16_as_ushort(h[1][t]) << 16);
      pk.y = (uint32_t)__bfloat16_as_ushort(h[2][t]) | ((uint32_t)__bfloat16_as_ushort(h[3][t]) << 16);
      *reinterpret_cast<uint2*>(J.dst + ((int64_t)t * J.rows_alloc + grow) * EK + 4 * lane) = pk;
    }
    // max = f 2^E with f in [1/2, 1): E = ex_max - 1022; values are 2^{E-8} sum a_t 2^{-8t}
    if (lane == 0) J.e[grow] = ex_max ? ex_max - 1022 - 8 : 0;
  }
}

cudaError_t launch_emu_split(const EmuSplitParams& P, cudaStream_t st) {
  if (P.njobs <= 0 || P.total_blocks <= 0) return cudaSuccess;
  const int ns = P.job[0].ns;
  if (ns == 6)
    k_emu_split<6><<<P.total_blocks, 256, 0, st>>>(P);
  else if (ns == 5)
    k_emu_split<5><<<P.total_blocks, 256, 0, st>>>(P);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <int NS>
static cudaError_t emu_launch(const EmuParams& P, DevStatus* status, int64_t limit_ns, cudaStream_t st,
                              int max_ctas) {
  static std::atomic<unsigned long long> done{0};
  if (device_needs_setup(done)) {
    cudaError_t e = cudaFuncSetAttribute(k_emu_gemm<NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         emu::Cfg<NS>::SMEM);
    if (e != cudaSuccess) return e;
    mark_device_done(done);
  }
  int grid = (int)std::min<int64_t>(P.total_tiles, tc_num_sms());
  if (max_ctas > 0 && grid > max_ctas) grid = max_ctas;
  k_emu_gemm<NS><<<grid, emu::THREADS, emu::Cfg<NS>::SMEM, st>>>(P, status, (uint64_t)limit_ns);
  return cudaGetLastError();
}

cudaError_t launch_emu_gemm(const EmuParams& P, int ns, DevStatus* status, int64_t limit_ns, cudaStream_t st,
                            int max_ctas) {
  if (P.total_tiles <= 0) return cudaSuccess;
  if (ns == 5) return emu_launch<5>(P, status, limit_ns, st, max_ctas);
  if (ns == 6) return emu_launch<6>(P, status, limit_ns, st, max_ctas);
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- host helpers
td_status slice_buf(SliceBuf& b, int rows, int ns) {
  b.rows = rows;
  b.v = nullptr;
  b.e = nullptr;
  if (cudaMalloc((void**)&b.v, (size_t)ns * rows * EK * sizeof(__nv_bfloat16)) != cudaSuccess ||
      cudaMalloc((void**)&b.e, (size_t)rows * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    free_slice_buf(b);
    return fail(TD_ERR_OOM, "device allocation failed: operand slices");
  }
  td_status r = encode_3d(&b.boxA, b.v, EK, (uint64_t)rows, (uint64_t)ns, EK * 2, (uint64_t)rows * EK * 2, 32,
                          128, (uint32_t)ns);
  if (r == TD_OK)
    r = encode_3d(&b.boxB, b.v, EK, (uint64_t)rows, (uint64_t)ns, EK * 2, (uint64_t)rows * EK * 2, 32, 64,
                  (uint32_t)ns);
  return r;
}

void free_slice_buf(SliceBuf& b) {
  if (b.v) cudaFree(b.v);
  if (b.e) cudaFree(b.e);
  b.v = nullptr;
  b.e = nullptr;
}

void add_split_job(EmuSplitParams& P, const void* src, int64_t rs, int64_t ks, int rows, SliceBuf& dst, int ns,
                   bool src_f32, int rows_valid, bool lower, int k_valid) {
  if (rows <= 0) return;
  EmuSplitJob& j = P.job[P.njobs++];
  j.src = src;
  j.rs = rs;
  j.ks = ks;
  j.rows = rows;
  j.rows_alloc = dst.rows;
  j.dst = dst.v;
  j.e = dst.e;
  j.ns = ns;
  j.src_f32 = src_f32 ? 1 : 0;
  j.rows_valid = rows_valid < 0 ? rows : rows_valid;
  j.lower = lower ? 1 : 0;
  j.k_valid = k_valid;
  j.block0 = P.total_blocks;
  P.total_blocks += (rows + 31) / 32;
}

void add_product(EmuParams& P, const SliceBuf& A, const SliceBuf& B, double* C, int64_t ldc, double alpha,
                 double beta, int m_tiles, int n_tiles, bool lower, int a_row0, int b_row0) {
  if (m_tiles <= 0 || n_tiles <= 0) return;
  EmuProb& q = P.p[P.nprob++];
  q.mapA = A.boxA;
  q.mapB = B.boxB;
  q.ea = A.e;
  q.eb = B.e;
  q.C = C;
  q.ldc = ldc;
  q.alpha = alpha;
  q.beta = beta;
  q.a_row0 = a_row0;
  q.b_row0 = b_row0;
  q.m_tiles = m_tiles;
  q.n_tiles = n_tiles;
  q.lower = lower ? 1 : 0;
  q.tile_begin = P.total_tiles;
  P.total_tiles += emu_tiles(q);
}

}  // namespace td
