// bf16 slicing of the whitening operator and of residual batches.
//
// Both operands are held as four bf16 slices x = s0 + s1 + s2 + s3: s0 is a
// fixed-point "hi" slice, an integer multiple (|.| <= 255) of a power-of-two
// quantum shared by the whole operator row (resp. residual column), and
// s1..s3 are floating bf16 slices of the remainder.  The hi*hi products of
// one output element are then all multiples of one quantum and their FP32
// tensor-core sum is exact; the remaining products carry the small rest.
//
// Operator: L^{-1} (FP64, computed once per segment), lower triangle packed as
// 256 x 32 blocks: row tile m (256 rows) holds k-blocks kb = 0 .. 8(m+1)-1 of
// 32 columns, at block offset 8 m (m+1) / 2 + kb; each block stores its four
// slices one after another ([block][slice][256][32], row-major) -- the
// tensor-core B operand, read by TMA one k-block (64 KB) at a time.
//
// Residuals: float32 R (N' x K, column-major) -> four bf16 slices laid out
// [slice][k][j] (j contiguous, row stride nkp8): the tensor-core A operand.
// The four slices hold each float32 exactly.
#include <cooperative_groups.h>

#include "td_internal.h"

namespace cg = cooperative_groups;

namespace td {

// Per-row power-of-two quantum q_i of the operator's fixed-point hi slice:
// the smallest 2^e with max_j |Linv_ij| <= 255 q_i, made coarser if needed so
// that sum_j |round(Linv_ij / q_i)| <= 2^16.  Any residual column whose hi
// slice is an integer multiple of its own quantum with magnitude <= 255 then
// gives hi*hi partial sums that are integer multiples of q_i p_k below 2^24
// of them: exactly representable in FP32, so the tensor-core accumulation of
// that product is exact.  (Integers up to 256 are exact in bf16.)
// Column-major L^-1: a block of 32 rows x 8 column groups (warps), so a warp
// reads 32 consecutive rows of one column; the maximum as an integer compare
// of the magnitude bits (exact), the sum of integers |round(x / q_i)| in FP64
// (exact: below 2^53), both in any order -- the same q_i as a row-at-a-time
// scan.  q_i is a power of two, so x / q_i is x * (1 / q_i) exactly.
__global__ void __launch_bounds__(256) k_row_quantum(const double* __restrict__ Linv, int64_t ld, int64_t nk,
                                                     int64_t nkp, double* __restrict__ qrow) {
  __shared__ unsigned long long smx[8][32];
  __shared__ double sl1[8][32];
  __shared__ double sq[32];
  __shared__ int sbad;
  const int r = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * 32 + r;
  const int64_t jmax = (i < nk) ? i : -1;
  const double* row = Linv + i;
  unsigned long long mb = 0ull;
#pragma unroll 4
  for (int64_t j = g; j <= jmax; j += 8)
    mb = max(mb, (unsigned long long)__double_as_longlong(row[j * ld]) & 0x7fffffffffffffffull);
  smx[g][r] = mb;
  __syncthreads();
  if (g == 0) {
    unsigned long long m = smx[0][r];
#pragma unroll
    for (int h = 1; h < 8; ++h) m = max(m, smx[h][r]);
    const double mx = __longlong_as_double((long long)m);
    double q = 1.0;
    if (mx > 0.0) {
      q = ldexp(1.0, (int)ceil(log2(mx / 255.0)));
      if (mx / q > 255.0) q *= 2.0;
    }
    sq[r] = q;
  }
  __syncthreads();
  for (int it = 0; it < 64; ++it) {
    const double q = sq[r];
    const double iq = 1.0 / q;   // exact: q is a power of two
    double l1 = 0.0;
#pragma unroll 4
    for (int64_t j = g; j <= jmax; j += 8) l1 += fabs(rint(row[j * ld] * iq));
    sl1[g][r] = l1;
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    if (g == 0) {
      double t = 0.0;
#pragma unroll
      for (int h = 0; h < 8; ++h) t += sl1[h][r];
      if (t > 65536.0) {
        sq[r] = q * 2.0;
        sbad = 1;
      }
    }
    __syncthreads();
    const int bad = sbad;
    __syncthreads();   // sbad and sl1 are rewritten by the next pass
    if (!bad) break;
  }
  if (g == 0 && i < nkp) qrow[i] = sq[r];
}

// The same quantum for an operator stored row-major (row i at Linv + i ld):
// one warp per row, lanes on consecutive columns.  The maximum and the sum of
// integers are exact in any order, so both layouts give the same q_i.
__global__ void k_row_quantum_rm(const double* __restrict__ Linv, int64_t ld, int64_t nk, int64_t nkp,
                                 double* __restrict__ qrow) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < nkp; i += nw) {
    const double* row = Linv + i * ld;
    const int64_t jmax = (i < nk) ? i : -1;
    double mx = 0.0;
    for (int64_t j = lane; j <= jmax; j += 32) mx = fmax(mx, fabs(row[j]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    double q = 1.0;
    if (mx > 0.0) {
      q = ldexp(1.0, (int)ceil(log2(mx / 255.0)));
      if (mx / q > 255.0) q *= 2.0;
      for (int it = 0; it < 64; ++it) {
        double l1 = 0.0;
        const double iq = 1.0 / q;   // exact: q is a power of two
        for (int64_t j = lane; j <= jmax; j += 32) l1 += fabs(rint(row[j] * iq));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) l1 += __shfl_xor_sync(0xffffffffu, l1, off);
        if (l1 <= 65536.0) break;
        q *= 2.0;
      }
    }
    if (lane == 0) qrow[i] = q;
  }
}

cudaError_t launch_row_quantum(const double* Linv, int64_t ld, int64_t nk, int64_t nkp, double* qrow,
                               cudaStream_t st, bool row_major) {
  if (row_major) {
    const int64_t blocks = ceil_div(nkp, 8);
    k_row_quantum_rm<<<(unsigned)(blocks < 65535 * 4 ? blocks : 65535 * 4), 256, 0, st>>>(Linv, ld, nk, nkp, qrow);
  } else {
    k_row_quantum<<<(unsigned)ceil_div(nkp, 32), 256, 0, st>>>(Linv, ld, nk, nkp, qrow);
  }
  return cudaGetLastError();
}

// x = q a0 + r,  a0 = rint(x / q) (|a0| <= 255, exact in bf16 as q a0),
// r = x - q a0 split into three floating bf16 slices.
__device__ __forceinline__ void split4_fixed_f64(double x, double q, double iq, __nv_bfloat16 (&s)[4]) {
  const double hi = q * rint(x * iq);   // iq = 1 / q exactly (q a power of two)
  s[0] = __double2bfloat16(hi);
  split3_f64(x - hi, s[1], s[2], s[3]);
}

template <bool RM>
__global__ void __launch_bounds__(256) k_op_slices(const double* __restrict__ Linv, int64_t ld, int64_t nk,
                                                    const double* __restrict__ qrow,
                                                    __nv_bfloat16* __restrict__ op) {
  const int m = blockIdx.y, kb = blockIdx.x;
  if (kb >= (OP_ROWS / OP_KB) * (m + 1)) return;
  const int r = threadIdx.x;
  const int64_t i = (int64_t)m * OP_ROWS + r;
  const int64_t blk = (OP_ROWS / OP_KB) * (int64_t)m * (m + 1) / 2 + kb;
  const double q = qrow[i];
  const double iq = 1.0 / q;
  __align__(16) __nv_bfloat16 sl[OP_SLICES][OP_KB];
#pragma unroll 4
  for (int c = 0; c < OP_KB; ++c) {
    const int64_t j = (int64_t)kb * OP_KB + c;
    const double x = (i < nk && j < nk && j <= i) ? Linv[RM ? i * ld + j : i + j * ld] : 0.0;
    __nv_bfloat16 s4[4];
    split4_fixed_f64(x, q, iq, s4);
#pragma unroll
    for (int u = 0; u < OP_SLICES; ++u) sl[u][c] = s4[u];
  }
  __nv_bfloat16* base = op + (blk * OP_SLICES) * (OP_ROWS * OP_KB) + (int64_t)r * OP_KB;
#pragma unroll
  for (int u = 0; u < OP_SLICES; ++u) {
    const uint4* v = reinterpret_cast<const uint4*>(sl[u]);
    uint4* d = reinterpret_cast<uint4*>(base + (int64_t)u * OP_ROWS * OP_KB);
#pragma unroll
    for (int w = 0; w < OP_KB * 2 / 16; ++w) d[w] = v[w];
  }
}

cudaError_t launch_op_slices(const double* Linv, int64_t ld, int64_t nk, int64_t nkp, const double* qrow,
                             __nv_bfloat16* op, cudaStream_t st, bool row_major) {
  const int nm = (int)(nkp / OP_ROWS);
  dim3 grid((OP_ROWS / OP_KB) * nm, nm);
  if (row_major)
    k_op_slices<true><<<grid, OP_ROWS, 0, st>>>(Linv, ld, nk, qrow, op);
  else
    k_op_slices<false><<<grid, OP_ROWS, 0, st>>>(Linv, ld, nk, qrow, op);
  return cudaGetLastError();
}

// Residual slices (r_quantum, r_slice_value): rows j0 .. j1-1 of one column.
__device__ __forceinline__ void r_slice_rows(const float* __restrict__ col, int64_t j0, int64_t j1, float p,
                                             __nv_bfloat16* __restrict__ dst, int64_t slice_stride, int nslices) {
  for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
    __nv_bfloat16 o[4];
    r_slice_value(col[j], p, o);
    dst[j] = o[0];
    dst[j + slice_stride] = o[1];
    if (nslices > 2) dst[j + 2 * slice_stride] = o[2];
    if (nslices > 3) dst[j + 3 * slice_stride] = o[3];
  }
}

__device__ __forceinline__ float block_max256(float mx, float* red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  mx = red[0];
#pragma unroll
  for (int w = 1; w < 8; ++w) mx = fmaxf(mx, red[w]);
  __syncthreads();
  return mx;
}

// The dependent kernel (the tensor-core product) may start streaming the
// operator while this one runs; it waits for this grid before reading rs.
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
// Launched as a programmatic dependent (small batches), the kernel may start
// while the preceding launch runs: nothing is read or written before this
// wait (a no-op otherwise).
__device__ __forceinline__ void pdl_wait_prior() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// one CTA per column (large batches)
__global__ void __launch_bounds__(256) k_r_slices(const float* __restrict__ R, int64_t ldr, int64_t nk, int64_t K,
                                                   int64_t nkp8, int64_t capK, __nv_bfloat16* __restrict__ rs,
                                                   int nslices, int* __restrict__ zero, int nzero) {
  __shared__ float red[8];
  pdl_launch_dependents();
  pdl_wait_prior();
  if (zero && blockIdx.x == 0)
    for (int i = threadIdx.x; i < nzero; i += blockDim.x) zero[i] = 0;
  const int64_t slice_stride = capK * nkp8;
  for (int64_t k = blockIdx.x; k < K; k += gridDim.x) {
    const float* col = R + k * ldr;
    float mx = 0.f;
    for (int64_t j = threadIdx.x; j < nk; j += blockDim.x) mx = fmaxf(mx, fabsf(col[j]));
    const float p = r_quantum(block_max256(mx, red));
    r_slice_rows(col, 0, nk, p, rs + k * nkp8, slice_stride, nslices);
  }
}

// one CTA per column, the column held in registers (one read of R): THREADS
// threads x V float4 each cover up to 4 V THREADS rows; 16-byte loads, 8-byte
// stores of four bf16 per slice.  Needs ldr, N' multiples of 4 and R 16-byte
// aligned (the launcher checks).
template <int THREADS, int V>
__global__ void __launch_bounds__(THREADS) k_r_slices_reg(const float* __restrict__ R, int64_t ldr, int64_t nk,
                                                          int64_t K, int64_t nkp8, int64_t capK,
                                                          __nv_bfloat16* __restrict__ rs, int nslices,
                                                          int* __restrict__ zero, int nzero) {
  __shared__ float red[THREADS / 32];
  pdl_launch_dependents();
  pdl_wait_prior();
  if (zero && blockIdx.x == 0)
    for (int i = threadIdx.x; i < nzero; i += blockDim.x) zero[i] = 0;
  const int64_t k = blockIdx.x;
  const float4* col = reinterpret_cast<const float4*>(R + k * ldr);
  const int64_t nv = nk / 4;
  float4 x[V];
  float mx = 0.f;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int64_t i = threadIdx.x + (int64_t)v * THREADS;
    x[v] = i < nv ? col[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    mx = fmaxf(mx, fmaxf(fmaxf(fabsf(x[v].x), fabsf(x[v].y)), fmaxf(fabsf(x[v].z), fabsf(x[v].w))));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  mx = red[0];
#pragma unroll
  for (int w = 1; w < THREADS / 32; ++w) mx = fmaxf(mx, red[w]);
  const float p = r_quantum(mx);
  const int64_t slice_stride = capK * nkp8;
  __nv_bfloat16* dst = rs + k * nkp8;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int64_t i = threadIdx.x + (int64_t)v * THREADS;
    if (i >= nv) break;
    const float xs[4] = {x[v].x, x[v].y, x[v].z, x[v].w};
    __align__(8) __nv_bfloat16 o[4][4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      __nv_bfloat16 t[4];
      r_slice_value(xs[e], p, t);
#pragma unroll
      for (int u = 0; u < 4; ++u) o[u][e] = t[u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (u < nslices) *reinterpret_cast<uint2*>(dst + u * slice_stride + 4 * i) = *reinterpret_cast<const uint2*>(o[u]);
  }
}

// a cluster of RS_CL CTAs per column (small batches: more SMs on the few
// columns); the column maximum is combined through distributed shared memory.
// The maximum is exact in any order, so p_k equals the one-CTA kernel's.
constexpr int RS_CL = 8;
__global__ void __cluster_dims__(RS_CL, 1, 1) __launch_bounds__(256)
    k_r_slices_cl(const float* __restrict__ R, int64_t ldr, int64_t nk, int64_t K, int64_t nkp8, int64_t capK,
                  __nv_bfloat16* __restrict__ rs, int nslices, int* __restrict__ zero, int nzero) {
  __shared__ float red[8];
  __shared__ float cmax;
  pdl_launch_dependents();
  pdl_wait_prior();
  if (zero && blockIdx.x == 0)
    for (int i = threadIdx.x; i < nzero; i += blockDim.x) zero[i] = 0;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int64_t k = blockIdx.x / RS_CL;
  const int64_t per = (nk + RS_CL - 1) / RS_CL;
  const int64_t j0 = rank * per, j1 = (j0 + per < nk) ? j0 + per : nk;
  const float* col = R + k * ldr;
  float mx = 0.f;
  for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) mx = fmaxf(mx, fabsf(col[j]));
  mx = block_max256(mx, red);
  if (threadIdx.x == 0) cmax = mx;
  cl.sync();
  float g = 0.f;
#pragma unroll
  for (int r = 0; r < RS_CL; ++r) g = fmaxf(g, *cl.map_shared_rank(&cmax, r));
  cl.sync();   // every CTA has read its peers' maxima before any of them exits
  r_slice_rows(col, j0, j1, r_quantum(g), rs + k * nkp8, capK * nkp8, nslices);
}

cudaError_t launch_r_slices(const float* R, int64_t ldr, int64_t nk, int64_t K, int64_t nkp8, int64_t capK,
                            __nv_bfloat16* rs, int nslices, cudaStream_t st, int* zero, int nzero, bool pdl) {
  if (K <= 0) return cudaSuccess;
  const bool reg_ok = K <= 2147483647LL && ldr % 4 == 0 && nk % 4 == 0 &&
                      (reinterpret_cast<uintptr_t>(R) & 15) == 0 && nk <= 4 * 8 * 1024;
  auto launch_pdl = [&](auto kern, unsigned grid, unsigned block) -> cudaError_t {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, R, ldr, nk, K, nkp8, capK, rs, nslices, zero, nzero);
  };
  if (K <= 64 && reg_ok) {
    // up to 64 columns: one 1024-thread CTA per column, the column in
    // registers (one read, one block barrier, no cluster barriers); measured
    // at N' = 8192 a call of 4 columns 49.1 against 50.1 us with the cluster
    // form, of 32 columns 56.7 against 60
    if (pdl) return launch_pdl(k_r_slices_reg<1024, 8>, (unsigned)K, 1024u);
    k_r_slices_reg<1024, 8><<<(unsigned)K, 1024, 0, st>>>(R, ldr, nk, K, nkp8, capK, rs, nslices, zero, nzero);
  } else if (K <= 64 || (K <= 256 && !reg_ok)) {
    // few columns, unaligned or longer than 32768 rows: a cluster per column
    // puts more SMs on them
    if (pdl) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(K * RS_CL));
      cfg.blockDim = dim3(256);
      cfg.dynamicSmemBytes = 0;
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      return cudaLaunchKernelEx(&cfg, k_r_slices_cl, R, ldr, nk, K, nkp8, capK, rs, nslices, zero, nzero);
    }
    k_r_slices_cl<<<(unsigned)(K * RS_CL), 256, 0, st>>>(R, ldr, nk, K, nkp8, capK, rs, nslices, zero, nzero);
  } else if (reg_ok) {
    // column in registers: 8 float4 per thread (at K = 256, N' = 8192: one
    // read of R instead of the cluster form's two, and no cluster barriers)
    const unsigned grid = (unsigned)K;
    if (nk <= 4 * 8 * 256)
      k_r_slices_reg<256, 8><<<grid, 256, 0, st>>>(R, ldr, nk, K, nkp8, capK, rs, nslices, zero, nzero);
    else if (nk <= 4 * 8 * 512)
      k_r_slices_reg<512, 8><<<grid, 512, 0, st>>>(R, ldr, nk, K, nkp8, capK, rs, nslices, zero, nzero);
    else
      k_r_slices_reg<1024, 8><<<grid, 1024, 0, st>>>(R, ldr, nk, K, nkp8, capK, rs, nslices, zero, nzero);
  } else {
    const int grid = (int)(K < 4096 ? K : 4096);
    k_r_slices<<<grid, 256, 0, st>>>(R, ldr, nk, K, nkp8, capK, rs, nslices, zero, nzero);
  }
  return cudaGetLastError();
}

}  // namespace td
