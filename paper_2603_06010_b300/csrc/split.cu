// bf16 slicing of the whitening operator and of residual batches.
//
// Operator: L^{-1} (FP64, computed once per segment) is stored as three
// bf16 slices x = s0 + s1 + s2 of its lower triangle, packed as 256 x 32
// blocks: row tile m (256 rows) holds k-blocks kb = 0 .. 8(m+1)-1 of 32
// columns, at block offset 8 m (m+1) / 2 + kb; each block stores its three
// slices one after another ([block][slice][256][32], row-major).  This is the
// tensor-core B operand, read by TMA one k-block (48 KB) at a time.
//
// Residuals: float32 R (N' x K, column-major) -> three bf16 slices laid out
// [slice][k][j] (j contiguous, row stride nkp8): the tensor-core A operand.
// Three slices hold a float32 exactly.
#include "td_internal.h"

namespace td {

__global__ void __launch_bounds__(256) k_op_slices(const double* __restrict__ Linv, int64_t ld, int64_t nk,
                                                    __nv_bfloat16* __restrict__ op) {
  const int m = blockIdx.y, kb = blockIdx.x;
  if (kb >= (OP_ROWS / OP_KB) * (m + 1)) return;
  const int r = threadIdx.x;
  const int64_t i = (int64_t)m * OP_ROWS + r;
  const int64_t blk = (OP_ROWS / OP_KB) * (int64_t)m * (m + 1) / 2 + kb;
  __align__(16) __nv_bfloat16 s0[OP_KB], s1[OP_KB], s2[OP_KB];
#pragma unroll 4
  for (int c = 0; c < OP_KB; ++c) {
    const int64_t j = (int64_t)kb * OP_KB + c;
    const double x = (i < nk && j < nk && j <= i) ? Linv[i + j * ld] : 0.0;
    split3_f64(x, s0[c], s1[c], s2[c]);
  }
  __nv_bfloat16* base = op + (blk * 3) * (OP_ROWS * OP_KB) + (int64_t)r * OP_KB;
  const uint4* v0 = reinterpret_cast<const uint4*>(s0);
  const uint4* v1 = reinterpret_cast<const uint4*>(s1);
  const uint4* v2 = reinterpret_cast<const uint4*>(s2);
  uint4* d0 = reinterpret_cast<uint4*>(base);
  uint4* d1 = reinterpret_cast<uint4*>(base + OP_ROWS * OP_KB);
  uint4* d2 = reinterpret_cast<uint4*>(base + 2 * OP_ROWS * OP_KB);
#pragma unroll
  for (int u = 0; u < OP_KB * 2 / 16; ++u) {
    d0[u] = v0[u];
    d1[u] = v1[u];
    d2[u] = v2[u];
  }
}

cudaError_t launch_op_slices(const double* Linv, int64_t ld, int64_t nk, int64_t nkp, __nv_bfloat16* op,
                             cudaStream_t st) {
  const int nm = (int)(nkp / OP_ROWS);
  dim3 grid((OP_ROWS / OP_KB) * nm, nm);
  k_op_slices<<<grid, OP_ROWS, 0, st>>>(Linv, ld, nk, op);
  return cudaGetLastError();
}

__global__ void k_r_slices(const float* __restrict__ R, int64_t ldr, int64_t nk, int64_t K, int64_t nkp8,
                           int64_t capK, __nv_bfloat16* __restrict__ rs, int nslices) {
  const int64_t slice_stride = capK * nkp8;
  for (int64_t k = blockIdx.y; k < K; k += gridDim.y)
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nk; j += (int64_t)gridDim.x * blockDim.x) {
    const float x = R[j + k * ldr];
    __nv_bfloat16 a, b, c;
    split3_f32(x, a, b, c);
    __nv_bfloat16* p = rs + k * nkp8 + j;
    p[0] = a;
    p[slice_stride] = b;
    if (nslices > 2) p[2 * slice_stride] = c;
  }
}

cudaError_t launch_r_slices(const float* R, int64_t ldr, int64_t nk, int64_t K, int64_t nkp8, int64_t capK,
                            __nv_bfloat16* rs, int nslices, cudaStream_t st) {
  if (K <= 0) return cudaSuccess;
  int gx = (int)ceil_div(nk, 256);
  if (gx > 32) gx = 32;
  dim3 grid(gx, (unsigned)(K < 65535 ? K : 65535));
  k_r_slices<<<grid, 256, 0, st>>>(R, ldr, nk, K, nkp8, capK, rs, nslices);
  return cudaGetLastError();
}

}  // namespace td
