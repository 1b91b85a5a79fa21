// Plain FP64 blocked forward substitution W = L^{-1} R (Sec. II.A, the
// whitening operator W = L^{-1}; Sec. III.A, the triangular-solve form of
// the whitening), the FP64 chi2 / logL reduction, and the bounded-wait probe.
//
// One launch per 64-row block row I (the dependency chain of the solve):
//   W_I = L_II^{-1} (R_I - sum_{J<I} L_IJ W_J)
// Each CTA owns 32 columns.  With no right-hand side given, R is the
// identity and the launches build L^{-1} itself (columns right of the
// diagonal block are zero and skipped).
#include <algorithm>

#include "td_internal.h"

namespace td {


__global__ void __launch_bounds__(256) k_trsm_f64_row(const double* __restrict__ L, int64_t ld,
                                                       const double* __restrict__ dinv, int I,
                                                       const float* __restrict__ rhs32, int64_t ldr, int64_t nk,
                                                       int64_t ncols, double* __restrict__ W, int64_t ldw,
                                                       double* __restrict__ partials, int64_t ldp) {
  __shared__ double Ls[FT * FT];   // Ls[k*64 + r] = L_IJ[r][k]
  __shared__ double Ws[FT * 32];   // Ws[k*32 + c] = W_J[k][c]; later the reduction scratch
  const int tid = threadIdx.x;
  const int r = tid & 63, cg = tid >> 6;   // 4 groups of 8 columns
  const int64_t col0 = (int64_t)blockIdx.x * 32;
  const bool ident = (rhs32 == nullptr);
  int Jstart = 0;
  if (ident) {
    if (col0 >= (int64_t)(I + 1) * FT) return;   // strictly upper part of L^{-1}: zero
    Jstart = (int)(col0 / FT);
  }
  const int64_t row = (int64_t)I * FT + r;
  double acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int64_t col = col0 + cg * 8 + q;
    if (ident)
      acc[q] = (row == col) ? 1.0 : 0.0;
    else
      acc[q] = (row < nk && col < ncols) ? (double)rhs32[row + col * ldr] : 0.0;
  }
  for (int J = Jstart; J < I; ++J) {
    for (int e = tid; e < FT * FT; e += 256) {
      const int rr = e % FT, k = e / FT;
      Ls[e] = L[((int64_t)I * FT + rr) + ((int64_t)J * FT + k) * ld];
    }
    for (int e = tid; e < FT * 32; e += 256) {
      const int k = e % FT, c = e / FT;
      const int64_t col = col0 + c;
      Ws[k * 32 + c] = (col < ncols) ? W[((int64_t)J * FT + k) + col * ldw] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < FT; ++k) {
      const double a = Ls[k * FT + r];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = fma(-a, Ws[k * 32 + cg * 8 + q], acc[q]);
    }
    __syncthreads();
  }
  // W_I = Dinv_I * T  (T = acc, staged through shared memory)
#pragma unroll
  for (int q = 0; q < 8; ++q) Ws[r * 32 + cg * 8 + q] = acc[q];
  const double* D = dinv + (int64_t)I * FT * FT;   // column-major: D[rr + 64 k] = Dinv[rr][k]
  for (int e = tid; e < FT * FT; e += 256) Ls[e] = D[e];
  __syncthreads();
  double out[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) out[q] = 0.0;
  for (int k = 0; k <= r; ++k) {
    const double a = Ls[k * FT + r];
#pragma unroll
    for (int q = 0; q < 8; ++q) out[q] = fma(a, Ws[k * 32 + cg * 8 + q], out[q]);
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int64_t col = col0 + cg * 8 + q;
    if (col < ncols) W[row + col * ldw] = out[q];
  }
  if (partials != nullptr) {
    // chi2 share of these 64 rows, per column: fixed shuffle tree, then 2 warps
    __syncthreads();   // Ws is free again
    double (*red)[8] = reinterpret_cast<double (*)[8]>(Ws);
    const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      double v = out[q] * out[q];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();
    if (tid < 32) {
      const int g = tid >> 3, q = tid & 7;
      const int64_t col = col0 + g * 8 + q;
      const double s = red[2 * g][q] + red[2 * g + 1][q];
      if (col < ncols) partials[(int64_t)I * ldp + col] = s;
    }
  }
}

// Right-looking FP64 forward substitution for residual batches (the plain
// FP64 evaluation path), T = R in FP64 first, then per 64-row block I:
//   W_I = L_II^{-1} T_I            (k_f64_diag: up to 32 columns per CTA)
//   T_J -= L_JI W_I for J > I      (k_f64_update: one thread per row and 1 to
//                                   8 columns, all rows below block I at once)
// so every step spreads over the rows below it, whatever K is.  (The row-wise
// kernel above takes one CTA per 32 columns and loops over the blocks left of
// its row: at K <= 32 a single CTA per step, hundreds of times slower.)
__global__ void k_f64_init(const float* __restrict__ R, int64_t ldr, int64_t nk, int64_t nkp, int64_t K,
                           double* __restrict__ T, int64_t ldw) {
  const int64_t n = nkp * K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % nkp, c = e / nkp;
    T[i + c * ldw] = i < nk ? (double)R[i + c * ldr] : 0.0;
  }
}

// W_I = Dinv_I T_I in place (rows 64 I .. 64 I + 63 of T), and the chi2 share
// of these rows per column (fixed shuffle tree over each warp's 32 rows, then
// the two warps of a column group in order).  256 threads load Dinv_I and T_I
// (16-byte loads, all in flight at once); the first 64 CG compute: row
// r = tid & 63, columns CT cg .. + CT - 1 of the CTA's CT CG.  The column
// counts follow K, since every idle multiply-add still costs FP64 issue slots.
template <int CT, int CG>
__global__ void __launch_bounds__(256) k_f64_diag(const double* __restrict__ dinv, int I, int64_t K,
                                                  double* __restrict__ T, int64_t ldw, double* __restrict__ partials,
                                                  int64_t ldp) {
  constexpr int NC = CT * CG;
  __shared__ __align__(16) double Ds[FT * FT];
  __shared__ double Ts[FT * NC];
  __shared__ double red[2 * CG][CT];
  const int tid = threadIdx.x;
  const int64_t col0 = (int64_t)blockIdx.x * NC;
  const double2* D = reinterpret_cast<const double2*>(dinv + (int64_t)I * FT * FT);   // D[rr + 64 k]
#pragma unroll
  for (int v = 0; v < FT * FT / 2 / 256; ++v) reinterpret_cast<double2*>(Ds)[tid + 256 * v] = D[tid + 256 * v];
  for (int e = tid; e < FT * NC; e += 256) {
    const int k = e % FT, c = e / FT;
    const int64_t col = col0 + c;
    Ts[k * NC + c] = col < K ? T[(int64_t)I * FT + k + col * ldw] : 0.0;
  }
  __syncthreads();
  if (tid >= 64 * CG) return;
  const int r = tid & 63, cg = tid >> 6;
  double out[CT];
#pragma unroll
  for (int q = 0; q < CT; ++q) out[q] = 0.0;
  for (int k = 0; k <= r; ++k) {
    const double a = Ds[k * FT + r];
#pragma unroll
    for (int q = 0; q < CT; ++q) out[q] = fma(a, Ts[k * NC + cg * CT + q], out[q]);
  }
  const int64_t row = (int64_t)I * FT + r;
#pragma unroll
  for (int q = 0; q < CT; ++q) {
    const int64_t col = col0 + cg * CT + q;
    if (col < K) T[row + col * ldw] = out[q];
  }
  const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
  for (int q = 0; q < CT; ++q) {
    double v = out[q] * out[q];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp][q] = v;
  }
  asm volatile("bar.sync 1, %0;" ::"r"(64 * CG) : "memory");   // the computing threads only
  if (tid < NC) {
    const int g = tid / CT, q = tid % CT;
    const int64_t col = col0 + tid;
    if (col < K) partials[(int64_t)I * ldp + col] = red[2 * g][q] + red[2 * g + 1][q];
  }
}

// T_J -= L_JI W_I for the rows below block I.  128 threads = 32 rows x 4
// quarters of the 64-long contraction (16 loads of L in flight per thread,
// consecutive rows per warp); the quarters' partial sums are added in a fixed
// order.  The CTA's CT columns (blockIdx.y) of W_I sit in shared memory.
template <int CT>
__global__ void __launch_bounds__(128) k_f64_update(const double* __restrict__ L, int64_t ld, int I, int64_t nkp,
                                                    int64_t K, double* __restrict__ T, int64_t ldw) {
  __shared__ double Ws[FT * CT];
  __shared__ double part[4][32][CT];
  const int64_t c0 = (int64_t)blockIdx.y * CT;
  for (int e = threadIdx.x; e < FT * CT; e += 128) {
    const int k = e / CT, q = e % CT;
    Ws[e] = c0 + q < K ? T[(int64_t)I * FT + k + (c0 + q) * ldw] : 0.0;
  }
  __syncthreads();
  const int rr = threadIdx.x & 31, kq = threadIdx.x >> 5;
  const int64_t i = (int64_t)(I + 1) * FT + (int64_t)blockIdx.x * 32 + rr;
  double acc[CT];
#pragma unroll
  for (int q = 0; q < CT; ++q) acc[q] = 0.0;
  if (i < nkp) {
    const double* Lrow = L + i + ((int64_t)I * FT + kq * 16) * ld;
    double a[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = Lrow[(int64_t)k * ld];
#pragma unroll
    for (int k = 0; k < 16; ++k)
#pragma unroll
      for (int q = 0; q < CT; ++q) acc[q] = fma(a[k], Ws[(kq * 16 + k) * CT + q], acc[q]);
  }
#pragma unroll
  for (int q = 0; q < CT; ++q) part[kq][rr][q] = acc[q];
  __syncthreads();
  if (kq == 0 && i < nkp) {
#pragma unroll
    for (int q = 0; q < CT; ++q)
      if (c0 + q < K)
        T[i + (c0 + q) * ldw] -= ((part[0][rr][q] + part[1][rr][q]) + part[2][rr][q]) + part[3][rr][q];
  }
}

template <int CT, int CG>
static void fp64_steps(const double* L, int64_t ld, const double* dinv, int64_t nkp, int64_t K, double* T,
                       int64_t ldw, double* partials, int64_t ldp, cudaStream_t st) {
  const int nt = (int)(nkp / FT);
  for (int I = 0; I < nt; ++I) {
    k_f64_diag<CT, CG><<<(unsigned)ceil_div(K, CT * CG), 256, 0, st>>>(dinv, I, K, T, ldw, partials, ldp);
    const int64_t rows = nkp - (int64_t)(I + 1) * FT;
    if (rows > 0)
      k_f64_update<CT><<<dim3((unsigned)ceil_div(rows, 32), (unsigned)ceil_div(K, CT)), 128, 0, st>>>(
          L, ld, I, nkp, K, T, ldw);
  }
}

cudaError_t launch_fp64_solve(const double* L, int64_t ld, const double* dinv, const float* R, int64_t ldr,
                              int64_t nk, int64_t nkp, int64_t K, double* T, int64_t ldw, double* partials,
                              int64_t ldp, cudaStream_t st) {
  if (K <= 0) return cudaSuccess;
  const int64_t n = nkp * K;
  k_f64_init<<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 4096), 256, 0, st>>>(R, ldr, nk, nkp, K, T, ldw);
  if (K == 1)
    fp64_steps<1, 1>(L, ld, dinv, nkp, K, T, ldw, partials, ldp, st);
  else if (K == 2)
    fp64_steps<2, 1>(L, ld, dinv, nkp, K, T, ldw, partials, ldp, st);
  else if (K <= 4)
    fp64_steps<4, 1>(L, ld, dinv, nkp, K, T, ldw, partials, ldp, st);
  else if (K <= 8)
    fp64_steps<8, 1>(L, ld, dinv, nkp, K, T, ldw, partials, ldp, st);
  else if (K <= 16)
    fp64_steps<8, 2>(L, ld, dinv, nkp, K, T, ldw, partials, ldp, st);
  else
    fp64_steps<8, 4>(L, ld, dinv, nkp, K, T, ldw, partials, ldp, st);
  return cudaGetLastError();
}

cudaError_t launch_trsm_f64_row(const double* L, int64_t ld, const double* dinv, int I, const float* rhs32,
                                int64_t ldr, int64_t nk, int64_t ncols, double* W, int64_t ldw,
                                double* partials, int64_t ldp, cudaStream_t st) {
  const int64_t grid = ceil_div(ncols, 32);
  if (grid <= 0) return cudaSuccess;
  k_trsm_f64_row<<<(unsigned)grid, 256, 0, st>>>(L, ld, dinv, I, rhs32, ldr, nk, ncols, W, ldw, partials,
                                                  ldp);
  return cudaGetLastError();
}

// chi2_k = sum over row groups of the partials, then
// logL_k = -chi2_k/2 - logdet/2 - (N'/2) log 2 pi   (Eq. eqn:lik with the
// constant written out).  One warp per column: lane l adds groups l, l+32, ...
// in order, then a fixed shuffle tree -- the same order for every batch.
__global__ void k_finalize(const double* __restrict__ partials, int64_t ldp, int nparts, int64_t K,
                           double logdet, int64_t nk, double* __restrict__ logL, double* __restrict__ chi2) {
  // launched as a programmatic dependent: the partials are complete once the
  // producing grid is
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int lane = threadIdx.x & 31;
  const int64_t col = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (col >= K) return;
  double s = 0.0;
  for (int p0 = lane; p0 < nparts; p0 += 32 * 8) {
    double v[8];   // eight loads in flight (clamped addresses), then the additions in order
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = partials[(int64_t)min(p0 + 32 * i, nparts - 1) * ldp + col];
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (p0 + 32 * i < nparts) s += v[i];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane == 0) {
    if (chi2) chi2[col] = s;
    logL[col] = -0.5 * s - 0.5 * logdet - 0.5 * (double)nk * LOG2PI;
  }
}

cudaError_t launch_finalize(const double* partials, int64_t ldp, int nparts, int64_t K, double logdet,
                            int64_t nk, double* logL, double* chi2, cudaStream_t st) {
  if (K <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ceil_div(K, 8));
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_finalize, partials, ldp, nparts, K, logdet, nk, logL, chi2);
}

// A wait on an mbarrier that nothing arrives at: must give up after limit_ns
// and report TD_ERR_TIMEOUT, leaving the context usable.
__global__ void k_wait_probe(DevStatus* status, int64_t limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!mbar_wait(&bar, 0, (uint64_t)limit_ns)) set_status(status, ST_TIMEOUT, 1);
  }
}

cudaError_t launch_bounded_wait_probe(DevStatus* status, int64_t limit_ns, cudaStream_t st) {
  k_wait_probe<<<1, 32, 0, st>>>(status, limit_ns);
  return cudaGetLastError();
}

}  // namespace td
