// Covariance build and blocked right-looking Cholesky, FP64 (Sec. II.A,
// C = L L^T; Sec. III.A, "Factorization of the covariance matrix": O(N^3),
// once per segment, result cached).
//
// Storage: A is nkp x nkp column-major FP64 (nkp = N' rounded up to 256).
// The padding is the identity, so the factor of the padded matrix is
// blockdiag(L, I) and every 64 x 64 tile is full.
#include <cstdio>
#include <string>
#include <vector>

#include "td_internal.h"

namespace td {

// ---------------------------------------------------------------- K1 gather
// A[i, j] = acf[|t_i - t_j|] for i, j < N' (Sec. II, C_ij = rho(|i - j|) on
// the kept sample times; Sec. II.B item 2, gaps delete rows and columns).
__global__ void k_gather(const double* __restrict__ acf, const int32_t* __restrict__ t, int64_t nk,
                         int64_t nkp, double* __restrict__ A) {
  for (int64_t j = blockIdx.y; j < nkp; j += gridDim.y)
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nkp; i += (int64_t)gridDim.x * blockDim.x) {
    double v;
    if (i < nk && j < nk) {
      int d = t[i] - t[j];
      v = acf[d < 0 ? -d : d];
    } else {
      v = (i == j) ? 1.0 : 0.0;
    }
    A[i + j * nkp] = v;
  }
}

cudaError_t launch_gather(const double* acf, const int32_t* t, int64_t nk, int64_t nkp, double* A,
                          cudaStream_t st) {
  dim3 grid((unsigned)ceil_div(nkp, 256), (unsigned)(nkp < 65535 ? nkp : 65535));
  if (grid.x > 64) grid.x = 64;
  k_gather<<<grid, 256, 0, st>>>(acf, t, nk, nkp, A);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- K2 potrf
// Unblocked Cholesky of the 64 x 64 diagonal tile j in shared memory, its
// triangular inverse (used by the panel update and the forward
// substitution), and the tile's share of log det C = 2 sum log L_ii.
__global__ void __launch_bounds__(256) k_potrf_diag(double* __restrict__ A, int64_t ld, int64_t nk, int j,
                                                     double* __restrict__ dinv, double* __restrict__ ldpart,
                                                     DevStatus* status) {
  __shared__ double a[FT][FT + 1];   // a[col][row]
  __shared__ double x[FT][FT + 1];   // inverse, x[col][row]
  __shared__ double logd[FT];
  const int tid = threadIdx.x;
  const int64_t base = (int64_t)j * FT;
  for (int e = tid; e < FT * FT; e += 256) {
    int r = e % FT, c = e / FT;
    a[c][r] = A[(base + r) + (base + c) * ld];
  }
  __syncthreads();
  for (int k = 0; k < FT; ++k) {
    if (tid == 0) {
      double p = a[k][k];
      if (!(p > 0.0) || !isfinite(p)) {
        long long g = base + k;
        if (g < nk) {
          atomicMin((unsigned long long*)&status->pivot, (unsigned long long)g);
          atomicCAS(&status->code, 0, ST_NOT_PD);
        }
        p = nan("");
      }
      double d = sqrt(p);
      a[k][k] = d;
      logd[k] = log(d);
    }
    __syncthreads();
    if (tid > k && tid < FT) a[k][tid] /= a[k][k];
    __syncthreads();
    const int rem = FT - 1 - k;   // trailing size
    for (int e = tid; e < rem * rem; e += 256) {
      int r = k + 1 + e % rem, c = k + 1 + e / rem;
      if (r >= c) a[c][r] -= a[k][r] * a[k][c];
    }
    __syncthreads();
  }
  // inverse of the lower-triangular tile, one column per thread
  if (tid < FT) {
    const int c = tid;
    for (int r = 0; r < c; ++r) x[c][r] = 0.0;
    x[c][c] = 1.0 / a[c][c];
    for (int r = c + 1; r < FT; ++r) {
      double s = 0.0;
      for (int k = c; k < r; ++k) s += a[k][r] * x[c][k];
      x[c][r] = -s / a[r][r];
    }
  }
  __syncthreads();
  for (int e = tid; e < FT * FT; e += 256) {
    int r = e % FT, c = e / FT;
    A[(base + r) + (base + c) * ld] = (r >= c) ? a[c][r] : 0.0;
    dinv[(int64_t)j * FT * FT + e] = x[c][r];   // column-major 64 x 64
  }
  if (tid == 0) {
    double s = 0.0;
    for (int k = 0; k < FT; ++k)
      if (base + k < nk) s += logd[k];
    ldpart[j] = 2.0 * s;
  }
}

cudaError_t launch_potrf_diag(double* A, int64_t ld, int64_t nk, int j, double* dinv, double* ldpart,
                              DevStatus* status, cudaStream_t st) {
  k_potrf_diag<<<1, 256, 0, st>>>(A, ld, nk, j, dinv, ldpart, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- K3 panel
// L_ij = A_ij L_jj^{-T} for the tiles i > j below the diagonal tile.
__global__ void __launch_bounds__(256) k_panel(double* __restrict__ A, int64_t ld, int j,
                                                const double* __restrict__ dinv) {
  __shared__ double As[FT * FT];   // As[k*64 + r] = A_ij[r][k]
  __shared__ double Ds[FT * FT];   // Ds[c*64 + k] = Dinv[c][k]
  const int i = j + 1 + blockIdx.x;
  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)i * FT, c0 = (int64_t)j * FT;
  const double* D = dinv + (int64_t)j * FT * FT;
  for (int e = tid; e < FT * FT; e += 256) {
    int r = e % FT, k = e / FT;
    As[e] = A[(r0 + r) + (c0 + k) * ld];
    Ds[r * FT + k] = D[e];   // D is column-major: D[e] = Dinv[r][k]
  }
  __syncthreads();
  // out[r][c] = sum_k A_ij[r][k] Dinv[c][k]   (= A_ij Dinv^T)
  const int r = tid & 63, cg = tid >> 6;   // 4 groups of 16 columns
  double acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = 0.0;
  for (int k = 0; k < FT; ++k) {
    double av = As[k * FT + r];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = fma(av, Ds[(cg * 16 + q) * FT + k], acc[q]);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 16; ++q) A[(r0 + r) + (c0 + cg * 16 + q) * ld] = acc[q];
}

cudaError_t launch_panel(double* A, int64_t ld, int j, int nt, const double* dinv, cudaStream_t st) {
  if (nt - j - 1 <= 0) return cudaSuccess;
  k_panel<<<nt - j - 1, 256, 0, st>>>(A, ld, j, dinv);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- K4 trailing update
// A_ik -= L_ij L_kj^T for j < k <= i (lower triangle of the trailing matrix).
__global__ void __launch_bounds__(256) k_syrk(double* __restrict__ A, int64_t ld, int j, int nt) {
  __shared__ double Ls[FT * FT];   // Ls[q*64 + r] = L_ij[r][q]
  __shared__ double Ks[FT * FT];   // Ks[q*64 + c] = L_kj[c][q]
  // decode the triangular tile index
  const int m = nt - j - 1;
  int64_t b = blockIdx.x;
  // rows ii in [0, m), cols kk in [0, ii]; b = ii*(ii+1)/2 + kk
  int ii = (int)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
  while ((int64_t)(ii + 1) * (ii + 2) / 2 <= b) ++ii;
  while ((int64_t)ii * (ii + 1) / 2 > b) --ii;
  const int kk = (int)(b - (int64_t)ii * (ii + 1) / 2);
  const int i = j + 1 + ii, k = j + 1 + kk;
  (void)m;
  const int tid = threadIdx.x;
  const int64_t ri = (int64_t)i * FT, rk = (int64_t)k * FT, cj = (int64_t)j * FT;
  for (int e = tid; e < FT * FT; e += 256) {
    int r = e % FT, q = e / FT;
    Ls[e] = A[(ri + r) + (cj + q) * ld];
    Ks[e] = A[(rk + r) + (cj + q) * ld];
  }
  __syncthreads();
  const int r0 = (tid & 15) * 4, c0 = (tid >> 4) * 4;
  double acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
  for (int q = 0; q < FT; ++q) {
    double a0 = Ls[q * FT + r0], a1 = Ls[q * FT + r0 + 1], a2 = Ls[q * FT + r0 + 2], a3 = Ls[q * FT + r0 + 3];
    double b0 = Ks[q * FT + c0], b1 = Ks[q * FT + c0 + 1], b2 = Ks[q * FT + c0 + 2], b3 = Ks[q * FT + c0 + 3];
    double av[4] = {a0, a1, a2, a3}, bv[4] = {b0, b1, b2, b3};
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = fma(av[u], bv[v], acc[u][v]);
  }
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int64_t idx = (ri + r0 + u) + (rk + c0 + v) * ld;
      A[idx] -= acc[u][v];
    }
}

cudaError_t launch_syrk(double* A, int64_t ld, int j, int nt, cudaStream_t st) {
  const int64_t m = nt - j - 1;
  if (m <= 0) return cudaSuccess;
  const int64_t blocks = m * (m + 1) / 2;
  k_syrk<<<(unsigned)blocks, 256, 0, st>>>(A, ld, j, nt);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- host drivers
template <class T>
static td_status falloc(T** p, size_t count, const char* what) {
  *p = nullptr;
  if (count == 0) return TD_OK;
  if (cudaMalloc((void**)p, count * sizeof(T)) != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(TD_ERR_OOM, std::string("device allocation failed: ") + what);
  }
  return TD_OK;
}

td_status factor_begin(td_segment* s, cudaStream_t st) {
  s->factored = false;
  s->pivot = -1;
  free_refine_state(s);   // slices of the old L
  const int64_t nkp = s->nkp;
  const int nt = (int)(nkp / FT);
  td_status r;
  if (!s->L && (r = falloc(&s->L, (size_t)(nkp * nkp), "factor L")) != TD_OK) return r;
  if (!s->dinv && (r = falloc(&s->dinv, (size_t)nt * FT * FT, "diagonal inverses")) != TD_OK) return r;
  if (!s->ldpart && (r = falloc(&s->ldpart, (size_t)nt, "logdet partials")) != TD_OK) return r;
  if ((r = reset_status(s, st)) != TD_OK) return r;
  TD_CUDA(launch_gather(s->acf, s->t, s->nk, nkp, s->L, st));
  return TD_OK;
}

td_status factor_end(td_segment* s, double* linv, cudaStream_t st) {
  const int64_t nkp = s->nkp;
  const int nt = (int)(nkp / FT);
  DevStatus hs;
  td_status r = read_status(s, st, &hs);
  if (r != TD_OK || hs.code == ST_NOT_PD) {
    cudaFree(linv);
    if (r != TD_OK) return r;
    s->pivot = hs.pivot;
    char buf[128];
    snprintf(buf, sizeof buf, "covariance not positive definite at kept sample %lld", (long long)hs.pivot);
    return fail(TD_ERR_NOT_PD, buf);
  }
  if (hs.code == ST_TIMEOUT) {
    cudaFree(linv);
    reset_status(s, st);
    return fail(TD_ERR_TIMEOUT, "a bounded in-kernel wait of the factor ran out");
  }
  std::vector<double> ld((size_t)nt);
  cudaError_t e = cudaMemcpy(ld.data(), s->ldpart, (size_t)nt * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    cudaFree(linv);
    return cuda_fail(e, "log det shares");
  }
  double logdet = 0.0;
  for (int j = 0; j < nt; ++j) logdet += ld[(size_t)j];
  // bf16 slices of the whitening operator
  const int64_t nm = nkp / OP_ROWS;
  s->op_blocks = op_row_offset(nm);
  if (!s->op && (r = falloc(&s->op, (size_t)(s->op_blocks * OP_SLICES * OP_ROWS * OP_KB), "operator slices")) != TD_OK) {
    cudaFree(linv);
    return r;
  }
  double* qrow = nullptr;
  if ((r = falloc(&qrow, (size_t)nkp, "row quanta")) != TD_OK) {
    cudaFree(linv);
    return r;
  }
  e = launch_row_quantum(linv, nkp, s->nk, nkp, qrow, st);
  if (e == cudaSuccess) e = launch_op_slices(linv, nkp, s->nk, nkp, qrow, s->op, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(linv);
  cudaFree(qrow);
  if (e != cudaSuccess) return cuda_fail(e, "td_factor operator build");
  s->logdet = logdet;
  s->factored = true;
  return TD_OK;
}

// The FP64 CUDA-core route: 64-wide blocked right-looking Cholesky, then L^{-1}
// by forward substitution of the identity (both O(N'^3) on DFMA).
td_status factor_fp64_cores(td_segment* s, cudaStream_t st) {
  td_status r = factor_begin(s, st);
  if (r != TD_OK) return r;
  const int64_t nkp = s->nkp;
  const int nt = (int)(nkp / FT);
  for (int j = 0; j < nt; ++j) {
    TD_CUDA(launch_potrf_diag(s->L, nkp, s->nk, j, s->dinv, s->ldpart, s->status, st));
    TD_CUDA(launch_panel(s->L, nkp, j, nt, s->dinv, st));
    TD_CUDA(launch_syrk(s->L, nkp, j, nt, st));
  }
  double* linv = nullptr;
  if ((r = falloc(&linv, (size_t)(nkp * nkp), "L^{-1} (temporary)")) != TD_OK) return r;
  cudaError_t e = cudaMemsetAsync(linv, 0, (size_t)(nkp * nkp) * sizeof(double), st);
  for (int I = 0; I < nt && e == cudaSuccess; ++I)
    e = launch_trsm_f64_row(s->L, nkp, s->dinv, I, nullptr, 0, s->nk, nkp, linv, nkp, nullptr, 0, st);
  if (e != cudaSuccess) {
    cudaFree(linv);
    return cuda_fail(e, "FP64 inverse");
  }
  return factor_end(s, linv, st);
}

}  // namespace td
