// The covariance factor C = L L^T and the whitening operator L^{-1} with the
// O(N'^3) work on the tensor cores (Sec. II.A, C = L L^T and W = L^{-1};
// Sec. III.A, "Factorization of the covariance matrix": once per segment).
//
// Blocked right-looking Cholesky in blocks of b = 128, carrying the identity
// along so that the same eliminations turn it into L^{-1} (forward
// substitution of the identity, block row by block row).  Step p:
//   1. L_pp = chol(A_pp) and X_pp = L_pp^{-1}: one CTA, double-float (k_potrf_blk)
//   2. panel   L_{>p,p} = A_{>p,p} X_pp^T                   (split product)
//      block row of the inverse  X_{p,<p} = X_pp B_{p,<p}   (split product)
//   3. trailing A_{>p,>p} -= L_{>p,p} L_{>p,p}^T (lower tiles) and
//      B_{>p,<=p} -= L_{>p,p} X_{p,<=p}                      (split products)
// where B starts as the identity and block row p of B, once updated by the
// steps before it, is X_pp^{-1} times block row p of L^{-1}.  The split
// products are the FP64-accurate emulation on bf16 tensor cores of
// emu_gemm.cu (contraction 128 = b, so every product is one exact pass);
// the block factor and its inverse run in double-float (FP32 pairs, about 48
// significant bits, the split products' precision) on the CUDA cores.
//
// Storage: L (in place of C) and X = L^{-1} are nkp x nkp column-major FP64
// (nkp = N' rounded up to 256; identity padding, so both factor as blockdiag
// with an identity).  Operand slices [ns][rows][128] bf16 per product.
#include <algorithm>
#include <cstdio>
#include <string>
#include <vector>

#include "emu_gemm.h"

namespace td {

namespace {
constexpr int PB = EK;                      // block size of the factor (128)
constexpr int PK_ELEMS = PB * (PB + 1) / 2; // packed lower triangle
__device__ __forceinline__ int pk(int r, int c) { return c * (2 * PB - 1 - c) / 2 + r; }   // r >= c
constexpr size_t POTRF_SMEM = (size_t)(2 * PK_ELEMS + 64 * 64) * sizeof(float2);

// Double-float arithmetic: a value is an unevaluated pair h + l of FP32
// numbers with |l| <= ulp(h)/2, about 48 significant bits.  The sums and
// products below are the classical error-free transformations (Knuth's
// two-sum, Dekker's fast two-sum, the FMA form of the exact product), written
// with the _rn intrinsics so the compiler neither contracts nor reorders them.
struct df {
  float h, l;
};
__device__ __forceinline__ df df_make(float h, float l) {
  df r;
  r.h = h;
  r.l = l;
  return r;
}
__device__ __forceinline__ df df_from(double x) {
  const float h = __double2float_rn(x);
  return df_make(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ double df_to(df a) { return (double)a.h + (double)a.l; }
// s + e = a + b exactly
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df_make(s, e);
}
// s + e = a + b exactly, given |a| >= |b| (or a = 0)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);   // p + e = a.h b.h exactly
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ df df_add(df a, df b) {
  const df s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ df df_neg(df a) { return df_make(-a.h, -a.l); }
// (double)f * 2^e2, the double's bits assembled from the float's (exponent
// rebiased, significand shifted) on the integer pipe; a subnormal float is
// first scaled by 2^64 (exact), and only infinite and NaN floats take the
// FP64 route
__device__ __forceinline__ double f2d_pow2(float f, int e2) {
  unsigned u = __float_as_uint(f);
  unsigned ex = (u >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  if ((u & 0x7fffffffu) == 0u) return __longlong_as_double((long long)sign);
  if (ex == 0xffu) return ldexp((double)f, e2);
  if (ex == 0u) {
    u = __float_as_uint(__fmul_rn(f, 18446744073709551616.0f));   // 2^64
    ex = (u >> 23) & 0xffu;
    e2 -= 64;
  }
  return __longlong_as_double(
      (long long)(sign | ((unsigned long long)(ex + 896u + (unsigned)e2) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
}
// h + l scaled by 2^e2, in FP64 (one addition)
__device__ __forceinline__ double df_to_pow2(df a, int e2) { return f2d_pow2(a.h, e2) + f2d_pow2(a.l, e2); }
// c - a b
__device__ __forceinline__ df df_fnms(df c, df a, df b) { return df_add(c, df_neg(df_mul(a, b))); }
}  // namespace

// One CTA of 512 threads on the diagonal block p of A (column-major, ld), in
// double-float arithmetic on the FP32 pipe (B300 issues about two FP64
// multiply-adds per clock per SM; the FP32 pipe 128): the block is scaled by
// an exact power of two 4^-m (so strain-scale covariances stay inside FP32's
// range), factored by an unblocked right-looking Cholesky in shared memory
// (packed lower triangle), and inverted by 64-row halves (X11 = L11^{-1} and
// X22 = L22^{-1} by forward substitution of the identity, row by row, then
// X21 = -X22 L21 X11).  Then, unscaled (L = 2^m L_s, X = 2^-m X_s):
//   A_pp <- L_pp (upper part zero),  X_pp <- L_pp^{-1},  linv <- L_pp^{-1}
//   (128 x 128 column-major), dinv tiles 2p, 2p+1 <- the two 64 x 64 diagonal
//   inverses (the FP64 path's tiles), ldpart[2p + h] <- 2 sum log L_ii over the
//   kept rows of half h.
// Pivots, their square roots and reciprocals are formed in double-float as
// well (one thread on the critical path of every column).  About 48
// significant bits throughout, the precision of the six-slice split products
// that use L_pp and X_pp.  A pivot that is not positive and finite records
// TD_ERR_NOT_PD with its kept-sample index (the smallest over the factor) and
// continues with NaN.
__global__ void __launch_bounds__(512) k_potrf_blk(double* __restrict__ A, double* __restrict__ X, int64_t ld,
                                                    int64_t nk, int p, double* __restrict__ linv,
                                                    double* __restrict__ dinv, double* __restrict__ ldpart,
                                                    DevStatus* status) {
  extern __shared__ float2 smf[];
  df* a = reinterpret_cast<df*>(smf);   // L, packed
  df* x = a + PK_ELEMS;                 // L^{-1}, packed
  df* t = x + PK_ELEMS;                 // 64 x 64 scratch, t[r + 64 c]
  __shared__ double logd[PB];
  __shared__ df ipv[PB], idg[PB];
  __shared__ double smax[4];
  __shared__ int sm_m;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t o = (int64_t)p * PB;
  // scale 4^-m with m from the largest diagonal entry of the kept rows (an
  // integer exponent: the scaling and its inverse are exact).  Padding rows
  // (the identity past N') stay unscaled: they are decoupled from the kept
  // rows, and scaled by a strain-scale 4^-m they would overflow FP32.
  if (tid < PB) {
    const double v = (o + tid < nk) ? A[(o + tid) + (o + tid) * ld] : 0.0;
    double dmax = (v > 0.0 && isfinite(v)) ? v : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, off));
    if (lane == 0) smax[warp] = dmax;
  }
  __syncthreads();
  if (tid == 0) {
    const double mx = fmax(fmax(smax[0], smax[1]), fmax(smax[2], smax[3]));
    sm_m = mx > 0.0 ? ilogb(mx) / 2 : 0;
  }
  __syncthreads();
  const int m = sm_m;
  const double down = ldexp(1.0, -2 * m);
  for (int e0 = tid; e0 < PB * PB; e0 += 8 * 512) {   // eight loads in flight, then the conversions
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + 512 * u, r = e % PB, c = e / PB;
      v[u] = (r >= c && o + r < nk) ? A[(o + r) + (o + c) * ld] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + 512 * u, r = e % PB, c = e / PB;
      if (r >= c) a[pk(r, c)] = (o + r < nk) ? df_from(v[u] * down) : df_make(r == c ? 1.f : 0.f, 0.f);
    }
  }
  for (int e = tid; e < PK_ELEMS; e += 512) x[e] = df_make(0.f, 0.f);
  __syncthreads();
  // Right-looking elimination on the unscaled columns, one barrier per
  // column: column k stays as A's values (l_rk d_k) until the end, and the
  // trailing update uses a_rk a_ck / p_k.  The pivot p_{k+1} is final as soon
  // as element (k+1, k+1) has had its update in step k; the thread that makes
  // that update (warp 0, lane 0) prepares 1/p_{k+1} and 1/sqrt(p_{k+1}) for
  // step k+1.  That thread is on the critical path of every step, so it
  // works in double-float too: y = 1/sqrt(p) from the FP32 reciprocal square
  // root and two Newton steps y <- y + y (1 - p y^2) / 2 (each doubles the
  // correct bits), then sqrt(p) = p y and 1/p = y^2 (FP64 square roots and
  // divisions are long sequences on a part with few FP64 units).
  auto pivot = [&](int k) {
    const df pv = a[pk(k, k)];
    if (!(pv.h > 0.f) || !isfinite(pv.h)) {
      const long long g = o + k;
      if (g < nk) {
        atomicMin((unsigned long long*)&status->pivot, (unsigned long long)g);
        atomicCAS(&status->code, 0, ST_NOT_PD);
      }
      const float qn = __int_as_float(0x7fc00000);
      a[pk(k, k)] = ipv[k] = idg[k] = df_make(qn, qn);
      return;
    }
    df y = df_make(rsqrtf(pv.h), 0.f);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      const df rr = df_fnms(df_make(1.f, 0.f), pv, df_mul(y, y));   // 1 - p y^2
      y = df_add(y, df_mul(y, df_make(0.5f * rr.h, 0.5f * rr.l)));
    }
    a[pk(k, k)] = df_mul(pv, y);
    ipv[k] = df_mul(y, y);
    idg[k] = y;
  };
  if (tid == 0) pivot(0);
  __syncthreads();
  for (int k = 0; k < PB - 1; ++k) {
    const df ip = ipv[k];
    for (int c = k + 1 + warp; c < PB; c += 16) {
      const df lck = df_mul(a[pk(c, k)], ip);
      for (int r = c + lane; r < PB; r += 32) a[pk(r, c)] = df_fnms(a[pk(r, c)], a[pk(r, k)], lck);
      if (c == k + 1 && lane == 0) pivot(k + 1);   // (k+1, k+1) was this thread's first element
    }
    __syncthreads();
  }
  // scale the columns: l_rk = a_rk / d_k; log d_k of the scaled block, one
  // column per thread
  if (tid < PB) logd[tid] = log(df_to(a[pk(tid, tid)]));
  for (int c = warp; c < PB; c += 16) {
    const df s = idg[c];
    for (int r = c + 1 + lane; r < PB; r += 32) a[pk(r, c)] = df_mul(a[pk(r, c)], s);
  }
  __syncthreads();
  // inverses of the two 64 x 64 diagonal halves: forward substitution of the
  // identity, one row of each half per step.  A row not yet final holds
  // acc_rc = -sum_{i < k} l_ri x_ic; row k becomes x_kc = (delta_kc + acc_kc) / l_kk
  // (the reciprocals the pivots formed: an FP64 division is a long sequence
  // on this part), then the rows below it take their share of it.
  for (int j = 0; j < 64; ++j) {
    if (tid < PB) {
      const int h = tid >> 6, cc = tid & 63;
      if (cc <= j) {
        const int k = 64 * h + j, c = 64 * h + cc;
        df v = x[pk(k, c)];
        if (cc == j) v = df_add(v, df_make(1.f, 0.f));
        x[pk(k, c)] = df_mul(v, idg[k]);
      }
    }
    __syncthreads();
    const int nr = 63 - j, ncc = j + 1, per = nr * ncc;
    for (int e = tid; e < 2 * per; e += 512) {
      const int h = e / per, q = e - h * per;
      const int rr = q % nr, cc = q / nr;
      const int k = 64 * h + j, r = k + 1 + rr, c = 64 * h + cc;
      x[pk(r, c)] = df_fnms(x[pk(r, c)], a[pk(r, k)], x[pk(k, c)]);
    }
    __syncthreads();
  }
  // t = L21 X11   (t[r][c] = sum_{k >= c} L[64 + r][k] X[k][c])
  for (int e = tid; e < 64 * 64; e += 512) {
    const int r = e & 63, c = e >> 6;
    df s0 = df_make(0.f, 0.f), s1 = s0;   // two interleaved partial sums
    int k = c;
    for (; k + 1 < 64; k += 2) {
      s0 = df_add(s0, df_mul(a[pk(64 + r, k)], x[pk(k, c)]));
      s1 = df_add(s1, df_mul(a[pk(64 + r, k + 1)], x[pk(k + 1, c)]));
    }
    if (k < 64) s0 = df_add(s0, df_mul(a[pk(64 + r, k)], x[pk(k, c)]));
    t[r + 64 * c] = df_add(s0, s1);
  }
  __syncthreads();
  // X21 = -X22 t   (X21[r][c] = -sum_{k <= r} X[64 + r][64 + k] t[k][c])
  for (int e = tid; e < 64 * 64; e += 512) {
    const int r = e & 63, c = e >> 6;
    df s0 = df_make(0.f, 0.f), s1 = s0;   // two interleaved partial sums
    int k = 0;
    for (; k + 1 <= r; k += 2) {
      s0 = df_add(s0, df_mul(x[pk(64 + r, 64 + k)], t[k + 64 * c]));
      s1 = df_add(s1, df_mul(x[pk(64 + r, 65 + k)], t[k + 1 + 64 * c]));
    }
    if (k <= r) s0 = df_add(s0, df_mul(x[pk(64 + r, 64 + k)], t[k + 64 * c]));
    x[pk(64 + r, c)] = df_neg(df_add(s0, s1));
  }
  __syncthreads();
  for (int e = tid; e < PB * PB; e += 512) {   // L = 2^m L_s, X = 2^-m X_s
    const int r = e % PB, c = e / PB;
    const bool lo = r >= c, pad = o + r >= nk;   // a padding row's only entry is its diagonal 1
    const double lv = lo ? df_to_pow2(a[pk(r, c)], pad ? 0 : m) : 0.0;
    const double xv = lo ? df_to_pow2(x[pk(r, c)], pad ? 0 : -m) : 0.0;
    A[(o + r) + (o + c) * ld] = lv;
    X[(o + r) + (o + c) * ld] = xv;
    linv[e] = xv;
    if ((r < 64) == (c < 64)) {   // the two 64 x 64 diagonal tiles, column-major
      const int h = r >> 6;
      dinv[(int64_t)(2 * p + h) * 64 * 64 + (r & 63) + 64 * (c & 63)] = xv;
    }
  }
  if (tid < 2) {
    const double shift = (double)m * 0.69314718055994530942;   // log 2^m
    double sacc = 0.0;
    for (int k = 64 * tid; k < 64 * tid + 64; ++k)
      if (o + k < nk) sacc += logd[k] + shift;
    ldpart[2 * p + tid] = 2.0 * sacc;
  }
}

// X = identity (nkp x nkp column-major)
__global__ void k_eye(double* __restrict__ X, int64_t nkp) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nkp; i += (int64_t)gridDim.x * blockDim.x)
    X[i + i * nkp] = 1.0;
}

namespace {
template <class T>
td_status talloc(T** p, size_t count, const char* what) {
  *p = nullptr;
  if (count == 0) return TD_OK;
  if (cudaMalloc((void**)p, count * sizeof(T)) != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(TD_ERR_OOM, std::string("device allocation failed: ") + what);
  }
  return TD_OK;
}

}  // namespace

td_status factor_tensor(td_segment* s, cudaStream_t st, int ns) {
  td_status r = factor_begin(s, st);
  if (r != TD_OK) return r;
  static std::atomic<unsigned long long> attr_done{0};
  if (device_needs_setup(attr_done)) {
    TD_CUDA(cudaFuncSetAttribute(k_potrf_blk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)POTRF_SMEM));
    mark_device_done(attr_done);
  }
  const int64_t nkp = s->nkp, ld = nkp;
  const int nb = (int)(nkp / PB);
  double* X = nullptr;
  double* lblk = nullptr;
  SliceBuf sAP, sLI, sBP, sP, sX;
  auto cleanup = [&]() {
    free_slice_buf(sAP);
    free_slice_buf(sLI);
    free_slice_buf(sBP);
    free_slice_buf(sP);
    free_slice_buf(sX);
    if (lblk) cudaFree(lblk);
  };
  if ((r = talloc(&X, (size_t)(nkp * nkp), "L^{-1} (temporary)")) != TD_OK ||
      (r = talloc(&lblk, (size_t)PB * PB, "block inverse")) != TD_OK ||
      (r = slice_buf(sAP, (int)nkp, ns)) != TD_OK || (r = slice_buf(sLI, PB, ns)) != TD_OK ||
      (r = slice_buf(sBP, (int)nkp, ns)) != TD_OK || (r = slice_buf(sP, (int)nkp, ns)) != TD_OK ||
      (r = slice_buf(sX, (int)nkp, ns)) != TD_OK) {
    cleanup();
    if (X) cudaFree(X);
    return r;
  }
  const int64_t lim = 2000000000LL;   // bound on each in-kernel wait
  cudaError_t e = cudaMemsetAsync(X, 0, (size_t)(nkp * nkp) * sizeof(double), st);
  if (e == cudaSuccess) {
    k_eye<<<(unsigned)std::min<int64_t>(1024, ceil_div(nkp, 256)), 256, 0, st>>>(X, nkp);
    e = cudaGetLastError();
  }
  // Lookahead: step p's trailing update is issued in two parts.  The first
  // (G2a) covers what step p+1 reads -- block column p+1 of the Schur
  // complement and block row p+1 of the inverse --; the block factor of step
  // p+1 (one CTA, FP64) then runs on a second stream while the rest (G2b,
  // one SM short of the full grid) runs on the first.  G2b touches neither
  // the diagonal block p+1 nor anything the block factor writes.
  cudaStream_t la = nullptr;
  cudaEvent_t ev_a = nullptr, ev_p = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&la, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_a, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_p, cudaEventDisableTiming);
  if (e == cudaSuccess) {
    k_potrf_blk<<<1, 512, POTRF_SMEM, st>>>(s->L, X, ld, s->nk, 0, lblk, s->dinv, s->ldpart, s->status);
    e = cudaGetLastError();
  }
  const int nsm = tc_num_sms();
  for (int p = 0; p < nb && e == cudaSuccess; ++p) {
    const int64_t o = (int64_t)p * PB;
    const int64_t T = nkp - o - PB;   // rows below the block
    double* Lp = s->L + (o + PB) + o * ld;   // panel A_{>p,p}, then L_{>p,p}
    if (p > 0 && (e = cudaStreamWaitEvent(st, ev_p, 0)) != cudaSuccess) break;   // block factor p done
    // slices of X_pp (rows), of the panel (rows) and of block row p of B (columns)
    EmuSplitParams S1{};
    add_split_job(S1, lblk, 1, PB, PB, sLI, ns);
    add_split_job(S1, Lp, 1, ld, (int)T, sAP, ns);
    add_split_job(S1, X + o, ld, 1, (int)o, sBP, ns);
    if ((e = launch_emu_split(S1, st)) != cudaSuccess) break;
    EmuParams G1{};
    add_product(G1, sAP, sLI, Lp, ld, 1.0, 0.0, (int)(T / PB), PB / 64, false);
    add_product(G1, sLI, sBP, X + o, ld, 1.0, 0.0, 1, (int)(o / 64), false);
    if ((e = launch_emu_gemm(G1, ns, s->status, lim, st)) != cudaSuccess) break;
    if (T == 0) break;
    // slices of L_{>p,p} (rows) and of block row p of L^{-1} up to the diagonal (columns)
    EmuSplitParams S2{};
    add_split_job(S2, Lp, 1, ld, (int)T, sP, ns);
    add_split_job(S2, X + o, ld, 1, (int)(o + PB), sX, ns);
    if ((e = launch_emu_split(S2, st)) != cudaSuccess) break;
    // G2a: the first 128 columns of the Schur complement (all its rows) and
    // block row p+1 of the inverse
    EmuParams G2a{};
    add_product(G2a, sP, sP, s->L + (o + PB) * (1 + ld), ld, -1.0, 1.0, (int)(T / PB), PB / 64, false);
    add_product(G2a, sP, sX, X + (o + PB), ld, -1.0, 1.0, 1, (int)((o + PB) / 64), false);
    if ((e = launch_emu_gemm(G2a, ns, s->status, lim, st)) != cudaSuccess) break;
    if ((e = cudaEventRecord(ev_a, st)) != cudaSuccess) break;
    // block factor of step p+1 beside G2b
    if ((e = cudaStreamWaitEvent(la, ev_a, 0)) != cudaSuccess) break;
    k_potrf_blk<<<1, 512, POTRF_SMEM, la>>>(s->L, X, ld, s->nk, p + 1, lblk, s->dinv, s->ldpart, s->status);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = cudaEventRecord(ev_p, la)) != cudaSuccess) break;
    // G2b: the rest of the Schur complement (lower tiles) and of the inverse
    const int64_t T2 = T - PB;
    EmuParams G2b{};
    add_product(G2b, sP, sP, s->L + (o + 2 * PB) * (1 + ld), ld, -1.0, 1.0, (int)(T2 / PB), (int)(T2 / 64), true,
             PB, PB);
    add_product(G2b, sP, sX, X + (o + 2 * PB), ld, -1.0, 1.0, (int)(T2 / PB), (int)((o + PB) / 64), false, PB, 0);
    if ((e = launch_emu_gemm(G2b, ns, s->status, lim, st, nsm - 1)) != cudaSuccess) break;
  }
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_p, 0);
  if (la) cudaStreamDestroy(la);
  if (ev_a) cudaEventDestroy(ev_a);
  if (ev_p) cudaEventDestroy(ev_p);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) {
    cudaFree(X);
    return cuda_fail(e, "tensor-core factor");
  }
  return factor_end(s, X, st);
}

}  // namespace td
