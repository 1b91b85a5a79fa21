// Gohberg-Semencul evaluation of chi2 for gap-free (Toeplitz) segments
// (Sec. III.A: the GS formula for the inverse of a Toeplitz matrix and the
// circulant-embedded FFT products, Eq. eq:toeplitz_fft).
//
// With x = C^{-1} e_1, the inverse of the symmetric Toeplitz C is
//   C^{-1} = (L_x L_x^T - R_x^T R_x) / x_0,
// L_x lower-triangular Toeplitz with first column x, R_x upper-triangular
// Toeplitz with first row (0, x_{N-1}, ..., x_1).  So
//   chi2 = r^T C^{-1} r = (|L_x^T r|^2 - |R_x r|^2) / x_0,
// two triangular Toeplitz products, each the first N entries of a circular
// convolution of length M = 2^m >= 2N: O(N log N) per residual instead of the
// O(N^2) of a dense whitening operator, and O(N) memory per segment.
//
// Setup (td_gs_prepare, once per segment): x from the Levinson-Durbin chain
// (FP64, rows of L^{-1} not stored), the two embedding vectors' spectra by an
// FP64 radix-2 FFT, scaled by 1 / (M x_0) and rounded to FP32 (x_0 times the
// sums then gives chi2; the scaled spectra are 1 + small in the white-noise
// limit, so their rounding does not act as one common scale error).
//
// Per batch (k_gs_chi2): one thread-block cluster of eight CTAs per pair of
// residual columns, the pair packed as one complex signal r_a + i r_b (both
// convolution kernels are real, so the real and imaginary parts of the result
// stay the two columns' own).  CTA r holds M/8 consecutive values in shared
// memory, FP32.  A radix-2 decimation-in-frequency FFT (natural order in,
// bit-reversed out): its first three stages pair values M/2, M/4, M/8 apart,
// so they form one radix-8 pass across the cluster through distributed
// shared memory; the other stages stay inside each CTA (three per register
// pass).  Then the pointwise products with the two spectra (kept in the same
// bit-reversed order), and for each product the inverse network (decimation
// in time, bit-reversed in, natural out).  The sums of squares over the first
// N outputs run in double-float, each CTA's four sums in FP64 added by rank 0
// in rank order, which writes chi2 and logL.  The two terms hardly
// cancel (|R_x r|^2 is about 1% of |L_x^T r|^2 at N = 1024 for these
// covariances), so the FP32 FFTs' rounding carries over to chi2 about as is.
//
// Twiddles are applied as rotations built from three shears (lifting):
//   x1 = x + a y,  y1 = y + b x1,  x2 = x1 + a y1,   a = -tan(theta/2), b = sin(theta)
// (a quarter turn, exact, first when |theta| > pi/2).  Each shear has
// determinant one whatever the rounding of a and b, so the rotation keeps the
// signal's energy to second order; a complex product with (cos, sin) rounded
// to FP32 has |w|^2 - 1 of one sign at the stages with few distinct twiddles
// and biased chi2 by about -1.3e-7 (forward and inverse transform together),
// while the sheared form leaves about 2e-9.  The residual error is FP32
// rounding that averages over the N terms: ~1.5e-8 rms of chi2 at N = 1024,
// which sets the path's lower limit N >= 1024 (below it the dense paths are
// cheap anyway).
//
// A column shares its FFTs with its partner column, so its last bits depend
// on the partner: results agree within rounding, not bitwise, across batches.
#include <algorithm>
#include <climits>
#include <cmath>
#include <string>

#include <cooperative_groups.h>

#include "td_internal.h"

namespace cg = cooperative_groups;

namespace td {

constexpr int GS_CL = 8;          // CTAs per column pair: one thread-block cluster
constexpr int GS_MAX_LOGM = 16;   // M <= 65536 (N <= 32768): M/8 <= 8192 values per CTA
constexpr int64_t GS_MIN_N = 1024;
constexpr int GS_TWO_SIGNAL_LOGM = 16;

// one spare slot per 16: every register pass of the 2^14 network then reads and
// writes its groups at the two-wavefront minimum of 8-byte accesses
__device__ __forceinline__ int gpad(int i) { return i + (i >> 4); }

__device__ __forceinline__ float2 c_mul(float2 a, float2 w) {
  return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}

// Sign flips and swaps: (x, y) times (-i)^qd (forward) or (+i)^qd (inverse), exact.
template <bool INV>
__device__ __forceinline__ float2 quarter_turns(float x, float y, int qd) {
  const bool sw = qd & 1;
  const unsigned n1 = (unsigned)((qd ^ (qd >> 1)) & 1) << 31, n2 = (unsigned)((qd >> 1) & 1) << 31;
  const unsigned nr = INV ? n1 : n2, ns = INV ? n2 : n1;
  const float r = sw ? y : x, s = sw ? x : y;
  return make_float2(__uint_as_float(__float_as_uint(r) ^ nr), __uint_as_float(__float_as_uint(s) ^ ns));
}

// (x + i y) exp(-+ 2 pi i idx / L) for 0 <= idx < L: idx mod L/4 by three shears
// with lift[j] = (-tan(theta/2), sin(theta)), theta = -2 pi j / L, then the
// quarter turns idx div L/4
template <bool INV>
__device__ __forceinline__ float2 twiddle(float2 v, int idx, int logl, const float2* lift) {
  const float2 ab = lift[idx & ((1 << (logl - 2)) - 1)];
  const float a = INV ? -ab.x : ab.x, b = INV ? -ab.y : ab.y;
  const float x1 = fmaf(a, v.y, v.x);
  const float y1 = fmaf(b, x1, v.y);
  const float x2 = fmaf(a, y1, x1);
  return quarter_turns<INV>(x2, y1, idx >> (logl - 2));
}

// exp(-+ i pi/4) by three shears with constant coefficients
template <bool INV>
__device__ __forceinline__ float2 rot_eighth(float2 v) {
  const float a = INV ? -0.41421356237309503f : 0.41421356237309503f;   // tan(pi/8)
  const float b = INV ? 0.70710678118654752f : -0.70710678118654752f;   // sin(-+pi/4)
  const float x1 = fmaf(a, v.y, v.x);
  const float y1 = fmaf(b, x1, v.y);
  return make_float2(fmaf(a, y1, x1), y1);
}

template <int R>
__device__ __forceinline__ constexpr int brev(int m) {
  return R == 3 ? (((m & 1) << 2) | (m & 2) | ((m >> 2) & 1)) : (R == 2 ? (((m & 1) << 1) | ((m >> 1) & 1)) : m);
}

// R radix-2 stages s0 .. s0+R-1 of a length-L network on one group held in
// registers: v[k] is the element at o + k q of its block, q = L >> (s0+R).
// Stage s pairs elements h = L >> (s+1) apart inside blocks of 2h and gives the
// element at position p < h of its block the twiddle exp(-2 pi i p 2^s / L).
// Grouped, the R stages are a length-2^R DFT with constant twiddles (bit-
// reversed output) followed by exp(-2 pi i theta m / L) on output m, theta =
// o 2^s0: 2^R - 1 general twiddles per group instead of R 2^(R-1).
//   forward (DIF):  (a, b) -> (a + b, (a - b) w)
//   inverse (DIT):  the inverse of the forward group, times 2^R: conjugate
//                   twiddles first, then (u, t) -> (u + t conj(w), u - t conj(w))
//                   in decreasing stage order
template <int R, bool INV>
__device__ __forceinline__ void group_op(float2 (&v)[1 << R], int theta, int logl, const float2* lift) {
  constexpr int N = 1 << R;
  if (INV) {
#pragma unroll
    for (int m = 1; m < N; ++m) v[brev<R>(m)] = twiddle<true>(v[brev<R>(m)], theta * m, logl, lift);
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int st = INV ? R - 1 - i : i;
    const int d = 1 << (R - 1 - st);       // pair distance; the constant twiddle of pair k is exp(-2 pi i (k mod d) / 2d)
#pragma unroll
    for (int k = 0; k < N; ++k) {
      if (k & d) continue;
      const int e = (k & (d - 1)) * (8 / (2 * d));   // in eighths of a turn: 0, 1, 2 or 3
      if (!INV) {
        const float2 a = v[k], b = v[k + d];
        v[k] = make_float2(a.x + b.x, a.y + b.y);
        float2 t = make_float2(a.x - b.x, a.y - b.y);
        if (e & 1) t = rot_eighth<false>(t);
        if (e & 2) t = quarter_turns<false>(t.x, t.y, 1);
        v[k + d] = t;
      } else {
        float2 t = v[k + d];
        if (e & 2) t = quarter_turns<true>(t.x, t.y, 1);
        if (e & 1) t = rot_eighth<true>(t);
        const float2 a = v[k];
        v[k] = make_float2(a.x + t.x, a.y + t.y);
        v[k + d] = make_float2(a.x - t.x, a.y - t.y);
      }
    }
  }
  if (!INV) {
#pragma unroll
    for (int m = 1; m < N; ++m) v[brev<R>(m)] = twiddle<false>(v[brev<R>(m)], theta * m, logl, lift);
  }
}

// One register pass of the local length-2^logl networks of NSIG signals kept
// one after another in this CTA's buffer (signal j's value l at index
// j 2^logl + l); a thread takes the same group of every signal, so their
// arithmetic interleaves.
template <int R, bool INV, int NSIG>
__device__ __forceinline__ void fft_pass(float2* buf, const float2* lift, int logl, int s0) {
  const int lq = logl - s0 - R;
  const int q = 1 << lq;
  const int groups = 1 << (logl - R);
  for (int g = threadIdx.x; g < groups; g += blockDim.x) {
    const int o = g & (q - 1);
    const int base = ((g >> lq) << (logl - s0)) + o;
    float2 v[NSIG][1 << R];
#pragma unroll
    for (int j = 0; j < NSIG; ++j)
#pragma unroll
      for (int k = 0; k < (1 << R); ++k) v[j][k] = buf[gpad((j << logl) + base + k * q)];
#pragma unroll
    for (int j = 0; j < NSIG; ++j) group_op<R, INV>(v[j], o << s0, logl, lift);
#pragma unroll
    for (int j = 0; j < NSIG; ++j)
#pragma unroll
      for (int k = 0; k < (1 << R); ++k) buf[gpad((j << logl) + base + k * q)] = v[j][k];
  }
}

template <bool INV, int NSIG>
__device__ __forceinline__ void fft_run_pass(float2* buf, const float2* lift, int logl, int s0) {
  const int R = min(3, logl - s0);
  if (R == 3)
    fft_pass<3, INV, NSIG>(buf, lift, logl, s0);
  else if (R == 2)
    fft_pass<2, INV, NSIG>(buf, lift, logl, s0);
  else
    fft_pass<1, INV, NSIG>(buf, lift, logl, s0);
  __syncthreads();
}

template <int NSIG>
__device__ void fft_forward(float2* buf, const float2* lift, int logl) {
  for (int s0 = 0; s0 < logl; s0 += 3) fft_run_pass<false, NSIG>(buf, lift, logl, s0);
}
template <int NSIG>
__device__ void fft_inverse(float2* buf, const float2* lift, int logl) {
  for (int s0 = ((logl - 1) / 3) * 3; s0 >= 0; s0 -= 3) fft_run_pass<true, NSIG>(buf, lift, logl, s0);
}

// Stages 0..2 of the length-M network: elements M/2, M/4, M/8 apart, i.e. the
// group (o + k M/8, k = 0..7) holds local value o of every CTA of the
// cluster.  CTA r owns the groups o in [r ml/8, (r+1) ml/8) of every signal:
// it reads the eight values from the eight CTAs' shared memory, runs the three
// stages and writes them back; every value has one owner, so the pass needs
// no other ordering than the cluster barriers around it.
template <bool INV, int NSIG>
__device__ __forceinline__ void cross_pass(float2* buf, int logm, const float2* __restrict__ lift_g) {
  cg::cluster_group cl = cg::this_cluster();
  const int logml = logm - 3, per = (1 << logml) / GS_CL;
  const int o0 = (int)cl.block_rank() * per;
  float2* peer[GS_CL];
#pragma unroll
  for (int k = 0; k < GS_CL; ++k) peer[k] = cl.map_shared_rank(buf, k);
  for (int t = threadIdx.x; t < per; t += blockDim.x) {
    const int o = o0 + t;
    float2 v[NSIG][GS_CL];
#pragma unroll
    for (int j = 0; j < NSIG; ++j)
#pragma unroll
      for (int k = 0; k < GS_CL; ++k) v[j][k] = peer[k][gpad((j << logml) + o)];
#pragma unroll
    for (int j = 0; j < NSIG; ++j) group_op<3, INV>(v[j], o, logm, lift_g);
#pragma unroll
    for (int j = 0; j < NSIG; ++j)
#pragma unroll
      for (int k = 0; k < GS_CL; ++k) peer[k][gpad((j << logml) + o)] = v[j][k];
  }
}

// (hi, lo) double-float sums of a block, fixed order: shuffle tree per warp,
// then the warps in order; the result is valid in thread 0.  NV values per
// thread; red holds 32 x NV x 2 floats.
template <int NV>
__device__ __forceinline__ void block_sum_ff(float (&h)[NV], float (&l)[NV], float* red, double (&out)[NV]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float oh = __shfl_down_sync(0xffffffffu, h[j], off);
      const float ol = __shfl_down_sync(0xffffffffu, l[j], off);
      ff_add(oh, h[j], l[j]);
      l[j] += ol;
    }
    if (lane == 0) {
      red[(w * NV + j) * 2] = h[j];
      red[(w * NV + j) * 2 + 1] = l[j];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {   // FP64 is a slow pipe here: one thread adds the warps' pairs
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double s = 0.0;
      for (int i = 0; i < nw; ++i) s += (double)red[(i * NV + j) * 2] + (double)red[(i * NV + j) * 2 + 1];
      out[j] = s;
    }
  }
  __syncthreads();   // red is free again
}

__device__ __forceinline__ void sum_squares(const float2* buf, int base, int ml, int n, float& ha, float& la,
                                            float& hb, float& lb) {
  for (int l = threadIdx.x; l < ml && base + l < n; l += blockDim.x) {
    const float2 p = buf[gpad(l)];
    ff_add_square(p.x, ha, la);
    ff_add_square(p.y, hb, lb);
  }
}

// One cluster of GS_CL CTAs per NSIG column pairs (persistent over pairs).
// CTA r holds values [r ml, (r+1) ml) of each length-M signal, ml = M / GS_CL:
// cluster barrier, the cross pass (stages 0..2), cluster barrier, the local
// stages 3..m-1 (a length-ml network), the spectral products, and for each
// product the inverse in the opposite order.  Each CTA's partial sums are
// added by rank 0 in rank order.
template <int NSIG>
__global__ void __cluster_dims__(GS_CL, 1, 1) __launch_bounds__(NSIG == 1 ? 1024 : 512)
    k_gs_chi2(const float* __restrict__ R, int64_t ldr, int n, int K, int logm, const float2* __restrict__ S1,
              const float2* __restrict__ S2, const float2* __restrict__ lift_g, float2* __restrict__ scr, double x0,
              double logdet, double* __restrict__ logL, double* __restrict__ chi2, float rscale) {
  extern __shared__ float2 buf[];   // NSIG signals (gpad(NSIG ml) slots), then the ml/4 local twiddle shears
  __shared__ float red[32 * 4 * NSIG * 2];
  __shared__ double part[4 * NSIG];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int logml = logm - 3, ml = 1 << logml;
  const int npairs = (K + 1) / 2;
  const int cid = blockIdx.x / GS_CL, ncl = gridDim.x / GS_CL;
  const int base = rank * ml;
  float2* my = scr + ((int64_t)cid * GS_CL + rank) * ml * NSIG;
  float2* tws = buf + gpad(NSIG * ml);
  for (int i = threadIdx.x; i < ml / 4; i += blockDim.x) tws[i] = lift_g[GS_CL * i];   // exp(-2 pi i j / ml)
  for (int p0 = cid * NSIG; p0 < npairs; p0 += ncl * NSIG) {
#pragma unroll
    for (int j = 0; j < NSIG; ++j) {
      const int ca = 2 * (p0 + j), cb = ca + 1;
      const bool has_a = ca < K, has_b = cb < K;
      const float* ra = R + (int64_t)(has_a ? ca : 0) * ldr;
      const float* rb = R + (int64_t)(has_b ? cb : 0) * ldr;
      for (int l = threadIdx.x; l < ml; l += blockDim.x) {
        const int i = base + l;
        buf[gpad(j * ml + l)] =
            make_float2((i < n && has_a) ? ra[i] * rscale : 0.f, (i < n && has_b) ? rb[i] * rscale : 0.f);
      }
    }
    cl.sync();
    cross_pass<false, NSIG>(buf, logm, lift_g);
    cl.sync();
    fft_forward<NSIG>(buf, tws, logml);
    for (int l = threadIdx.x; l < NSIG * ml; l += blockDim.x) {
      const int g = base + (l & (ml - 1));
      const float2 y = buf[gpad(l)];
      buf[gpad(l)] = c_mul(y, __ldg(&S1[g]));
      my[l] = c_mul(y, __ldg(&S2[g]));   // the same thread reads it back below
    }
    __syncthreads();
    float h[4 * NSIG], lo[4 * NSIG];
#pragma unroll
    for (int j = 0; j < 4 * NSIG; ++j) h[j] = lo[j] = 0.f;
    fft_inverse<NSIG>(buf, tws, logml);
    cl.sync();
    cross_pass<true, NSIG>(buf, logm, lift_g);
    cl.sync();
#pragma unroll
    for (int j = 0; j < NSIG; ++j)
      sum_squares(buf + gpad(j * ml), base, ml, n, h[4 * j], lo[4 * j], h[4 * j + 1], lo[4 * j + 1]);
    __syncthreads();
    for (int l = threadIdx.x; l < NSIG * ml; l += blockDim.x) buf[gpad(l)] = my[l];
    __syncthreads();
    fft_inverse<NSIG>(buf, tws, logml);
    cl.sync();
    cross_pass<true, NSIG>(buf, logm, lift_g);
    cl.sync();
#pragma unroll
    for (int j = 0; j < NSIG; ++j)
      sum_squares(buf + gpad(j * ml), base, ml, n, h[4 * j + 2], lo[4 * j + 2], h[4 * j + 3], lo[4 * j + 3]);
    double s[4 * NSIG];
#pragma unroll
    for (int j = 0; j < 4 * NSIG; ++j) s[j] = 0.0;
    block_sum_ff<4 * NSIG>(h, lo, red, s);
    if (threadIdx.x == 0)
      for (int j = 0; j < 4 * NSIG; ++j) part[j] = s[j];
    cl.sync();
    if (rank == 0 && threadIdx.x == 0) {
      double t[4 * NSIG];
      for (int j = 0; j < 4 * NSIG; ++j) t[j] = 0.0;
      for (int r = 0; r < GS_CL; ++r) {
        const double* pr = cl.map_shared_rank(part, r);
        for (int j = 0; j < 4 * NSIG; ++j) t[j] += pr[j];
      }
      for (int j = 0; j < NSIG; ++j) {
        const int ca = 2 * (p0 + j), cb = ca + 1;
        for (int c = 0; c < 2; ++c) {
          const int col = c == 0 ? ca : cb;
          if (col >= K) continue;
          const double c2 = x0 * (t[4 * j + c] - t[4 * j + 2 + c]);
          logL[col] = -0.5 * c2 - 0.5 * logdet - 0.5 * (double)n * LOG2PI;
          if (chi2) chi2[col] = c2;
        }
      }
    }
    // the next iteration's first cluster barrier orders rank 0's reads of
    // part[] before any CTA writes it again
  }
  cl.sync();   // no CTA leaves while rank 0 may still read its partial sums
}

// ---------------------------------------------------------------- setup

// the two circulant embeddings (length M) of the GS factors' products:
//   c1: L_x^T (upper Toeplitz, first row x):        c1[0] = x_0, c1[M - i] = x_i
//   c2: R_x   (upper Toeplitz, first row (0, x_{N-1}, ..., x_1)): c2[M - j] = x_{N-j}
__global__ void k_gs_embed(const double* __restrict__ x, int n, int logm, double2* __restrict__ c) {
  const int M = 1 << logm;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    double v1 = 0.0, v2 = 0.0;
    if (i == 0) v1 = x[0];
    const int j = M - i;   // i = M - j
    if (i > 0 && j >= 1 && j <= n - 1) {
      v1 = x[j];
      v2 = x[n - j];
    }
    c[i] = make_double2(v1, 0.0);
    c[M + i] = make_double2(v2, 0.0);
  }
}

// one radix-2 DIF stage in FP64, in global memory, on the two arrays (blockIdx.y)
__global__ void k_fft64_stage(double2* __restrict__ X, int logm, int s) {
  const int M = 1 << logm;
  const int lh = logm - s - 1;
  double2* A = X + (int64_t)blockIdx.y * M;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < M / 2; t += gridDim.x * blockDim.x) {
    const int p = t & ((1 << lh) - 1);
    const int i = ((t >> lh) << (lh + 1)) + p, j = i + (1 << lh);
    double sn, cs;
    sincospi(-(double)p * (double)(1 << (s + 1)) / (double)M, &sn, &cs);
    const double2 a = A[i], b = A[j];
    const double dx = a.x - b.x, dy = a.y - b.y;
    A[i] = make_double2(a.x + b.x, a.y + b.y);
    A[j] = make_double2(dx * cs - dy * sn, dx * sn + dy * cs);
  }
}

__global__ void k_gs_spectra(const double2* __restrict__ X, const double* __restrict__ x, int logm,
                             float2* __restrict__ S1, float2* __restrict__ S2, float2* __restrict__ lift) {
  const int M = 1 << logm;
  const double scale = 1.0 / ((double)M * x[0]);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    const double2 a = X[i], b = X[M + i];
    S1[i] = make_float2((float)(a.x * scale), (float)(a.y * scale));
    S2[i] = make_float2((float)(b.x * scale), (float)(b.y * scale));
    if (i < M / 4) {   // theta = -2 pi i / M in (-pi/2, 0]: a = -tan(theta/2) = tan(pi i / M), b = sin(theta)
      double sh, ch, sn, cs;
      sincospi((double)i / (double)M, &sh, &ch);
      sincospi(-2.0 * (double)i / (double)M, &sn, &cs);
      lift[i] = make_float2((float)(sh / ch), (float)sn);
    }
  }
}

template <class T>
static void gs_free(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

bool gs_supported(const td_segment* s) {
  return s->nk == s->n && s->n >= GS_MIN_N && s->n <= ((int64_t)1 << (GS_MAX_LOGM - 1));
}

void free_gs_state(td_segment* s) {
  GsState& g = s->gs;
  gs_free(g.S1);
  gs_free(g.S2);
  gs_free(g.tw);
  gs_free(g.scr);
  g.scr_elems = 0;
  g.ready = false;
}

// per CTA: ml = M / GS_CL values per signal; one thread per radix-8 group of the local passes
static int gs_threads(int logm, int nsig) {
  return std::max(32, std::min(nsig == 1 ? 1024 : 512, (1 << (logm - 3)) / 8));
}
static size_t gs_smem(int logm, int nsig) {
  const int ml = 1 << (logm - 3), tot = nsig * ml;
  return (size_t)(tot + (tot >> 4) + (ml >> 2)) * sizeof(float2);
}

template <int NSIG>
static td_status gs_launch(GsState& g, const float* R, int64_t ldr, int n, int64_t K, double* logL, double* chi2,
                           cudaStream_t st, bool query_only, int* clusters_out) {
  const int threads = gs_threads(g.logm, NSIG);
  const size_t smem = gs_smem(g.logm, NSIG);
  static std::atomic<unsigned long long> attr_done{0};
  if (device_needs_setup(attr_done)) {
    TD_CUDA(cudaFuncSetAttribute(k_gs_chi2<NSIG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)gs_smem(GS_MAX_LOGM, NSIG)));
    // small CTAs (22 KB at N = 8192): let as many share an SM as the registers allow
    TD_CUDA(cudaFuncSetAttribute(k_gs_chi2<NSIG>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    mark_device_done(attr_done);
  }
  const int64_t npairs = (K + 1) / 2, units = (npairs + NSIG - 1) / NSIG;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(GS_CL * std::min<int64_t>(units, 4096)));
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  int max_clusters = 0;
  TD_CUDA(cudaOccupancyMaxActiveClusters(&max_clusters, k_gs_chi2<NSIG>, &cfg));
  if (max_clusters < 1) return fail(TD_ERR_CUDA, "GSCE cluster does not fit the device");
  const int clusters = (int)std::min<int64_t>(units, max_clusters);
  *clusters_out = clusters;
  if (query_only) return TD_OK;
  const int64_t need = ((int64_t)clusters * NSIG) << g.logm;   // NSIG length-M product buffers per cluster
  if (need > g.scr_elems) {
    cudaStreamSynchronize(st);
    gs_free(g.scr);
    g.scr_elems = 0;
    if (cudaMalloc((void**)&g.scr, (size_t)need * sizeof(float2)) != cudaSuccess) {
      cudaGetLastError();
      return fail(TD_ERR_OOM, "GSCE product buffer");
    }
    g.scr_elems = need;
  }
  // Residuals enter the FP32 transforms multiplied by 2^k with 2^{2k} ~ x_0
  // (so the whitened values are of order one whatever the units of the
  // data: strain-scale residuals of ~1e-21 would otherwise square into FP32
  // subnormals); chi2 takes x_0 / 2^{2k}.  A power of two scales every FP32
  // step exactly, so the result's bits do not depend on k.
  const int k = (int)std::max(-120L, std::min(120L, std::lround(0.5 * std::log2(g.x0))));
  const float rscale = std::ldexp(1.0f, k);
  k_gs_chi2<NSIG><<<clusters * GS_CL, threads, smem, st>>>(R, ldr, n, (int)K, g.logm, g.S1, g.S2, g.tw, g.scr,
                                                           std::ldexp(g.x0, -2 * k), g.logdet, logL, chi2,
                                                           rscale);
  TD_CUDA(cudaGetLastError());
  return TD_OK;
}

// Two signals per CTA halve the barriers per column pair and let each thread
// interleave two groups, at 127 registers a thread.  Measured at K = 2048-4096:
// N = 32768 (M = 65536) 4.8 ms against 5.9 ms with one signal; N = 16384 2.8 ms
// against 2.1 ms and N = 8192 2.0 ms against 1.4 ms (the registers then halve
// the resident CTAs).  So two
// signals from M = 2^GS_TWO_SIGNAL_LOGM on, and only once the pairs outnumber
// the clusters one signal keeps resident (small batches keep one pair per
// cluster, for latency).
td_status gs_batch(td_segment* s, const float* R, int64_t ldr, int64_t K, double* logL, double* chi2,
                   cudaStream_t st) {
  GsState& g = s->gs;
  if (K > INT_MAX - 1) return fail(TD_ERR_INVALID, "K too large for the GSCE path");
  int resident1 = 0;
  td_status r = gs_launch<1>(g, R, ldr, (int)s->n, K, logL, chi2, st, true, &resident1);
  if (r != TD_OK) return r;
  const int64_t npairs = (K + 1) / 2;
  int used = 0;
  r = (g.logm >= GS_TWO_SIGNAL_LOGM && npairs > (int64_t)resident1) ? gs_launch<2>(g, R, ldr, (int)s->n, K, logL, chi2, st, false, &used)
                                  : gs_launch<1>(g, R, ldr, (int)s->n, K, logL, chi2, st, false, &used);
  if (r != TD_OK) return r;
  s->prof_kernels += 1;
  return TD_OK;
}

}  // namespace td

using namespace td;

extern "C" td_status td_gs_prepare(td_segment* s, void* stream) {
  if (!s) return fail(TD_ERR_INVALID, "segment is NULL");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != s->device) return fail(TD_ERR_INVALID, "segment belongs to another device; set it current first");
  if (s->nk != s->n) return fail(TD_ERR_UNSUPPORTED, "GSCE needs a gap-free (Toeplitz) segment");
  int logm = 4;
  while ((1LL << logm) < 2 * s->n) ++logm;
  if (logm > GS_MAX_LOGM) return fail(TD_ERR_UNSUPPORTED, "GSCE takes N <= 32768 samples in this version");
  if (s->n < GS_MIN_N)
    return fail(TD_ERR_UNSUPPORTED, "GSCE takes N >= 1024 samples (FP32 FFT rounding is not averaged enough below)");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  free_gs_state(s);
  const int M = 1 << logm;
  double *a0 = nullptr, *a1 = nullptr, *x = nullptr, *ld = nullptr, *vh = nullptr;
  double2* c = nullptr;
  LevJob* dj = nullptr;
  GsState& g = s->gs;
  td_status r = TD_OK;
  auto cleanup = [&]() {
    for (double** p : {&a0, &a1, &x, &ld, &vh}) gs_free(*p);
    gs_free(c);
    gs_free(dj);
  };
  if (cudaMalloc((void**)&a0, (size_t)s->n * 8) != cudaSuccess || cudaMalloc((void**)&a1, (size_t)s->n * 8) != cudaSuccess ||
      cudaMalloc((void**)&x, (size_t)s->n * 8) != cudaSuccess || cudaMalloc((void**)&ld, 8) != cudaSuccess ||
      cudaMalloc((void**)&vh, (size_t)s->n * 8) != cudaSuccess ||
      cudaMalloc((void**)&c, (size_t)2 * M * sizeof(double2)) != cudaSuccess ||
      cudaMalloc((void**)&dj, sizeof(LevJob)) != cudaSuccess ||
      cudaMalloc((void**)&g.S1, (size_t)M * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&g.S2, (size_t)M * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&g.tw, (size_t)(M / 4) * sizeof(float2)) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    free_gs_state(s);
    return fail(TD_ERR_OOM, "GSCE setup buffers");
  }
  const LevJob job{s->acf, s->n, a0, a1, nullptr, 0, ld, s->status, x, vh};
  DevStatus h0{0, 0, LLONG_MAX};
  cudaError_t e = cudaMemcpyAsync(s->status, &h0, sizeof h0, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dj, &job, sizeof job, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_levinson_rows(dj, 1, st);
  const int blocks = (int)std::min<int64_t>(1024, ceil_div(M, 256));
  if (e == cudaSuccess) {
    k_gs_embed<<<blocks, 256, 0, st>>>(x, (int)s->n, logm, c);
    e = cudaGetLastError();
  }
  for (int stg = 0; stg < logm && e == cudaSuccess; ++stg) {
    k_fft64_stage<<<dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>(1024, ceil_div(M / 2, 256))), 2), 256, 0,
                    st>>>(c, logm, stg);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_gs_spectra<<<blocks, 256, 0, st>>>(c, x, logm, g.S1, g.S2, g.tw);
    e = cudaGetLastError();
  }
  DevStatus hs{0, 0, 0};
  double logdet = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, s->status, sizeof hs, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&logdet, ld, 8, cudaMemcpyDeviceToHost, st);
  double x0 = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&x0, x, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) {
    free_gs_state(s);
    return cuda_fail(e, "GSCE setup");
  }
  if (hs.code == ST_NOT_PD) {
    free_gs_state(s);
    s->pivot = hs.pivot;
    char buf[128];
    snprintf(buf, sizeof buf, "covariance not positive definite at kept sample %lld", (long long)hs.pivot);
    return fail(TD_ERR_NOT_PD, buf);
  }
  g.logm = logm;
  g.logdet = logdet;
  g.x0 = x0;
  g.ready = true;
  return r;
}
