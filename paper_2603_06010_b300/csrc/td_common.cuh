// Device-side helpers shared by the kernels: inline-PTX wrappers for mbarrier,
// TMA (cp.async.bulk.tensor), tcgen05 (TMEM alloc / MMA / commit / ld), a
// bounded wait on the global nanosecond timer, and bf16 slicing.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace td {

// device status word codes (mirror td_status)
enum : int { ST_OK = 0, ST_NOT_PD = 2, ST_TIMEOUT = 5 };

struct DevStatus {
  int code;          // first error code (atomicCAS from 0)
  int where;         // which wait ran out (kernel-specific tag)
  long long pivot;   // min failing pivot (factor)
  // measurement: SM cycles and global-timer nanoseconds over the spans the
  // split-product kernel's MMA-issuing threads ran (summed over CTAs); their
  // ratio is the SM clock the kernel actually ran at
  unsigned long long mma_cycles;
  unsigned long long mma_ns;
};

__device__ __forceinline__ void set_status(DevStatus* st, int code, int where) {
  if (atomicCAS(&st->code, 0, code) == 0) st->where = where;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of parity `parity` to complete, giving up after limit_ns.
// Returns false when the bound ran out (the caller records TD_ERR_TIMEOUT).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

// ---------------------------------------------------------------- TMA
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}
__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ---------------------------------------------------------------- tcgen05
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D[tmem] (+)= A[smem desc] * B[smem desc]^T, kind::f16 (bf16 inputs, fp32 accumulate)
__device__ __forceinline__ void tc_mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// The same MMA with a collector-buffer hint for A (USE 1: fill, 2: use, 3:
// last use): consecutive MMAs of one thread that share their A operand read it
// from shared memory once.
template <int USE>
__device__ __forceinline__ void tc_mma_f16_a(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                             uint32_t accumulate) {
  static_assert(USE >= 1 && USE <= 3, "collector usage");
  if constexpr (USE == 1)
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  else if constexpr (USE == 2)
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16.collector::a::use [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// arrive on an mbarrier once every MMA issued so far by this thread has completed
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
// 32 lanes x 32 consecutive 32-bit columns -> 32 registers per thread
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
        "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
        "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor (tcgen05): K-major operand, rows of 64 B
// (32 bf16) stored contiguously, 64-byte swizzle; 8-row core groups are
// 512 B apart (stride byte offset); the leading byte offset is unused for a
// swizzled K-major operand whose MMA K extent (32 B) fits the 64 B atom.
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);        // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused) = 16 B
  d |= (uint64_t)((512 >> 4) & 0x3FFF) << 32;      // stride byte offset = 512 B
  d |= (uint64_t)1 << 46;                          // descriptor version (0b001)
  d |= (uint64_t)4 << 61;                          // swizzle: 64 B
  return d;
}
// Instruction descriptor, kind::f16: bf16 x bf16 -> f32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4)                       // D format f32
         | (1u << 7)                     // A format bf16
         | (1u << 10)                    // B format bf16
         | ((uint32_t)(N >> 3) << 17)    // N / 8
         | ((uint32_t)(M >> 4) << 24);   // M / 16
}

// The split products of one 16-deep step (both operands K-major, 64-byte
// swizzle, slices a_slice / b_slice bytes apart, kofs the step's byte offset
// in the 64-byte rows): A slice a against B slices b = NSL-1-a ... 0, the
// smaller products first.  (0, 0) is the exact hi*hi sum and goes to d_hi,
// every other product to d_lo; `first` = 0 starts both accumulators.  The
// MMAs of one A slice follow each other, so the collector buffer keeps that
// slice and shared memory delivers each A slice once per step instead of once
// per product.
template <int NSL>
__device__ __forceinline__ void split_products_step(uint32_t d_hi, uint32_t d_lo, uint32_t sa, uint32_t a_slice,
                                                    uint32_t sb, uint32_t b_slice, uint32_t kofs, uint32_t idesc,
                                                    uint32_t first) {
#pragma unroll
  for (int a = 0; a < NSL; ++a) {
    const uint64_t ad = smem_desc_sw64(sa + a * a_slice + kofs);
#pragma unroll
    for (int b = NSL - 1 - a; b >= 0; --b) {
      const int n = NSL - a;           // MMAs sharing this A slice
      const int i = NSL - 1 - a - b;   // position among them
      const uint64_t bd = smem_desc_sw64(sb + b * b_slice + kofs);
      const bool hh = a == 0 && b == 0;
      const uint32_t d = hh ? d_hi : d_lo;
      const uint32_t acc = (hh || (a == 0 && b == NSL - 1)) ? first : 1u;
      if (n == 1)
        tc_mma_f16(d, ad, bd, idesc, acc);
      else if (i == 0)
        tc_mma_f16_a<1>(d, ad, bd, idesc, acc);
      else if (i == n - 1)
        tc_mma_f16_a<3>(d, ad, bd, idesc, acc);
      else
        tc_mma_f16_a<2>(d, ad, bd, idesc, acc);
    }
  }
}
// ---------------------------------------------------------------- slicing
// x = s0 + s1 + s2 with each s a bf16 (round-to-nearest on the running
// remainder, computed exactly in the wider type).
__device__ __forceinline__ void split3_f64(double x, __nv_bfloat16& s0, __nv_bfloat16& s1, __nv_bfloat16& s2) {
  s0 = __double2bfloat16(x);
  double r = x - (double)__bfloat162float(s0);
  s1 = __double2bfloat16(r);
  r = r - (double)__bfloat162float(s1);
  s2 = __double2bfloat16(r);
}
__device__ __forceinline__ void split3_f32(float x, __nv_bfloat16& s0, __nv_bfloat16& s1, __nv_bfloat16& s2) {
  s0 = __float2bfloat16_rn(x);
  float r = x - __bfloat162float(s0);   // exact: s0 is x rounded to 8 significant bits
  s1 = __float2bfloat16_rn(r);
  r = r - __bfloat162float(s1);         // exact
  s2 = __float2bfloat16_rn(r);
}

// Residual slices: the column's power-of-two quantum p_k
// (max_j |R_jk| <= 255 p_k), then R = p_k b0 + r with r in up to three
// floating bf16 slices (all four slices hold a float32 exactly).
__device__ __forceinline__ float r_quantum(float mx) {
  float p = 1.f;
  if (mx > 0.f) {
    p = exp2f(ceilf(log2f(mx / 255.f)));
    if (mx / p > 255.f) p *= 2.f;
  }
  return p;
}
__device__ __forceinline__ void r_slice_value(float x, float p, __nv_bfloat16 (&o)[4]) {
  const float hi = p * rintf(x / p);
  o[0] = __float2bfloat16_rn(hi);
  split3_f32(x - hi, o[1], o[2], o[3]);
}

// exact square w*w = p + e and compensated accumulation into (hi, lo)
__device__ __forceinline__ void ff_add_square(float w, float& hi, float& lo) {
  float p = w * w;
  float e = fmaf(w, w, -p);
  float t = hi + p;
  float bp = t - hi;
  float err = (hi - (t - bp)) + (p - bp);
  hi = t;
  lo += err + e;
}

// (hi, lo) += a, compensated (two-sum on the head)
__device__ __forceinline__ void ff_add(float a, float& hi, float& lo) {
  float t = hi + a;
  float bp = t - hi;
  float err = (hi - (t - bp)) + (a - bp);
  hi = t;
  lo += err;
}

// (a + b)^2 for an FP32 pair whose sum is the value: two-sum first, then the
// exact square of the head and the cross term, accumulated into (hi, lo)
__device__ __forceinline__ void ff_add_square2(float a, float b, float& hi, float& lo) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);   // a + b = s + e exactly
  float p = s * s;
  float pe = fmaf(s, s, -p);             // s*s = p + pe exactly
  float t = hi + p;
  float bp = t - hi;
  float err = (hi - (t - bp)) + (p - bp);
  hi = t;
  lo += err + pe + 2.f * s * e;
}

}  // namespace td
