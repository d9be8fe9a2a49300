// Device helpers of the tensor-core evaluation kernels: shared-memory and
// instruction descriptors of tcgen05.mma kind::f16, tensor-memory loads,
// mbarriers with a bounded wait, bulk copies, packed FP32 pairs, and the two
// arithmetic steps every form of the mixed evaluation shares bit for bit:
// the log coordinates of a point (op. 1 of Algorithm 2) and the complex
// exponential of eight monomials split into BF16 operand parts (eq. (8)).
// Internal to libhpt.
#pragma once

#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

namespace hpt {
namespace {

__device__ __forceinline__ uint32_t su32(const void* ptr) {
  return (uint32_t)__cvta_generic_to_shared(ptr);
}

// Shared-memory matrix descriptor: canonical K-major layout, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);           // start address
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;       // leading byte offset (K)
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;       // stride byte offset (M/N)
  d |= (uint64_t)1 << 46;                            // descriptor version
  return d;                                          // no swizzle, base offset 0
}

// kind::f16 instruction descriptor: FP32 D, BF16 A and B, both K-major.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// The coefficient GEMM [D_z h | D_tau h | h] = E B^T in three passes per
// K-slice, hi*hi, hi*lo and lo*hi.  a_hi, a_lo, b_hi, b_lo are the
// descriptors of the first 256-byte K-slice (B_lo's rows follow B_hi's, so
// b_hi with N = 2 NJ spans both); a K-slice adds 16 to a descriptor's address
// field.  Grouped (MixedSys::jst): J in three column groups, E_hi [B_hi;
// B_lo]^T into columns [tj, tj + 2 NJ) by coef_gemm_hi and E_lo B_hi^T into
// [tj + 2 NJ, tj + 3 NJ) by coef_gemm_lo, J = (hh + hl) + lh; two MMAs per
// K-slice, and the two parts can be issued by two threads at once (an MMA
// costs its issuing thread about a hundred cycles whatever its N).  Else
// three MMAs per K-slice into one accumulator of NJ columns.  The whole warp
// calls these; lane 0 issues.
__device__ __forceinline__ void coef_gemm_hi(uint32_t tj, uint64_t a_hi, uint64_t b_hi, int NJ, int kslices);
__device__ __forceinline__ void coef_gemm_lo(uint32_t tj, uint64_t a_lo, uint64_t b_hi, int NJ, int kslices);
__device__ __forceinline__ void coef_gemm(uint32_t tj, uint64_t a_hi, uint64_t a_lo, uint64_t b_hi, uint64_t b_lo,
                                          int NJ, int kslices, bool grouped);

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

// The same two instructions for a whole warp that runs the issue loop
// together: the operands stay warp-uniform (no per-thread copies into the
// uniform datapath on every MMA) and lane 0 issues.  Always the same lane:
// a commit tracks the MMAs its own thread issued before it, and the
// pipelined evaluation relies on that order.
__device__ __forceinline__ void mma_bf16_w(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                           uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p, e;\n .reg .u32 l;\n setp.ne.b32 p, %4, 0;\n mov.u32 l, %%laneid;\n"
      " setp.eq.u32 e, l, 0;\n"
      " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit_w(uint32_t mbar) {
  asm volatile(
      "{\n .reg .pred e;\n .reg .u32 l;\n mov.u32 l, %%laneid;\n setp.eq.u32 e, l, 0;\n"
      " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(mbar)
      : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void coef_gemm_hi(uint32_t tj, uint64_t a_hi, uint64_t b_hi, int NJ, int kslices) {
  const uint32_t id = idesc_bf16(128, 2 * NJ);
  for (int s = 0; s < kslices; ++s) mma_bf16_w(tj, a_hi + 16 * s, b_hi + 16 * s, id, s > 0);
}
__device__ __forceinline__ void coef_gemm_lo(uint32_t tj, uint64_t a_lo, uint64_t b_hi, int NJ, int kslices) {
  const uint32_t id = idesc_bf16(128, NJ);
  for (int s = 0; s < kslices; ++s) mma_bf16_w(tj + 2 * (uint32_t)NJ, a_lo + 16 * s, b_hi + 16 * s, id, s > 0);
}
__device__ __forceinline__ void coef_gemm(uint32_t tj, uint64_t a_hi, uint64_t a_lo, uint64_t b_hi, uint64_t b_lo,
                                          int NJ, int kslices, bool grouped) {
  if (grouped) {
    coef_gemm_hi(tj, a_hi, b_hi, NJ, kslices);
    coef_gemm_lo(tj, a_lo, b_hi, NJ, kslices);
    return;
  }
  const uint32_t id = idesc_bf16(128, NJ);
  for (int s = 0; s < kslices; ++s) {
    mma_bf16_w(tj, a_hi + 16 * s, b_hi + 16 * s, id, s > 0);
    mma_bf16_w(tj, a_hi + 16 * s, b_lo + 16 * s, id, 1);
    mma_bf16_w(tj, a_lo + 16 * s, b_hi + 16 * s, id, 1);
  }
}

// Eight J columns from c0 of the coefficient accumulator at taddr (grouped:
// the three column groups added, (hh + hl) + lh).
__device__ __forceinline__ void tmem_ld8_j(uint32_t taddr, int NJ, bool grouped, float (&v)[8]) {
  uint32_t a[8], b[8], c[8];
  tmem_ld8(taddr, a);
  if (grouped) {
    tmem_ld8(taddr + (uint32_t)NJ, b);
    tmem_ld8(taddr + 2 * (uint32_t)NJ, c);
  }
  tmem_wait_ld();
#pragma unroll
  for (int q = 0; q < 8; ++q)
    v[q] = grouped ? (__uint_as_float(a[q]) + __uint_as_float(b[q])) + __uint_as_float(c[q]) : __uint_as_float(a[q]);
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}
// One potentially blocking test of phase `parity`: the thread may be
// suspended until the phase completes or about 0.1 ms have passed (the time
// hint), so a waiting warp does not spin through issue slots.
__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity), "r"(100000u)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Non-blocking test of phase `parity` (the cheap path when it has completed).
__device__ __forceinline__ bool mbar_test(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after ~2 s of global time.
__device__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  if (mbar_test(mbar, parity)) return true;
  const uint64_t t0 = gtimer();
  for (;;) {
    if (mbar_try(mbar, parity)) return true;
    if (gtimer() - t0 > 2000000000ull) return false;
  }
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ int canon(int r, int k, int K) {
  return (r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint16_t bf16_rn(float v) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
__device__ __forceinline__ float bf16_f(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }

// Packed FP32 pairs (sm_100 family): one instruction rounds each half exactly
// as the scalar operation would, so the results are those of the scalar code.
__device__ __forceinline__ uint64_t f2pk(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2up(uint64_t v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {   // a * b + c
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

constexpr float kLog2E = 1.44269504088896341f;     // log2(e)
constexpr float kInvTwoPi = 0.159154943091895336f;
constexpr float kTwoPi = 6.28318530717958648f;

// Op. 1 in the units of the exponential below: Re z = log2 |y| and
// Im z = arg(y) / (2 pi) (principal branch, revolutions), so that Re W is an
// exponent of 2 and Im W a phase in revolutions, whose reduction modulo 1 is
// one exact subtraction.  The t-exponent term of Re W is (tau / D) log2(e) e.
__device__ __forceinline__ void log_coords(float2 v, float& zr, float& zi) {
  zr = log2f(hypotf(v.x, v.y));
  zi = atan2f(v.y, v.x) * kInvTwoPi;
}

// A point's angle arg(y) / (2 pi) (revolutions, the Im z of log_coords) in
// 32-bit fixed point, units of 2^-32 revolution (rounded to the nearest unit,
// an error far below the FP32 angle's own for any angle above 2^-8); sums of
// integer multiples of such angles reduce modulo one revolution exactly by
// wrapping.
__device__ __forceinline__ uint32_t fixed_angle(float zi) {
  return (uint32_t)(unsigned long long)llrintf(zi * 4294967296.f);
}

// E = 2^(Re W + tau2 e) (cos 2 pi r, sin 2 pi r), r = Im W - rint(Im W), for
// the eight monomials of one 8-column chunk (wre, wim: the chunk's exponent
// accumulators, texp: their t-exponents); returns Re E and Im E each split
// into BF16 hi + lo (hi = RN(E), lo = RN(E - hi)), eight values to a uint4.
// Monomials whose bit is set in big8 (sum |a_j| above kBigPhase, whose FP32
// phase accumulation would lose accuracy) take r = (sum_j a_j q_j mod 2^32)
// 2^-32 instead: aint their int16 exponent vectors (n per monomial), zq the
// point's fixed angles with stride 128.
__device__ __forceinline__ void cexp_split8(const uint32_t (&wre)[8], const uint32_t (&wim)[8],
                                            const float* __restrict__ texp, float tau2, uint32_t big8,
                                            const int16_t* __restrict__ aint, const uint32_t* __restrict__ zq,
                                            int n, uint4& hre, uint4& lre, uint4& him, uint4& lim) {
  const uint64_t TAU = f2pk(tau2, tau2), TWO_PI = f2pk(kTwoPi, kTwoPi);
  float rr[8];
#pragma unroll
  for (int q = 0; q < 8; q += 2) {
    const float i0 = __uint_as_float(wim[q]), i1 = __uint_as_float(wim[q + 1]);
    f2up(sub2(f2pk(i0, i1), f2pk(rintf(i0), rintf(i1))), rr[q], rr[q + 1]);
  }
  if (big8) {   // the same for every point of the tile: a uniform branch
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (big8 & (1u << q)) {
        uint32_t ph = 0;
        for (int j = 0; j < n; ++j) ph += (uint32_t)(int32_t)aint[q * n + j] * zq[j * 128];
        rr[q] = (float)(int32_t)ph * 2.3283064365386963e-10f;   // 2^-32
      }
    }
  }
  uint32_t hr[4], hi_[4], lr[4], li[4];
#pragma unroll
  for (int q = 0; q < 8; q += 2) {
    const float2 te = *(const float2*)&texp[q];
    const uint64_t wr = fma2(TAU, f2pk(te.x, te.y), f2pk(__uint_as_float(wre[q]), __uint_as_float(wre[q + 1])));
    float x0, x1;
    f2up(mul2(f2pk(rr[q], rr[q + 1]), TWO_PI), x0, x1);
    float s0, c0, s1, c1;
    __sincosf(x0, &s0, &c0);
    __sincosf(x1, &s1, &c1);
    float w0, w1;
    f2up(wr, w0, w1);
    const uint64_t m = f2pk(ex2_approx(w0), ex2_approx(w1));
    float er0, er1, ei0, ei1;
    const uint64_t er = mul2(m, f2pk(c0, c1)), ei = mul2(m, f2pk(s0, s1));
    f2up(er, er0, er1);
    f2up(ei, ei0, ei1);
    const __nv_bfloat162 hre2 = __floats2bfloat162_rn(er0, er1);
    const __nv_bfloat162 him2 = __floats2bfloat162_rn(ei0, ei1);
    const float2 fre = __bfloat1622float2(hre2), fim = __bfloat1622float2(him2);
    float lr0, lr1, li0, li1;
    f2up(sub2(er, f2pk(fre.x, fre.y)), lr0, lr1);
    f2up(sub2(ei, f2pk(fim.x, fim.y)), li0, li1);
    const __nv_bfloat162 lre2 = __floats2bfloat162_rn(lr0, lr1);
    const __nv_bfloat162 lim2 = __floats2bfloat162_rn(li0, li1);
    hr[q / 2] = *(const uint32_t*)&hre2;
    hi_[q / 2] = *(const uint32_t*)&him2;
    lr[q / 2] = *(const uint32_t*)&lre2;
    li[q / 2] = *(const uint32_t*)&lim2;
  }
  hre = make_uint4(hr[0], hr[1], hr[2], hr[3]);
  lre = make_uint4(lr[0], lr[1], lr[2], lr[3]);
  him = make_uint4(hi_[0], hi_[1], hi_[2], hi_[3]);
  lim = make_uint4(li[0], li[1], li[2], li[3]);
}

}  // namespace
}  // namespace hpt
