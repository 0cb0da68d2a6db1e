// Fifth-generation tensor-core primitives (sm_103a, inline PTX) and the split of
// FP64 values into bf16 slices used by the tensor-core leaf solves (tc.cu).
//
// Split (an error-free transformation in the style of Ozaki et al.): a real value v
// with |v| < 2^(e-1) is written as v = 2^e * sum_{i=1..S} t_i 2^(-7 i) + r with
// integers |t_1| <= 64, |t_i| <= 127 (truncation of the fixed-point expansion of
// v / 2^e, sign carried by every t_i) and |r| < 2^(e - 7 S).  Each slice
// t_i 2^(-7 i) is exact in bf16.  A product of two slices is t_i u_j 2^(-7 (i+j));
// all products of one level l = i + j share the factor 2^(-7 l), so their sum over
// K terms is an integer multiple of it, exact in an FP32 accumulator while that
// integer stays below 2^24 (levels 2 and 3 for K <= 1040).  Deeper levels carry
// 2^-21 and less of the leading level and are summed in one FP32 accumulator.
#pragma once

#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>

namespace eo {
namespace tc {

constexpr int MT = 128;   // operator rows per tile (TMEM lanes)
constexpr int NT = 32;    // right-hand-side columns per tile
constexpr int KS = 16;    // K of one MMA instruction (16-bit operands)
constexpr int BITS = 7;   // bits per slice

// bytes of one slice block of one K step: A (MT x KS), B (NT x KS), bf16, in the
// canonical K-major layout without swizzle: core matrices of 8 rows x 16 bytes,
// core (r8, k8) at byte (r8 * 2 + k8) * 128, row r % 8 of a core at 16 * (r % 8)
constexpr int A_BLK = MT * KS * 2;
constexpr int B_BLK = NT * KS * 2;

__host__ __device__ __forceinline__ int core_off(int r, int k) {   // element offset in a block
  return ((r >> 3) * 2 + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

// Exponent e with |v| < 2^(e-1) for the largest magnitude m of a row or column
// (m = 0: 0).  Works on the bit pattern, so no FP64 arithmetic is issued.
__host__ __device__ __forceinline__ int split_exponent(double m) {
  if (!(m > 0)) return 0;
  int ex;
#ifdef __CUDA_ARCH__
  ex = (int)((__double_as_longlong(m) >> 52) & 0x7FF) - 1022;   // m in [2^(ex-1), 2^ex)
#else
  std::frexp(m, &ex);
#endif
  return ex + 1;
}

// The S slices of v relative to 2^e (|v| < 2^(e-1)), as floats t_i 2^(-7 i).
template <int S>
__device__ __forceinline__ void split_value(double v, int e, float* out) {
  const long long bits = __double_as_longlong(v);
  const int E = (int)((bits >> 52) & 0x7FF);
  long long T = 0;
  if (E != 0) {   // subnormals (below 2^-1022) count as zero
    const long long m = (bits & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;   // |v| = m 2^(E - 1075)
    const int sh = E - 1075 - e + BITS * S;                                 // T = floor(|v| 2^(7S - e))
    if (sh >= 0) T = m << sh;                                               // |v| < 2^(e-1): T < 2^(7S-1)
    else if (sh > -64) T = m >> (-sh);
  }
  const float sg = bits < 0 ? -1.0f : 1.0f;
#pragma unroll
  for (int i = 1; i <= S; ++i) {
    const int t = (int)((T >> (BITS * (S - i))) & 127);
    out[i - 1] = sg * __int2float_rn(t) * __int_as_float((127 - BITS * i) << 23);   // t 2^(-7 i)
  }
}

// Exponent e with |x| < 2^(e-1) for a float magnitude x > 0 (0: INT_MIN / 2, below
// every other exponent).
__device__ __forceinline__ int split_exponent_f(float x) {
  const int b = __float_as_int(x) & 0x7FFFFFFF;
  if (b == 0) return -(1 << 30);
  return ((b >> 23) & 0xFF) - 126 + 1;   // x in [2^(E-127), 2^(E-126))
}

// The S slices of the FP32 pair value hi + lo relative to 2^e (|hi + lo| < 2^(e-1),
// up to a relative 2^-20), by rounding to nearest instead of truncation: digit i is
// y rounded to a multiple of 2^(-7 i) by adding and subtracting 1.5 * 2^(23 - 7 i)
// (exact in FP32 for |y| below 2^(22 - 7 i)), and the remainder y - digit is exact.
// The low part joins the remainder after the third digit (rounding there is below
// 2^-46 of 2^e).  |t_i| <= 64 for every digit.  FP32 additions only.
template <int S>
__device__ __forceinline__ void split_pair_rn(float hi, float lo, int e, float* out) {
  float y = ldexpf(hi, -e);
  const float yl = ldexpf(lo, -e);
#pragma unroll
  for (int i = 1; i <= S; ++i) {
    if (i == 4) y = __fadd_rn(y, yl);
    const float c = __int_as_float((127 + 23 - BITS * i) << 23) * 1.5f;   // 1.5 * 2^(23 - 7 i)
    const float t = __fsub_rn(__fadd_rn(y, c), c);
    y = __fsub_rn(y, t);
    out[i - 1] = t;
  }
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, K-major, leading (K) core stride
// lbo, strided (M/N) 8-row stride sbo, descriptor version 1 (bits 46-47)
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: FP32 D, bf16 A and B, both K-major, N, M, negate A
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int negA) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)negA << 13) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar)));
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes));
}

// bounded wait for the phase with parity `phase`; false when it gave up
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t phase, long long limit) {
  uint32_t done = 0;
  for (long long it = 0; it < limit; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(phase));
    if (done) return true;
  }
  return false;
}

// bulk copy (TMA engine, no tensor map) of `bytes` (multiple of 16, both addresses
// 16-byte aligned) from global to shared memory, completing on mbar
__device__ __forceinline__ void bulk_g2s(void* smem_dst, const void* gsrc, uint32_t bytes, uint64_t* mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(smem_dst)),
               "l"(gsrc), "r"(bytes), "r"(smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane (warp w reads lanes 32 (w % 4) ..)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace tc
}  // namespace eo
