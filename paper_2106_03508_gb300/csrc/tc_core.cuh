// tcgen05 / TMA / mbarrier building blocks for sm_103a (inline PTX).
//
// Conventions of the split-BF16 GEMM mainloop used by the moment build:
//  - operands are K-major BF16 tiles loaded by TMA with 64-byte swizzling
//    (32 K elements per row, 8-row atoms of 512 B);
//  - one elected thread issues tcgen05.mma (kind::f16, BF16 inputs, FP32
//    accumulator in tensor memory), M = 128 rows, N = BN columns, K = 16 per
//    instruction;
//  - every wait on an mbarrier is bounded: on timeout the CTA raises an abort
//    flag, records an error code in global memory and leaves its loops.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cstdint>

namespace agf2 {
namespace tc {

// Wait limit, in ns of the global timer (2 s).  The global timer is the time
// base of every bounded wait: a thread suspended in mbarrier.try_wait or in
// a sleep does not keep an SM-clock counter advancing at its nominal rate.
constexpr unsigned long long kWaitNs = 2000000000ULL;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
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
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity.  Returns false (and sets
// *abort) if the CTA is aborting or the limit is reached.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort) return false;
    if (global_ns() - t0 > kWaitNs) {
      *abort = 1;
      return false;
    }
  }
  return true;
}

// ---- TMA (tensor maps are __grid_constant__ kernel parameters) ----
__device__ __forceinline__ void tma_prefetch(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2),
      "r"(c3)
      : "memory");
}

// ---- tensor memory ----
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ---- MMA ----
// Instruction descriptor, kind::f16 with BF16 A/B, FP32 D, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4)                              // D format: F32
         | (1u << 7)                            // A format: BF16
         | (1u << 10)                           // B format: BF16
         | ((uint32_t)(N >> 3) << 17)           // N / 8
         | ((uint32_t)(M >> 4) << 24);          // M / 16
}

// Shared-memory matrix descriptor: K-major tile, 64-byte swizzle, rows of 64 B
// (32 BF16), 8-row atoms 512 B apart (stride byte offset), sm_100 version bits.
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for this layout)
  d |= (uint64_t)(512u >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)4 << 61;             // SWIZZLE_64B
  return d;
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// Arrive on `bar` once all previously issued tcgen05.mma of this thread are done.
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 8 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive FP32 columns of this thread's TMEM lane (32x32b shape: warp
// w of a warpgroup reads lanes 32 (w % 4) .. 32 (w % 4) + 31).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- fixed-point three-limb BF16 slicing ----
// With a per-row power-of-two unit s (|x| < R s on that row, R = 2^rbits,
// rbits <= 8),
//   x / s ~ h0 + h1 + h2,  h0 an integer in [-R, R], h1 in 2^-8 Z,
//   h2 in 2^-16 Z (|h1|, |h2| <= 128 units of their grid),
// all exactly representable in BF16.  Products h0*h0' are integers of
// magnitude <= R^2, so a sum of K of them is exact in the FP32 tensor-core
// accumulator whenever R^2 K <= 2^24 (or, for any K, under a row
// certificate: certified_unit).  The remaining limb products are kept in a
// separate accumulator.  slice3f cuts FP32 values; slice3_int cuts FP64
// values on the integer pipe (fixed_digits).

// |x| as its IEEE bit pattern: non-negative doubles order like their bits as
// unsigned integers, so a running max |x| runs on the integer pipe.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
}

// ---- integer-pipe helpers (the FP64 pipe of this part issues about two
// operations per clock per SM, so per-element FP64 work in a memory-bound
// kernel or an epilogue costs more than the memory traffic itself) ----

// Exponent returned for a unit that underflowed to zero in FP32 (rows whose
// values lie below 2^-149 times their digits, e.g. far tails of decaying DF
// factors): far below the double range, and small enough that a sum of two
// such exponents cannot overflow an int.
constexpr int kZeroUnitExp = -100000;

// Exponent k of a power-of-two float u = 2^k (kZeroUnitExp for u = 0).
__device__ __forceinline__ int pow2_exp(float u) {
  const unsigned b = __float_as_uint(u);
  const unsigned e = (b >> 23) & 0xffu;
  if (e) return (int)e - 127;
  return (b & 0x7fffffu) ? ilogbf(u) : kZeroUnitExp;
}

// Exponent k of a power-of-two double u = 2^k (u normal).
__device__ __forceinline__ int pow2_exp(double u) {
  return (int)(((unsigned long long)__double_as_longlong(u) >> 52) & 0x7ffULL) - 1023;
}

// f 2^k as a double, exactly: a float converts to a double by re-biasing the
// exponent and widening the significand, done here on the integer pipe.
// Zero (or k below the double range) gives 0; subnormal, non-finite or
// out-of-range results take FP64 ldexp.
__device__ __forceinline__ double scale_to_double(float f, int k) {
  const unsigned b = __float_as_uint(f);
  if ((b & 0x7fffffffu) == 0u || k < -1400) return 0.0;  // |f 2^k| < 2^-1270: zero
  const int e = (int)((b >> 23) & 0xffu);
  const int ed = e + 896 + k;  // 1023 - 127 = 896
  if (e == 0 || e == 0xff || ed <= 0 || ed >= 0x7ff) return ldexp((double)f, k);
  const unsigned hi = (b & 0x80000000u) | ((unsigned)ed << 20) | ((b & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)(b << 29));
}

// An FP32 upper bound of |x| (round toward +infinity of the significand, on the
// integer pipe); |x| below the smallest normal float gives 2^-126, above the
// float range +infinity.
__device__ __forceinline__ float abs_up_float(double x) {
  const unsigned long long b = abs_bits(x);
  if (b == 0) return 0.0f;
  const int ef = (int)(b >> 52) - 896;
  if (ef >= 255) return __int_as_float(0x7f800000);
  if (ef <= 0) return 1.17549435e-38f;  // 2^-126
  unsigned fb = ((unsigned)ef << 23) | (unsigned)((b >> 29) & 0x7fffffULL);
  if (b & 0x1fffffffULL) fb += 1u;  // a carry into the exponent is the right bound
  return __uint_as_float(fb);
}

// Balanced base-256 fixed-point digits of v = x / 2^ku (the caller's unit
// keeps |v| < 2^9): d0 the nearest integer to v, then each d_i the nearest
// integer to 256 x the exact remainder, so v = d0 + d1/256 + ... + d_{ND-1}
// 256^(1-ND) up to the last digit's rounding (<= 2^-(8 ND - 7)); ties round
// away from zero.  Exact 64-bit integer arithmetic on the significand
// (x = +-m 2^(e-1075)), no FP64 instruction; |d0| <= |v| + 1/2 as with rint,
// and |d_i| <= 128 for i >= 1.
template <int ND>
__device__ __forceinline__ void fixed_digits(double x, int ku, int (&d)[ND]) {
#pragma unroll
  for (int i = 0; i < ND; ++i) d[i] = 0;
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ffULL);
  if (e == 0 || e == 0x7ff) return;  // zero, subnormal (< 2^-1022) or non-finite
  long long m = (long long)((b & 0xfffffffffffffULL) | (1ULL << 52));
  int t = 1075 + ku - e;  // v = m 2^-t, t >= 45 when |v| < 2^9
  if (t > 62) {
    if (t - 62 > 53) return;  // |v| < 2^-62: every digit rounds to zero
    m >>= (t - 62);           // dropped bits could only decide exact ties
    t = 62;
  }
  if (t < 8 * ND) t = 8 * ND;  // outside the caller's contract; keeps the shifts defined
  long long q = (m + (1LL << (t - 1))) >> t;
  long long r = m - q * (1LL << t);
  d[0] = (int)q;
#pragma unroll
  for (int i = 1; i < ND; ++i) {
    t -= 8;
    q = (r + (1LL << (t - 1))) >> t;  // arithmetic shift: floor(r / 2^t + 1/2)
    r -= q * (1LL << t);
    d[i] = (int)q;
  }
  if (b >> 63) {
#pragma unroll
    for (int i = 0; i < ND; ++i) d[i] = -d[i];
  }
}

__device__ __forceinline__ void slice3f(float u, __nv_bfloat16& h0, __nv_bfloat16& h1,
                                        __nv_bfloat16& h2) {
  const float a0 = rintf(u);
  const float r1 = (u - a0) * 256.0f;
  const float a1 = rintf(r1);
  const float a2 = rintf((r1 - a1) * 256.0f);
  h0 = __float2bfloat16_rn(a0);
  h1 = __float2bfloat16_rn(a1 * (1.0f / 256.0f));
  h2 = __float2bfloat16_rn(a2 * (1.0f / 65536.0f));
}

// Slicing unit of a row with max |x| = m: the power of two 2^(E - rbits)
// with m < 2^E, so that |x| / unit < 2^rbits.
__host__ __device__ __forceinline__ double slice_unit(double m, int rbits) {
  if (!(m > 0.0)) return 1.0;
  int E;
  frexp(m, &E);  // m = f 2^E, f in [0.5, 1)
  return ldexp(1.0, E - rbits);
}

__device__ __forceinline__ float slice_unitf(float m, int rbits) {
  if (!(m > 0.0f)) return 1.0f;
  int E;
  frexpf(m, &E);
  return ldexpf(1.0f, E - rbits);
}

// Row unit with an exactness certificate: start from slice_unit(m, 8) and
// double it until sum_k (|x_k|/u + 1/2)^2 <= 2^24, bounded above by
// s2/u^2 + s1/u + n/4 (s2 = sum x^2, s1 = sum |x|, n entries).  Then the
// row's integer limbs satisfy sum_k h0_k^2 <= 2^24, so by Cauchy-Schwarz
// every partial sum of h0 h0' products between two such rows -- over any
// K range -- is an integer of magnitude <= 2^24, exact in FP32.  Doubling
// the unit is needed only for rows whose entries are nearly all of the
// row's maximum size, where a coarser grid costs little.
__host__ __device__ __forceinline__ double certified_unit(double m, double s2, double s1,
                                                          double n) {
  double u = slice_unit(m, 8);
  while (s2 / (u * u) + s1 / u + 0.25 * n > 16777216.0) u *= 2.0;
  return u;
}

// Row statistics for certified_unit on the integer and FP32 pipes: max |x|
// (bits), and upper bounds of sum x^2 and sum |x| (FP32, every operation
// rounded toward +infinity, so the bounds hold however the sums are split).
struct RowStats {
  unsigned long long mb = 0;
  float s2 = 0.0f, s1 = 0.0f;
  __device__ __forceinline__ void add(double x) {
    mb = max(mb, abs_bits(x));
    const float a = abs_up_float(x);
    s2 = __fadd_ru(s2, __fmul_ru(a, a));
    s1 = __fadd_ru(s1, a);
  }
  __device__ __forceinline__ void merge(unsigned long long mb2, float s22, float s12) {
    mb = max(mb, mb2);
    s2 = __fadd_ru(s2, s22);
    s1 = __fadd_ru(s1, s12);
  }
  __device__ __forceinline__ void warp_reduce() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      merge((unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)mb, o),
            __shfl_xor_sync(0xffffffffu, s2, o), __shfl_xor_sync(0xffffffffu, s1, o));
  }
  // certified_unit from the bounds; false if a bound overflowed the float
  // range (|x| >= 2^64 somewhere), where the caller recomputes in FP64
  __device__ __forceinline__ bool unit(double n, double& u) const {
    if (!(s2 <= 3.4e38f) || !(s1 <= 3.4e38f)) return false;
    u = certified_unit(__longlong_as_double((long long)mb), (double)s2, (double)s1, n);
    return true;
  }
};

// Three limbs of x / 2^ku (slice3's layout: h0 integer, h1 in 2^-8 Z, h2 in
// 2^-16 Z) from fixed_digits<3>.
__device__ __forceinline__ void slice3_int(double x, int ku, __nv_bfloat16& h0,
                                           __nv_bfloat16& h1, __nv_bfloat16& h2) {
  int d[3];
  fixed_digits<3>(x, ku, d);
  h0 = __float2bfloat16_rn((float)d[0]);
  h1 = __float2bfloat16_rn((float)d[1] * (1.0f / 256.0f));
  h2 = __float2bfloat16_rn((float)d[2] * (1.0f / 65536.0f));
}

}  // namespace tc
}  // namespace agf2
