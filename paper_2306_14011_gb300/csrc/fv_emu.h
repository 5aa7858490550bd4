// IEEE-754 binary64 arithmetic on the integer pipe.
//
// On GB300 the FP64 pipe retires about two lane-operations per clock per SM,
// so a warp-wide FP64 instruction holds a sub-partition's FP64 unit for ~64
// cycles, while the same sub-partition can issue one integer instruction per
// cycle.  A double-precision product written out in 32-bit integer operations
// (~30 instructions) therefore costs fewer issue cycles than the FP64 pipe
// spends on it, and runs beside the FP64 pipe's own work.
//
// emu_dmul_bits computes the correctly rounded (round to nearest, ties to
// even) product of two doubles, bit for bit what the FP64 multiplier
// returns, on the common path: both operands normal and a normal result.
// Everything else (zero, subnormal, infinite or NaN operands, subnormal
// results) is flagged for the caller to evaluate in FP64.
//
// The construction is the schoolbook one.  With the implicit leading one, a
// normal double is m * 2^(e - 1075) with a 53-bit integer significand m and
// biased exponent e.  The exact product of the significands,
// P = ma * mb, lies in [2^104, 2^106) and is formed from 32-bit halves with
// four 32x32 -> 64-bit multiply-adds.  With s = 1 when P >= 2^105, the
// result's significand is P >> (52 + s) rounded to nearest-even on the bits
// shifted out, and its biased exponent is ea + eb - 1023 + s; a rounding
// carry out of the significand moves into the exponent field by itself when
// the two are packed by addition.
//
// Host and device: the same source is checked against the host's IEEE
// multiplication on the CPU and against the GPU's FP64 multiplier.
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define FV_EMU_HD __host__ __device__ __forceinline__
#else
#define FV_EMU_HD inline
#endif

namespace fvk {

// 32 x 32 -> 64-bit unsigned product.
FV_EMU_HD uint64_t emu_mul_wide(uint32_t a, uint32_t b) { return (uint64_t)a * (uint64_t)b; }

// The low word of (hi:lo) >> n for 0 < n < 32 (a funnel shift on the GPU).
FV_EMU_HD uint32_t emu_shr_pair(uint32_t lo, uint32_t hi, uint32_t n) {
#ifdef __CUDA_ARCH__
  return __funnelshift_r(lo, hi, n);
#else
  return (uint32_t)((((uint64_t)hi << 32) | lo) >> n);
#endif
}

// Product of the doubles with bit patterns (ha:la) and (hb:lb) into (hr:lr).
// Returns false when the operands or the result leave the fast path -- a
// zero, subnormal, infinite or NaN operand, or a result below the normal
// range -- and the returned bits are then meaningless.  A result that rounds
// past the largest double comes out as the correctly signed infinity.
FV_EMU_HD bool emu_dmul_bits(uint32_t ha, uint32_t la, uint32_t hb, uint32_t lb, uint32_t &hr, uint32_t &lr) {
  const uint32_t ea = (ha >> 20) & 0x7ffu, eb = (hb >> 20) & 0x7ffu;
  // significand halves: a = a1 2^32 + la with a1 = 2^20 + the top 20 stored bits
  const uint32_t a1 = (ha & 0xfffffu) | 0x100000u, b1 = (hb & 0xfffffu) | 0x100000u;
  // P = w 2^64 + zl 2^32 + xl, exactly
  const uint64_t x = emu_mul_wide(la, lb);
  const uint64_t y = emu_mul_wide(a1, lb) + (x >> 32);  // < 2^54
  const uint64_t z = emu_mul_wide(la, b1) + y;          // < 2^55
  const uint64_t w = emu_mul_wide(a1, b1) + (z >> 32);  // < 2^42
  const uint32_t xl = (uint32_t)x, zl = (uint32_t)z, wh = (uint32_t)(w >> 32);
  const uint32_t s = wh >> 9;                           // bit 105 of P: 1 when P >= 2^105
  const uint32_t k = 20u + s;                           // the significand is P >> (32 + k)
  // Round to nearest, ties to even, by adding 2^(31+k) - 1 + lsb to P and
  // truncating: the carry into bit 32 + k happens exactly when the bits
  // below it exceed one half, or equal one half with an odd lsb.  The
  // addend's words: low lsb - 1 (all ones, or 0 when lsb = 1), high
  // 2^(k-1) - 1 + lsb.
  const uint32_t lsb = (zl >> k) & 1u;
  const uint32_t c0 = (xl + (lsb - 1u)) < xl ? 1u : 0u;  // carry out of the low word (lsb - 1 = 0 adds none)
  const uint64_t mid = (uint64_t)zl + ((0x80000u << s) - 1u + lsb) + c0;
  const uint32_t zr = (uint32_t)mid;
  const uint64_t wr = w + (mid >> 32);
  // the rounded significand (P + addend) >> (32 + k), leading one at bit 52
  const uint32_t ml = emu_shr_pair(zr, (uint32_t)wr, k);
  const uint32_t mh = emu_shr_pair((uint32_t)wr, (uint32_t)(wr >> 32), k);
  const uint32_t e1 = ea + eb + s - 1024u;              // biased exponent - 1 (wraps below the range)
  hr = (mh + (e1 << 20)) | ((ha ^ hb) & 0x80000000u);   // the leading one lands in the exponent
  lr = ml;
  // normal operands (exponent fields 1..2046) and e1 <= 2045; a rounding
  // carry from e1 = 2045 gives exponent field 2047 and a zero significand:
  // the infinity IEEE rounding returns
  const uint32_t big = (ea - 1u) > (eb - 1u) ? (ea - 1u) : (eb - 1u);
  return (big > e1 ? big : e1) < 2046u;
}

// The same product with signed zeros on the fast path as well: a zero
// operand times a finite double gives the zero of the product's sign.
FV_EMU_HD bool emu_dmul_bits_z(uint32_t ha, uint32_t la, uint32_t hb, uint32_t lb, uint32_t &hr, uint32_t &lr) {
  const bool ok = emu_dmul_bits(ha, la, hb, lb, hr, lr);
  const bool za = ((ha << 1) | la) == 0u, zb = ((hb << 1) | lb) == 0u;
  const bool zero = za || zb;
  hr = zero ? ((ha ^ hb) & 0x80000000u) : hr;
  lr = zero ? 0u : lr;
  // a zero times a zero, or times a normal or subnormal number (exponent
  // field below 2047): no infinity or NaN operand
  const bool finite = ((ha >> 20) & 0x7ffu) != 0x7ffu && ((hb >> 20) & 0x7ffu) != 0x7ffu;
  return zero ? finite : ok;
}

// The second-order series term of the reciprocal and reciprocal square-root
// refinements: w = 2^-k e + c e^2 (k = 0 or 1, c > 0 an FP32 constant), as
// the bits of a double, for the small residual e = 1 - x y^n of a seed y
// (1/x = y (1 + e + e^2 + ...), 1/sqrt(x) = y (1 + e/2 + 3 e^2/8 + ...)).
// 2^-k e is exact (an exponent decrement); c e^2 is formed in FP32 (e
// truncated to FP32: relative error below 2^-21) and added to it as an
// integer number of its units in the last place, so w carries an absolute
// error below 2^-21 c e^2 + one unit in the last place of w -- below 2^-60
// for |e| < 2^-19, far below the rounding of the refined result y (1 + w).
// Binade crossings of the addition are handled exactly; |e| below 2^-959
// gives w = 0.  The same integer steps on the host and the GPU, so the FP64
// and integer-pipe evaluations of the flux that use it agree bit for bit.
FV_EMU_HD float emu_f32_from_bits(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  __builtin_memcpy(&f, &b, 4);
  return f;
#endif
}
FV_EMU_HD uint32_t emu_bits_from_f32(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t b;
  __builtin_memcpy(&b, &f, 4);
  return b;
#endif
}
FV_EMU_HD float emu_fmul_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}

FV_EMU_HD void emu_series2_bits(uint32_t he, uint32_t le, uint32_t k, float c, uint32_t &hw, uint32_t &lw) {
  const uint32_t Ee = (he >> 20) & 0x7ffu;
  const uint32_t neg = he & 0x80000000u;
  const uint32_t Eb = Ee - k;                                  // exponent field of 2^-k e
  const uint64_t f = ((uint64_t)(he & 0xfffffu) << 32) | le;  // its 52-bit fraction
  // e^2 c in FP32 from e truncated to FP32 (|e| < 2^-126 makes it 0)
  const uint32_t e32b = Ee > 896u ? (((Ee - 896u) << 23) | ((he & 0xfffffu) << 3) | (le >> 29)) : 0u;
  const float e32 = emu_f32_from_bits(e32b);
  const uint32_t qb = emu_bits_from_f32(emu_fmul_rn(emu_fmul_rn(c, e32), e32));
  const uint32_t Eq = qb >> 23;                                // q >= 0
  const uint64_t mq = Eq != 0u ? (uint64_t)((qb & 0x7fffffu) | 0x800000u) : 0u;
  // K = q / ulp(2^-k e) = mq 2^(Eq - 150 - (Eb - 1075))
  const int sh = (int)Eq + 925 - (int)Eb;
  const uint64_t K = sh >= 0 ? (sh < 40 ? mq << sh : 0xffffffffffull) : (-sh < 32 ? mq >> (-sh) : 0ull);
  const uint64_t one = 1ull << 52;
  uint64_t bits;
  if (!neg) {  // |w| = |2^-k e| + K
    const uint64_t S = f + K;
    bits = S < one ? (((uint64_t)Eb << 52) | S) : (((uint64_t)(Eb + 1u) << 52) | ((S - one) >> 1));
  } else {     // |w| = |2^-k e| - K, into the binade below when K > f
    bits = f >= K ? (((uint64_t)Eb << 52) | (f - K)) : (((uint64_t)(Eb - 1u) << 52) | (one - 2u * (K - f)));
  }
  const bool tiny = Ee < 64u;
  hw = tiny ? 0u : ((uint32_t)(bits >> 32) | neg);
  lw = tiny ? 0u : (uint32_t)bits;
}

}  // namespace fvk
