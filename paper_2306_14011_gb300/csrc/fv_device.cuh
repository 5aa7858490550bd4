// Device-side building blocks of the FP64 Euler kernels (sm_103a).
//
// Design note.  On GB300 the FP64 pipe retires about two lane-operations per
// clock per SM (~0.6 T FP64 instructions/s per GPU), roughly sixty times less
// than what HBM can feed to this stencil; the FP64 pipe, not memory, bounds
// every kernel here.  So:
//   * comparisons, absolute values, min/max and the minmod limiter run on the
//     integer pipe, on IEEE-754 bit patterns (exact for finite doubles);
//   * reciprocals and reciprocal square roots start from the PTX
//     rcp.approx.ftz.f64 / rsqrt.approx.ftz.f64 seeds (issued on the
//     special-function unit, relative error below 2^-20) and are refined to
//     full double precision by one third-order Householder step in FMA;
//   * the Roe flux is arranged so each quantity is formed once, and evaluated
//     one-sided (roe_F), without the flux of the right state;
//   * its products run on the integer pipe (pmul, fv_emu.h: the correctly
//     rounded product in 32-bit integer operations), which the FP64 pipe's
//     own work leaves idle; a warp whose operands leave that path evaluates
//     the flux again in FP64.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "fv_emu.h"

namespace fvk {

// ------------------------------------------------------------ device flags
enum : unsigned { FLAG_NONPHYSICAL = 1u, FLAG_TIMEOUT = 2u };

// ------------------------------------------------------------ integer-pipe helpers
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }

// The FP64 product for the rare inputs the integer-pipe replacements below
// leave to the FP64 multiplier.  Kept out of line: a multiply written inside
// their warp-uniform branches was speculated above the branch by the compiler
// and then occupied the FP64 pipe on every call.
static __device__ __noinline__ double dmul_fp64_slow(double a, double b) { return __dmul_rn(a, b); }

// |x| by clearing the sign bit.
__device__ __forceinline__ double iabs(double x) {
  return __hiloint2double(__double2hiint(x) & 0x7fffffff, __double2loint(x));
}

// a < b for non-negative finite doubles (bit patterns are ordered like the values).
__device__ __forceinline__ bool ilt_nonneg(double a, double b) { return dbits(a) < dbits(b); }

// Select between two doubles on the integer pipe (a double-typed ?: can be
// emitted as FP64 moves, which occupy the FP64 pipe).
__device__ __forceinline__ double isel(bool p, double a, double b) {
  return __longlong_as_double(p ? dbits(a) : dbits(b));
}

// minmod(a, b): 0 when the signs differ (or either is zero), else the argument
// of smaller magnitude (b on ties).  Bitwise equal to the branchy definition
// for finite inputs (a zero argument yields a signed zero, which adds as
// zero).  Integer compares and selects on the 32-bit halves only: written
// with 64-bit sign masks, the compiler forms |a| and |b| as FP64 absolute
// values, two FP64-pipe instructions per call.
__device__ __forceinline__ double minmod(double a, double b) {
  const int ha = __double2hiint(a), hb = __double2hiint(b);
  const unsigned la = (unsigned)__double2loint(a), lb = (unsigned)__double2loint(b);
  const unsigned ma = (unsigned)ha & 0x7fffffffu, mb = (unsigned)hb & 0x7fffffffu;
  const bool a_smaller = ma < mb || (ma == mb && la < lb);
  const bool opposite = (ha ^ hb) < 0;
  const int h = opposite ? 0 : (a_smaller ? ha : hb);
  const int l = opposite ? 0 : (int)(a_smaller ? la : lb);
  return __hiloint2double(h, l);
}

// true when x is +0 or -0 (32-bit halves, integer pipe).
__device__ __forceinline__ bool izero(double x) {
  return (((unsigned)__double2hiint(x) & 0x7fffffffu) | (unsigned)__double2loint(x)) == 0u;
}

// x / 2 for x >= 0 on the integer pipe: decrement the biased exponent.  Exact
// (bitwise equal to 0.5 * x) for x = 0, inf, NaN and every normal x of
// exponent field >= 2; the rest (0 < x < 2^-1021, never reached by the squared
// speeds and inverse squared sound speeds it is used on) take the FP64
// multiply in a warp-uniform branch.
__device__ __forceinline__ double half_nonneg(double x) {
  const long long b = dbits(x);
  const bool normal = b >= (2ll << 52) && b < 0x7ff0000000000000ll;
  const bool tiny = b > 0 && b < (2ll << 52);
  double h = __longlong_as_double(normal ? b - (1ll << 52) : (b <= 0 ? 0ll : b));
  if (__any_sync(__activemask(), tiny)) {
    if (tiny) h = dmul_fp64_slow(0.5, x);
  }
  return h;
}

// x * 2^K (K = -2, -1 or 1) on the integer pipe: add K to the biased
// exponent.  Exact (bitwise equal to the FP64 product) for x = +-0 and every
// x whose exponent field stays within 1..2046; the rest (results near the
// subnormal range or overflowing, inf, NaN) take the FP64 multiply in a
// warp-uniform branch.
template <int K>
__device__ __forceinline__ double scale_pow2(double x) {
  const int hi = __double2hiint(x);
  const int e = (int)(((unsigned)hi >> 20) & 0x7ffu);
  const bool fast = e >= 1 && e <= 2046 && e + K >= 1 && e + K <= 2046;
  const bool zero = izero(x);
  double q = __hiloint2double(fast ? hi + K * (1 << 20) : hi, __double2loint(x));
  if (__any_sync(__activemask(), !fast && !zero)) {
    if (!fast && !zero) q = dmul_fp64_slow(K == -2 ? 0.25 : (K == -1 ? 0.5 : 2.0), x);
  }
  return q;
}
__device__ __forceinline__ double quarter(double x) { return scale_pow2<-2>(x); }

// true when x is not a finite positive double (x <= 0, -0, inf or NaN).
__device__ __forceinline__ bool not_positive_finite(double x) {
  const long long ix = dbits(x);
  return ix <= 0 || ix >= 0x7ff0000000000000ll;
}

// ------------------------------------------------------------ products on the integer pipe
// a * b in the flux routines.  EMU: on the integer pipe without a branch --
// ok is cleared when the operands or the product leave the integer path
// (the value is then meaningless and the caller recomputes in FP64); ZERO
// also takes signed zeros on the integer path.  Otherwise the FP64 product,
// rounded on its own (__dmul_rn: never contracted into a neighbouring
// addition), so that both evaluations give the same bits.
template <bool EMU, bool ZERO = false>
__device__ __forceinline__ double pmul(double a, double b, bool &ok) {
  if (!EMU) return __dmul_rn(a, b);
  uint32_t hr, lr;
  const uint32_t ha = (uint32_t)__double2hiint(a), la = (uint32_t)__double2loint(a);
  const uint32_t hb = (uint32_t)__double2hiint(b), lb = (uint32_t)__double2loint(b);
  ok &= ZERO ? emu_dmul_bits_z(ha, la, hb, lb, hr, lr) : emu_dmul_bits(ha, la, hb, lb, hr, lr);
  return __hiloint2double((int)hr, (int)lr);
}

// ------------------------------------------------------------ reciprocal and rsqrt
__device__ __forceinline__ double rsqrt_seed(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  return y;
}
__device__ __forceinline__ double rcp_seed(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  return y;
}
// The same seeds as volatile asm, for the FP64 re-evaluation of the flux in
// a rarely taken branch: the compiler can then neither share them with the
// integer-path evaluation nor hoist the products that depend on them above
// the branch (where they would run on every call).
__device__ __forceinline__ double rsqrt_seed_v(double x) {
  double y;
  asm volatile("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  return y;
}
__device__ __forceinline__ double rcp_seed_v(double x) {
  double y;
  asm volatile("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  return y;
}

// The second-order series term w = 2^-k e + c e^2 of a refinement
// (emu_series2_bits: integer and FP32 operations, no FP64 instruction).
template <int K>
__device__ __forceinline__ double series2(double e, float c) {
  uint32_t hw, lw;
  emu_series2_bits((uint32_t)__double2hiint(e), (uint32_t)__double2loint(e), (uint32_t)K, c, hw, lw);
  return __hiloint2double((int)hw, (int)lw);
}

// 1/sqrt(x) for positive normal x.  With y0 the seed and e = 1 - x*y0^2,
// 1/sqrt(x) = y0 (1 - e)^(-1/2) = y0 (1 + e/2 + 3e^2/8 + O(e^3)); truncating
// the binomial series after e^2 is the third-order Householder step, so
// |e| < 2^-20 leaves a truncation error below 2^-59.  x*y0 is a product
// (integer pipe with EMU), e an FMA, the series term w = e/2 + 3e^2/8 is
// formed on the integer pipe (series2), and y0 (1 + w) one more FMA: two
// FP64 instructions.
template <bool EMU = false, bool VOLATILE_SEED = false>
__device__ __forceinline__ double rsqrt_fp64(double x, bool &ok) {
  const double y = VOLATILE_SEED ? rsqrt_seed_v(x) : rsqrt_seed(x);
  const double t = pmul<EMU>(x, y, ok);
  const double e = fma(-t, y, 1.0);
  return fma(y, series2<1>(e, 0.375f), y);
}
__device__ __forceinline__ double rsqrt_fp64(double x) {
  bool ok = true;
  return rsqrt_fp64<false>(x, ok);
}

// 1/x for normal x: 1/x = y0 / (1 - e) with e = 1 - x*y0, so
// 1/x = y0 (1 + e + e^2 + O(e^3)): e an FMA, w = e + e^2 on the integer
// pipe, y0 (1 + w) an FMA (same truncation order).
template <bool VOLATILE_SEED = false>
__device__ __forceinline__ double rcp_fp64(double x) {
  const double y = VOLATILE_SEED ? rcp_seed_v(x) : rcp_seed(x);
  const double e = fma(-x, y, 1.0);
  return fma(y, series2<0>(e, 1.0f), y);
}

// van Leer's limited slope, 2ab / (a + b) when a and b share one strict sign,
// else 0 (sign tests and the select on the integer pipe; 7 FP64 operations).
__device__ __forceinline__ double vanleer(double a, double b) {
  const bool ok = ((__double2hiint(a) ^ __double2hiint(b)) >= 0) && !izero(a) && !izero(b);
  const double r = (2.0 * a * b) * rcp_fp64(a + b);
  return isel(ok, r, 0.0);
}

// ---- FP32 pre-selection for the time-step reduction.
//
// FP64 -> FP32 on the integer pipe by truncating the mantissa: relative error
// below 2^-23 for |x| in the FP32 normal range; smaller values flush to
// (signed) zero, larger ones and NaN become infinite.
__device__ __forceinline__ float f32_trunc(double x) {
  const unsigned long long b = (unsigned long long)dbits(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  const unsigned sign = hi & 0x80000000u;
  unsigned f = sign | ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  f = e <= 0 ? sign : f;
  f = e >= 255 ? (sign | 0x7f800000u) : f;
  return __uint_as_float(f);
}

// The wave-speed sum s = sum_d (|u_d| + c) / dx_d of cell c (of N cells, SoA
// state U) evaluated in FP32 (round-to-nearest operations
// that are never contracted), and a certified relative error bound rel of it.
// Returns false when no bound is certified.  Certification needs rho, E in
// [2^-30, 2^30] and |m_d| <= 2^30 (no FP32 overflow or underflow on the way)
// and a pressure p = (gamma-1)(E - k) free of strong cancellation,
// kappa = (E + k)/(E - k) <= 1024.  A first-order bound of the FP32 error is
// then (6 kappa + 11) 2^-24 (conversions 2^-23 each, every operation 2^-24,
// the relative error of E - k amplified by kappa); rel = (16 kappa32 + 32)
// 2^-24 exceeds twice that, kappa32 being kappa evaluated in FP32 (within
// 0.1% of it when kappa <= 1024).
template <int DIM>
__device__ __forceinline__ bool wave_sum32(const double *U, long long N, long long c, float g1f, float gammaf,
                                           const float *inv_hf, float &s32, float &rel) {
  constexpr int NV = DIM + 2;
  const float rho = f32_trunc(U[c]);
  const float E = f32_trunc(U[(NV - 1) * N + c]);
  bool ok = rho >= 0x1p-30f && rho <= 0x1p30f && E >= 0x1p-30f && E <= 0x1p30f;
  const float r = __frcp_rn(rho);
  float u[DIM];
  float k = 0.0f;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const float m = f32_trunc(U[(1 + d) * N + c]);
    ok = ok && fabsf(m) <= 0x1p30f;
    u[d] = __fmul_rn(m, r);
    k = __fadd_rn(k, __fmul_rn(m, u[d]));
  }
  k = 0.5f * k;
  const float em = __fsub_rn(E, k), ep = __fadd_rn(E, k);
  ok = ok && em > 0.0f && ep <= __fmul_rn(1024.0f, em);
  const float c2 = __fmul_rn(__fmul_rn(gammaf, __fmul_rn(g1f, em)), r);
  const float cs = __fsqrt_rn(c2);
  float s = 0.0f;
#pragma unroll
  for (int d = 0; d < DIM; ++d) s = __fadd_rn(s, __fmul_rn(__fadd_rn(fabsf(u[d]), cs), inv_hf[d]));
  s32 = s;
  rel = __fmaf_ru(__fmul_ru(16.0f, __fmul_ru(ep, __frcp_ru(em))), 0x1p-24f, 32.0f * 0x1p-24f);
  return ok;
}

// ------------------------------------------------------------ Roe flux
// min(x, 0) on the integer pipe: x for x < 0, +0 for x >= 0 and for -0.
__device__ __forceinline__ double min0(double x) {
  const bool neg = __double2hiint(x) < 0 && !izero(x);
  return isel(neg, x, 0.0);
}

// -x by flipping the sign bit (integer pipe).
__device__ __forceinline__ double ineg(double x) {
  return __hiloint2double(__double2hiint(x) ^ (int)0x80000000u, __double2loint(x));
}

// The Roe flux across a face with unit normal along one axis.  States are
// ordered normal-first: q = (rho, m_n, m_t[0..NT-1], rho*e_t), where m_n is
// the momentum along the face normal and m_t the tangential momenta.
// The flux is  F = (F(QL) + F(QR))/2 - sum_w |lambda_w| alpha_w r_w / 2
// with acoustic waves alpha_{1,3} = (dp -+ rho~ c~ du_n) / (2 c~^2), entropy
// wave alpha_2 = drho - dp / c~^2, shear waves rho~ du_t, eigenvalues
// u~_n -+ c~ and u~_n; Harten's fix replaces |lambda| by (lambda^2 +
// delta^2)/(2 delta) for the acoustic waves when |lambda| < delta = efix c~.
// Roe's averages make F(QR) - F(QL) = sum_w lambda_w alpha_w r_w exactly (in
// exact arithmetic), so
//   F = F(QL) + sum_w (lambda_w - |lambda_w|)/2 alpha_w r_w
//     = F(QR) - sum_w (lambda_w + |lambda_w|)/2 alpha_w r_w.
// Taken from the upwind side of u~_n, every wave but one acoustic wave drops
// out: for u~_n >= 0 the entropy, shear and u~_n + c~ waves have lambda >= 0
// and (efix < 1) |lambda| >= c~ > delta, so only the u~_n - c~ wave is left;
// for u~_n < 0 symmetrically only u~_n + c~.  With x = |u~_n| - c~,
//   F = F(Q_upwind) + k alpha_s r_s,   k = (x - |x|*)/2  (= min(x, 0)),
// alpha_s = dp/(2 c~^2) -+ rho~ du_n/(2 c~), r_s = (1, u~_n -+ c~, u~_t,
// H~ - c~ |u~_n|) (upper signs for u~_n >= 0).  Free streams give F(Q)
// exactly; fully supersonic faces give the upwind physical flux exactly.
// g1 = gamma - 1; inv2efix = 1 / (2 efix) (unused when efix = 0); efix < 1.
// EMU: the products run on the integer pipe (pmul) and ok reports whether
// every one stayed on the integer path; the wrapper roe_F below recomputes
// the flux in FP64 when one did not.
template <int NT, bool EMU>
__device__ __forceinline__ void roe_F_impl(const double (&QL)[NT + 3], const double (&QR)[NT + 3], double g1,
                                           double efix, double inv2efix, double (&G)[NT + 3], bool &ok) {
  constexpr int E = NT + 2;
  // left primitives: 1/sqrt(rho) gives both sqrt(rho) and 1/rho
  const double tL = rsqrt_fp64<EMU, !EMU>(QL[0], ok);
  const double rL = pmul<EMU>(tL, tL, ok);
  const double sL = pmul<EMU>(QL[0], tL, ok);
  const double unL = pmul<EMU, true>(QL[1], rL, ok);
  double utL[NT];
  double kL = pmul<EMU, true>(QL[1], unL, ok);  // rho |u|^2
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    utL[t] = pmul<EMU, true>(QL[2 + t], rL, ok);
    kL = fma(QL[2 + t], utL[t], kL);
  }
  const double pL = pmul<EMU>(g1, fma(-0.5, kL, QL[E]), ok);
  const double eL = QL[E] + pL;  // rho h_t
  // right primitives
  const double tR = rsqrt_fp64<EMU, !EMU>(QR[0], ok);
  const double rR = pmul<EMU>(tR, tR, ok);
  const double sR = pmul<EMU>(QR[0], tR, ok);
  const double unR = pmul<EMU, true>(QR[1], rR, ok);
  double utR[NT];
  double kR = pmul<EMU, true>(QR[1], unR, ok);
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    utR[t] = pmul<EMU, true>(QR[2 + t], rR, ok);
    kR = fma(QR[2 + t], utR[t], kR);
  }
  const double pR = pmul<EMU>(g1, fma(-0.5, kR, QR[E]), ok);
  const double eR = QR[E] + pR;

  // Roe averages with sqrt(rho) weights wL = sL / (sL + sR), wR = 1 - wL:
  // u~ = uR - wL (uR - uL), and H~ = (sL HL + sR HR) / (sL + sR) with
  // sL HL = eL / sL = eL tL
  const double inv = rcp_fp64<!EMU>(sL + sR);
  const double wL = pmul<EMU>(sL, inv, ok);
  const double dun = unR - unL;
  const double un = fma(-wL, dun, unR);
  double ut[NT];
  double q2 = pmul<EMU, true>(un, un, ok);
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    ut[t] = fma(-wL, utR[t] - utL[t], utR[t]);
    q2 = fma(ut[t], ut[t], q2);
  }
  const double H = pmul<EMU>(fma(eL, tL, pmul<EMU>(eR, tR, ok)), inv, ok);
  const double rho = pmul<EMU>(sL, sR, ok);
  const double c2 = pmul<EMU>(g1, H - half_nonneg(q2), ok);
  const double tc = rsqrt_fp64<EMU, !EMU>(c2, ok);  // 1/c~
  const double c = pmul<EMU>(c2, tc, ok);

  // the acoustic wave that crosses from downwind (upper signs: u~_n >= 0)
  const bool up_left = __double2hiint(un) >= 0;
  const double aun = iabs(un);
  const double sc = isel(up_left, c, ineg(c));
  const double dp = pR - pL;
  const double alpha =
      pmul<EMU, true>(pmul<EMU, true>(fma(-pmul<EMU>(rho, sc, ok), dun, dp), tc, ok), half_nonneg(tc), ok);  // (dp -+ rho~ c~ du_n) / (2 c~^2)
  const double x = aun - c;
  // k = (x - |x|*)/2 with the entropy fix.  Whether |x| < delta = efix c~ is
  // decided in FP32 (operands truncated on the integer pipe).  The fixed |x|
  // equals delta at |x| = delta and differs from |x| by (|x| - delta)^2 /
  // (2 delta), and FP32 truncation can only flip the decision where
  // | |x|/delta - 1 | < ~2^-22, so a flipped decision changes k by at most
  // ~delta 2^-46: about a hundred FP64 roundings of k, far below the 1e-12
  // the results are held to.  Near sonic points only: a warp-uniform branch
  // keeps the (rare) fix from being computed unconditionally.
  double k = min0(x);
  const float deltaf = __fmul_rn(f32_trunc(efix), f32_trunc(c));
  const bool fix = f32_trunc(iabs(x)) < deltaf;
  if (__any_sync(__activemask(), fix)) {
    const double delta = efix * c;
    const double d2 = delta * delta, s4 = 0.5 * (tc * inv2efix);  // s4 = 1 / (4 delta)
    k = isel(fix, fma(-fma(x, x, d2), s4, 0.5 * x), k);
  }
  const double g = pmul<EMU, true>(k, alpha, ok);

  // F(Q_upwind) + g r_s (selects on the integer pipe)
  const double m = isel(up_left, QL[1], QR[1]);
  const double u_n = isel(up_left, unL, unR);
  G[0] = m + g;
  G[1] = fma(m, u_n, isel(up_left, pL, pR) + pmul<EMU, true>(g, un - sc, ok));
#pragma unroll
  for (int t = 0; t < NT; ++t) G[2 + t] = fma(m, isel(up_left, utL[t], utR[t]), pmul<EMU, true>(g, ut[t], ok));
  G[E] = fma(u_n, isel(up_left, eL, eR), pmul<EMU, true>(g, fma(-c, aun, H), ok));
}

// The Roe flux above with its products on the integer pipe; a warp in which
// any lane's product left the integer path (a zero, subnormal, infinite or
// NaN operand or result outside the cases pmul takes) evaluates it again in
// FP64.  Both give the same bits wherever the integer path applies.
template <int NT>
__device__ __forceinline__ void roe_F(const double (&QL)[NT + 3], const double (&QR)[NT + 3], double g1,
                                      double efix, double inv2efix, double (&G)[NT + 3]) {
  bool ok = true;
  roe_F_impl<NT, true>(QL, QR, g1, efix, inv2efix, G, ok);
  if (__any_sync(__activemask(), !ok)) roe_F_impl<NT, false>(QL, QR, g1, efix, inv2efix, G, ok);
}

// ------------------------------------------------------------ mbarrier / TMA (inline PTX)
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// One double from global to shared memory without a register round trip
// (cp.async, completion per thread with cp_async_wait_all).
__device__ __forceinline__ void cp_async8(uint32_t dst, const double *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Orders this thread's generic-proxy shared-memory accesses before later
// async-proxy (TMA) accesses of the same locations.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `parity` of the barrier, giving up after limit_ns of wall
// time (checked every 256 polls).  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0u && globaltimer_ns() - t0 > limit_ns) return false;
  }
}

// Spin while *word == value, giving up after limit_ns of wall time (checked
// every poll, with a short sleep between polls).  Returns false on timeout.
__device__ __forceinline__ bool spin_while_equal(const volatile unsigned *word, unsigned value, uint64_t limit_ns) {
  const uint64_t t0 = globaltimer_ns();
  while (*word == value) {
    if (globaltimer_ns() - t0 > limit_ns) return false;
    __nanosleep(64);
  }
  return true;
}

// TMA tiled loads into shared memory, completing on an mbarrier.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

}  // namespace fvk
