// Reverse mode (vector-Jacobian products) of the face flux and of the MUSCL
// reconstruction, for the discrete adjoint of the residual (paper Eq. (5) with
// the fluxes of Eq. (2) and states of Eq. (6)).
//
// roe_F_vjp recomputes the forward quantities of roe_F (fv_device.cuh), with
// its products on the integer pipe like roe_F: the
// upwind physical flux plus the one acoustic wave that crosses from downwind,
// which equals the central Roe flux (F(QL) + F(QR))/2 - sum |lambda| alpha r/2
// as a function; it propagates a cotangent Gb of F back to the two states,
// line by line in reverse.  Conventions at the non-differentiable points
// follow the forward-mode reference: |x| has derivative sign(x) with
// sign(+0) = +1 (the upwind side of u~_n = +0 is the left one, where the
// contact and shear waves drop out, as sign(+0) = +1 gives), the entropy fix
// takes the branch the forward pass took, and the limited slope minmod(a, b)
// passes the derivative of the argument it returned (b on ties) and none when
// the arguments do not have one strict sign.
#pragma once
#include "fv_device.cuh"

namespace fvk {

// x with the sign of x flipped when s < 0 (or s is -0): x * sign(s), exact, integer pipe.
__device__ __forceinline__ double mul_sign(double x, double s) {
  return __hiloint2double(__double2hiint(x) ^ (__double2hiint(s) & (int)0x80000000u), __double2loint(x));
}

// EMU: every product runs on the integer pipe (pmul, signed zeros included)
// and ok reports whether all stayed on the integer path; the wrapper below
// re-evaluates in FP64 (products rounded on their own, so both evaluations
// give the same bits) when one did not.
template <int NT, bool EMU>
__device__ __forceinline__ void roe_F_vjp_impl(const double (&QL)[NT + 3], const double (&QR)[NT + 3], double g1,
                                               double efix, double inv2efix, const double (&Gb)[NT + 3],
                                               double (&QLb)[NT + 3], double (&QRb)[NT + 3], bool &ok) {
  constexpr int E = NT + 2;
  auto M = [&ok](double a, double b) { return pmul<EMU, true>(a, b, ok); };
  // ---------------- forward: the quantities of roe_F
  const double tL = rsqrt_fp64<EMU, !EMU>(QL[0], ok);
  const double rL = M(tL, tL);
  const double sL = M(QL[0], tL);
  const double unL = M(QL[1], rL);
  double utL[NT];
  double kL = M(QL[1], unL);
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    utL[t] = M(QL[2 + t], rL);
    kL = fma(QL[2 + t], utL[t], kL);
  }
  const double pL = M(g1, fma(-0.5, kL, QL[E]));
  const double eL = QL[E] + pL;
  const double tR = rsqrt_fp64<EMU, !EMU>(QR[0], ok);
  const double rR = M(tR, tR);
  const double sR = M(QR[0], tR);
  const double unR = M(QR[1], rR);
  double utR[NT];
  double kR = M(QR[1], unR);
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    utR[t] = M(QR[2 + t], rR);
    kR = fma(QR[2 + t], utR[t], kR);
  }
  const double pR = M(g1, fma(-0.5, kR, QR[E]));
  const double eR = QR[E] + pR;
  const double inv = rcp_fp64<!EMU>(sL + sR);
  const double wL = M(sL, inv), wR = M(sR, inv);
  const double dun = unR - unL;
  const double un = fma(-wL, dun, unR);
  double ut[NT], dut[NT];
  double q2 = M(un, un);
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    dut[t] = utR[t] - utL[t];
    ut[t] = fma(-wL, dut[t], utR[t]);
    q2 = fma(ut[t], ut[t], q2);
  }
  const double Hn = fma(eL, tL, M(eR, tR));
  const double H = M(Hn, inv);
  const double rho = M(sL, sR);
  const double c2 = M(g1, H - half_nonneg(q2));
  const double tc = rsqrt_fp64<EMU, !EMU>(c2, ok);
  const double c = M(c2, tc);
  const bool up_left = __double2hiint(un) >= 0;
  const double aun = iabs(un);
  const double sc = isel(up_left, c, ineg(c));
  const double dp = pR - pL;
  const double rsc = M(rho, sc);
  const double num = fma(-rsc, dun, dp);
  const double tc2h = M(tc, half_nonneg(tc));  // 1 / (2 c~^2)
  const double alpha = M(num, tc2h);
  const double x = aun - c;
  const bool neg = __double2hiint(x) < 0 && !izero(x);
  double k = isel(neg, x, 0.0);
  // the fix decision of roe_F (FP32 copies), so both differentiate one function
  const float deltaf = __fmul_rn(f32_trunc(efix), f32_trunc(c));
  const bool fix = f32_trunc(iabs(x)) < deltaf;
  const bool anyfix = __any_sync(__activemask(), fix);
  double delta = 0.0, s2 = 0.0;
  if (anyfix) {
    delta = __dmul_rn(efix, c);
    s2 = __dmul_rn(tc, inv2efix);  // 1 / (2 delta)
    k = isel(fix, fma(-fma(x, x, __dmul_rn(delta, delta)), __dmul_rn(0.5, s2), __dmul_rn(0.5, x)), k);
  }
  const double g = M(k, alpha);
  const double lam = un - sc;
  const double hr = fma(-c, aun, H);
  const double m = isel(up_left, QL[1], QR[1]);
  const double u_n = isel(up_left, unL, unR);
  const double e = isel(up_left, eL, eR);

  // ---------------- reverse
  // G0 = m + g; G1 = m u_n + p_up + g lam; G2+t = m ut_up + g ut; GE = u_n e + g hr
  double mb = fma(Gb[1], u_n, Gb[0]);
  double u_nb = fma(Gb[E], e, M(Gb[1], m));
  const double pupb = Gb[1];
  const double eupb = M(Gb[E], u_n);
  double gb = fma(Gb[E], hr, fma(Gb[1], lam, Gb[0]));
  double utupb[NT], utb[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    mb = fma(Gb[2 + t], isel(up_left, utL[t], utR[t]), mb);
    utupb[t] = M(Gb[2 + t], m);
    gb = fma(Gb[2 + t], ut[t], gb);
    utb[t] = M(Gb[2 + t], g);
  }
  const double lamb = M(Gb[1], g);
  const double hrb = M(Gb[E], g);
  // hr = H - c aun ; lam = un - sc
  double Hb = hrb;
  double cb = M(-hrb, aun);
  double aunb = M(-hrb, c);
  double unb = lamb;
  double scb = -lamb;
  // g = k alpha
  const double kb = M(gb, alpha);
  const double alphab = M(gb, k);
  // k = min(x, 0), or with the fix x/2 - (x^2 + delta^2) / (4 delta)
  double xb = isel(neg, kb, 0.0);
  if (anyfix) {
    const double xs = __dmul_rn(x, s2);  // x / (2 delta)
    xb = isel(fix, __dmul_rn(kb, 0.5 - xs), xb);
    cb = fma(isel(fix, __dmul_rn(kb, fma(xs, xs, -0.25)), 0.0), efix, cb);  // delta = efix c
  }
  // x = aun - c ; aun = |un|
  aunb += xb;
  cb -= xb;
  unb += mul_sign(aunb, un);
  // alpha = num tc2h ; num = dp - rsc dun ; rsc = rho sc ; tc2h = tc^2 / 2 ; sc = +-c
  const double numb = M(alphab, tc2h);
  double tcb = M(M(alphab, num), tc);
  const double dpb = numb;
  const double rscb = M(-numb, dun);
  const double dunb = M(-numb, rsc);
  const double rhob = M(rscb, sc);
  scb = fma(rscb, rho, scb);
  cb += isel(up_left, scb, ineg(scb));
  // c = c2 tc ; tc = c2^(-1/2)
  tcb = fma(cb, c2, tcb);
  double c2b = M(cb, tc);
  c2b = fma(tcb, -M(half_nonneg(tc), M(tc, tc)), c2b);
  // c2 = g1 (H - q2/2) ; q2 = un^2 + sum ut^2
  Hb = fma(c2b, g1, Hb);
  const double q2b2 = M(-g1, c2b);  // 2 q2b
  unb = fma(q2b2, un, unb);
  // H = Hn inv ; Hn = eL tL + eR tR
  double invb = M(Hb, Hn);
  const double Hnb = M(Hb, inv);
  double eLb = M(Hnb, tL), eRb = M(Hnb, tR);
  double tLb = M(Hnb, eL), tRb = M(Hnb, eR);
  // rho = sL sR
  double sLb = M(rhob, sR), sRb = M(rhob, sL);
  // ut = utR - wL dut = wL utL + wR utR ; un = unR - wL dun ; dun = unR - unL
  double wLb = M(-unb, dun);
  double utLb[NT], utRb[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    utb[t] = fma(q2b2, ut[t], utb[t]);
    wLb = fma(-utb[t], dut[t], wLb);
    utLb[t] = fma(utb[t], wL, isel(up_left, utupb[t], 0.0));
    utRb[t] = fma(utb[t], wR, isel(up_left, 0.0, utupb[t]));
  }
  double unLb = fma(unb, wL, isel(up_left, u_nb, 0.0)) - dunb;
  double unRb = fma(unb, wR, isel(up_left, 0.0, u_nb)) + dunb;
  // wL = sL inv (wR = 1 - wL) ; inv = 1 / (sL + sR)
  sLb = fma(wLb, inv, sLb);
  invb = fma(wLb, sL, invb);
  const double Sb = M(M(-invb, inv), inv);
  sLb += Sb;
  sRb += Sb;
  // dp = pR - pL ; the upwind side's m, p, e
  double pLb = isel(up_left, pupb - dpb, -dpb), pRb = isel(up_left, dpb, pupb + dpb);
  eLb += isel(up_left, eupb, 0.0);
  eRb += isel(up_left, 0.0, eupb);
  double mnLb = isel(up_left, mb, 0.0), mnRb = isel(up_left, 0.0, mb);

  // left side: eL = E + pL ; pL = g1 (E - kL/2) ; kL = mn unL + sum mt utL ;
  // unL = mn rL ; utL = mt rL ; sL = rho tL ; rL = tL^2 ; tL = rho^(-1/2)
  double ELb = eLb;
  pLb += eLb;
  ELb = fma(pLb, g1, ELb);
  const double kLb = M(M(-0.5, g1), pLb);
  mnLb = fma(kLb, unL, mnLb);
  unLb = fma(kLb, QL[1], unLb);
  double rLb = 0.0;
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    double mtb = M(kLb, utL[t]);
    utLb[t] = fma(kLb, QL[2 + t], utLb[t]);
    mtb = fma(utLb[t], rL, mtb);
    rLb = fma(utLb[t], QL[2 + t], rLb);
    QLb[2 + t] = mtb;
  }
  mnLb = fma(unLb, rL, mnLb);
  rLb = fma(unLb, QL[1], rLb);
  tLb = fma(sLb, QL[0], tLb);
  double rhoLb = M(sLb, tL);
  tLb = fma(rLb, scale_pow2<1>(tL), tLb);
  rhoLb = fma(tLb, -M(half_nonneg(tL), rL), rhoLb);
  QLb[0] = rhoLb;
  QLb[1] = mnLb;
  QLb[E] = ELb;

  // right side
  double ERb = eRb;
  pRb += eRb;
  ERb = fma(pRb, g1, ERb);
  const double kRb = M(M(-0.5, g1), pRb);
  mnRb = fma(kRb, unR, mnRb);
  unRb = fma(kRb, QR[1], unRb);
  double rRb = 0.0;
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    double mtb = M(kRb, utR[t]);
    utRb[t] = fma(kRb, QR[2 + t], utRb[t]);
    mtb = fma(utRb[t], rR, mtb);
    rRb = fma(utRb[t], QR[2 + t], rRb);
    QRb[2 + t] = mtb;
  }
  mnRb = fma(unRb, rR, mnRb);
  rRb = fma(unRb, QR[1], rRb);
  tRb = fma(sRb, QR[0], tRb);
  double rhoRb = M(sRb, tR);
  tRb = fma(rRb, scale_pow2<1>(tR), tRb);
  rhoRb = fma(tRb, -M(half_nonneg(tR), rR), rhoRb);
  QRb[0] = rhoRb;
  QRb[1] = mnRb;
  QRb[E] = ERb;
}

// The face flux VJP with its products on the integer pipe; a warp in which a
// product left the integer path evaluates it again in FP64.
template <int NT>
__device__ __forceinline__ void roe_F_vjp(const double (&QL)[NT + 3], const double (&QR)[NT + 3], double g1,
                                          double efix, double inv2efix, const double (&Gb)[NT + 3],
                                          double (&QLb)[NT + 3], double (&QRb)[NT + 3]) {
  bool ok = true;
  roe_F_vjp_impl<NT, true>(QL, QR, g1, efix, inv2efix, Gb, QLb, QRb, ok);
  if (__any_sync(__activemask(), !ok)) roe_F_vjp_impl<NT, false>(QL, QR, g1, efix, inv2efix, Gb, QLb, QRb, ok);
}

// Which argument the limited slope minmod(a, b) passes a derivative through:
// 1 = a, 2 = b, 0 = none (signs differ or an argument is zero; ties -> b).
__device__ __forceinline__ int minmod_pick(double a, double b) {
  const int ha = __double2hiint(a), hb = __double2hiint(b);
  const unsigned la = (unsigned)__double2loint(a), lb = (unsigned)__double2loint(b);
  const unsigned ma = (unsigned)ha & 0x7fffffffu, mb = (unsigned)hb & 0x7fffffffu;
  if (((ha ^ hb) < 0) || (ma | la) == 0u || (mb | lb) == 0u) return 0;
  return (ma < mb || (ma == mb && la < lb)) ? 1 : 2;
}

}  // namespace fvk
