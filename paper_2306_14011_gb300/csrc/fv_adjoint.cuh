// Reverse mode (vector-Jacobian products) of the face flux and of the MUSCL
// reconstruction, for the discrete adjoint of the residual (paper Eq. (5) with
// the fluxes of Eq. (2) and states of Eq. (6)).
//
// roe_2F_vjp recomputes the forward quantities of twice the flux of roe_F
// (fv_device.cuh), in the central form (F(QL) + F(QR)) - sum |lambda| alpha r,
// and propagates a cotangent Gb of that output (2F) back to its inputs, line
// by line in reverse.  Conventions at the non-differentiable points follow the
// forward-mode reference: |x| has derivative sign(x) with sign(+0) = +1, the
// entropy fix takes the branch the forward pass took, and the limited slope
// minmod(a, b) passes the derivative of the argument it returned (b on ties)
// and none when the arguments do not have one strict sign.
#pragma once
#include "fv_device.cuh"

namespace fvk {

// x with the sign of x flipped when s < 0 (or s is -0): x * sign(s), exact, integer pipe.
__device__ __forceinline__ double mul_sign(double x, double s) {
  return __hiloint2double(__double2hiint(x) ^ (__double2hiint(s) & (int)0x80000000u), __double2loint(x));
}

template <int NT>
__device__ __forceinline__ void roe_2F_vjp(const double (&QL)[NT + 3], const double (&QR)[NT + 3], double g1,
                                           double efix, double inv2efix, const double (&Gb)[NT + 3],
                                           double (&QLb)[NT + 3], double (&QRb)[NT + 3]) {
  constexpr int E = NT + 2;
  // ---------------- forward: 2F in the central form, with the Roe averages
  // in their two-weight form u~ = wL uL + wR uR, H~ = wL HL + wR HR (the same
  // function as roe_F, which evaluates it one-sided to save FP64 operations)
  const double tL = rsqrt_fp64(QL[0]);
  const double rL = tL * tL;
  const double sL = QL[0] * tL;
  const double unL = QL[1] * rL;
  double utL[NT];
  double kL = QL[1] * unL;
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    utL[t] = QL[2 + t] * rL;
    kL = fma(QL[2 + t], utL[t], kL);
  }
  const double pL = g1 * fma(-0.5, kL, QL[E]);
  const double eL = QL[E] + pL;
  const double HL = eL * rL;
  const double tR = rsqrt_fp64(QR[0]);
  const double rR = tR * tR;
  const double sR = QR[0] * tR;
  const double unR = QR[1] * rR;
  double utR[NT];
  double kR = QR[1] * unR;
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    utR[t] = QR[2 + t] * rR;
    kR = fma(QR[2 + t], utR[t], kR);
  }
  const double pR = g1 * fma(-0.5, kR, QR[E]);
  const double eR = QR[E] + pR;
  const double HR = eR * rR;
  const double inv = rcp_fp64(sL + sR);
  const double wL = sL * inv, wR = sR * inv;
  const double un = fma(wL, unL, wR * unR);
  double ut[NT];
  double q2 = un * un;
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    ut[t] = fma(wL, utL[t], wR * utR[t]);
    q2 = fma(ut[t], ut[t], q2);
  }
  const double H = fma(wL, HL, wR * HR);
  const double rho = sL * sR;
  const double hq = half_nonneg(q2);
  const double c2 = g1 * (H - hq);
  const double tc = rsqrt_fp64(c2);
  const double c = c2 * tc;
  const double ic2 = tc * tc;
  const double dp = pR - pL;
  const double dun = unR - unL;
  const double rc = rho * c;
  const double rcdun = rc * dun;
  const double hic2 = half_nonneg(ic2);
  const double a1 = (dp - rcdun) * hic2;
  const double a3 = (dp + rcdun) * hic2;
  const double a2 = fma(-dp, ic2, QR[0] - QL[0]);
  const double x1 = un - c, x3 = un + c;
  const double m1 = iabs(x1), m3 = iabs(x3), l2 = iabs(un);
  // the fix decision of roe_F (FP32 copies), so both differentiate one function
  const float deltaf = __fmul_rn(f32_trunc(efix), f32_trunc(c));
  const bool fix1 = f32_trunc(m1) < deltaf, fix3 = f32_trunc(m3) < deltaf;
  double l1 = m1, l3 = m3, delta = 0.0, s2 = 0.0;
  const bool anyfix = __any_sync(__activemask(), fix1 || fix3);
  if (anyfix) {
    delta = efix * c;
    s2 = tc * inv2efix;
    const double d2 = delta * delta;
    l1 = isel(fix1, fma(m1, m1, d2) * s2, m1);
    l3 = isel(fix3, fma(m3, m3, d2) * s2, m3);
  }
  const double A1 = l1 * a1, A2 = l2 * a2, A3 = l3 * a3;
  const double lr = l2 * rho;
  const double s13 = A1 + A3;
  const double d13 = A3 - A1;
  const double cd13 = c * d13;
  const double D0 = s13 + A2;
  double B[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) B[t] = lr * (utR[t] - utL[t]);

  // ---------------- reverse
  double mnLb = Gb[0] + Gb[1] * unL, mnRb = Gb[0] + Gb[1] * unR;
  double unLb = Gb[1] * QL[1] + Gb[E] * eL, unRb = Gb[1] * QR[1] + Gb[E] * eR;
  double pLb = Gb[1], pRb = Gb[1];
  double eLb = Gb[E] * unL, eRb = Gb[E] * unR;
  double utLb[NT], utRb[NT], utb[NT], Bb[NT];
  double D0b = -Gb[0];
  const double Dnb = -Gb[1];
  const double DEb = -Gb[E];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    mnLb = fma(Gb[2 + t], utL[t], mnLb);
    mnRb = fma(Gb[2 + t], utR[t], mnRb);
    utLb[t] = Gb[2 + t] * QL[1];
    utRb[t] = Gb[2 + t] * QR[1];
    const double Dtb = -Gb[2 + t];
    // DE += ut B; Dt = ut D0 + B
    utb[t] = fma(DEb, B[t], Dtb * D0);
    Bb[t] = fma(DEb, ut[t], Dtb);
    D0b = fma(Dtb, ut[t], D0b);
  }
  // DE = hq A2 + sum ut B + un cd13 + H s13
  double hqb = DEb * A2;
  double A2b = DEb * hq;
  double unb = DEb * cd13;
  double cd13b = DEb * un;
  double Hb = DEb * s13;
  double s13b = DEb * H;
  // B = lr (utR - utL)
  double lrb = 0.0;
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    lrb = fma(Bb[t], utR[t] - utL[t], lrb);
    utRb[t] = fma(Bb[t], lr, utRb[t]);
    utLb[t] = fma(-Bb[t], lr, utLb[t]);
  }
  // Dn = un D0 + cd13
  unb = fma(Dnb, D0, unb);
  D0b = fma(Dnb, un, D0b);
  cd13b += Dnb;
  // D0 = s13 + A2
  s13b += D0b;
  A2b += D0b;
  // cd13 = c d13; d13 = A3 - A1; s13 = A1 + A3
  double cb = cd13b * d13;
  const double d13b = cd13b * c;
  const double A3b = s13b + d13b, A1b = s13b - d13b;
  // lr = l2 rho
  double l2b = lrb * rho;
  double rhob = lrb * l2;
  // A_w = l_w a_w
  const double l1b = A1b * a1, a1b = A1b * l1;
  l2b = fma(A2b, a2, l2b);
  const double a2b = A2b * l2;
  const double l3b = A3b * a3, a3b = A3b * l3;
  // eigenvalue magnitudes, entropy fix
  double m1b = l1b, m3b = l3b, deltab = 0.0, tcb = 0.0;
  if (anyfix) {
    const double s2b = isel(fix1, l1b * fma(m1, m1, delta * delta), 0.0) +
                       isel(fix3, l3b * fma(m3, m3, delta * delta), 0.0);
    m1b = isel(fix1, 2.0 * m1 * s2 * l1b, l1b);
    m3b = isel(fix3, 2.0 * m3 * s2 * l3b, l3b);
    deltab = isel(fix1, 2.0 * delta * s2 * l1b, 0.0) + isel(fix3, 2.0 * delta * s2 * l3b, 0.0);
    tcb = s2b * inv2efix;
  }
  cb = fma(deltab, efix, cb);
  const double x1b = mul_sign(m1b, x1), x3b = mul_sign(m3b, x3);
  unb += mul_sign(l2b, un) + x1b + x3b;
  cb += x3b - x1b;
  // a2 = drho - dp ic2 ; a1, a3 = (dp -+ rcdun) hic2
  const double drhob = a2b;
  double dpb = fma(a1b + a3b, hic2, -a2b * ic2);
  double ic2b = -a2b * dp;
  const double rcdunb = (a3b - a1b) * hic2;
  const double hic2b = fma(a1b, dp - rcdun, a3b * (dp + rcdun));
  ic2b = fma(0.5, hic2b, ic2b);
  // rcdun = rc dun ; rc = rho c
  const double rcb = rcdunb * dun;
  const double dunb = rcdunb * rc;
  rhob = fma(rcb, c, rhob);
  cb = fma(rcb, rho, cb);
  unRb += dunb;
  unLb -= dunb;
  pRb += dpb;
  pLb -= dpb;
  // ic2 = tc^2 ; c = c2 tc ; tc = c2^(-1/2)
  tcb = fma(ic2b, scale_pow2<1>(tc), tcb);
  tcb = fma(cb, c2, tcb);
  double c2b = cb * tc;
  c2b = fma(tcb, -(scale_pow2<-1>(tc) * ic2), c2b);
  // c2 = g1 (H - hq)
  Hb = fma(c2b, g1, Hb);
  hqb = fma(-c2b, g1, hqb);
  // q2b = hqb / 2 enters as 2 q2b un = hqb un and 2 q2b ut = hqb ut
  // rho = sL sR
  double sLb = rhob * sR, sRb = rhob * sL;
  // H = wL HL + wR HR
  double wLb = Hb * HL, wRb = Hb * HR;
  const double HLb = Hb * wL, HRb = Hb * wR;
  // q2 = un^2 + sum ut^2
  unb = fma(hqb, un, unb);
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    utb[t] = fma(hqb, ut[t], utb[t]);
    // ut = wL utL + wR utR
    wLb = fma(utb[t], utL[t], wLb);
    wRb = fma(utb[t], utR[t], wRb);
    utLb[t] = fma(utb[t], wL, utLb[t]);
    utRb[t] = fma(utb[t], wR, utRb[t]);
  }
  // un = wL unL + wR unR
  wLb = fma(unb, unL, wLb);
  wRb = fma(unb, unR, wRb);
  unLb = fma(unb, wL, unLb);
  unRb = fma(unb, wR, unRb);
  // wL = sL inv ; wR = sR inv ; inv = 1 / (sL + sR)
  sLb = fma(wLb, inv, sLb);
  sRb = fma(wRb, inv, sRb);
  const double invb = fma(wLb, sL, wRb * sR);
  const double Sb = -invb * inv * inv;
  sLb += Sb;
  sRb += Sb;

  // left side: HL = eL rL ; eL = E + pL ; pL = g1 (E - kL/2) ; kL = mn unL + sum mt utL
  double rLb = HLb * eL;
  eLb = fma(HLb, rL, eLb);
  double ELb = eLb;
  pLb += eLb;
  ELb = fma(pLb, g1, ELb);
  const double kLb = -0.5 * g1 * pLb;
  mnLb = fma(kLb, unL, mnLb);
  unLb = fma(kLb, QL[1], unLb);
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    double mtb = kLb * utL[t];
    utLb[t] = fma(kLb, QL[2 + t], utLb[t]);
    // utL = mt rL
    mtb = fma(utLb[t], rL, mtb);
    rLb = fma(utLb[t], QL[2 + t], rLb);
    QLb[2 + t] = mtb;
  }
  // unL = mn rL ; sL = rho tL ; rL = tL^2 ; tL = rho^(-1/2)
  mnLb = fma(unLb, rL, mnLb);
  rLb = fma(unLb, QL[1], rLb);
  double tLb = sLb * QL[0];
  double rhoLb = sLb * tL;
  tLb = fma(rLb, scale_pow2<1>(tL), tLb);
  rhoLb = fma(tLb, -(scale_pow2<-1>(tL) * rL), rhoLb);
  QLb[0] = rhoLb - drhob;
  QLb[1] = mnLb;
  QLb[E] = ELb;

  // right side
  double rRb = HRb * eR;
  eRb = fma(HRb, rR, eRb);
  double ERb = eRb;
  pRb += eRb;
  ERb = fma(pRb, g1, ERb);
  const double kRb = -0.5 * g1 * pRb;
  mnRb = fma(kRb, unR, mnRb);
  unRb = fma(kRb, QR[1], unRb);
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    double mtb = kRb * utR[t];
    utRb[t] = fma(kRb, QR[2 + t], utRb[t]);
    mtb = fma(utRb[t], rR, mtb);
    rRb = fma(utRb[t], QR[2 + t], rRb);
    QRb[2 + t] = mtb;
  }
  mnRb = fma(unRb, rR, mnRb);
  rRb = fma(unRb, QR[1], rRb);
  double tRb = sRb * QR[0];
  double rhoRb = sRb * tR;
  tRb = fma(rRb, scale_pow2<1>(tR), tRb);
  rhoRb = fma(tRb, -(scale_pow2<-1>(tR) * rR), rhoRb);
  QRb[0] = rhoRb + drhob;
  QRb[1] = mnRb;
  QRb[E] = ERb;
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
