// q(1) q~(2) -> t(3) t~(4): the per-event amplitude arithmetic (helicity
// amplitudes -> the three constants of the helicity-summed |M|^2 as a polynomial
// in the top mass squared).  Device routines templated on the arithmetic type;
// the tile that runs them is in qq_kernel.cuh.
#pragma once

#include "helas.cuh"

namespace rex {

// S^mu = b^dag sigma^mu a (sigma = (1, sigma_x, sigma_y, sigma_z)); the sigmabar
// bilinear is (S^0, -S^vec).
template <typename R>
__device__ __forceinline__ void sigma_bilinear(const cx<R>* b, const cx<R>* a, cx<R>* S) {
  const cx<R> b0a0 = cdot1(b[0], a[0]), b0a1 = cdot1(b[0], a[1]);
  const cx<R> b1a0 = cdot1(b[1], a[0]), b1a1 = cdot1(b[1], a[1]);
  S[0] = b0a0 + b1a1;
  S[1] = b0a1 + b1a0;
  const cx<R> d = b1a0 - b0a1;          // b^dag sigma_y a = -i b0* a1 + i b1* a0
  S[2] = cx<R>{-d.im, d.re};
  S[3] = b0a0 - b1a1;
}

// chi_-, chi_+ of p and E + |p| (= w+^2)
template <typename R>
__device__ __forceinline__ R chis(const R* p, cx<R>* chim, cx<R>* chip) {
  const R a = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
  chi_pair(p, a, chip, chim);
  return p[0] + a;
}

// The helicity sum of one event as C0 + C2 m^2 + C4 m^4 (c[0..2]) times the
// incoming scale w+(1)^2 w+(2)^2 (*e12) times g^4 colour / (avg s^2), which the
// caller applies where it needs |M|^2 itself (the ratio does not).
template <typename R>
__device__ __forceinline__ void qq_ttx_coefficients(const R (&p)[4][4], R* c, R* e12) {
  cx<R> x1[2][2], x2[2][2], x3[2][2], x4[2][2];   // [0] = chi-, [1] = chi+
  const R e1 = chis(p[0], x1[0], x1[1]);
  const R e2 = chis(p[1], x2[0], x2[1]);
  const R e3 = chis(p[2], x3[0], x3[1]);
  const R e4 = chis(p[3], x4[0], x4[1]);

  // J_in / (w+(1) w+(2)) for (l1, l2) = (+, -): -chi2+^dag sigma chi1+ (the sign drops
  // out of every |.|^2 and DL* DR) and (-, +): chi2-^dag sigmabar chi1-.
  cx<R> J[2][4];
  sigma_bilinear(x2[1], x1[1], J[0]);
  sigma_bilinear(x2[0], x1[0], J[1]);
#pragma unroll
  for (int m = 1; m < 4; ++m) J[1][m] = cx<R>{-J[1][m].re, -J[1][m].im};

  // top-helicity pairs q = (l3, l4) in the order (+,+), (+,-), (-,+), (-,-):
  // xi = chi3_{l3}, eta = chi4_{-l4}
  R pll[4], prr[4], plr[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int l3p = q < 2, l4p = (q & 1) == 0;
    cx<R> S[4];
    sigma_bilinear(x3[l3p ? 1 : 0], x4[l4p ? 0 : 1], S);
    R ll = R(0), rr = R(0), lr = R(0);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const cx<R> t0 = J[h][0] * S[0];
      const cx<R> t1 = J[h][1] * S[1] + J[h][2] * S[2] + J[h][3] * S[3];
      const cx<R> dl = t0 + t1, dr = t0 - t1;   // J.BL, J.BR (Minkowski)
      ll += dl.re * dl.re + dl.im * dl.im;
      rr += dr.re * dr.re + dr.im * dr.im;
      lr += dl.re * dr.re + dl.im * dr.im;
    }
    pll[q] = ll;
    prr[q] = rr;
    plr[q] = lr;
  }
  // W^2 = e3 e4, r^2 = e4 / e3, with one reciprocal
  const R w2 = e3 * e4;
  const R iw2 = R(1) / w2;
  const R r2 = e4 * e4 * iw2, ir2 = e3 * e3 * iw2;
  c[0] = w2 * (prr[1] + pll[2]);
  c[1] = r2 * (pll[0] + prr[3]) + ir2 * (prr[0] + pll[3]) - R(2) * (plr[0] + plr[1] + plr[2] + plr[3]);
  c[2] = iw2 * (pll[1] + prr[2]);
  *e12 = e1 * e2;
}

// Helicity-exclusive form: the term of one configuration (l1, l2, l3, l4) (positive:
// +1, otherwise -1) as C0 + C2 m^2 + C4 m^4 in the same normalisation.  Equal q, q~
// helicities give exact zeros (chirality).  For the top pair q = (l3, l4):
//   (+,+): C2 = r^2 LL + RR / r^2 - 2 LR;   (-,-): C2 = LL / r^2 + r^2 RR - 2 LR;
//   (+,-): C0 = W^2 RR, C2 = -2 LR, C4 = LL / W^2;   (-,+): C0 = W^2 LL, C2 = -2 LR, C4 = RR / W^2,
// with LL = |DL|^2, RR = |DR|^2, LR = Re(DL* DR) of the one incoming current.
template <typename R>
__device__ __forceinline__ void qq_ttx_coefficients_h(const R (&p)[4][4], int l1, int l2, int l3, int l4, R* c,
                                                      R* e12) {
  cx<R> x1[2][2], x2[2][2], x3[2][2], x4[2][2];   // [0] = chi-, [1] = chi+
  const R e1 = chis(p[0], x1[0], x1[1]);
  const R e2 = chis(p[1], x2[0], x2[1]);
  const R e3 = chis(p[2], x3[0], x3[1]);
  const R e4 = chis(p[3], x4[0], x4[1]);
  *e12 = e1 * e2;
  c[0] = c[1] = c[2] = R(0);
  if ((l1 > 0) == (l2 > 0)) return;
  cx<R> J[4], S[4];
  if (l1 > 0) {
    sigma_bilinear(x2[1], x1[1], J);            // (+, -): sigma
  } else {
    sigma_bilinear(x2[0], x1[0], J);            // (-, +): sigmabar
#pragma unroll
    for (int m = 1; m < 4; ++m) J[m] = cx<R>{-J[m].re, -J[m].im};
  }
  sigma_bilinear(x3[l3 > 0 ? 1 : 0], x4[l4 > 0 ? 0 : 1], S);
  const cx<R> t0 = J[0] * S[0];
  const cx<R> t1 = J[1] * S[1] + J[2] * S[2] + J[3] * S[3];
  const cx<R> dl = t0 + t1, dr = t0 - t1;
  const R ll = dl.re * dl.re + dl.im * dl.im;
  const R rr = dr.re * dr.re + dr.im * dr.im;
  const R lr = dl.re * dr.re + dl.im * dr.im;
  const R w2 = e3 * e4;
  const R iw2 = R(1) / w2;
  const R r2 = e4 * e4 * iw2, ir2 = e3 * e3 * iw2;
  if ((l3 > 0) == (l4 > 0)) {
    c[1] = (l3 > 0 ? r2 * ll + ir2 * rr : ir2 * ll + r2 * rr) - R(2) * lr;
  } else if (l3 > 0) {
    c[0] = w2 * rr;
    c[1] = R(-2) * lr;
    c[2] = iw2 * ll;
  } else {
    c[0] = w2 * ll;
    c[1] = R(-2) * lr;
    c[2] = iw2 * rr;
  }
}

}  // namespace rex
