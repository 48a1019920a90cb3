// q(1) q~(2) -> t(3) t~(4) g(5): helicity amplitudes of one lane (device routines,
// templated on the arithmetic type; the tile that runs them is in qqg_kernel.cuh).
//
// Diagrams (light line read from vbar(p2) to u(p1), top line from ubar(p3) to v(p4);
// s = (p1 + p2)^2, s' = (p3 + p4)^2, k = p5, eps a real linear polarisation):
//   a1 = C1 . J_out / s',   C1 = vbar2 gamma^mu (p1 - k)-slash eps-slash u1 / (p1 - k)^2
//   a2 = C2 . J_out / s',   C2 = vbar2 eps-slash (k - p2)-slash gamma^mu u1 / (k - p2)^2
//   a3 = ubar3 eps-slash ((p3 + k)-slash + m) J_in-slash v4 / (((p3 + k)^2 - m^2 + i m G) s)
//   a4 = ubar3 J_in-slash ((-p4 - k)-slash + m) eps-slash v4 / (((p4 + k)^2 - m^2 + i m G) s)
//   a5 = E . J_out / (s s'),  E = (J_in.eps)(q + k) + (J_in.(q' - k)) eps - (eps.(q' + q)) J_in
// with J_in = vbar2 gamma u1, J_out = ubar3 gamma v4, q = p1 + p2, q' = p3 + p4 (the
// three-gluon vertex with every momentum incoming).  The Feynman-rule factors are
// -i g^3 for a1..a4 and g^3 for a5; the -i is moved into the colour matrix, which
// then is the real symmetric N / 3 below, and g^6, 1/3 and the 1/36 average go into
// the per-point factor.  N = 3 sum over colours of conj(K_d) K_d' for the colour
// structures (t^b t^a)(t^b), (t^a t^b)(t^b), (t^b)(t^a t^b), (t^b)(t^b t^a) and
// f^{bac}(t^b)(t^c), with the i of the last one's relative phase included; from
// Tr(t^a t^b) = delta/2, sum_a t^a t^a = C_F = 4/3, sum_a t^a t^b t^a = -t^b / 6,
// f^{acd} f^{bcd} = 3 delta: e.g. N_11 = 3 (N C_F^2 / 2) = 8, N_55 = 3 (C_A (N^2-1)/4) = 18.
//
// A lane holds one light-quark helicity pair (the two with equal helicities vanish
// for massless quarks) and one gluon polarisation: 4 lanes per event.  Everything
// the parameters do not touch (C1, C2, E, J_in) is built once per event; per mass
// slot the lane builds the top spinors, the two top-line chains and the 5 amplitudes
// of its 4 top-helicity pairs.
#pragma once

#include "helas.cuh"
#include "qq_amplitude.cuh"

namespace rex {

// psibar gamma^mu chi of Dirac spinors (chiral basis):
// psi_L^dag sigmabar^mu chi_L + psi_R^dag sigma^mu chi_R
template <typename R>
__device__ __forceinline__ void dirac_current(const cx<R>* psi, const cx<R>* chi, cx<R>* J) {
  cx<R> sl[4], sr[4];
  sigma_bilinear(psi, chi, sl);
  sigma_bilinear(psi + 2, chi + 2, sr);
  J[0] = sl[0] + sr[0];
#pragma unroll
  for (int m = 1; m < 4; ++m) J[m] = sr[m] - sl[m];
}

// out = J-slash psi for a complex 4-vector J
template <typename R>
__device__ __forceinline__ void cslash(const cx<R>* J, const cx<R>* psi, cx<R>* out) {
  R jr[4], ji[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    jr[m] = J[m].re;
    ji[m] = J[m].im;
  }
  cx<R> t[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    out[i] = cx<R>{R(0), R(0)};
    t[i] = cx<R>{R(0), R(0)};
  }
  slash_acc(R(1), jr, psi, out);
  slash_acc(R(1), ji, psi, t);
#pragma unroll
  for (int i = 0; i < 4; ++i) out[i] = out[i] + cx<R>{-t[i].im, t[i].re};
}

// Minkowski product of complex 4-vectors (no conjugation)
template <typename R>
__device__ __forceinline__ cx<R> cdotm(const cx<R>* a, const cx<R>* b) {
  return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}

// Minkowski product of a complex and a real 4-vector
template <typename R>
__device__ __forceinline__ cx<R> cdotr(const cx<R>* a, const R* b) {
  return cx<R>{a[0].re * b[0] - a[1].re * b[1] - a[2].re * b[2] - a[3].re * b[3],
               a[0].im * b[0] - a[1].im * b[1] - a[2].im * b[2] - a[3].im * b[3]};
}

// 3 x the colour matrix of a1..a5 (real symmetric; see the header comment)
__device__ __forceinline__ constexpr int qqg_colour(int i, int j) {
  constexpr int N[5][5] = {{8, -1, 7, -2, -9}, {-1, 8, -2, 7, 9}, {7, -2, 8, -1, -9},
                           {-2, 7, -1, 8, 9}, {-9, 9, -9, 9, 18}};
  return N[i][j];
}

template <typename R>
struct QqgLane {
  cx<R> jin[4], c1[4], c2[4], e[4];
  R eps[4], a3[4], a4[4];
  cx<R> chi3[2][2], chi4[2][2];   // [0] = chi-, [1] = chi+
  R wp3, wp4;
  R is, isp;                      // 1/s, 1/s'
  R d3, d4;                       // (p3 + k)^2 - m0^2, (p4 + k)^2 - m0^2
  bool split;                     // gauge split of J_in taken (jin holds J', QqgSplit the rest)
};

// The rest of a lane's gauge split (qqg_lane_gauge_split), kept in shared memory; a
// lane without the split holds zeros here, which leave its amplitudes unchanged.
template <typename R>
struct QqgSplit {
  cx<R> al;                       // J_in = J' + al q
  R qpe;                          // q'.eps
  R n3[4], n4[4];                 // (1, -p-hat) of top and antitop
  R h3, h4;                       // (p^2 - m0^2) / (2 (E + |p|)) of top and antitop
  R g3, g4;                       // 1 / (2 (E + |p|))
};

template <typename R>
__device__ __forceinline__ void qqg_split_clear(QqgSplit<R>& S) {
#pragma unroll
  for (int m = 0; m < 4; ++m) S.n3[m] = S.n4[m] = R(0);
  S.al = cx<R>{R(0), R(0)};
  S.qpe = S.h3 = S.h4 = S.g3 = S.g4 = R(0);
}

// The event's invariants, taken in FP64 by the caller (once per event): 1/s, 1/s',
// 1/(p1 - k)^2, 1/(k - p2)^2 and the top-propagator denominators at a reference mass
// m0, (p3 + k)^2 - m0^2 and (p4 + k)^2 - m0^2; a slot at mass m adds m0^2 - m^2.
template <typename R>
struct QqgInvariants {
  R is, isp, ia1, ia2, d3, d4;
};

// Lane set-up: light-quark helicities (l1, l2) = h12 ? (-, +) : (+, -), gluon
// polarisation pol; p: the event's momenta in R along the fermion-number flow of
// the q q~ -> t t~ g slots.  C1 and C2 are left without their propagator factors
// and the invariants unset: qqg_lane_scale applies them.
//
// Crossed channels: bit 0, 1, 2 of neg marks slot 0, 1, 4 as holding a negated
// physical momentum (an outgoing antiquark, an outgoing quark, an incoming gluon).
// Their wavefunctions are built from the physical momentum with the direct
// channel's functions: summed over helicities only sum_h psi psibar enters, and for
// a massless momentum that is p-slash for u and for v alike, while the two real
// linear polarisations of a gluon sum to the same transverse projector whether it
// is incoming or outgoing.  (The helicity-exclusive form has no such freedom and
// takes the direct channel only.)
template <typename R>
__device__ __forceinline__ void qqg_lane_setup(const R (&p)[5][4], int h12, int pol, QqgLane<R>& L, int neg = 0) {
  const int l1 = h12 ? -1 : 1;
  R k0[4], k1[4], k4[4];   // physical momenta of the light partons
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    k0[m] = (neg & 1) ? -p[0][m] : p[0][m];
    k1[m] = (neg & 2) ? -p[1][m] : p[1][m];
    k4[m] = (neg & 4) ? -p[4][m] : p[4][m];
  }
  cx<R> u1[4], v2[4];
  spinor_u(k0, R(0), l1, u1);
  spinor_v(k1, R(0), -l1, v2);
  pol_linear(k4, pol, L.eps);
  dirac_current(v2, u1, L.jin);
  R a1[4], a2[4], qk[4], qpk[4], qq2[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    a1[m] = p[0][m] - p[4][m];
    a2[m] = p[4][m] - p[1][m];
    L.a3[m] = p[2][m] + p[4][m];
    L.a4[m] = -p[3][m] - p[4][m];
    const R q = p[0][m] + p[1][m], qp = p[2][m] + p[3][m];
    qk[m] = q + p[4][m];
    qpk[m] = qp - p[4][m];
    qq2[m] = qp + q;
  }
  // C1 = vbar2 gamma^mu a1-slash eps-slash u1 / a1^2
  cx<R> t1[4], t2[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) t1[i] = cx<R>{R(0), R(0)};
  slash_acc(R(1), L.eps, u1, t1);
#pragma unroll
  for (int i = 0; i < 4; ++i) t2[i] = cx<R>{R(0), R(0)};
  slash_acc(R(1), a1, t1, t2);
  dirac_current(v2, t2, L.c1);
  // C2 = vbar2 eps-slash a2-slash gamma^mu u1 / a2^2 = bar(a2-slash eps-slash v2) gamma^mu u1 / a2^2
#pragma unroll
  for (int i = 0; i < 4; ++i) t1[i] = cx<R>{R(0), R(0)};
  slash_acc(R(1), L.eps, v2, t1);
#pragma unroll
  for (int i = 0; i < 4; ++i) t2[i] = cx<R>{R(0), R(0)};
  slash_acc(R(1), a2, t1, t2);
  dirac_current(t2, u1, L.c2);
  // E = (J_in.eps)(q + k) + (J_in.(q' - k)) eps - (eps.(q' + q)) J_in
  const cx<R> je = cdotr(L.jin, L.eps), jq = cdotr(L.jin, qpk);
  const R eq = mdot(L.eps, qq2);
#pragma unroll
  for (int m = 0; m < 4; ++m) L.e[m] = qk[m] * je + L.eps[m] * jq - eq * L.jin[m];
  // top helicity 2-spinors (mass independent)
  L.wp3 = sqrt(chis(p[2], L.chi3[0], L.chi3[1]));
  L.wp4 = sqrt(chis(p[3], L.chi4[0], L.chi4[1]));
  L.split = false;
}

// Gauge split of the light-quark current for a gluon of small virtuality s = q^2
// (the crossed channels' t-channel gluon of a forward light quark, |s| << s').
//
// There a3, a4 and a5 each grow like 1/|s| while their colour sum grows like
// 1/sqrt|s|: J_in points along q up to O(sqrt|s|), and the part along q cancels
// between the three (Ward identity), which in FP32 costs a relative error of about
// 2^-24 s'/|s|.  Writing J_in = J' + al q with J'.q' = 0 (q' = p3 + p4, al =
// J_in.q' / q.q'), linearity gives a_i(J_in) = a_i(J') + al a_i(q), and with the
// propagator identities S(P) q-slash = c3 + S(P)(p4-slash + m) (P = p3 + k, q = P +
// p4), ubar3 q-slash S(Q) = ubar3 (p3-slash - m) S(Q) - c4 ubar3 (Q = -p4 - k), with
// c = (P^2 - m^2) / (P^2 - m^2 + i m Gamma) (1 at zero width), and the three-gluon
// vertex contracted with q:
//     s a3(q) =  c3 X + ubar3 eps-slash S(P) d4-slash v4
//     s a4(q) = -c4 X + ubar3 d3-slash S(Q) eps-slash v4
//     s a5(q) =     X - (q'.eps) ubar3 (d3 + d4)-slash v4 / s',     X = ubar3 eps-slash v4,
// where d = p - p~ = (p^2 - m^2) / (2 (E + |p|)) (1, -p-hat) is the difference between
// a top momentum and the on-shell momentum its spinor is built on at mass m (zero at
// the event's own mass).  X (0, 0, 1, -1, 1) is a null vector of the colour matrix
// (its rows 2..4 against (1, -1, 1) sum to 0), so dropping it leaves |M|^2 unchanged:
// the lane evaluates a3..a5 with J' in place of J_in plus al times the d terms and
// X (c - 1), none of which cancels.  J' = J_in - al q itself cancels, so it is formed in FP64
// from the FP64 momenta (once per event, for the events that take the split).
// pd: the event's slot momenta in FP64; e3, e4: p3^2 - m0^2 and p4^2 - m0^2 in FP64.
template <typename R>
__device__ __forceinline__ void qqg_lane_gauge_split(const double (&pd)[5][4], int h12, int neg, R e3, R e4,
                                                     QqgLane<R>& L, QqgSplit<R>& S) {
  const int l1 = h12 ? -1 : 1;
  double k0[4], k1[4], q[4], qp[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    k0[m] = (neg & 1) ? -pd[0][m] : pd[0][m];
    k1[m] = (neg & 2) ? -pd[1][m] : pd[1][m];
    q[m] = pd[0][m] + pd[1][m];
    qp[m] = pd[2][m] + pd[3][m];
  }
  cx<double> u1[4], v2[4], j[4];
  spinor_u(k0, 0.0, l1, u1);
  spinor_v(k1, 0.0, -l1, v2);
  dirac_current(v2, u1, j);
  const cx<double> jq = cdotr(j, qp);
  const double iqq = 1.0 / mdot(q, qp);
  const cx<double> al = cx<double>{jq.re * iqq, jq.im * iqq};
  cx<R> jp[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) jp[m] = cx<R>{R(j[m].re - al.re * q[m]), R(j[m].im - al.im * q[m])};
  // E with J' (the same vertex as qqg_lane_setup)
  R qk[4], qpk[4], qq2[4], r3[4], r4[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    qk[m] = R(q[m] + pd[4][m]);
    qpk[m] = R(qp[m] - pd[4][m]);
    qq2[m] = R(qp[m] + q[m]);
    r3[m] = R(pd[2][m]);
    r4[m] = R(pd[3][m]);
  }
  const cx<R> je = cdotr(jp, L.eps), jqk = cdotr(jp, qpk);
  const R eq = mdot(L.eps, qq2);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    L.jin[m] = jp[m];
    L.e[m] = qk[m] * je + L.eps[m] * jqk - eq * jp[m];
  }
  S.al = cx<R>{R(al.re), R(al.im)};
  R qpr[4] = {R(qp[0]), R(qp[1]), R(qp[2]), R(qp[3])};
  S.qpe = mdot(qpr, L.eps);
  const R a3 = sqrt(r3[1] * r3[1] + r3[2] * r3[2] + r3[3] * r3[3]);
  const R a4 = sqrt(r4[1] * r4[1] + r4[2] * r4[2] + r4[3] * r4[3]);
  S.n3[0] = R(1);
  S.n4[0] = R(1);
#pragma unroll
  for (int m = 1; m < 4; ++m) {
    S.n3[m] = -r3[m] / a3;
    S.n4[m] = -r4[m] / a4;
  }
  S.g3 = R(0.5) / (L.wp3 * L.wp3);
  S.g4 = R(0.5) / (L.wp4 * L.wp4);
  S.h3 = e3 * S.g3;
  S.h4 = e4 * S.g4;
  L.split = true;
}

// The event's invariants into the lane: 1/s, 1/s', the top denominators and the
// light-quark propagator factors of C1, C2.
template <typename R>
__device__ __forceinline__ void qqg_lane_scale(const QqgInvariants<R>& inv, QqgLane<R>& L) {
  L.is = inv.is;
  L.isp = inv.isp;
  L.d3 = inv.d3;
  L.d4 = inv.d4;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    L.c1[m] = inv.ia1 * L.c1[m];
    L.c2[m] = inv.ia2 * L.c2[m];
  }
}

// Re(a^dag C a) for the lane's five amplitudes, C = 3 x the colour matrix
// (double-float has its own form: one sum of products)
template <typename R>
__device__ __forceinline__ R qqg_form(const cx<R> (&a)[5]) {
  R form = R(0);
#pragma unroll
  for (int d = 0; d < 5; ++d) {
    form += R(qqg_colour(d, d)) * (a[d].re * a[d].re + a[d].im * a[d].im);
#pragma unroll
    for (int d2 = d + 1; d2 < 5; ++d2)
      form += R(2 * qqg_colour(d, d2)) * (a[d].re * a[d2].re + a[d].im * a[d2].im);
  }
  return form;
}

// The lane's colour-summed |amplitude|^2 summed over the 4 top-helicity pairs at top
// mass mr, with dm2 = m0^2 - m^2 and mw = m Gamma (g, colour 1/3 and averaging not
// applied).
// The lane's colour-summed |amplitude|^2 summed over the 4 top-helicity pairs at top
// mass mr, with dm2 = m0^2 - m^2 and mw = m Gamma (g, colour 1/3 and averaging not
// applied).
template <typename R>
__device__ __forceinline__ R qqg_slot(const QqgLane<R>& L, R mr, R dm2, R mw) {
  cx<R> u3[2][4], v4[2][4];
  spinor_u_from(L.chi3, L.wp3, mr / L.wp3, u3);
  spinor_v_from(L.chi4, L.wp4, mr / L.wp4, v4);
  // 1 / (d + i m Gamma)
  const R d3 = L.d3 + dm2, d4 = L.d4 + dm2;
  const R n3 = R(1) / (d3 * d3 + mw * mw), n4 = R(1) / (d4 * d4 + mw * mw);
  const cx<R> f3 = L.is * cx<R>{d3 * n3, -mw * n3}, f4 = L.is * cx<R>{d4 * n4, -mw * n4};
  const R f5 = L.is * L.isp;
  R sum = R(0);
  constexpr int UNROLL_HEL = expensive_arith<R>::value ? 1 : 2;   // the helicity loops
#pragma unroll UNROLL_HEL
  for (int l4 = 0; l4 < 2; ++l4) {
    cx<R> t1[4], t2[4], t3[4], s1[4], s2[4], s3[4];
    // eps-slash (a3-slash + m) J_in-slash v4
    cslash(L.jin, v4[l4], t1);
    slash_plus_scalar(L.a3, mr, t1, t2);
#pragma unroll
    for (int i = 0; i < 4; ++i) t3[i] = cx<R>{R(0), R(0)};
    slash_acc(R(1), L.eps, t2, t3);
    // J_in-slash (a4-slash + m) eps-slash v4
#pragma unroll
    for (int i = 0; i < 4; ++i) s1[i] = cx<R>{R(0), R(0)};
    slash_acc(R(1), L.eps, v4[l4], s1);
    slash_plus_scalar(L.a4, mr, s1, s2);
    cslash(L.jin, s2, s3);
#pragma unroll UNROLL_HEL
    for (int l3 = 0; l3 < 2; ++l3) {
      cx<R> jout[4];
      dirac_current(u3[l3], v4[l4], jout);
      cx<R> a[5];
      a[0] = L.isp * cdotm(L.c1, jout);
      a[1] = L.isp * cdotm(L.c2, jout);
      a[2] = f3 * ubar_dot(u3[l3], t3);
      a[3] = f4 * ubar_dot(u3[l3], s3);
      a[4] = f5 * cdotm(L.e, jout);
      sum += qqg_form(a);
    }
  }
  return sum;
}

// qqg_slot for a tile of crossed channels (a light line with a t-channel gluon): L.jin
// and L.e hold J' and E(J'), sp the rest of the lane's gauge split (zeros without one).
template <typename R>
__device__ __forceinline__ R qqg_slot_split(const QqgLane<R>& L, R mr, R dm2, R mw, const QqgSplit<R>* sp) {
  cx<R> u3[2][4], v4[2][4];
  spinor_u_from(L.chi3, L.wp3, mr / L.wp3, u3);
  spinor_v_from(L.chi4, L.wp4, mr / L.wp4, v4);
  // 1 / (d + i m Gamma)
  const R d3 = L.d3 + dm2, d4 = L.d4 + dm2;
  const R n3 = R(1) / (d3 * d3 + mw * mw), n4 = R(1) / (d4 * d4 + mw * mw);
  const cx<R> f3 = L.is * cx<R>{d3 * n3, -mw * n3}, f4 = L.is * cx<R>{d4 * n4, -mw * n4};
  const R f5 = L.is * L.isp;
  // al d3 and al d4 at this mass, d = delta (1, -p-hat)
  const R del3 = sp->h3 + dm2 * sp->g3, del4 = sp->h4 + dm2 * sp->g4;
  R sum = R(0);
  constexpr int UNROLL_HEL = expensive_arith<R>::value ? 1 : 2;   // the helicity loops
#pragma unroll UNROLL_HEL
  for (int l4 = 0; l4 < 2; ++l4) {
    cx<R> t1[4], t2[4], t3[4], s1[4], s2[4], s3[4];
    {  // eps-slash (a3-slash + m) (J' + al d4)-slash v4
      cx<R> j4[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) j4[m] = L.jin[m] + (del4 * sp->n4[m]) * sp->al;
      cslash(j4, v4[l4], t1);
    }
    slash_plus_scalar(L.a3, mr, t1, t2);
#pragma unroll
    for (int i = 0; i < 4; ++i) t3[i] = cx<R>{R(0), R(0)};
    slash_acc(R(1), L.eps, t2, t3);
    // (J' + al d3)-slash (a4-slash + m) eps-slash v4
#pragma unroll
    for (int i = 0; i < 4; ++i) s1[i] = cx<R>{R(0), R(0)};
    slash_acc(R(1), L.eps, v4[l4], s1);
    slash_plus_scalar(L.a4, mr, s1, s2);
    {
      cx<R> j3[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) j3[m] = L.jin[m] + (del3 * sp->n3[m]) * sp->al;
      cslash(j3, s2, s3);
    }
#pragma unroll UNROLL_HEL
    for (int l3 = 0; l3 < 2; ++l3) {
      cx<R> jout[4];
      dirac_current(u3[l3], v4[l4], jout);
      cx<R> a[5];
      a[0] = L.isp * cdotm(L.c1, jout);
      a[1] = L.isp * cdotm(L.c2, jout);
      a[2] = f3 * ubar_dot(u3[l3], t3);
      a[3] = f4 * ubar_dot(u3[l3], s3);
      {  // E(J') - (q'.eps) al (d3 + d4), with ubar3 D-slash v4 = D . J_out
        R dv[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) dv[m] = del3 * sp->n3[m] + del4 * sp->n4[m];
        a[4] = f5 * (cdotm(L.e, jout) - sp->qpe * (sp->al * cdotr(jout, dv)));
      }
      if (mw != R(0)) {
        // a width leaves X (c - 1) of the null part, c = D / (D + i m Gamma):
        // -(i m Gamma al X) f3 in a3 and +(i m Gamma al X) f4 in a4
        const cx<R> ax = sp->al * cdotr(jout, L.eps);
        const cx<R> iwx = cx<R>{-mw * ax.im, mw * ax.re};
        a[2] = a[2] - f3 * iwx;
        a[3] = a[3] + f4 * iwx;
      }
      sum += qqg_form(a);
    }
  }
  return sum;
}

// ---- helicity-exclusive form: the event's own configuration (l1, l2, l3, l4, lg) ----
// The gluon in the helicity basis, eps*(lg) = -(lg e_theta - i e_phi) / sqrt(2), with
// e_theta, e_phi the two linear polarisations of pol_linear; the light-line and
// top-line chains as above with a complex polarisation, and C2's adjoint taken with
// conj(eps) (vbar eps-slash b-slash = bar(b-slash conj(eps)-slash v)).
template <typename R>
struct QqgLaneH {
  cx<R> jin[4], c1[4], c2[4], e[4], eps[4];
  R a3[4], a4[4];
  cx<R> chi3[2][2], chi4[2][2];
  R wp3, wp4;
  R is, isp, d3, d4;
  int i3, i4;      // top spinor index: 1 for helicity +, 0 for -
  bool zero;       // equal light-quark helicities: the configuration vanishes
};

template <typename R>
__device__ __forceinline__ void qqg_lane_setup_h(const R (&p)[5][4], const signed char* hel, QqgLaneH<R>& L) {
  const int l1 = hel[0] > 0 ? 1 : -1, l2 = hel[1] > 0 ? 1 : -1, lg = hel[4] > 0 ? 1 : -1;
  L.i3 = hel[2] > 0 ? 1 : 0;
  L.i4 = hel[3] > 0 ? 1 : 0;
  L.zero = l1 == l2;
  cx<R> u1[4], v2[4];
  spinor_u(p[0], R(0), l1, u1);
  spinor_v(p[1], R(0), l2, v2);
  R e1[4], e2[4];
  pol_linear(p[4], 0, e1);
  pol_linear(p[4], 1, e2);
  const R r = R(0.70710678118654752440);
  cx<R> epsc[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    L.eps[m] = cx<R>{-R(lg) * e1[m] * r, e2[m] * r};
    epsc[m] = cx<R>{L.eps[m].re, -L.eps[m].im};
  }
  dirac_current(v2, u1, L.jin);
  R a1[4], a2[4], qk[4], qpk[4], qq2[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    a1[m] = p[0][m] - p[4][m];
    a2[m] = p[4][m] - p[1][m];
    L.a3[m] = p[2][m] + p[4][m];
    L.a4[m] = -p[3][m] - p[4][m];
    const R q = p[0][m] + p[1][m], qp = p[2][m] + p[3][m];
    qk[m] = q + p[4][m];
    qpk[m] = qp - p[4][m];
    qq2[m] = qp + q;
  }
  cx<R> t1[4], t2[4];
  cslash(L.eps, u1, t1);                       // C1 = vbar2 gamma^mu a1-slash eps-slash u1
#pragma unroll
  for (int i = 0; i < 4; ++i) t2[i] = cx<R>{R(0), R(0)};
  slash_acc(R(1), a1, t1, t2);
  dirac_current(v2, t2, L.c1);
  cslash(epsc, v2, t1);                        // C2 = bar(a2-slash conj(eps)-slash v2) gamma^mu u1
#pragma unroll
  for (int i = 0; i < 4; ++i) t2[i] = cx<R>{R(0), R(0)};
  slash_acc(R(1), a2, t1, t2);
  dirac_current(t2, u1, L.c2);
  const cx<R> je = cdotm(L.jin, L.eps), jq = cdotr(L.jin, qpk), eq = cdotr(L.eps, qq2);
#pragma unroll
  for (int m = 0; m < 4; ++m) L.e[m] = qk[m] * je + L.eps[m] * jq - eq * L.jin[m];
  L.wp3 = sqrt(chis(p[2], L.chi3[0], L.chi3[1]));
  L.wp4 = sqrt(chis(p[3], L.chi4[0], L.chi4[1]));
}

template <typename R>
__device__ __forceinline__ void qqg_lane_scale_h(const QqgInvariants<R>& inv, QqgLaneH<R>& L) {
  L.is = inv.is;
  L.isp = inv.isp;
  L.d3 = inv.d3;
  L.d4 = inv.d4;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    L.c1[m] = inv.ia1 * L.c1[m];
    L.c2[m] = inv.ia2 * L.c2[m];
  }
}

// The colour-summed |amplitude|^2 of the lane's one configuration at top mass mr.
template <typename R>
__device__ __forceinline__ R qqg_slot_h(const QqgLaneH<R>& L, R mr, R dm2, R mw) {
  if (L.zero) return R(0);
  cx<R> u3[2][4], v4[2][4];
  spinor_u_from(L.chi3, L.wp3, mr / L.wp3, u3);
  spinor_v_from(L.chi4, L.wp4, mr / L.wp4, v4);
  const cx<R>* u = u3[L.i3];
  const cx<R>* v = v4[L.i4];
  const R d3 = L.d3 + dm2, d4 = L.d4 + dm2;
  const R n3 = R(1) / (d3 * d3 + mw * mw), n4 = R(1) / (d4 * d4 + mw * mw);
  const cx<R> f3 = L.is * cx<R>{d3 * n3, -mw * n3}, f4 = L.is * cx<R>{d4 * n4, -mw * n4};
  cx<R> t1[4], t2[4], t3[4], s1[4], s2[4], s3[4], jout[4];
  cslash(L.jin, v, t1);                        // eps-slash (a3-slash + m) J_in-slash v4
  slash_plus_scalar(L.a3, mr, t1, t2);
  cslash(L.eps, t2, t3);
  cslash(L.eps, v, s1);                        // J_in-slash (a4-slash + m) eps-slash v4
  slash_plus_scalar(L.a4, mr, s1, s2);
  cslash(L.jin, s2, s3);
  dirac_current(u, v, jout);
  cx<R> a[5];
  a[0] = L.isp * cdotm(L.c1, jout);
  a[1] = L.isp * cdotm(L.c2, jout);
  a[2] = f3 * ubar_dot(u, t3);
  a[3] = f4 * ubar_dot(u, s3);
  a[4] = (L.is * L.isp) * cdotm(L.e, jout);
  R form = R(0);
#pragma unroll
  for (int d = 0; d < 5; ++d) {
    form += R(qqg_colour(d, d)) * (a[d].re * a[d].re + a[d].im * a[d].im);
#pragma unroll
    for (int d2 = d + 1; d2 < 5; ++d2)
      form += R(2 * qqg_colour(d, d2)) * (a[d].re * a[d2].re + a[d].im * a[d2].im);
  }
  return form;
}

}  // namespace rex
