// Colour-ordered Berends-Giele amplitudes for g g -> t t~ + k g (k = 0, 1, 2).
// Generated by paper_2510_05100_b300/codegen/qcd_bg.py (python -m
// paper_2510_05100_b300.codegen); do not edit.
#pragma once
#include "../helas.cuh"

namespace rex {

// ---- gg_ttx: g g -> t t~ + 0 g, 2 gluons, 2 colour flows
// Generated by paper_2510_05100_b300/codegen/qcd_bg.py; do not edit.
struct gg_ttx_info {
  static constexpr int NGLUON = 2;
  static constexpr int NFLOW = 2;
  static constexpr int NGHEL = 4;
  static constexpr int COLOUR_DEN = 3;
};

// exact flow colour matrix C = gg_ttx_colour / 3; flows (top end first):
//   flow 0: (0, 1)
//   flow 1: (1, 0)
constexpr int gg_ttx_colour[2][2] = {
  {16, -2},
  {-2, 16},
};

template <typename R>
struct gg_ttx_gluons {
  R J0[4];
  R J1[4];
  R J01[4];
  R Q0[4];   // -(p_tbar + P)
  R Q1[4];   // -(p_tbar + P)
};

// gluon currents for one gluon polarisation configuration (mass independent)
template <typename R>
__device__ __forceinline__ void gg_ttx_gluon_state(const R (&pg)[2][4], const R (&eps)[2][4], const R (&ptb)[4], gg_ttx_gluons<R>& st) {
  const R* P0 = pg[0];
#pragma unroll
  for (int m = 0; m < 4; ++m) st.J0[m] = eps[0][m];
  const R* P1 = pg[1];
#pragma unroll
  for (int m = 0; m < 4; ++m) st.J1[m] = eps[1][m];
  R P01[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) P01[m] = pg[0][m] + pg[1][m];
  {  // J(0,1)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J0, P0, st.J1, P1, t);
    const R f = R(-1) / mdot(P01, P01);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J01[m] = f * t[m];
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) st.Q0[m] = -(ptb[m] + pg[0][m]);
#pragma unroll
  for (int m = 0; m < 4; ++m) st.Q1[m] = -(ptb[m] + pg[1][m]);
}

// sum over top and antitop helicities of sum_{s,s'} conj(A_s) Cint_{ss'} A_s'
// for one (mass, width); Cint = C * COLOUR_DEN.  WIDTH selects complex denominators.
// The quadratic form of one helicity is evaluated in CS (a positive-definite form:
// no cancellation), and the helicity sum is accumulated in ACC.
template <typename R, typename ACC, bool WIDTH, typename CS = ACC>
__device__ __forceinline__ ACC gg_ttx_quark_line(const gg_ttx_gluons<R>& st, const R (&pt)[4], const R (&ptb)[4], R mt, R wt) {
  ACC total = ACC(0);
  const R d0 = mdot(st.Q0, st.Q0) - mt * mt;
  R id0r, id0i;
  if (WIDTH) { const R im = mt * wt; const R nn = R(1) / (d0 * d0 + im * im); id0r = d0 * nn; id0i = -im * nn; } else { id0r = R(1) / d0; id0i = R(0); }
  const R d1 = mdot(st.Q1, st.Q1) - mt * mt;
  R id1r, id1i;
  if (WIDTH) { const R im = mt * wt; const R nn = R(1) / (d1 * d1 + im * im); id1r = d1 * nn; id1i = -im * nn; } else { id1r = R(1) / d1; id1i = R(0); }
  cx<R> ut[2][4];
  spinor_u(pt, mt, -1, ut[0]);
  spinor_u(pt, mt, +1, ut[1]);
#pragma unroll 1
  for (int hb = 0; hb < 2; ++hb) {
    cx<R> v[4];
    spinor_v(ptb, mt, hb == 0 ? -1 : +1, v);
    cx<R> psi0[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J0, v, t);
      if (WIDTH) fermion_prop(st.Q0, mt, cx<R>{id0r, id0i}, t, psi0);
      else fermion_prop_real(st.Q0, mt, id0r, t, psi0);
    }
    cx<R> psi1[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J1, v, t);
      if (WIDTH) fermion_prop(st.Q1, mt, cx<R>{id1r, id1i}, t, psi1);
      else fermion_prop_real(st.Q1, mt, id1r, t, psi1);
    }
    cx<R> A[2][2];
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J0, psi1, x);
      slash_acc(R(1), st.J01, v, x);
      A[0][0] = ubar_dot(ut[0], x);
      A[1][0] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J1, psi0, x);
      slash_acc(R(-1), st.J01, v, x);
      A[0][1] = ubar_dot(ut[0], x);
      A[1][1] = ubar_dot(ut[1], x);
    }
#pragma unroll
    for (int ht = 0; ht < 2; ++ht) {
      CS s = CS(0);
      s += CS(16) * (CS(A[ht][0].re) * CS(A[ht][0].re) + CS(A[ht][0].im) * CS(A[ht][0].im));
      s += CS(16) * (CS(A[ht][1].re) * CS(A[ht][1].re) + CS(A[ht][1].im) * CS(A[ht][1].im));
      s += CS(-4) * (CS(A[ht][0].re) * CS(A[ht][1].re) + CS(A[ht][0].im) * CS(A[ht][1].im));
      total += ACC(s);
    }
  }
  return total;
}

// ---- gg_ttxg: g g -> t t~ + 1 g, 3 gluons, 6 colour flows
// Generated by paper_2510_05100_b300/codegen/qcd_bg.py; do not edit.
struct gg_ttxg_info {
  static constexpr int NGLUON = 3;
  static constexpr int NFLOW = 6;
  static constexpr int NGHEL = 8;
  static constexpr int COLOUR_DEN = 9;
};

// exact flow colour matrix C = gg_ttxg_colour / 9; flows (top end first):
//   flow 0: (0, 1, 2)
//   flow 1: (0, 2, 1)
//   flow 2: (1, 0, 2)
//   flow 3: (1, 2, 0)
//   flow 4: (2, 0, 1)
//   flow 5: (2, 1, 0)
constexpr int gg_ttxg_colour[6][6] = {
  {64, -8, -8, 1, 1, 10},
  {-8, 64, 1, 10, -8, 1},
  {-8, 1, 64, -8, 10, 1},
  {1, 10, -8, 64, 1, -8},
  {1, -8, 10, 1, 64, -8},
  {10, 1, 1, -8, -8, 64},
};

template <typename R>
struct gg_ttxg_gluons {
  R J0[4];
  R J1[4];
  R J2[4];
  R J01[4];
  R J02[4];
  R J12[4];
  R J012[4];
  R J021[4];
  R J102[4];
  R Q0[4];   // -(p_tbar + P)
  R Q1[4];   // -(p_tbar + P)
  R Q2[4];   // -(p_tbar + P)
  R Q01[4];   // -(p_tbar + P)
  R Q02[4];   // -(p_tbar + P)
  R Q12[4];   // -(p_tbar + P)
};

// gluon currents for one gluon polarisation configuration (mass independent)
template <typename R>
__device__ __forceinline__ void gg_ttxg_gluon_state(const R (&pg)[3][4], const R (&eps)[3][4], const R (&ptb)[4], gg_ttxg_gluons<R>& st) {
  const R* P0 = pg[0];
#pragma unroll
  for (int m = 0; m < 4; ++m) st.J0[m] = eps[0][m];
  const R* P1 = pg[1];
#pragma unroll
  for (int m = 0; m < 4; ++m) st.J1[m] = eps[1][m];
  const R* P2 = pg[2];
#pragma unroll
  for (int m = 0; m < 4; ++m) st.J2[m] = eps[2][m];
  R P01[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) P01[m] = pg[0][m] + pg[1][m];
  R P02[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) P02[m] = pg[0][m] + pg[2][m];
  R P12[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) P12[m] = pg[1][m] + pg[2][m];
  R P012[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) P012[m] = pg[0][m] + pg[1][m] + pg[2][m];
  {  // J(0,1)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J0, P0, st.J1, P1, t);
    const R f = R(-1) / mdot(P01, P01);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J01[m] = f * t[m];
  }
  {  // J(0,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J0, P0, st.J2, P2, t);
    const R f = R(-1) / mdot(P02, P02);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J02[m] = f * t[m];
  }
  {  // J(1,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J1, P1, st.J2, P2, t);
    const R f = R(-1) / mdot(P12, P12);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J12[m] = f * t[m];
  }
  {  // J(0,1,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J0, P0, st.J12, P12, t);
    vvv_acc(R(1), st.J01, P01, st.J2, P2, t);
    vvvv_acc(R(1), st.J0, st.J1, st.J2, t);
    const R f = R(-1) / mdot(P012, P012);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J012[m] = f * t[m];
  }
  {  // J(0,2,1)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(-1), st.J0, P0, st.J12, P12, t);
    vvv_acc(R(1), st.J02, P02, st.J1, P1, t);
    vvvv_acc(R(1), st.J0, st.J2, st.J1, t);
    const R f = R(-1) / mdot(P012, P012);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J021[m] = f * t[m];
  }
  {  // J(1,0,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J1, P1, st.J02, P02, t);
    vvv_acc(R(-1), st.J01, P01, st.J2, P2, t);
    vvvv_acc(R(1), st.J1, st.J0, st.J2, t);
    const R f = R(-1) / mdot(P012, P012);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J102[m] = f * t[m];
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) st.Q0[m] = -(ptb[m] + pg[0][m]);
#pragma unroll
  for (int m = 0; m < 4; ++m) st.Q1[m] = -(ptb[m] + pg[1][m]);
#pragma unroll
  for (int m = 0; m < 4; ++m) st.Q2[m] = -(ptb[m] + pg[2][m]);
#pragma unroll
  for (int m = 0; m < 4; ++m) st.Q01[m] = -(ptb[m] + pg[0][m] + pg[1][m]);
#pragma unroll
  for (int m = 0; m < 4; ++m) st.Q02[m] = -(ptb[m] + pg[0][m] + pg[2][m]);
#pragma unroll
  for (int m = 0; m < 4; ++m) st.Q12[m] = -(ptb[m] + pg[1][m] + pg[2][m]);
}

// sum over top and antitop helicities of sum_{s,s'} conj(A_s) Cint_{ss'} A_s'
// for one (mass, width); Cint = C * COLOUR_DEN.  WIDTH selects complex denominators.
// The quadratic form of one helicity is evaluated in CS (a positive-definite form:
// no cancellation), and the helicity sum is accumulated in ACC.
template <typename R, typename ACC, bool WIDTH, typename CS = ACC>
__device__ __forceinline__ ACC gg_ttxg_quark_line(const gg_ttxg_gluons<R>& st, const R (&pt)[4], const R (&ptb)[4], R mt, R wt) {
  ACC total = ACC(0);
  const R d0 = mdot(st.Q0, st.Q0) - mt * mt;
  R id0r, id0i;
  if (WIDTH) { const R im = mt * wt; const R nn = R(1) / (d0 * d0 + im * im); id0r = d0 * nn; id0i = -im * nn; } else { id0r = R(1) / d0; id0i = R(0); }
  const R d1 = mdot(st.Q1, st.Q1) - mt * mt;
  R id1r, id1i;
  if (WIDTH) { const R im = mt * wt; const R nn = R(1) / (d1 * d1 + im * im); id1r = d1 * nn; id1i = -im * nn; } else { id1r = R(1) / d1; id1i = R(0); }
  const R d2 = mdot(st.Q2, st.Q2) - mt * mt;
  R id2r, id2i;
  if (WIDTH) { const R im = mt * wt; const R nn = R(1) / (d2 * d2 + im * im); id2r = d2 * nn; id2i = -im * nn; } else { id2r = R(1) / d2; id2i = R(0); }
  const R d01 = mdot(st.Q01, st.Q01) - mt * mt;
  R id01r, id01i;
  if (WIDTH) { const R im = mt * wt; const R nn = R(1) / (d01 * d01 + im * im); id01r = d01 * nn; id01i = -im * nn; } else { id01r = R(1) / d01; id01i = R(0); }
  const R d02 = mdot(st.Q02, st.Q02) - mt * mt;
  R id02r, id02i;
  if (WIDTH) { const R im = mt * wt; const R nn = R(1) / (d02 * d02 + im * im); id02r = d02 * nn; id02i = -im * nn; } else { id02r = R(1) / d02; id02i = R(0); }
  const R d12 = mdot(st.Q12, st.Q12) - mt * mt;
  R id12r, id12i;
  if (WIDTH) { const R im = mt * wt; const R nn = R(1) / (d12 * d12 + im * im); id12r = d12 * nn; id12i = -im * nn; } else { id12r = R(1) / d12; id12i = R(0); }
  cx<R> ut[2][4];
  spinor_u(pt, mt, -1, ut[0]);
  spinor_u(pt, mt, +1, ut[1]);
#pragma unroll 1
  for (int hb = 0; hb < 2; ++hb) {
    cx<R> v[4];
    spinor_v(ptb, mt, hb == 0 ? -1 : +1, v);
    cx<R> psi0[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J0, v, t);
      if (WIDTH) fermion_prop(st.Q0, mt, cx<R>{id0r, id0i}, t, psi0);
      else fermion_prop_real(st.Q0, mt, id0r, t, psi0);
    }
    cx<R> psi1[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J1, v, t);
      if (WIDTH) fermion_prop(st.Q1, mt, cx<R>{id1r, id1i}, t, psi1);
      else fermion_prop_real(st.Q1, mt, id1r, t, psi1);
    }
    cx<R> psi2[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J2, v, t);
      if (WIDTH) fermion_prop(st.Q2, mt, cx<R>{id2r, id2i}, t, psi2);
      else fermion_prop_real(st.Q2, mt, id2r, t, psi2);
    }
    cx<R> psi01[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J0, psi1, t);
      slash_acc(R(1), st.J01, v, t);
      if (WIDTH) fermion_prop(st.Q01, mt, cx<R>{id01r, id01i}, t, psi01);
      else fermion_prop_real(st.Q01, mt, id01r, t, psi01);
    }
    cx<R> psi02[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J0, psi2, t);
      slash_acc(R(1), st.J02, v, t);
      if (WIDTH) fermion_prop(st.Q02, mt, cx<R>{id02r, id02i}, t, psi02);
      else fermion_prop_real(st.Q02, mt, id02r, t, psi02);
    }
    cx<R> psi10[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J1, psi0, t);
      slash_acc(R(-1), st.J01, v, t);
      if (WIDTH) fermion_prop(st.Q01, mt, cx<R>{id01r, id01i}, t, psi10);
      else fermion_prop_real(st.Q01, mt, id01r, t, psi10);
    }
    cx<R> psi12[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J1, psi2, t);
      slash_acc(R(1), st.J12, v, t);
      if (WIDTH) fermion_prop(st.Q12, mt, cx<R>{id12r, id12i}, t, psi12);
      else fermion_prop_real(st.Q12, mt, id12r, t, psi12);
    }
    cx<R> psi20[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J2, psi0, t);
      slash_acc(R(-1), st.J02, v, t);
      if (WIDTH) fermion_prop(st.Q02, mt, cx<R>{id02r, id02i}, t, psi20);
      else fermion_prop_real(st.Q02, mt, id02r, t, psi20);
    }
    cx<R> psi21[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J2, psi1, t);
      slash_acc(R(-1), st.J12, v, t);
      if (WIDTH) fermion_prop(st.Q12, mt, cx<R>{id12r, id12i}, t, psi21);
      else fermion_prop_real(st.Q12, mt, id12r, t, psi21);
    }
    cx<R> A[2][6];
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J0, psi12, x);
      slash_acc(R(1), st.J01, psi2, x);
      slash_acc(R(1), st.J012, v, x);
      A[0][0] = ubar_dot(ut[0], x);
      A[1][0] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J0, psi21, x);
      slash_acc(R(1), st.J02, psi1, x);
      slash_acc(R(1), st.J021, v, x);
      A[0][1] = ubar_dot(ut[0], x);
      A[1][1] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J1, psi02, x);
      slash_acc(R(-1), st.J01, psi2, x);
      slash_acc(R(1), st.J102, v, x);
      A[0][2] = ubar_dot(ut[0], x);
      A[1][2] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J1, psi20, x);
      slash_acc(R(1), st.J12, psi0, x);
      slash_acc(R(1), st.J021, v, x);
      A[0][3] = ubar_dot(ut[0], x);
      A[1][3] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J2, psi01, x);
      slash_acc(R(-1), st.J02, psi1, x);
      slash_acc(R(1), st.J102, v, x);
      A[0][4] = ubar_dot(ut[0], x);
      A[1][4] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J2, psi10, x);
      slash_acc(R(-1), st.J12, psi0, x);
      slash_acc(R(1), st.J012, v, x);
      A[0][5] = ubar_dot(ut[0], x);
      A[1][5] = ubar_dot(ut[1], x);
    }
#pragma unroll
    for (int ht = 0; ht < 2; ++ht) {
      CS s = CS(0);
      s += CS(64) * (CS(A[ht][0].re) * CS(A[ht][0].re) + CS(A[ht][0].im) * CS(A[ht][0].im));
      s += CS(64) * (CS(A[ht][1].re) * CS(A[ht][1].re) + CS(A[ht][1].im) * CS(A[ht][1].im));
      s += CS(64) * (CS(A[ht][2].re) * CS(A[ht][2].re) + CS(A[ht][2].im) * CS(A[ht][2].im));
      s += CS(64) * (CS(A[ht][3].re) * CS(A[ht][3].re) + CS(A[ht][3].im) * CS(A[ht][3].im));
      s += CS(64) * (CS(A[ht][4].re) * CS(A[ht][4].re) + CS(A[ht][4].im) * CS(A[ht][4].im));
      s += CS(64) * (CS(A[ht][5].re) * CS(A[ht][5].re) + CS(A[ht][5].im) * CS(A[ht][5].im));
      s += CS(-16) * (CS(A[ht][0].re) * CS(A[ht][1].re) + CS(A[ht][0].im) * CS(A[ht][1].im));
      s += CS(-16) * (CS(A[ht][0].re) * CS(A[ht][2].re) + CS(A[ht][0].im) * CS(A[ht][2].im));
      s += CS(2) * (CS(A[ht][0].re) * CS(A[ht][3].re) + CS(A[ht][0].im) * CS(A[ht][3].im));
      s += CS(2) * (CS(A[ht][0].re) * CS(A[ht][4].re) + CS(A[ht][0].im) * CS(A[ht][4].im));
      s += CS(20) * (CS(A[ht][0].re) * CS(A[ht][5].re) + CS(A[ht][0].im) * CS(A[ht][5].im));
      s += CS(2) * (CS(A[ht][1].re) * CS(A[ht][2].re) + CS(A[ht][1].im) * CS(A[ht][2].im));
      s += CS(20) * (CS(A[ht][1].re) * CS(A[ht][3].re) + CS(A[ht][1].im) * CS(A[ht][3].im));
      s += CS(-16) * (CS(A[ht][1].re) * CS(A[ht][4].re) + CS(A[ht][1].im) * CS(A[ht][4].im));
      s += CS(2) * (CS(A[ht][1].re) * CS(A[ht][5].re) + CS(A[ht][1].im) * CS(A[ht][5].im));
      s += CS(-16) * (CS(A[ht][2].re) * CS(A[ht][3].re) + CS(A[ht][2].im) * CS(A[ht][3].im));
      s += CS(20) * (CS(A[ht][2].re) * CS(A[ht][4].re) + CS(A[ht][2].im) * CS(A[ht][4].im));
      s += CS(2) * (CS(A[ht][2].re) * CS(A[ht][5].re) + CS(A[ht][2].im) * CS(A[ht][5].im));
      s += CS(2) * (CS(A[ht][3].re) * CS(A[ht][4].re) + CS(A[ht][3].im) * CS(A[ht][4].im));
      s += CS(-16) * (CS(A[ht][3].re) * CS(A[ht][5].re) + CS(A[ht][3].im) * CS(A[ht][5].im));
      s += CS(-16) * (CS(A[ht][4].re) * CS(A[ht][5].re) + CS(A[ht][4].im) * CS(A[ht][5].im));
      total += ACC(s);
    }
  }
  return total;
}

// ---- gg_ttxgg: g g -> t t~ + 2 g, 4 gluons, 24 colour flows
// Generated by paper_2510_05100_b300/codegen/qcd_bg.py; do not edit.
struct gg_ttxgg_info {
  static constexpr int NGLUON = 4;
  static constexpr int NFLOW = 24;
  static constexpr int NGHEL = 16;
  static constexpr int COLOUR_DEN = 54;
};

// exact flow colour matrix C = gg_ttxgg_colour / 54; flows (top end first):
//   flow 0: (0, 1, 2, 3)
//   flow 1: (0, 1, 3, 2)
//   flow 2: (0, 2, 1, 3)
//   flow 3: (0, 2, 3, 1)
//   flow 4: (0, 3, 1, 2)
//   flow 5: (0, 3, 2, 1)
//   flow 6: (1, 0, 2, 3)
//   flow 7: (1, 0, 3, 2)
//   flow 8: (1, 2, 0, 3)
//   flow 9: (1, 2, 3, 0)
//   flow 10: (1, 3, 0, 2)
//   flow 11: (1, 3, 2, 0)
//   flow 12: (2, 0, 1, 3)
//   flow 13: (2, 0, 3, 1)
//   flow 14: (2, 1, 0, 3)
//   flow 15: (2, 1, 3, 0)
//   flow 16: (2, 3, 0, 1)
//   flow 17: (2, 3, 1, 0)
//   flow 18: (3, 0, 1, 2)
//   flow 19: (3, 0, 2, 1)
//   flow 20: (3, 1, 0, 2)
//   flow 21: (3, 1, 2, 0)
//   flow 22: (3, 2, 0, 1)
//   flow 23: (3, 2, 1, 0)
constexpr int gg_ttxgg_colour[24][24] = {
  {512, -64, -64, 8, 8, 80, -64, 8, 8, -1, -1, -10, 8, -1, 80, -10, 71, 62, -1, -10, -10, 62, 62, -28},
  {-64, 512, 8, 80, -64, 8, 8, -64, -1, -10, 8, -1, -1, -10, -10, 62, 62, -28, 8, -1, 80, -10, 71, 62},
  {-64, 8, 512, -64, 80, 8, 8, -1, 80, -10, 71, 62, -64, 8, 8, -1, -1, -10, -10, -1, 62, -28, -10, 62},
  {8, 80, -64, 512, 8, -64, -1, -10, -10, 62, 62, -28, 8, -64, -1, -10, 8, -1, -1, 8, 71, 62, 80, -10},
  {8, -64, 80, 8, 512, -64, -1, 8, 71, 62, 80, -10, -10, -1, 62, -28, -10, 62, -64, 8, 8, -1, -1, -10},
  {80, 8, 8, -64, -64, 512, -10, -1, 62, -28, -10, 62, -1, 8, 71, 62, 80, -10, 8, -64, -1, -10, 8, -1},
  {-64, 8, 8, -1, -1, -10, 512, -64, -64, 8, 8, 80, 80, -10, 8, -1, 62, 71, -10, 62, -1, -10, -28, 62},
  {8, -64, -1, -10, 8, -1, -64, 512, 8, 80, -64, 8, -10, 62, -1, -10, -28, 62, 80, -10, 8, -1, 62, 71},
  {8, -1, 80, -10, 71, 62, -64, 8, 512, -64, 80, 8, 8, -1, -64, 8, -10, -1, 62, -28, -10, -1, 62, -10},
  {-1, -10, -10, 62, 62, -28, 8, 80, -64, 512, 8, -64, -1, -10, 8, -64, -1, 8, 71, 62, -1, 8, -10, 80},
  {-1, 8, 71, 62, 80, -10, 8, -64, 80, 8, 512, -64, 62, -28, -10, -1, 62, -10, 8, -1, -64, 8, -10, -1},
  {-10, -1, 62, -28, -10, 62, 80, 8, 8, -64, -64, 512, 71, 62, -1, 8, -10, 80, -1, -10, 8, -64, -1, 8},
  {8, -1, -64, 8, -10, -1, 80, -10, 8, -1, 62, 71, 512, -64, -64, 8, 8, 80, 62, -10, -28, 62, -1, -10},
  {-1, -10, 8, -64, -1, 8, -10, 62, -1, -10, -28, 62, -64, 512, 8, 80, -64, 8, -10, 80, 62, 71, 8, -1},
  {80, -10, 8, -1, 62, 71, 8, -1, -64, 8, -10, -1, -64, 8, 512, -64, 80, 8, -28, 62, 62, -10, -10, -1},
  {-10, 62, -1, -10, -28, 62, -1, -10, 8, -64, -1, 8, 8, 80, -64, 512, 8, -64, 62, 71, -10, 80, -1, 8},
  {71, 62, -1, 8, -10, 80, 62, -28, -10, -1, 62, -10, 8, -64, 80, 8, 512, -64, -1, 8, -10, -1, -64, 8},
  {62, -28, -10, -1, 62, -10, 71, 62, -1, 8, -10, 80, 80, 8, 8, -64, -64, 512, -10, -1, -1, 8, 8, -64},
  {-1, 8, -10, -1, -64, 8, -10, 80, 62, 71, 8, -1, 62, -10, -28, 62, -1, -10, 512, -64, -64, 8, 8, 80},
  {-10, -1, -1, 8, 8, -64, 62, -10, -28, 62, -1, -10, -10, 80, 62, 71, 8, -1, -64, 512, 8, 80, -64, 8},
  {-10, 80, 62, 71, 8, -1, -1, 8, -10, -1, -64, 8, -28, 62, 62, -10, -10, -1, -64, 8, 512, -64, 80, 8},
  {62, -10, -28, 62, -1, -10, -10, -1, -1, 8, 8, -64, 62, 71, -10, 80, -1, 8, 8, 80, -64, 512, 8, -64},
  {62, 71, -10, 80, -1, 8, -28, 62, 62, -10, -10, -1, -1, 8, -10, -1, -64, 8, 8, -64, 80, 8, 512, -64},
  {-28, 62, 62, -10, -10, -1, 62, 71, -10, 80, -1, 8, -10, -1, -1, 8, 8, -64, 80, 8, 8, -64, -64, 512},
};

template <typename R>
struct gg_ttxgg_gluons {
  R J0[4];
  R J1[4];
  R J2[4];
  R J3[4];
  R J01[4];
  R J02[4];
  R J03[4];
  R J12[4];
  R J13[4];
  R J23[4];
  R J012[4];
  R J013[4];
  R J021[4];
  R J023[4];
  R J031[4];
  R J032[4];
  R J102[4];
  R J103[4];
  R J123[4];
  R J132[4];
  R J203[4];
  R J213[4];
  R J0123[4];
  R J0132[4];
  R J0213[4];
  R J0231[4];
  R J0312[4];
  R J0321[4];
  R J1023[4];
  R J1032[4];
  R J1203[4];
  R J1302[4];
  R J2013[4];
  R J2103[4];
  R Q0[4];   // -(p_tbar + P)
  R Q1[4];   // -(p_tbar + P)
  R Q2[4];   // -(p_tbar + P)
  R Q3[4];   // -(p_tbar + P)
  R Q01[4];   // -(p_tbar + P)
  R Q02[4];   // -(p_tbar + P)
  R Q03[4];   // -(p_tbar + P)
  R Q12[4];   // -(p_tbar + P)
  R Q13[4];   // -(p_tbar + P)
  R Q23[4];   // -(p_tbar + P)
  R Q012[4];   // -(p_tbar + P)
  R Q013[4];   // -(p_tbar + P)
  R Q023[4];   // -(p_tbar + P)
  R Q123[4];   // -(p_tbar + P)
};

// gluon currents for one gluon polarisation configuration (mass independent)
template <typename R>
__device__ __forceinline__ void gg_ttxgg_gluon_state(const R (&pg)[4][4], const R (&eps)[4][4], const R (&ptb)[4], gg_ttxgg_gluons<R>& st) {
  const R* P0 = pg[0];
#pragma unroll
  for (int m = 0; m < 4; ++m) st.J0[m] = eps[0][m];
  const R* P1 = pg[1];
#pragma unroll
  for (int m = 0; m < 4; ++m) st.J1[m] = eps[1][m];
  const R* P2 = pg[2];
#pragma unroll
  for (int m = 0; m < 4; ++m) st.J2[m] = eps[2][m];
  const R* P3 = pg[3];
#pragma unroll
  for (int m = 0; m < 4; ++m) st.J3[m] = eps[3][m];
  R P01[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) P01[m] = pg[0][m] + pg[1][m];
  R P02[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) P02[m] = pg[0][m] + pg[2][m];
  R P03[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) P03[m] = pg[0][m] + pg[3][m];
  R P12[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) P12[m] = pg[1][m] + pg[2][m];
  R P13[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) P13[m] = pg[1][m] + pg[3][m];
  R P23[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) P23[m] = pg[2][m] + pg[3][m];
  R P012[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) P012[m] = pg[0][m] + pg[1][m] + pg[2][m];
  R P013[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) P013[m] = pg[0][m] + pg[1][m] + pg[3][m];
  R P023[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) P023[m] = pg[0][m] + pg[2][m] + pg[3][m];
  R P123[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) P123[m] = pg[1][m] + pg[2][m] + pg[3][m];
  R P0123[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) P0123[m] = pg[0][m] + pg[1][m] + pg[2][m] + pg[3][m];
  {  // J(0,1)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J0, P0, st.J1, P1, t);
    const R f = R(-1) / mdot(P01, P01);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J01[m] = f * t[m];
  }
  {  // J(0,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J0, P0, st.J2, P2, t);
    const R f = R(-1) / mdot(P02, P02);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J02[m] = f * t[m];
  }
  {  // J(0,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J0, P0, st.J3, P3, t);
    const R f = R(-1) / mdot(P03, P03);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J03[m] = f * t[m];
  }
  {  // J(1,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J1, P1, st.J2, P2, t);
    const R f = R(-1) / mdot(P12, P12);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J12[m] = f * t[m];
  }
  {  // J(1,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J1, P1, st.J3, P3, t);
    const R f = R(-1) / mdot(P13, P13);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J13[m] = f * t[m];
  }
  {  // J(2,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J2, P2, st.J3, P3, t);
    const R f = R(-1) / mdot(P23, P23);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J23[m] = f * t[m];
  }
  {  // J(0,1,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J0, P0, st.J12, P12, t);
    vvv_acc(R(1), st.J01, P01, st.J2, P2, t);
    vvvv_acc(R(1), st.J0, st.J1, st.J2, t);
    const R f = R(-1) / mdot(P012, P012);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J012[m] = f * t[m];
  }
  {  // J(0,1,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J0, P0, st.J13, P13, t);
    vvv_acc(R(1), st.J01, P01, st.J3, P3, t);
    vvvv_acc(R(1), st.J0, st.J1, st.J3, t);
    const R f = R(-1) / mdot(P013, P013);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J013[m] = f * t[m];
  }
  {  // J(0,2,1)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(-1), st.J0, P0, st.J12, P12, t);
    vvv_acc(R(1), st.J02, P02, st.J1, P1, t);
    vvvv_acc(R(1), st.J0, st.J2, st.J1, t);
    const R f = R(-1) / mdot(P012, P012);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J021[m] = f * t[m];
  }
  {  // J(0,2,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J0, P0, st.J23, P23, t);
    vvv_acc(R(1), st.J02, P02, st.J3, P3, t);
    vvvv_acc(R(1), st.J0, st.J2, st.J3, t);
    const R f = R(-1) / mdot(P023, P023);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J023[m] = f * t[m];
  }
  {  // J(0,3,1)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(-1), st.J0, P0, st.J13, P13, t);
    vvv_acc(R(1), st.J03, P03, st.J1, P1, t);
    vvvv_acc(R(1), st.J0, st.J3, st.J1, t);
    const R f = R(-1) / mdot(P013, P013);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J031[m] = f * t[m];
  }
  {  // J(0,3,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(-1), st.J0, P0, st.J23, P23, t);
    vvv_acc(R(1), st.J03, P03, st.J2, P2, t);
    vvvv_acc(R(1), st.J0, st.J3, st.J2, t);
    const R f = R(-1) / mdot(P023, P023);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J032[m] = f * t[m];
  }
  {  // J(1,0,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J1, P1, st.J02, P02, t);
    vvv_acc(R(-1), st.J01, P01, st.J2, P2, t);
    vvvv_acc(R(1), st.J1, st.J0, st.J2, t);
    const R f = R(-1) / mdot(P012, P012);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J102[m] = f * t[m];
  }
  {  // J(1,0,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J1, P1, st.J03, P03, t);
    vvv_acc(R(-1), st.J01, P01, st.J3, P3, t);
    vvvv_acc(R(1), st.J1, st.J0, st.J3, t);
    const R f = R(-1) / mdot(P013, P013);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J103[m] = f * t[m];
  }
  {  // J(1,2,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J1, P1, st.J23, P23, t);
    vvv_acc(R(1), st.J12, P12, st.J3, P3, t);
    vvvv_acc(R(1), st.J1, st.J2, st.J3, t);
    const R f = R(-1) / mdot(P123, P123);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J123[m] = f * t[m];
  }
  {  // J(1,3,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(-1), st.J1, P1, st.J23, P23, t);
    vvv_acc(R(1), st.J13, P13, st.J2, P2, t);
    vvvv_acc(R(1), st.J1, st.J3, st.J2, t);
    const R f = R(-1) / mdot(P123, P123);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J132[m] = f * t[m];
  }
  {  // J(2,0,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J2, P2, st.J03, P03, t);
    vvv_acc(R(-1), st.J02, P02, st.J3, P3, t);
    vvvv_acc(R(1), st.J2, st.J0, st.J3, t);
    const R f = R(-1) / mdot(P023, P023);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J203[m] = f * t[m];
  }
  {  // J(2,1,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J2, P2, st.J13, P13, t);
    vvv_acc(R(-1), st.J12, P12, st.J3, P3, t);
    vvvv_acc(R(1), st.J2, st.J1, st.J3, t);
    const R f = R(-1) / mdot(P123, P123);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J213[m] = f * t[m];
  }
  {  // J(0,1,2,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J0, P0, st.J123, P123, t);
    vvv_acc(R(1), st.J01, P01, st.J23, P23, t);
    vvv_acc(R(1), st.J012, P012, st.J3, P3, t);
    vvvv_acc(R(1), st.J0, st.J1, st.J23, t);
    vvvv_acc(R(1), st.J0, st.J12, st.J3, t);
    vvvv_acc(R(1), st.J01, st.J2, st.J3, t);
    const R f = R(-1) / mdot(P0123, P0123);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J0123[m] = f * t[m];
  }
  {  // J(0,1,3,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J0, P0, st.J132, P123, t);
    vvv_acc(R(-1), st.J01, P01, st.J23, P23, t);
    vvv_acc(R(1), st.J013, P013, st.J2, P2, t);
    vvvv_acc(R(-1), st.J0, st.J1, st.J23, t);
    vvvv_acc(R(1), st.J0, st.J13, st.J2, t);
    vvvv_acc(R(1), st.J01, st.J3, st.J2, t);
    const R f = R(-1) / mdot(P0123, P0123);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J0132[m] = f * t[m];
  }
  {  // J(0,2,1,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J0, P0, st.J213, P123, t);
    vvv_acc(R(1), st.J02, P02, st.J13, P13, t);
    vvv_acc(R(1), st.J021, P012, st.J3, P3, t);
    vvvv_acc(R(1), st.J0, st.J2, st.J13, t);
    vvvv_acc(R(-1), st.J0, st.J12, st.J3, t);
    vvvv_acc(R(1), st.J02, st.J1, st.J3, t);
    const R f = R(-1) / mdot(P0123, P0123);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J0213[m] = f * t[m];
  }
  {  // J(0,2,3,1)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J0, P0, st.J132, P123, t);
    vvv_acc(R(-1), st.J02, P02, st.J13, P13, t);
    vvv_acc(R(1), st.J023, P023, st.J1, P1, t);
    vvvv_acc(R(-1), st.J0, st.J2, st.J13, t);
    vvvv_acc(R(1), st.J0, st.J23, st.J1, t);
    vvvv_acc(R(1), st.J02, st.J3, st.J1, t);
    const R f = R(-1) / mdot(P0123, P0123);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J0231[m] = f * t[m];
  }
  {  // J(0,3,1,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J0, P0, st.J213, P123, t);
    vvv_acc(R(1), st.J03, P03, st.J12, P12, t);
    vvv_acc(R(1), st.J031, P013, st.J2, P2, t);
    vvvv_acc(R(1), st.J0, st.J3, st.J12, t);
    vvvv_acc(R(-1), st.J0, st.J13, st.J2, t);
    vvvv_acc(R(1), st.J03, st.J1, st.J2, t);
    const R f = R(-1) / mdot(P0123, P0123);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J0312[m] = f * t[m];
  }
  {  // J(0,3,2,1)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J0, P0, st.J123, P123, t);
    vvv_acc(R(-1), st.J03, P03, st.J12, P12, t);
    vvv_acc(R(1), st.J032, P023, st.J1, P1, t);
    vvvv_acc(R(-1), st.J0, st.J3, st.J12, t);
    vvvv_acc(R(-1), st.J0, st.J23, st.J1, t);
    vvvv_acc(R(1), st.J03, st.J2, st.J1, t);
    const R f = R(-1) / mdot(P0123, P0123);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J0321[m] = f * t[m];
  }
  {  // J(1,0,2,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J1, P1, st.J023, P023, t);
    vvv_acc(R(-1), st.J01, P01, st.J23, P23, t);
    vvv_acc(R(1), st.J102, P012, st.J3, P3, t);
    vvvv_acc(R(1), st.J1, st.J0, st.J23, t);
    vvvv_acc(R(1), st.J1, st.J02, st.J3, t);
    vvvv_acc(R(-1), st.J01, st.J2, st.J3, t);
    const R f = R(-1) / mdot(P0123, P0123);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J1023[m] = f * t[m];
  }
  {  // J(1,0,3,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J1, P1, st.J032, P023, t);
    vvv_acc(R(1), st.J01, P01, st.J23, P23, t);
    vvv_acc(R(1), st.J103, P013, st.J2, P2, t);
    vvvv_acc(R(-1), st.J1, st.J0, st.J23, t);
    vvvv_acc(R(1), st.J1, st.J03, st.J2, t);
    vvvv_acc(R(-1), st.J01, st.J3, st.J2, t);
    const R f = R(-1) / mdot(P0123, P0123);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J1032[m] = f * t[m];
  }
  {  // J(1,2,0,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J1, P1, st.J203, P023, t);
    vvv_acc(R(1), st.J12, P12, st.J03, P03, t);
    vvv_acc(R(1), st.J021, P012, st.J3, P3, t);
    vvvv_acc(R(1), st.J1, st.J2, st.J03, t);
    vvvv_acc(R(-1), st.J1, st.J02, st.J3, t);
    vvvv_acc(R(1), st.J12, st.J0, st.J3, t);
    const R f = R(-1) / mdot(P0123, P0123);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J1203[m] = f * t[m];
  }
  {  // J(1,3,0,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J1, P1, st.J203, P023, t);
    vvv_acc(R(1), st.J13, P13, st.J02, P02, t);
    vvv_acc(R(1), st.J031, P013, st.J2, P2, t);
    vvvv_acc(R(1), st.J1, st.J3, st.J02, t);
    vvvv_acc(R(-1), st.J1, st.J03, st.J2, t);
    vvvv_acc(R(1), st.J13, st.J0, st.J2, t);
    const R f = R(-1) / mdot(P0123, P0123);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J1302[m] = f * t[m];
  }
  {  // J(2,0,1,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J2, P2, st.J013, P013, t);
    vvv_acc(R(-1), st.J02, P02, st.J13, P13, t);
    vvv_acc(R(1), st.J102, P012, st.J3, P3, t);
    vvvv_acc(R(1), st.J2, st.J0, st.J13, t);
    vvvv_acc(R(1), st.J2, st.J01, st.J3, t);
    vvvv_acc(R(-1), st.J02, st.J1, st.J3, t);
    const R f = R(-1) / mdot(P0123, P0123);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J2013[m] = f * t[m];
  }
  {  // J(2,1,0,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), st.J2, P2, st.J103, P013, t);
    vvv_acc(R(-1), st.J12, P12, st.J03, P03, t);
    vvv_acc(R(1), st.J012, P012, st.J3, P3, t);
    vvvv_acc(R(1), st.J2, st.J1, st.J03, t);
    vvvv_acc(R(-1), st.J2, st.J01, st.J3, t);
    vvvv_acc(R(-1), st.J12, st.J0, st.J3, t);
    const R f = R(-1) / mdot(P0123, P0123);
#pragma unroll
    for (int m = 0; m < 4; ++m) st.J2103[m] = f * t[m];
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) st.Q0[m] = -(ptb[m] + pg[0][m]);
#pragma unroll
  for (int m = 0; m < 4; ++m) st.Q1[m] = -(ptb[m] + pg[1][m]);
#pragma unroll
  for (int m = 0; m < 4; ++m) st.Q2[m] = -(ptb[m] + pg[2][m]);
#pragma unroll
  for (int m = 0; m < 4; ++m) st.Q3[m] = -(ptb[m] + pg[3][m]);
#pragma unroll
  for (int m = 0; m < 4; ++m) st.Q01[m] = -(ptb[m] + pg[0][m] + pg[1][m]);
#pragma unroll
  for (int m = 0; m < 4; ++m) st.Q02[m] = -(ptb[m] + pg[0][m] + pg[2][m]);
#pragma unroll
  for (int m = 0; m < 4; ++m) st.Q03[m] = -(ptb[m] + pg[0][m] + pg[3][m]);
#pragma unroll
  for (int m = 0; m < 4; ++m) st.Q12[m] = -(ptb[m] + pg[1][m] + pg[2][m]);
#pragma unroll
  for (int m = 0; m < 4; ++m) st.Q13[m] = -(ptb[m] + pg[1][m] + pg[3][m]);
#pragma unroll
  for (int m = 0; m < 4; ++m) st.Q23[m] = -(ptb[m] + pg[2][m] + pg[3][m]);
#pragma unroll
  for (int m = 0; m < 4; ++m) st.Q012[m] = -(ptb[m] + pg[0][m] + pg[1][m] + pg[2][m]);
#pragma unroll
  for (int m = 0; m < 4; ++m) st.Q013[m] = -(ptb[m] + pg[0][m] + pg[1][m] + pg[3][m]);
#pragma unroll
  for (int m = 0; m < 4; ++m) st.Q023[m] = -(ptb[m] + pg[0][m] + pg[2][m] + pg[3][m]);
#pragma unroll
  for (int m = 0; m < 4; ++m) st.Q123[m] = -(ptb[m] + pg[1][m] + pg[2][m] + pg[3][m]);
}

// sum over top and antitop helicities of sum_{s,s'} conj(A_s) Cint_{ss'} A_s'
// for one (mass, width); Cint = C * COLOUR_DEN.  WIDTH selects complex denominators.
// The quadratic form of one helicity is evaluated in CS (a positive-definite form:
// no cancellation), and the helicity sum is accumulated in ACC.
template <typename R, typename ACC, bool WIDTH, typename CS = ACC>
__device__ __forceinline__ ACC gg_ttxgg_quark_line(const gg_ttxgg_gluons<R>& st, const R (&pt)[4], const R (&ptb)[4], R mt, R wt) {
  ACC total = ACC(0);
  const R d0 = mdot(st.Q0, st.Q0) - mt * mt;
  R id0r, id0i;
  if (WIDTH) { const R im = mt * wt; const R nn = R(1) / (d0 * d0 + im * im); id0r = d0 * nn; id0i = -im * nn; } else { id0r = R(1) / d0; id0i = R(0); }
  const R d1 = mdot(st.Q1, st.Q1) - mt * mt;
  R id1r, id1i;
  if (WIDTH) { const R im = mt * wt; const R nn = R(1) / (d1 * d1 + im * im); id1r = d1 * nn; id1i = -im * nn; } else { id1r = R(1) / d1; id1i = R(0); }
  const R d2 = mdot(st.Q2, st.Q2) - mt * mt;
  R id2r, id2i;
  if (WIDTH) { const R im = mt * wt; const R nn = R(1) / (d2 * d2 + im * im); id2r = d2 * nn; id2i = -im * nn; } else { id2r = R(1) / d2; id2i = R(0); }
  const R d3 = mdot(st.Q3, st.Q3) - mt * mt;
  R id3r, id3i;
  if (WIDTH) { const R im = mt * wt; const R nn = R(1) / (d3 * d3 + im * im); id3r = d3 * nn; id3i = -im * nn; } else { id3r = R(1) / d3; id3i = R(0); }
  const R d01 = mdot(st.Q01, st.Q01) - mt * mt;
  R id01r, id01i;
  if (WIDTH) { const R im = mt * wt; const R nn = R(1) / (d01 * d01 + im * im); id01r = d01 * nn; id01i = -im * nn; } else { id01r = R(1) / d01; id01i = R(0); }
  const R d02 = mdot(st.Q02, st.Q02) - mt * mt;
  R id02r, id02i;
  if (WIDTH) { const R im = mt * wt; const R nn = R(1) / (d02 * d02 + im * im); id02r = d02 * nn; id02i = -im * nn; } else { id02r = R(1) / d02; id02i = R(0); }
  const R d03 = mdot(st.Q03, st.Q03) - mt * mt;
  R id03r, id03i;
  if (WIDTH) { const R im = mt * wt; const R nn = R(1) / (d03 * d03 + im * im); id03r = d03 * nn; id03i = -im * nn; } else { id03r = R(1) / d03; id03i = R(0); }
  const R d12 = mdot(st.Q12, st.Q12) - mt * mt;
  R id12r, id12i;
  if (WIDTH) { const R im = mt * wt; const R nn = R(1) / (d12 * d12 + im * im); id12r = d12 * nn; id12i = -im * nn; } else { id12r = R(1) / d12; id12i = R(0); }
  const R d13 = mdot(st.Q13, st.Q13) - mt * mt;
  R id13r, id13i;
  if (WIDTH) { const R im = mt * wt; const R nn = R(1) / (d13 * d13 + im * im); id13r = d13 * nn; id13i = -im * nn; } else { id13r = R(1) / d13; id13i = R(0); }
  const R d23 = mdot(st.Q23, st.Q23) - mt * mt;
  R id23r, id23i;
  if (WIDTH) { const R im = mt * wt; const R nn = R(1) / (d23 * d23 + im * im); id23r = d23 * nn; id23i = -im * nn; } else { id23r = R(1) / d23; id23i = R(0); }
  const R d012 = mdot(st.Q012, st.Q012) - mt * mt;
  R id012r, id012i;
  if (WIDTH) { const R im = mt * wt; const R nn = R(1) / (d012 * d012 + im * im); id012r = d012 * nn; id012i = -im * nn; } else { id012r = R(1) / d012; id012i = R(0); }
  const R d013 = mdot(st.Q013, st.Q013) - mt * mt;
  R id013r, id013i;
  if (WIDTH) { const R im = mt * wt; const R nn = R(1) / (d013 * d013 + im * im); id013r = d013 * nn; id013i = -im * nn; } else { id013r = R(1) / d013; id013i = R(0); }
  const R d023 = mdot(st.Q023, st.Q023) - mt * mt;
  R id023r, id023i;
  if (WIDTH) { const R im = mt * wt; const R nn = R(1) / (d023 * d023 + im * im); id023r = d023 * nn; id023i = -im * nn; } else { id023r = R(1) / d023; id023i = R(0); }
  const R d123 = mdot(st.Q123, st.Q123) - mt * mt;
  R id123r, id123i;
  if (WIDTH) { const R im = mt * wt; const R nn = R(1) / (d123 * d123 + im * im); id123r = d123 * nn; id123i = -im * nn; } else { id123r = R(1) / d123; id123i = R(0); }
  cx<R> ut[2][4];
  spinor_u(pt, mt, -1, ut[0]);
  spinor_u(pt, mt, +1, ut[1]);
#pragma unroll 1
  for (int hb = 0; hb < 2; ++hb) {
    cx<R> v[4];
    spinor_v(ptb, mt, hb == 0 ? -1 : +1, v);
    cx<R> psi0[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J0, v, t);
      if (WIDTH) fermion_prop(st.Q0, mt, cx<R>{id0r, id0i}, t, psi0);
      else fermion_prop_real(st.Q0, mt, id0r, t, psi0);
    }
    cx<R> psi1[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J1, v, t);
      if (WIDTH) fermion_prop(st.Q1, mt, cx<R>{id1r, id1i}, t, psi1);
      else fermion_prop_real(st.Q1, mt, id1r, t, psi1);
    }
    cx<R> psi2[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J2, v, t);
      if (WIDTH) fermion_prop(st.Q2, mt, cx<R>{id2r, id2i}, t, psi2);
      else fermion_prop_real(st.Q2, mt, id2r, t, psi2);
    }
    cx<R> psi3[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J3, v, t);
      if (WIDTH) fermion_prop(st.Q3, mt, cx<R>{id3r, id3i}, t, psi3);
      else fermion_prop_real(st.Q3, mt, id3r, t, psi3);
    }
    cx<R> psi01[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J0, psi1, t);
      slash_acc(R(1), st.J01, v, t);
      if (WIDTH) fermion_prop(st.Q01, mt, cx<R>{id01r, id01i}, t, psi01);
      else fermion_prop_real(st.Q01, mt, id01r, t, psi01);
    }
    cx<R> psi02[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J0, psi2, t);
      slash_acc(R(1), st.J02, v, t);
      if (WIDTH) fermion_prop(st.Q02, mt, cx<R>{id02r, id02i}, t, psi02);
      else fermion_prop_real(st.Q02, mt, id02r, t, psi02);
    }
    cx<R> psi03[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J0, psi3, t);
      slash_acc(R(1), st.J03, v, t);
      if (WIDTH) fermion_prop(st.Q03, mt, cx<R>{id03r, id03i}, t, psi03);
      else fermion_prop_real(st.Q03, mt, id03r, t, psi03);
    }
    cx<R> psi10[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J1, psi0, t);
      slash_acc(R(-1), st.J01, v, t);
      if (WIDTH) fermion_prop(st.Q01, mt, cx<R>{id01r, id01i}, t, psi10);
      else fermion_prop_real(st.Q01, mt, id01r, t, psi10);
    }
    cx<R> psi12[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J1, psi2, t);
      slash_acc(R(1), st.J12, v, t);
      if (WIDTH) fermion_prop(st.Q12, mt, cx<R>{id12r, id12i}, t, psi12);
      else fermion_prop_real(st.Q12, mt, id12r, t, psi12);
    }
    cx<R> psi13[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J1, psi3, t);
      slash_acc(R(1), st.J13, v, t);
      if (WIDTH) fermion_prop(st.Q13, mt, cx<R>{id13r, id13i}, t, psi13);
      else fermion_prop_real(st.Q13, mt, id13r, t, psi13);
    }
    cx<R> psi20[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J2, psi0, t);
      slash_acc(R(-1), st.J02, v, t);
      if (WIDTH) fermion_prop(st.Q02, mt, cx<R>{id02r, id02i}, t, psi20);
      else fermion_prop_real(st.Q02, mt, id02r, t, psi20);
    }
    cx<R> psi21[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J2, psi1, t);
      slash_acc(R(-1), st.J12, v, t);
      if (WIDTH) fermion_prop(st.Q12, mt, cx<R>{id12r, id12i}, t, psi21);
      else fermion_prop_real(st.Q12, mt, id12r, t, psi21);
    }
    cx<R> psi23[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J2, psi3, t);
      slash_acc(R(1), st.J23, v, t);
      if (WIDTH) fermion_prop(st.Q23, mt, cx<R>{id23r, id23i}, t, psi23);
      else fermion_prop_real(st.Q23, mt, id23r, t, psi23);
    }
    cx<R> psi30[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J3, psi0, t);
      slash_acc(R(-1), st.J03, v, t);
      if (WIDTH) fermion_prop(st.Q03, mt, cx<R>{id03r, id03i}, t, psi30);
      else fermion_prop_real(st.Q03, mt, id03r, t, psi30);
    }
    cx<R> psi31[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J3, psi1, t);
      slash_acc(R(-1), st.J13, v, t);
      if (WIDTH) fermion_prop(st.Q13, mt, cx<R>{id13r, id13i}, t, psi31);
      else fermion_prop_real(st.Q13, mt, id13r, t, psi31);
    }
    cx<R> psi32[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J3, psi2, t);
      slash_acc(R(-1), st.J23, v, t);
      if (WIDTH) fermion_prop(st.Q23, mt, cx<R>{id23r, id23i}, t, psi32);
      else fermion_prop_real(st.Q23, mt, id23r, t, psi32);
    }
    cx<R> psi012[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J0, psi12, t);
      slash_acc(R(1), st.J01, psi2, t);
      slash_acc(R(1), st.J012, v, t);
      if (WIDTH) fermion_prop(st.Q012, mt, cx<R>{id012r, id012i}, t, psi012);
      else fermion_prop_real(st.Q012, mt, id012r, t, psi012);
    }
    cx<R> psi013[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J0, psi13, t);
      slash_acc(R(1), st.J01, psi3, t);
      slash_acc(R(1), st.J013, v, t);
      if (WIDTH) fermion_prop(st.Q013, mt, cx<R>{id013r, id013i}, t, psi013);
      else fermion_prop_real(st.Q013, mt, id013r, t, psi013);
    }
    cx<R> psi021[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J0, psi21, t);
      slash_acc(R(1), st.J02, psi1, t);
      slash_acc(R(1), st.J021, v, t);
      if (WIDTH) fermion_prop(st.Q012, mt, cx<R>{id012r, id012i}, t, psi021);
      else fermion_prop_real(st.Q012, mt, id012r, t, psi021);
    }
    cx<R> psi023[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J0, psi23, t);
      slash_acc(R(1), st.J02, psi3, t);
      slash_acc(R(1), st.J023, v, t);
      if (WIDTH) fermion_prop(st.Q023, mt, cx<R>{id023r, id023i}, t, psi023);
      else fermion_prop_real(st.Q023, mt, id023r, t, psi023);
    }
    cx<R> psi031[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J0, psi31, t);
      slash_acc(R(1), st.J03, psi1, t);
      slash_acc(R(1), st.J031, v, t);
      if (WIDTH) fermion_prop(st.Q013, mt, cx<R>{id013r, id013i}, t, psi031);
      else fermion_prop_real(st.Q013, mt, id013r, t, psi031);
    }
    cx<R> psi032[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J0, psi32, t);
      slash_acc(R(1), st.J03, psi2, t);
      slash_acc(R(1), st.J032, v, t);
      if (WIDTH) fermion_prop(st.Q023, mt, cx<R>{id023r, id023i}, t, psi032);
      else fermion_prop_real(st.Q023, mt, id023r, t, psi032);
    }
    cx<R> psi102[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J1, psi02, t);
      slash_acc(R(-1), st.J01, psi2, t);
      slash_acc(R(1), st.J102, v, t);
      if (WIDTH) fermion_prop(st.Q012, mt, cx<R>{id012r, id012i}, t, psi102);
      else fermion_prop_real(st.Q012, mt, id012r, t, psi102);
    }
    cx<R> psi103[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J1, psi03, t);
      slash_acc(R(-1), st.J01, psi3, t);
      slash_acc(R(1), st.J103, v, t);
      if (WIDTH) fermion_prop(st.Q013, mt, cx<R>{id013r, id013i}, t, psi103);
      else fermion_prop_real(st.Q013, mt, id013r, t, psi103);
    }
    cx<R> psi120[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J1, psi20, t);
      slash_acc(R(1), st.J12, psi0, t);
      slash_acc(R(1), st.J021, v, t);
      if (WIDTH) fermion_prop(st.Q012, mt, cx<R>{id012r, id012i}, t, psi120);
      else fermion_prop_real(st.Q012, mt, id012r, t, psi120);
    }
    cx<R> psi123[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J1, psi23, t);
      slash_acc(R(1), st.J12, psi3, t);
      slash_acc(R(1), st.J123, v, t);
      if (WIDTH) fermion_prop(st.Q123, mt, cx<R>{id123r, id123i}, t, psi123);
      else fermion_prop_real(st.Q123, mt, id123r, t, psi123);
    }
    cx<R> psi130[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J1, psi30, t);
      slash_acc(R(1), st.J13, psi0, t);
      slash_acc(R(1), st.J031, v, t);
      if (WIDTH) fermion_prop(st.Q013, mt, cx<R>{id013r, id013i}, t, psi130);
      else fermion_prop_real(st.Q013, mt, id013r, t, psi130);
    }
    cx<R> psi132[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J1, psi32, t);
      slash_acc(R(1), st.J13, psi2, t);
      slash_acc(R(1), st.J132, v, t);
      if (WIDTH) fermion_prop(st.Q123, mt, cx<R>{id123r, id123i}, t, psi132);
      else fermion_prop_real(st.Q123, mt, id123r, t, psi132);
    }
    cx<R> psi201[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J2, psi01, t);
      slash_acc(R(-1), st.J02, psi1, t);
      slash_acc(R(1), st.J102, v, t);
      if (WIDTH) fermion_prop(st.Q012, mt, cx<R>{id012r, id012i}, t, psi201);
      else fermion_prop_real(st.Q012, mt, id012r, t, psi201);
    }
    cx<R> psi203[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J2, psi03, t);
      slash_acc(R(-1), st.J02, psi3, t);
      slash_acc(R(1), st.J203, v, t);
      if (WIDTH) fermion_prop(st.Q023, mt, cx<R>{id023r, id023i}, t, psi203);
      else fermion_prop_real(st.Q023, mt, id023r, t, psi203);
    }
    cx<R> psi210[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J2, psi10, t);
      slash_acc(R(-1), st.J12, psi0, t);
      slash_acc(R(1), st.J012, v, t);
      if (WIDTH) fermion_prop(st.Q012, mt, cx<R>{id012r, id012i}, t, psi210);
      else fermion_prop_real(st.Q012, mt, id012r, t, psi210);
    }
    cx<R> psi213[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J2, psi13, t);
      slash_acc(R(-1), st.J12, psi3, t);
      slash_acc(R(1), st.J213, v, t);
      if (WIDTH) fermion_prop(st.Q123, mt, cx<R>{id123r, id123i}, t, psi213);
      else fermion_prop_real(st.Q123, mt, id123r, t, psi213);
    }
    cx<R> psi230[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J2, psi30, t);
      slash_acc(R(1), st.J23, psi0, t);
      slash_acc(R(1), st.J032, v, t);
      if (WIDTH) fermion_prop(st.Q023, mt, cx<R>{id023r, id023i}, t, psi230);
      else fermion_prop_real(st.Q023, mt, id023r, t, psi230);
    }
    cx<R> psi231[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J2, psi31, t);
      slash_acc(R(1), st.J23, psi1, t);
      slash_acc(R(1), st.J132, v, t);
      if (WIDTH) fermion_prop(st.Q123, mt, cx<R>{id123r, id123i}, t, psi231);
      else fermion_prop_real(st.Q123, mt, id123r, t, psi231);
    }
    cx<R> psi301[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J3, psi01, t);
      slash_acc(R(-1), st.J03, psi1, t);
      slash_acc(R(1), st.J103, v, t);
      if (WIDTH) fermion_prop(st.Q013, mt, cx<R>{id013r, id013i}, t, psi301);
      else fermion_prop_real(st.Q013, mt, id013r, t, psi301);
    }
    cx<R> psi302[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J3, psi02, t);
      slash_acc(R(-1), st.J03, psi2, t);
      slash_acc(R(1), st.J203, v, t);
      if (WIDTH) fermion_prop(st.Q023, mt, cx<R>{id023r, id023i}, t, psi302);
      else fermion_prop_real(st.Q023, mt, id023r, t, psi302);
    }
    cx<R> psi310[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J3, psi10, t);
      slash_acc(R(-1), st.J13, psi0, t);
      slash_acc(R(1), st.J013, v, t);
      if (WIDTH) fermion_prop(st.Q013, mt, cx<R>{id013r, id013i}, t, psi310);
      else fermion_prop_real(st.Q013, mt, id013r, t, psi310);
    }
    cx<R> psi312[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J3, psi12, t);
      slash_acc(R(-1), st.J13, psi2, t);
      slash_acc(R(1), st.J213, v, t);
      if (WIDTH) fermion_prop(st.Q123, mt, cx<R>{id123r, id123i}, t, psi312);
      else fermion_prop_real(st.Q123, mt, id123r, t, psi312);
    }
    cx<R> psi320[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J3, psi20, t);
      slash_acc(R(-1), st.J23, psi0, t);
      slash_acc(R(1), st.J023, v, t);
      if (WIDTH) fermion_prop(st.Q023, mt, cx<R>{id023r, id023i}, t, psi320);
      else fermion_prop_real(st.Q023, mt, id023r, t, psi320);
    }
    cx<R> psi321[4];
    {
      cx<R> t[4] = {};
      slash_acc(R(1), st.J3, psi21, t);
      slash_acc(R(-1), st.J23, psi1, t);
      slash_acc(R(1), st.J123, v, t);
      if (WIDTH) fermion_prop(st.Q123, mt, cx<R>{id123r, id123i}, t, psi321);
      else fermion_prop_real(st.Q123, mt, id123r, t, psi321);
    }
    cx<R> A[2][24];
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J0, psi123, x);
      slash_acc(R(1), st.J01, psi23, x);
      slash_acc(R(1), st.J012, psi3, x);
      slash_acc(R(1), st.J0123, v, x);
      A[0][0] = ubar_dot(ut[0], x);
      A[1][0] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J0, psi132, x);
      slash_acc(R(1), st.J01, psi32, x);
      slash_acc(R(1), st.J013, psi2, x);
      slash_acc(R(1), st.J0132, v, x);
      A[0][1] = ubar_dot(ut[0], x);
      A[1][1] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J0, psi213, x);
      slash_acc(R(1), st.J02, psi13, x);
      slash_acc(R(1), st.J021, psi3, x);
      slash_acc(R(1), st.J0213, v, x);
      A[0][2] = ubar_dot(ut[0], x);
      A[1][2] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J0, psi231, x);
      slash_acc(R(1), st.J02, psi31, x);
      slash_acc(R(1), st.J023, psi1, x);
      slash_acc(R(1), st.J0231, v, x);
      A[0][3] = ubar_dot(ut[0], x);
      A[1][3] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J0, psi312, x);
      slash_acc(R(1), st.J03, psi12, x);
      slash_acc(R(1), st.J031, psi2, x);
      slash_acc(R(1), st.J0312, v, x);
      A[0][4] = ubar_dot(ut[0], x);
      A[1][4] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J0, psi321, x);
      slash_acc(R(1), st.J03, psi21, x);
      slash_acc(R(1), st.J032, psi1, x);
      slash_acc(R(1), st.J0321, v, x);
      A[0][5] = ubar_dot(ut[0], x);
      A[1][5] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J1, psi023, x);
      slash_acc(R(-1), st.J01, psi23, x);
      slash_acc(R(1), st.J102, psi3, x);
      slash_acc(R(1), st.J1023, v, x);
      A[0][6] = ubar_dot(ut[0], x);
      A[1][6] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J1, psi032, x);
      slash_acc(R(-1), st.J01, psi32, x);
      slash_acc(R(1), st.J103, psi2, x);
      slash_acc(R(1), st.J1032, v, x);
      A[0][7] = ubar_dot(ut[0], x);
      A[1][7] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J1, psi203, x);
      slash_acc(R(1), st.J12, psi03, x);
      slash_acc(R(1), st.J021, psi3, x);
      slash_acc(R(1), st.J1203, v, x);
      A[0][8] = ubar_dot(ut[0], x);
      A[1][8] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J1, psi230, x);
      slash_acc(R(1), st.J12, psi30, x);
      slash_acc(R(1), st.J123, psi0, x);
      slash_acc(R(-1), st.J0321, v, x);
      A[0][9] = ubar_dot(ut[0], x);
      A[1][9] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J1, psi302, x);
      slash_acc(R(1), st.J13, psi02, x);
      slash_acc(R(1), st.J031, psi2, x);
      slash_acc(R(1), st.J1302, v, x);
      A[0][10] = ubar_dot(ut[0], x);
      A[1][10] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J1, psi320, x);
      slash_acc(R(1), st.J13, psi20, x);
      slash_acc(R(1), st.J132, psi0, x);
      slash_acc(R(-1), st.J0231, v, x);
      A[0][11] = ubar_dot(ut[0], x);
      A[1][11] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J2, psi013, x);
      slash_acc(R(-1), st.J02, psi13, x);
      slash_acc(R(1), st.J102, psi3, x);
      slash_acc(R(1), st.J2013, v, x);
      A[0][12] = ubar_dot(ut[0], x);
      A[1][12] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J2, psi031, x);
      slash_acc(R(-1), st.J02, psi31, x);
      slash_acc(R(1), st.J203, psi1, x);
      slash_acc(R(-1), st.J1302, v, x);
      A[0][13] = ubar_dot(ut[0], x);
      A[1][13] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J2, psi103, x);
      slash_acc(R(-1), st.J12, psi03, x);
      slash_acc(R(1), st.J012, psi3, x);
      slash_acc(R(1), st.J2103, v, x);
      A[0][14] = ubar_dot(ut[0], x);
      A[1][14] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J2, psi130, x);
      slash_acc(R(-1), st.J12, psi30, x);
      slash_acc(R(1), st.J213, psi0, x);
      slash_acc(R(-1), st.J0312, v, x);
      A[0][15] = ubar_dot(ut[0], x);
      A[1][15] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J2, psi301, x);
      slash_acc(R(1), st.J23, psi01, x);
      slash_acc(R(1), st.J032, psi1, x);
      slash_acc(R(-1), st.J1032, v, x);
      A[0][16] = ubar_dot(ut[0], x);
      A[1][16] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J2, psi310, x);
      slash_acc(R(1), st.J23, psi10, x);
      slash_acc(R(1), st.J132, psi0, x);
      slash_acc(R(-1), st.J0132, v, x);
      A[0][17] = ubar_dot(ut[0], x);
      A[1][17] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J3, psi012, x);
      slash_acc(R(-1), st.J03, psi12, x);
      slash_acc(R(1), st.J103, psi2, x);
      slash_acc(R(-1), st.J2103, v, x);
      A[0][18] = ubar_dot(ut[0], x);
      A[1][18] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J3, psi021, x);
      slash_acc(R(-1), st.J03, psi21, x);
      slash_acc(R(1), st.J203, psi1, x);
      slash_acc(R(-1), st.J1203, v, x);
      A[0][19] = ubar_dot(ut[0], x);
      A[1][19] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J3, psi102, x);
      slash_acc(R(-1), st.J13, psi02, x);
      slash_acc(R(1), st.J013, psi2, x);
      slash_acc(R(-1), st.J2013, v, x);
      A[0][20] = ubar_dot(ut[0], x);
      A[1][20] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J3, psi120, x);
      slash_acc(R(-1), st.J13, psi20, x);
      slash_acc(R(1), st.J213, psi0, x);
      slash_acc(R(-1), st.J0213, v, x);
      A[0][21] = ubar_dot(ut[0], x);
      A[1][21] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J3, psi201, x);
      slash_acc(R(-1), st.J23, psi01, x);
      slash_acc(R(1), st.J023, psi1, x);
      slash_acc(R(-1), st.J1023, v, x);
      A[0][22] = ubar_dot(ut[0], x);
      A[1][22] = ubar_dot(ut[1], x);
    }
    {
      cx<R> x[4] = {};
      slash_acc(R(1), st.J3, psi210, x);
      slash_acc(R(-1), st.J23, psi10, x);
      slash_acc(R(1), st.J123, psi0, x);
      slash_acc(R(-1), st.J0123, v, x);
      A[0][23] = ubar_dot(ut[0], x);
      A[1][23] = ubar_dot(ut[1], x);
    }
#pragma unroll
    for (int ht = 0; ht < 2; ++ht) {
      CS s = CS(0);
      s += CS(512) * (CS(A[ht][0].re) * CS(A[ht][0].re) + CS(A[ht][0].im) * CS(A[ht][0].im));
      s += CS(512) * (CS(A[ht][1].re) * CS(A[ht][1].re) + CS(A[ht][1].im) * CS(A[ht][1].im));
      s += CS(512) * (CS(A[ht][2].re) * CS(A[ht][2].re) + CS(A[ht][2].im) * CS(A[ht][2].im));
      s += CS(512) * (CS(A[ht][3].re) * CS(A[ht][3].re) + CS(A[ht][3].im) * CS(A[ht][3].im));
      s += CS(512) * (CS(A[ht][4].re) * CS(A[ht][4].re) + CS(A[ht][4].im) * CS(A[ht][4].im));
      s += CS(512) * (CS(A[ht][5].re) * CS(A[ht][5].re) + CS(A[ht][5].im) * CS(A[ht][5].im));
      s += CS(512) * (CS(A[ht][6].re) * CS(A[ht][6].re) + CS(A[ht][6].im) * CS(A[ht][6].im));
      s += CS(512) * (CS(A[ht][7].re) * CS(A[ht][7].re) + CS(A[ht][7].im) * CS(A[ht][7].im));
      s += CS(512) * (CS(A[ht][8].re) * CS(A[ht][8].re) + CS(A[ht][8].im) * CS(A[ht][8].im));
      s += CS(512) * (CS(A[ht][9].re) * CS(A[ht][9].re) + CS(A[ht][9].im) * CS(A[ht][9].im));
      s += CS(512) * (CS(A[ht][10].re) * CS(A[ht][10].re) + CS(A[ht][10].im) * CS(A[ht][10].im));
      s += CS(512) * (CS(A[ht][11].re) * CS(A[ht][11].re) + CS(A[ht][11].im) * CS(A[ht][11].im));
      s += CS(512) * (CS(A[ht][12].re) * CS(A[ht][12].re) + CS(A[ht][12].im) * CS(A[ht][12].im));
      s += CS(512) * (CS(A[ht][13].re) * CS(A[ht][13].re) + CS(A[ht][13].im) * CS(A[ht][13].im));
      s += CS(512) * (CS(A[ht][14].re) * CS(A[ht][14].re) + CS(A[ht][14].im) * CS(A[ht][14].im));
      s += CS(512) * (CS(A[ht][15].re) * CS(A[ht][15].re) + CS(A[ht][15].im) * CS(A[ht][15].im));
      s += CS(512) * (CS(A[ht][16].re) * CS(A[ht][16].re) + CS(A[ht][16].im) * CS(A[ht][16].im));
      s += CS(512) * (CS(A[ht][17].re) * CS(A[ht][17].re) + CS(A[ht][17].im) * CS(A[ht][17].im));
      s += CS(512) * (CS(A[ht][18].re) * CS(A[ht][18].re) + CS(A[ht][18].im) * CS(A[ht][18].im));
      s += CS(512) * (CS(A[ht][19].re) * CS(A[ht][19].re) + CS(A[ht][19].im) * CS(A[ht][19].im));
      s += CS(512) * (CS(A[ht][20].re) * CS(A[ht][20].re) + CS(A[ht][20].im) * CS(A[ht][20].im));
      s += CS(512) * (CS(A[ht][21].re) * CS(A[ht][21].re) + CS(A[ht][21].im) * CS(A[ht][21].im));
      s += CS(512) * (CS(A[ht][22].re) * CS(A[ht][22].re) + CS(A[ht][22].im) * CS(A[ht][22].im));
      s += CS(512) * (CS(A[ht][23].re) * CS(A[ht][23].re) + CS(A[ht][23].im) * CS(A[ht][23].im));
      s += CS(-128) * (CS(A[ht][0].re) * CS(A[ht][1].re) + CS(A[ht][0].im) * CS(A[ht][1].im));
      s += CS(-128) * (CS(A[ht][0].re) * CS(A[ht][2].re) + CS(A[ht][0].im) * CS(A[ht][2].im));
      s += CS(16) * (CS(A[ht][0].re) * CS(A[ht][3].re) + CS(A[ht][0].im) * CS(A[ht][3].im));
      s += CS(16) * (CS(A[ht][0].re) * CS(A[ht][4].re) + CS(A[ht][0].im) * CS(A[ht][4].im));
      s += CS(160) * (CS(A[ht][0].re) * CS(A[ht][5].re) + CS(A[ht][0].im) * CS(A[ht][5].im));
      s += CS(-128) * (CS(A[ht][0].re) * CS(A[ht][6].re) + CS(A[ht][0].im) * CS(A[ht][6].im));
      s += CS(16) * (CS(A[ht][0].re) * CS(A[ht][7].re) + CS(A[ht][0].im) * CS(A[ht][7].im));
      s += CS(16) * (CS(A[ht][0].re) * CS(A[ht][8].re) + CS(A[ht][0].im) * CS(A[ht][8].im));
      s += CS(-2) * (CS(A[ht][0].re) * CS(A[ht][9].re) + CS(A[ht][0].im) * CS(A[ht][9].im));
      s += CS(-2) * (CS(A[ht][0].re) * CS(A[ht][10].re) + CS(A[ht][0].im) * CS(A[ht][10].im));
      s += CS(-20) * (CS(A[ht][0].re) * CS(A[ht][11].re) + CS(A[ht][0].im) * CS(A[ht][11].im));
      s += CS(16) * (CS(A[ht][0].re) * CS(A[ht][12].re) + CS(A[ht][0].im) * CS(A[ht][12].im));
      s += CS(-2) * (CS(A[ht][0].re) * CS(A[ht][13].re) + CS(A[ht][0].im) * CS(A[ht][13].im));
      s += CS(160) * (CS(A[ht][0].re) * CS(A[ht][14].re) + CS(A[ht][0].im) * CS(A[ht][14].im));
      s += CS(-20) * (CS(A[ht][0].re) * CS(A[ht][15].re) + CS(A[ht][0].im) * CS(A[ht][15].im));
      s += CS(142) * (CS(A[ht][0].re) * CS(A[ht][16].re) + CS(A[ht][0].im) * CS(A[ht][16].im));
      s += CS(124) * (CS(A[ht][0].re) * CS(A[ht][17].re) + CS(A[ht][0].im) * CS(A[ht][17].im));
      s += CS(-2) * (CS(A[ht][0].re) * CS(A[ht][18].re) + CS(A[ht][0].im) * CS(A[ht][18].im));
      s += CS(-20) * (CS(A[ht][0].re) * CS(A[ht][19].re) + CS(A[ht][0].im) * CS(A[ht][19].im));
      s += CS(-20) * (CS(A[ht][0].re) * CS(A[ht][20].re) + CS(A[ht][0].im) * CS(A[ht][20].im));
      s += CS(124) * (CS(A[ht][0].re) * CS(A[ht][21].re) + CS(A[ht][0].im) * CS(A[ht][21].im));
      s += CS(124) * (CS(A[ht][0].re) * CS(A[ht][22].re) + CS(A[ht][0].im) * CS(A[ht][22].im));
      s += CS(-56) * (CS(A[ht][0].re) * CS(A[ht][23].re) + CS(A[ht][0].im) * CS(A[ht][23].im));
      s += CS(16) * (CS(A[ht][1].re) * CS(A[ht][2].re) + CS(A[ht][1].im) * CS(A[ht][2].im));
      s += CS(160) * (CS(A[ht][1].re) * CS(A[ht][3].re) + CS(A[ht][1].im) * CS(A[ht][3].im));
      s += CS(-128) * (CS(A[ht][1].re) * CS(A[ht][4].re) + CS(A[ht][1].im) * CS(A[ht][4].im));
      s += CS(16) * (CS(A[ht][1].re) * CS(A[ht][5].re) + CS(A[ht][1].im) * CS(A[ht][5].im));
      s += CS(16) * (CS(A[ht][1].re) * CS(A[ht][6].re) + CS(A[ht][1].im) * CS(A[ht][6].im));
      s += CS(-128) * (CS(A[ht][1].re) * CS(A[ht][7].re) + CS(A[ht][1].im) * CS(A[ht][7].im));
      s += CS(-2) * (CS(A[ht][1].re) * CS(A[ht][8].re) + CS(A[ht][1].im) * CS(A[ht][8].im));
      s += CS(-20) * (CS(A[ht][1].re) * CS(A[ht][9].re) + CS(A[ht][1].im) * CS(A[ht][9].im));
      s += CS(16) * (CS(A[ht][1].re) * CS(A[ht][10].re) + CS(A[ht][1].im) * CS(A[ht][10].im));
      s += CS(-2) * (CS(A[ht][1].re) * CS(A[ht][11].re) + CS(A[ht][1].im) * CS(A[ht][11].im));
      s += CS(-2) * (CS(A[ht][1].re) * CS(A[ht][12].re) + CS(A[ht][1].im) * CS(A[ht][12].im));
      s += CS(-20) * (CS(A[ht][1].re) * CS(A[ht][13].re) + CS(A[ht][1].im) * CS(A[ht][13].im));
      s += CS(-20) * (CS(A[ht][1].re) * CS(A[ht][14].re) + CS(A[ht][1].im) * CS(A[ht][14].im));
      s += CS(124) * (CS(A[ht][1].re) * CS(A[ht][15].re) + CS(A[ht][1].im) * CS(A[ht][15].im));
      s += CS(124) * (CS(A[ht][1].re) * CS(A[ht][16].re) + CS(A[ht][1].im) * CS(A[ht][16].im));
      s += CS(-56) * (CS(A[ht][1].re) * CS(A[ht][17].re) + CS(A[ht][1].im) * CS(A[ht][17].im));
      s += CS(16) * (CS(A[ht][1].re) * CS(A[ht][18].re) + CS(A[ht][1].im) * CS(A[ht][18].im));
      s += CS(-2) * (CS(A[ht][1].re) * CS(A[ht][19].re) + CS(A[ht][1].im) * CS(A[ht][19].im));
      s += CS(160) * (CS(A[ht][1].re) * CS(A[ht][20].re) + CS(A[ht][1].im) * CS(A[ht][20].im));
      s += CS(-20) * (CS(A[ht][1].re) * CS(A[ht][21].re) + CS(A[ht][1].im) * CS(A[ht][21].im));
      s += CS(142) * (CS(A[ht][1].re) * CS(A[ht][22].re) + CS(A[ht][1].im) * CS(A[ht][22].im));
      s += CS(124) * (CS(A[ht][1].re) * CS(A[ht][23].re) + CS(A[ht][1].im) * CS(A[ht][23].im));
      s += CS(-128) * (CS(A[ht][2].re) * CS(A[ht][3].re) + CS(A[ht][2].im) * CS(A[ht][3].im));
      s += CS(160) * (CS(A[ht][2].re) * CS(A[ht][4].re) + CS(A[ht][2].im) * CS(A[ht][4].im));
      s += CS(16) * (CS(A[ht][2].re) * CS(A[ht][5].re) + CS(A[ht][2].im) * CS(A[ht][5].im));
      s += CS(16) * (CS(A[ht][2].re) * CS(A[ht][6].re) + CS(A[ht][2].im) * CS(A[ht][6].im));
      s += CS(-2) * (CS(A[ht][2].re) * CS(A[ht][7].re) + CS(A[ht][2].im) * CS(A[ht][7].im));
      s += CS(160) * (CS(A[ht][2].re) * CS(A[ht][8].re) + CS(A[ht][2].im) * CS(A[ht][8].im));
      s += CS(-20) * (CS(A[ht][2].re) * CS(A[ht][9].re) + CS(A[ht][2].im) * CS(A[ht][9].im));
      s += CS(142) * (CS(A[ht][2].re) * CS(A[ht][10].re) + CS(A[ht][2].im) * CS(A[ht][10].im));
      s += CS(124) * (CS(A[ht][2].re) * CS(A[ht][11].re) + CS(A[ht][2].im) * CS(A[ht][11].im));
      s += CS(-128) * (CS(A[ht][2].re) * CS(A[ht][12].re) + CS(A[ht][2].im) * CS(A[ht][12].im));
      s += CS(16) * (CS(A[ht][2].re) * CS(A[ht][13].re) + CS(A[ht][2].im) * CS(A[ht][13].im));
      s += CS(16) * (CS(A[ht][2].re) * CS(A[ht][14].re) + CS(A[ht][2].im) * CS(A[ht][14].im));
      s += CS(-2) * (CS(A[ht][2].re) * CS(A[ht][15].re) + CS(A[ht][2].im) * CS(A[ht][15].im));
      s += CS(-2) * (CS(A[ht][2].re) * CS(A[ht][16].re) + CS(A[ht][2].im) * CS(A[ht][16].im));
      s += CS(-20) * (CS(A[ht][2].re) * CS(A[ht][17].re) + CS(A[ht][2].im) * CS(A[ht][17].im));
      s += CS(-20) * (CS(A[ht][2].re) * CS(A[ht][18].re) + CS(A[ht][2].im) * CS(A[ht][18].im));
      s += CS(-2) * (CS(A[ht][2].re) * CS(A[ht][19].re) + CS(A[ht][2].im) * CS(A[ht][19].im));
      s += CS(124) * (CS(A[ht][2].re) * CS(A[ht][20].re) + CS(A[ht][2].im) * CS(A[ht][20].im));
      s += CS(-56) * (CS(A[ht][2].re) * CS(A[ht][21].re) + CS(A[ht][2].im) * CS(A[ht][21].im));
      s += CS(-20) * (CS(A[ht][2].re) * CS(A[ht][22].re) + CS(A[ht][2].im) * CS(A[ht][22].im));
      s += CS(124) * (CS(A[ht][2].re) * CS(A[ht][23].re) + CS(A[ht][2].im) * CS(A[ht][23].im));
      s += CS(16) * (CS(A[ht][3].re) * CS(A[ht][4].re) + CS(A[ht][3].im) * CS(A[ht][4].im));
      s += CS(-128) * (CS(A[ht][3].re) * CS(A[ht][5].re) + CS(A[ht][3].im) * CS(A[ht][5].im));
      s += CS(-2) * (CS(A[ht][3].re) * CS(A[ht][6].re) + CS(A[ht][3].im) * CS(A[ht][6].im));
      s += CS(-20) * (CS(A[ht][3].re) * CS(A[ht][7].re) + CS(A[ht][3].im) * CS(A[ht][7].im));
      s += CS(-20) * (CS(A[ht][3].re) * CS(A[ht][8].re) + CS(A[ht][3].im) * CS(A[ht][8].im));
      s += CS(124) * (CS(A[ht][3].re) * CS(A[ht][9].re) + CS(A[ht][3].im) * CS(A[ht][9].im));
      s += CS(124) * (CS(A[ht][3].re) * CS(A[ht][10].re) + CS(A[ht][3].im) * CS(A[ht][10].im));
      s += CS(-56) * (CS(A[ht][3].re) * CS(A[ht][11].re) + CS(A[ht][3].im) * CS(A[ht][11].im));
      s += CS(16) * (CS(A[ht][3].re) * CS(A[ht][12].re) + CS(A[ht][3].im) * CS(A[ht][12].im));
      s += CS(-128) * (CS(A[ht][3].re) * CS(A[ht][13].re) + CS(A[ht][3].im) * CS(A[ht][13].im));
      s += CS(-2) * (CS(A[ht][3].re) * CS(A[ht][14].re) + CS(A[ht][3].im) * CS(A[ht][14].im));
      s += CS(-20) * (CS(A[ht][3].re) * CS(A[ht][15].re) + CS(A[ht][3].im) * CS(A[ht][15].im));
      s += CS(16) * (CS(A[ht][3].re) * CS(A[ht][16].re) + CS(A[ht][3].im) * CS(A[ht][16].im));
      s += CS(-2) * (CS(A[ht][3].re) * CS(A[ht][17].re) + CS(A[ht][3].im) * CS(A[ht][17].im));
      s += CS(-2) * (CS(A[ht][3].re) * CS(A[ht][18].re) + CS(A[ht][3].im) * CS(A[ht][18].im));
      s += CS(16) * (CS(A[ht][3].re) * CS(A[ht][19].re) + CS(A[ht][3].im) * CS(A[ht][19].im));
      s += CS(142) * (CS(A[ht][3].re) * CS(A[ht][20].re) + CS(A[ht][3].im) * CS(A[ht][20].im));
      s += CS(124) * (CS(A[ht][3].re) * CS(A[ht][21].re) + CS(A[ht][3].im) * CS(A[ht][21].im));
      s += CS(160) * (CS(A[ht][3].re) * CS(A[ht][22].re) + CS(A[ht][3].im) * CS(A[ht][22].im));
      s += CS(-20) * (CS(A[ht][3].re) * CS(A[ht][23].re) + CS(A[ht][3].im) * CS(A[ht][23].im));
      s += CS(-128) * (CS(A[ht][4].re) * CS(A[ht][5].re) + CS(A[ht][4].im) * CS(A[ht][5].im));
      s += CS(-2) * (CS(A[ht][4].re) * CS(A[ht][6].re) + CS(A[ht][4].im) * CS(A[ht][6].im));
      s += CS(16) * (CS(A[ht][4].re) * CS(A[ht][7].re) + CS(A[ht][4].im) * CS(A[ht][7].im));
      s += CS(142) * (CS(A[ht][4].re) * CS(A[ht][8].re) + CS(A[ht][4].im) * CS(A[ht][8].im));
      s += CS(124) * (CS(A[ht][4].re) * CS(A[ht][9].re) + CS(A[ht][4].im) * CS(A[ht][9].im));
      s += CS(160) * (CS(A[ht][4].re) * CS(A[ht][10].re) + CS(A[ht][4].im) * CS(A[ht][10].im));
      s += CS(-20) * (CS(A[ht][4].re) * CS(A[ht][11].re) + CS(A[ht][4].im) * CS(A[ht][11].im));
      s += CS(-20) * (CS(A[ht][4].re) * CS(A[ht][12].re) + CS(A[ht][4].im) * CS(A[ht][12].im));
      s += CS(-2) * (CS(A[ht][4].re) * CS(A[ht][13].re) + CS(A[ht][4].im) * CS(A[ht][13].im));
      s += CS(124) * (CS(A[ht][4].re) * CS(A[ht][14].re) + CS(A[ht][4].im) * CS(A[ht][14].im));
      s += CS(-56) * (CS(A[ht][4].re) * CS(A[ht][15].re) + CS(A[ht][4].im) * CS(A[ht][15].im));
      s += CS(-20) * (CS(A[ht][4].re) * CS(A[ht][16].re) + CS(A[ht][4].im) * CS(A[ht][16].im));
      s += CS(124) * (CS(A[ht][4].re) * CS(A[ht][17].re) + CS(A[ht][4].im) * CS(A[ht][17].im));
      s += CS(-128) * (CS(A[ht][4].re) * CS(A[ht][18].re) + CS(A[ht][4].im) * CS(A[ht][18].im));
      s += CS(16) * (CS(A[ht][4].re) * CS(A[ht][19].re) + CS(A[ht][4].im) * CS(A[ht][19].im));
      s += CS(16) * (CS(A[ht][4].re) * CS(A[ht][20].re) + CS(A[ht][4].im) * CS(A[ht][20].im));
      s += CS(-2) * (CS(A[ht][4].re) * CS(A[ht][21].re) + CS(A[ht][4].im) * CS(A[ht][21].im));
      s += CS(-2) * (CS(A[ht][4].re) * CS(A[ht][22].re) + CS(A[ht][4].im) * CS(A[ht][22].im));
      s += CS(-20) * (CS(A[ht][4].re) * CS(A[ht][23].re) + CS(A[ht][4].im) * CS(A[ht][23].im));
      s += CS(-20) * (CS(A[ht][5].re) * CS(A[ht][6].re) + CS(A[ht][5].im) * CS(A[ht][6].im));
      s += CS(-2) * (CS(A[ht][5].re) * CS(A[ht][7].re) + CS(A[ht][5].im) * CS(A[ht][7].im));
      s += CS(124) * (CS(A[ht][5].re) * CS(A[ht][8].re) + CS(A[ht][5].im) * CS(A[ht][8].im));
      s += CS(-56) * (CS(A[ht][5].re) * CS(A[ht][9].re) + CS(A[ht][5].im) * CS(A[ht][9].im));
      s += CS(-20) * (CS(A[ht][5].re) * CS(A[ht][10].re) + CS(A[ht][5].im) * CS(A[ht][10].im));
      s += CS(124) * (CS(A[ht][5].re) * CS(A[ht][11].re) + CS(A[ht][5].im) * CS(A[ht][11].im));
      s += CS(-2) * (CS(A[ht][5].re) * CS(A[ht][12].re) + CS(A[ht][5].im) * CS(A[ht][12].im));
      s += CS(16) * (CS(A[ht][5].re) * CS(A[ht][13].re) + CS(A[ht][5].im) * CS(A[ht][13].im));
      s += CS(142) * (CS(A[ht][5].re) * CS(A[ht][14].re) + CS(A[ht][5].im) * CS(A[ht][14].im));
      s += CS(124) * (CS(A[ht][5].re) * CS(A[ht][15].re) + CS(A[ht][5].im) * CS(A[ht][15].im));
      s += CS(160) * (CS(A[ht][5].re) * CS(A[ht][16].re) + CS(A[ht][5].im) * CS(A[ht][16].im));
      s += CS(-20) * (CS(A[ht][5].re) * CS(A[ht][17].re) + CS(A[ht][5].im) * CS(A[ht][17].im));
      s += CS(16) * (CS(A[ht][5].re) * CS(A[ht][18].re) + CS(A[ht][5].im) * CS(A[ht][18].im));
      s += CS(-128) * (CS(A[ht][5].re) * CS(A[ht][19].re) + CS(A[ht][5].im) * CS(A[ht][19].im));
      s += CS(-2) * (CS(A[ht][5].re) * CS(A[ht][20].re) + CS(A[ht][5].im) * CS(A[ht][20].im));
      s += CS(-20) * (CS(A[ht][5].re) * CS(A[ht][21].re) + CS(A[ht][5].im) * CS(A[ht][21].im));
      s += CS(16) * (CS(A[ht][5].re) * CS(A[ht][22].re) + CS(A[ht][5].im) * CS(A[ht][22].im));
      s += CS(-2) * (CS(A[ht][5].re) * CS(A[ht][23].re) + CS(A[ht][5].im) * CS(A[ht][23].im));
      s += CS(-128) * (CS(A[ht][6].re) * CS(A[ht][7].re) + CS(A[ht][6].im) * CS(A[ht][7].im));
      s += CS(-128) * (CS(A[ht][6].re) * CS(A[ht][8].re) + CS(A[ht][6].im) * CS(A[ht][8].im));
      s += CS(16) * (CS(A[ht][6].re) * CS(A[ht][9].re) + CS(A[ht][6].im) * CS(A[ht][9].im));
      s += CS(16) * (CS(A[ht][6].re) * CS(A[ht][10].re) + CS(A[ht][6].im) * CS(A[ht][10].im));
      s += CS(160) * (CS(A[ht][6].re) * CS(A[ht][11].re) + CS(A[ht][6].im) * CS(A[ht][11].im));
      s += CS(160) * (CS(A[ht][6].re) * CS(A[ht][12].re) + CS(A[ht][6].im) * CS(A[ht][12].im));
      s += CS(-20) * (CS(A[ht][6].re) * CS(A[ht][13].re) + CS(A[ht][6].im) * CS(A[ht][13].im));
      s += CS(16) * (CS(A[ht][6].re) * CS(A[ht][14].re) + CS(A[ht][6].im) * CS(A[ht][14].im));
      s += CS(-2) * (CS(A[ht][6].re) * CS(A[ht][15].re) + CS(A[ht][6].im) * CS(A[ht][15].im));
      s += CS(124) * (CS(A[ht][6].re) * CS(A[ht][16].re) + CS(A[ht][6].im) * CS(A[ht][16].im));
      s += CS(142) * (CS(A[ht][6].re) * CS(A[ht][17].re) + CS(A[ht][6].im) * CS(A[ht][17].im));
      s += CS(-20) * (CS(A[ht][6].re) * CS(A[ht][18].re) + CS(A[ht][6].im) * CS(A[ht][18].im));
      s += CS(124) * (CS(A[ht][6].re) * CS(A[ht][19].re) + CS(A[ht][6].im) * CS(A[ht][19].im));
      s += CS(-2) * (CS(A[ht][6].re) * CS(A[ht][20].re) + CS(A[ht][6].im) * CS(A[ht][20].im));
      s += CS(-20) * (CS(A[ht][6].re) * CS(A[ht][21].re) + CS(A[ht][6].im) * CS(A[ht][21].im));
      s += CS(-56) * (CS(A[ht][6].re) * CS(A[ht][22].re) + CS(A[ht][6].im) * CS(A[ht][22].im));
      s += CS(124) * (CS(A[ht][6].re) * CS(A[ht][23].re) + CS(A[ht][6].im) * CS(A[ht][23].im));
      s += CS(16) * (CS(A[ht][7].re) * CS(A[ht][8].re) + CS(A[ht][7].im) * CS(A[ht][8].im));
      s += CS(160) * (CS(A[ht][7].re) * CS(A[ht][9].re) + CS(A[ht][7].im) * CS(A[ht][9].im));
      s += CS(-128) * (CS(A[ht][7].re) * CS(A[ht][10].re) + CS(A[ht][7].im) * CS(A[ht][10].im));
      s += CS(16) * (CS(A[ht][7].re) * CS(A[ht][11].re) + CS(A[ht][7].im) * CS(A[ht][11].im));
      s += CS(-20) * (CS(A[ht][7].re) * CS(A[ht][12].re) + CS(A[ht][7].im) * CS(A[ht][12].im));
      s += CS(124) * (CS(A[ht][7].re) * CS(A[ht][13].re) + CS(A[ht][7].im) * CS(A[ht][13].im));
      s += CS(-2) * (CS(A[ht][7].re) * CS(A[ht][14].re) + CS(A[ht][7].im) * CS(A[ht][14].im));
      s += CS(-20) * (CS(A[ht][7].re) * CS(A[ht][15].re) + CS(A[ht][7].im) * CS(A[ht][15].im));
      s += CS(-56) * (CS(A[ht][7].re) * CS(A[ht][16].re) + CS(A[ht][7].im) * CS(A[ht][16].im));
      s += CS(124) * (CS(A[ht][7].re) * CS(A[ht][17].re) + CS(A[ht][7].im) * CS(A[ht][17].im));
      s += CS(160) * (CS(A[ht][7].re) * CS(A[ht][18].re) + CS(A[ht][7].im) * CS(A[ht][18].im));
      s += CS(-20) * (CS(A[ht][7].re) * CS(A[ht][19].re) + CS(A[ht][7].im) * CS(A[ht][19].im));
      s += CS(16) * (CS(A[ht][7].re) * CS(A[ht][20].re) + CS(A[ht][7].im) * CS(A[ht][20].im));
      s += CS(-2) * (CS(A[ht][7].re) * CS(A[ht][21].re) + CS(A[ht][7].im) * CS(A[ht][21].im));
      s += CS(124) * (CS(A[ht][7].re) * CS(A[ht][22].re) + CS(A[ht][7].im) * CS(A[ht][22].im));
      s += CS(142) * (CS(A[ht][7].re) * CS(A[ht][23].re) + CS(A[ht][7].im) * CS(A[ht][23].im));
      s += CS(-128) * (CS(A[ht][8].re) * CS(A[ht][9].re) + CS(A[ht][8].im) * CS(A[ht][9].im));
      s += CS(160) * (CS(A[ht][8].re) * CS(A[ht][10].re) + CS(A[ht][8].im) * CS(A[ht][10].im));
      s += CS(16) * (CS(A[ht][8].re) * CS(A[ht][11].re) + CS(A[ht][8].im) * CS(A[ht][11].im));
      s += CS(16) * (CS(A[ht][8].re) * CS(A[ht][12].re) + CS(A[ht][8].im) * CS(A[ht][12].im));
      s += CS(-2) * (CS(A[ht][8].re) * CS(A[ht][13].re) + CS(A[ht][8].im) * CS(A[ht][13].im));
      s += CS(-128) * (CS(A[ht][8].re) * CS(A[ht][14].re) + CS(A[ht][8].im) * CS(A[ht][14].im));
      s += CS(16) * (CS(A[ht][8].re) * CS(A[ht][15].re) + CS(A[ht][8].im) * CS(A[ht][15].im));
      s += CS(-20) * (CS(A[ht][8].re) * CS(A[ht][16].re) + CS(A[ht][8].im) * CS(A[ht][16].im));
      s += CS(-2) * (CS(A[ht][8].re) * CS(A[ht][17].re) + CS(A[ht][8].im) * CS(A[ht][17].im));
      s += CS(124) * (CS(A[ht][8].re) * CS(A[ht][18].re) + CS(A[ht][8].im) * CS(A[ht][18].im));
      s += CS(-56) * (CS(A[ht][8].re) * CS(A[ht][19].re) + CS(A[ht][8].im) * CS(A[ht][19].im));
      s += CS(-20) * (CS(A[ht][8].re) * CS(A[ht][20].re) + CS(A[ht][8].im) * CS(A[ht][20].im));
      s += CS(-2) * (CS(A[ht][8].re) * CS(A[ht][21].re) + CS(A[ht][8].im) * CS(A[ht][21].im));
      s += CS(124) * (CS(A[ht][8].re) * CS(A[ht][22].re) + CS(A[ht][8].im) * CS(A[ht][22].im));
      s += CS(-20) * (CS(A[ht][8].re) * CS(A[ht][23].re) + CS(A[ht][8].im) * CS(A[ht][23].im));
      s += CS(16) * (CS(A[ht][9].re) * CS(A[ht][10].re) + CS(A[ht][9].im) * CS(A[ht][10].im));
      s += CS(-128) * (CS(A[ht][9].re) * CS(A[ht][11].re) + CS(A[ht][9].im) * CS(A[ht][11].im));
      s += CS(-2) * (CS(A[ht][9].re) * CS(A[ht][12].re) + CS(A[ht][9].im) * CS(A[ht][12].im));
      s += CS(-20) * (CS(A[ht][9].re) * CS(A[ht][13].re) + CS(A[ht][9].im) * CS(A[ht][13].im));
      s += CS(16) * (CS(A[ht][9].re) * CS(A[ht][14].re) + CS(A[ht][9].im) * CS(A[ht][14].im));
      s += CS(-128) * (CS(A[ht][9].re) * CS(A[ht][15].re) + CS(A[ht][9].im) * CS(A[ht][15].im));
      s += CS(-2) * (CS(A[ht][9].re) * CS(A[ht][16].re) + CS(A[ht][9].im) * CS(A[ht][16].im));
      s += CS(16) * (CS(A[ht][9].re) * CS(A[ht][17].re) + CS(A[ht][9].im) * CS(A[ht][17].im));
      s += CS(142) * (CS(A[ht][9].re) * CS(A[ht][18].re) + CS(A[ht][9].im) * CS(A[ht][18].im));
      s += CS(124) * (CS(A[ht][9].re) * CS(A[ht][19].re) + CS(A[ht][9].im) * CS(A[ht][19].im));
      s += CS(-2) * (CS(A[ht][9].re) * CS(A[ht][20].re) + CS(A[ht][9].im) * CS(A[ht][20].im));
      s += CS(16) * (CS(A[ht][9].re) * CS(A[ht][21].re) + CS(A[ht][9].im) * CS(A[ht][21].im));
      s += CS(-20) * (CS(A[ht][9].re) * CS(A[ht][22].re) + CS(A[ht][9].im) * CS(A[ht][22].im));
      s += CS(160) * (CS(A[ht][9].re) * CS(A[ht][23].re) + CS(A[ht][9].im) * CS(A[ht][23].im));
      s += CS(-128) * (CS(A[ht][10].re) * CS(A[ht][11].re) + CS(A[ht][10].im) * CS(A[ht][11].im));
      s += CS(124) * (CS(A[ht][10].re) * CS(A[ht][12].re) + CS(A[ht][10].im) * CS(A[ht][12].im));
      s += CS(-56) * (CS(A[ht][10].re) * CS(A[ht][13].re) + CS(A[ht][10].im) * CS(A[ht][13].im));
      s += CS(-20) * (CS(A[ht][10].re) * CS(A[ht][14].re) + CS(A[ht][10].im) * CS(A[ht][14].im));
      s += CS(-2) * (CS(A[ht][10].re) * CS(A[ht][15].re) + CS(A[ht][10].im) * CS(A[ht][15].im));
      s += CS(124) * (CS(A[ht][10].re) * CS(A[ht][16].re) + CS(A[ht][10].im) * CS(A[ht][16].im));
      s += CS(-20) * (CS(A[ht][10].re) * CS(A[ht][17].re) + CS(A[ht][10].im) * CS(A[ht][17].im));
      s += CS(16) * (CS(A[ht][10].re) * CS(A[ht][18].re) + CS(A[ht][10].im) * CS(A[ht][18].im));
      s += CS(-2) * (CS(A[ht][10].re) * CS(A[ht][19].re) + CS(A[ht][10].im) * CS(A[ht][19].im));
      s += CS(-128) * (CS(A[ht][10].re) * CS(A[ht][20].re) + CS(A[ht][10].im) * CS(A[ht][20].im));
      s += CS(16) * (CS(A[ht][10].re) * CS(A[ht][21].re) + CS(A[ht][10].im) * CS(A[ht][21].im));
      s += CS(-20) * (CS(A[ht][10].re) * CS(A[ht][22].re) + CS(A[ht][10].im) * CS(A[ht][22].im));
      s += CS(-2) * (CS(A[ht][10].re) * CS(A[ht][23].re) + CS(A[ht][10].im) * CS(A[ht][23].im));
      s += CS(142) * (CS(A[ht][11].re) * CS(A[ht][12].re) + CS(A[ht][11].im) * CS(A[ht][12].im));
      s += CS(124) * (CS(A[ht][11].re) * CS(A[ht][13].re) + CS(A[ht][11].im) * CS(A[ht][13].im));
      s += CS(-2) * (CS(A[ht][11].re) * CS(A[ht][14].re) + CS(A[ht][11].im) * CS(A[ht][14].im));
      s += CS(16) * (CS(A[ht][11].re) * CS(A[ht][15].re) + CS(A[ht][11].im) * CS(A[ht][15].im));
      s += CS(-20) * (CS(A[ht][11].re) * CS(A[ht][16].re) + CS(A[ht][11].im) * CS(A[ht][16].im));
      s += CS(160) * (CS(A[ht][11].re) * CS(A[ht][17].re) + CS(A[ht][11].im) * CS(A[ht][17].im));
      s += CS(-2) * (CS(A[ht][11].re) * CS(A[ht][18].re) + CS(A[ht][11].im) * CS(A[ht][18].im));
      s += CS(-20) * (CS(A[ht][11].re) * CS(A[ht][19].re) + CS(A[ht][11].im) * CS(A[ht][19].im));
      s += CS(16) * (CS(A[ht][11].re) * CS(A[ht][20].re) + CS(A[ht][11].im) * CS(A[ht][20].im));
      s += CS(-128) * (CS(A[ht][11].re) * CS(A[ht][21].re) + CS(A[ht][11].im) * CS(A[ht][21].im));
      s += CS(-2) * (CS(A[ht][11].re) * CS(A[ht][22].re) + CS(A[ht][11].im) * CS(A[ht][22].im));
      s += CS(16) * (CS(A[ht][11].re) * CS(A[ht][23].re) + CS(A[ht][11].im) * CS(A[ht][23].im));
      s += CS(-128) * (CS(A[ht][12].re) * CS(A[ht][13].re) + CS(A[ht][12].im) * CS(A[ht][13].im));
      s += CS(-128) * (CS(A[ht][12].re) * CS(A[ht][14].re) + CS(A[ht][12].im) * CS(A[ht][14].im));
      s += CS(16) * (CS(A[ht][12].re) * CS(A[ht][15].re) + CS(A[ht][12].im) * CS(A[ht][15].im));
      s += CS(16) * (CS(A[ht][12].re) * CS(A[ht][16].re) + CS(A[ht][12].im) * CS(A[ht][16].im));
      s += CS(160) * (CS(A[ht][12].re) * CS(A[ht][17].re) + CS(A[ht][12].im) * CS(A[ht][17].im));
      s += CS(124) * (CS(A[ht][12].re) * CS(A[ht][18].re) + CS(A[ht][12].im) * CS(A[ht][18].im));
      s += CS(-20) * (CS(A[ht][12].re) * CS(A[ht][19].re) + CS(A[ht][12].im) * CS(A[ht][19].im));
      s += CS(-56) * (CS(A[ht][12].re) * CS(A[ht][20].re) + CS(A[ht][12].im) * CS(A[ht][20].im));
      s += CS(124) * (CS(A[ht][12].re) * CS(A[ht][21].re) + CS(A[ht][12].im) * CS(A[ht][21].im));
      s += CS(-2) * (CS(A[ht][12].re) * CS(A[ht][22].re) + CS(A[ht][12].im) * CS(A[ht][22].im));
      s += CS(-20) * (CS(A[ht][12].re) * CS(A[ht][23].re) + CS(A[ht][12].im) * CS(A[ht][23].im));
      s += CS(16) * (CS(A[ht][13].re) * CS(A[ht][14].re) + CS(A[ht][13].im) * CS(A[ht][14].im));
      s += CS(160) * (CS(A[ht][13].re) * CS(A[ht][15].re) + CS(A[ht][13].im) * CS(A[ht][15].im));
      s += CS(-128) * (CS(A[ht][13].re) * CS(A[ht][16].re) + CS(A[ht][13].im) * CS(A[ht][16].im));
      s += CS(16) * (CS(A[ht][13].re) * CS(A[ht][17].re) + CS(A[ht][13].im) * CS(A[ht][17].im));
      s += CS(-20) * (CS(A[ht][13].re) * CS(A[ht][18].re) + CS(A[ht][13].im) * CS(A[ht][18].im));
      s += CS(160) * (CS(A[ht][13].re) * CS(A[ht][19].re) + CS(A[ht][13].im) * CS(A[ht][19].im));
      s += CS(124) * (CS(A[ht][13].re) * CS(A[ht][20].re) + CS(A[ht][13].im) * CS(A[ht][20].im));
      s += CS(142) * (CS(A[ht][13].re) * CS(A[ht][21].re) + CS(A[ht][13].im) * CS(A[ht][21].im));
      s += CS(16) * (CS(A[ht][13].re) * CS(A[ht][22].re) + CS(A[ht][13].im) * CS(A[ht][22].im));
      s += CS(-2) * (CS(A[ht][13].re) * CS(A[ht][23].re) + CS(A[ht][13].im) * CS(A[ht][23].im));
      s += CS(-128) * (CS(A[ht][14].re) * CS(A[ht][15].re) + CS(A[ht][14].im) * CS(A[ht][15].im));
      s += CS(160) * (CS(A[ht][14].re) * CS(A[ht][16].re) + CS(A[ht][14].im) * CS(A[ht][16].im));
      s += CS(16) * (CS(A[ht][14].re) * CS(A[ht][17].re) + CS(A[ht][14].im) * CS(A[ht][17].im));
      s += CS(-56) * (CS(A[ht][14].re) * CS(A[ht][18].re) + CS(A[ht][14].im) * CS(A[ht][18].im));
      s += CS(124) * (CS(A[ht][14].re) * CS(A[ht][19].re) + CS(A[ht][14].im) * CS(A[ht][19].im));
      s += CS(124) * (CS(A[ht][14].re) * CS(A[ht][20].re) + CS(A[ht][14].im) * CS(A[ht][20].im));
      s += CS(-20) * (CS(A[ht][14].re) * CS(A[ht][21].re) + CS(A[ht][14].im) * CS(A[ht][21].im));
      s += CS(-20) * (CS(A[ht][14].re) * CS(A[ht][22].re) + CS(A[ht][14].im) * CS(A[ht][22].im));
      s += CS(-2) * (CS(A[ht][14].re) * CS(A[ht][23].re) + CS(A[ht][14].im) * CS(A[ht][23].im));
      s += CS(16) * (CS(A[ht][15].re) * CS(A[ht][16].re) + CS(A[ht][15].im) * CS(A[ht][16].im));
      s += CS(-128) * (CS(A[ht][15].re) * CS(A[ht][17].re) + CS(A[ht][15].im) * CS(A[ht][17].im));
      s += CS(124) * (CS(A[ht][15].re) * CS(A[ht][18].re) + CS(A[ht][15].im) * CS(A[ht][18].im));
      s += CS(142) * (CS(A[ht][15].re) * CS(A[ht][19].re) + CS(A[ht][15].im) * CS(A[ht][19].im));
      s += CS(-20) * (CS(A[ht][15].re) * CS(A[ht][20].re) + CS(A[ht][15].im) * CS(A[ht][20].im));
      s += CS(160) * (CS(A[ht][15].re) * CS(A[ht][21].re) + CS(A[ht][15].im) * CS(A[ht][21].im));
      s += CS(-2) * (CS(A[ht][15].re) * CS(A[ht][22].re) + CS(A[ht][15].im) * CS(A[ht][22].im));
      s += CS(16) * (CS(A[ht][15].re) * CS(A[ht][23].re) + CS(A[ht][15].im) * CS(A[ht][23].im));
      s += CS(-128) * (CS(A[ht][16].re) * CS(A[ht][17].re) + CS(A[ht][16].im) * CS(A[ht][17].im));
      s += CS(-2) * (CS(A[ht][16].re) * CS(A[ht][18].re) + CS(A[ht][16].im) * CS(A[ht][18].im));
      s += CS(16) * (CS(A[ht][16].re) * CS(A[ht][19].re) + CS(A[ht][16].im) * CS(A[ht][19].im));
      s += CS(-20) * (CS(A[ht][16].re) * CS(A[ht][20].re) + CS(A[ht][16].im) * CS(A[ht][20].im));
      s += CS(-2) * (CS(A[ht][16].re) * CS(A[ht][21].re) + CS(A[ht][16].im) * CS(A[ht][21].im));
      s += CS(-128) * (CS(A[ht][16].re) * CS(A[ht][22].re) + CS(A[ht][16].im) * CS(A[ht][22].im));
      s += CS(16) * (CS(A[ht][16].re) * CS(A[ht][23].re) + CS(A[ht][16].im) * CS(A[ht][23].im));
      s += CS(-20) * (CS(A[ht][17].re) * CS(A[ht][18].re) + CS(A[ht][17].im) * CS(A[ht][18].im));
      s += CS(-2) * (CS(A[ht][17].re) * CS(A[ht][19].re) + CS(A[ht][17].im) * CS(A[ht][19].im));
      s += CS(-2) * (CS(A[ht][17].re) * CS(A[ht][20].re) + CS(A[ht][17].im) * CS(A[ht][20].im));
      s += CS(16) * (CS(A[ht][17].re) * CS(A[ht][21].re) + CS(A[ht][17].im) * CS(A[ht][21].im));
      s += CS(16) * (CS(A[ht][17].re) * CS(A[ht][22].re) + CS(A[ht][17].im) * CS(A[ht][22].im));
      s += CS(-128) * (CS(A[ht][17].re) * CS(A[ht][23].re) + CS(A[ht][17].im) * CS(A[ht][23].im));
      s += CS(-128) * (CS(A[ht][18].re) * CS(A[ht][19].re) + CS(A[ht][18].im) * CS(A[ht][19].im));
      s += CS(-128) * (CS(A[ht][18].re) * CS(A[ht][20].re) + CS(A[ht][18].im) * CS(A[ht][20].im));
      s += CS(16) * (CS(A[ht][18].re) * CS(A[ht][21].re) + CS(A[ht][18].im) * CS(A[ht][21].im));
      s += CS(16) * (CS(A[ht][18].re) * CS(A[ht][22].re) + CS(A[ht][18].im) * CS(A[ht][22].im));
      s += CS(160) * (CS(A[ht][18].re) * CS(A[ht][23].re) + CS(A[ht][18].im) * CS(A[ht][23].im));
      s += CS(16) * (CS(A[ht][19].re) * CS(A[ht][20].re) + CS(A[ht][19].im) * CS(A[ht][20].im));
      s += CS(160) * (CS(A[ht][19].re) * CS(A[ht][21].re) + CS(A[ht][19].im) * CS(A[ht][21].im));
      s += CS(-128) * (CS(A[ht][19].re) * CS(A[ht][22].re) + CS(A[ht][19].im) * CS(A[ht][22].im));
      s += CS(16) * (CS(A[ht][19].re) * CS(A[ht][23].re) + CS(A[ht][19].im) * CS(A[ht][23].im));
      s += CS(-128) * (CS(A[ht][20].re) * CS(A[ht][21].re) + CS(A[ht][20].im) * CS(A[ht][21].im));
      s += CS(160) * (CS(A[ht][20].re) * CS(A[ht][22].re) + CS(A[ht][20].im) * CS(A[ht][22].im));
      s += CS(16) * (CS(A[ht][20].re) * CS(A[ht][23].re) + CS(A[ht][20].im) * CS(A[ht][23].im));
      s += CS(16) * (CS(A[ht][21].re) * CS(A[ht][22].re) + CS(A[ht][21].im) * CS(A[ht][22].im));
      s += CS(-128) * (CS(A[ht][21].re) * CS(A[ht][23].re) + CS(A[ht][21].im) * CS(A[ht][23].im));
      s += CS(-128) * (CS(A[ht][22].re) * CS(A[ht][23].re) + CS(A[ht][22].im) * CS(A[ht][23].im));
      total += ACC(s);
    }
  }
  return total;
}

}  // namespace rex
