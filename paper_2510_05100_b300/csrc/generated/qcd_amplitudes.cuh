// Colour-ordered Berends-Giele amplitudes for g g -> t t~ + k g (k = 0, 1, 2).
// Generated by paper_2510_05100_b300/codegen/qcd_bg.py (python -m
// paper_2510_05100_b300.codegen); do not edit.
//
// Per process: <name>_event (event-level data, filled once per event),
// <name>_mass (per event and mass slot), <name>_gluons (gluon currents of one
// polarisation configuration) and the routines that fill them, then
// <name>_quark_line: jamps and their colour form summed over top helicities.
#pragma once
#include <type_traits>

#include "../helas.cuh"

namespace rex {

// marker: no replacement colour form (use the scalar quadratic form)
struct NoColourForm {};

// ---- gg_ttx: g g -> t t~ + 0 g, 2 gluons, 2 colour flows
struct gg_ttx_info {
  static constexpr int NGLUON = 2;
  static constexpr int NFLOW = 2;
  static constexpr int NGHEL = 4;
  static constexpr int COLOUR_DEN = 3;
  static constexpr int NSUFFIX = 2;   // gluon sets absorbed on the antitop side
  static constexpr int NGSET = 1;      // gluon sets of two or more (internal gluons)
};

// exact flow colour matrix C = gg_ttx_colour / 3; flows (top end first):
//   flow 0: (0, 1)
//   flow 1: (1, 0)
constexpr int gg_ttx_colour[2][2] = {
  {16, -2},
  {-2, 16},
};
#if defined(__CUDACC__)
// device copy for lane-indexed reads (tensor-core colour form)
__constant__ int gg_ttx_colour_dev[2][2] = {
  {16, -2},
  {-2, 16},
};
#endif

// gluon sets (internal gluon lines): 0={01}
// suffix sets (off-shell antitop lines): 0={0}, 1={1}
template <typename R>
struct gg_ttx_event {
  R praw[16];     // particle momenta converted to R
  double dd[6];  // FP64 dot products of (pg_0..pg_1, p_tbar)
  R pg[2][4];          // outgoing-convention gluon momenta (incoming: -k)
  R pt[4], ptb[4];       // top, antitop
  R ps[1][4];        // momentum sum of each gluon set
  R fg[1];           // -1 / P^2 of each gluon set (P^2 in FP64)
  R q[2][4];        // -(p_tbar + P) of each suffix set
  double q2[2];     // q^2 in FP64 (the exact mode's mass slot subtracts m^2 in FP64)
  R qm[2];          // q^2 - m0^2 (FP64, then R): the mixed mode's slot adds m0^2 - m^2 in R
  cx<R> cht[2][2], chb[2][2];   // helicity 2-spinors chi-, chi+ of top / antitop
  R wpt, iwpt, wptb, iwptb;     // omega_+ and 1/omega_+ of top / antitop
};

template <typename R>
struct gg_ttx_mass {   // one (event, mass slot), shared memory
  cx<R> ut[2][4];        // u(p_t) for top helicity -, +
  cx<R> v[2][4];         // v(p_tbar) for antitop helicity -, +
  R idr[2], idi[2];   // 1/(q^2 - m^2 + i m Gamma), real and imaginary parts
  R m;
};

template <typename R>
struct gg_ttx_gluons {   // colour-ordered gluon currents of one polarisation configuration
  R J0[4];
  R J1[4];
  R J01[4];
};

// Event setup, phase 1, run by every lane l of nl lanes of the event: convert the
// FP64 momenta p (global, [npart][4], rows g g t t~ g..) to R and form the FP64
// dot products of the outgoing-convention vectors.  The invariants that cancel for
// soft or collinear gluons are built from these FP64 products.
template <typename R>
__device__ __forceinline__ void gg_ttx_event_phase1(const double* __restrict__ p, gg_ttx_event<R>& ev, int l, int nl) {
  for (int i = l; i < 16; i += nl) ev.praw[i] = to_r<R>(__ldg(p + i));
  for (int k = l; k < 6; k += nl) {
    int a = 0, b = 0;
    switch (k) {
      case 0: a = 0; b = 0; break;
      case 1: a = 0; b = 1; break;
      case 2: a = 0; b = 2; break;
      case 3: a = 1; b = 1; break;
      case 4: a = 1; b = 2; break;
      case 5: a = 2; b = 2; break;
    }
    // vector index -> (row, sign): gluons 0, 1 are incoming (-k), the antitop is row 3
    const int ra = a == 2 ? 3 : (a < 2 ? a : a + 2), rb = b == 2 ? 3 : (b < 2 ? b : b + 2);
    const double sa = (a < 2) ? -1.0 : 1.0, sb = (b < 2) ? -1.0 : 1.0;
    const double* x = p + 4 * ra;
    const double* y = p + 4 * rb;
    ev.dd[k] = sa * sb * (__ldg(x) * __ldg(y) - __ldg(x + 1) * __ldg(y + 1) - __ldg(x + 2) * __ldg(y + 2) - __ldg(x + 3) * __ldg(y + 3));
  }
}

// Event setup, phase 2 (after a barrier): lanes form the FP64 invariants (q^2 also
// less m02, the square of the launch's reference mass); lane 0 builds the R-typed
// vectors and the top/antitop spinor bases.
template <typename R>
__device__ __forceinline__ void gg_ttx_event_phase2(gg_ttx_event<R>& ev, double m02, int l, int nl) {
  for (int k = l; k < 3; k += nl) {
    switch (k) {
      case 0: ev.fg[0] = R(-1) / to_r<R>(ev.dd[0] + ev.dd[3] + 2.0 * ev.dd[1]); break;
      case 1: ev.q2[0] = ev.dd[0] + ev.dd[5] + 2.0 * ev.dd[2]; ev.qm[0] = to_r<R>(ev.q2[0] - m02); break;
      case 2: ev.q2[1] = ev.dd[3] + ev.dd[5] + 2.0 * ev.dd[4]; ev.qm[1] = to_r<R>(ev.q2[1] - m02); break;
    }
  }
  if (l == 0) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      ev.pg[0][m] = -ev.praw[0 + m];
      ev.pg[1][m] = -ev.praw[4 + m];
      ev.pt[m] = ev.praw[8 + m];
      ev.ptb[m] = ev.praw[12 + m];
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.ps[0][m] = ev.pg[0][m] + ev.pg[1][m];
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.q[0][m] = -(ev.ptb[m] + ev.pg[0][m]);
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.q[1][m] = -(ev.ptb[m] + ev.pg[1][m]);
    R pabs;
    omegas(ev.pt, R(0), &pabs, &ev.wpt, &ev.iwpt);
    ev.iwpt = R(1) / ev.wpt;
    chi_pair(ev.pt, pabs, ev.cht[1], ev.cht[0]);
    omegas(ev.ptb, R(0), &pabs, &ev.wptb, &ev.iwptb);
    ev.iwptb = R(1) / ev.wptb;
    chi_pair(ev.ptb, pabs, ev.chb[1], ev.chb[0]);
  }
}

// Per (event, mass), run by every lane l of nl: inverse propagator denominators,
// q^2 - m^2 in FP64 in the exact mode; in the mixed mode (R = float) (q^2 - m0^2) +
// (m0^2 - m^2) in R with dm2 = m0^2 - m^2 from the launch's slot table, so the slot
// loop issues no FP64 instruction (exact at the reference mass, where dm2 = 0, and
// free of cancellation elsewhere); lane 0 builds the top spinors.
template <typename R, bool WIDTH>
__device__ __forceinline__ void gg_ttx_mass_setup(const gg_ttx_event<R>& ev, double mt, double wt, R dm2, gg_ttx_mass<R>& mm, int l, int nl) {
  constexpr bool F32 = std::is_same<R, float>::value;
  const double m2 = mt * mt;
  const R mw = F32 ? to_r<R>(mt) * to_r<R>(wt) : R(mt * wt);
  for (int i = l; i < 2; i += nl) {
    const R d = F32 ? ev.qm[i] + dm2 : R(ev.q2[i] - m2);
    if (WIDTH) { const R nn = R(1) / (d * d + mw * mw); mm.idr[i] = d * nn; mm.idi[i] = -mw * nn; }
    else { mm.idr[i] = R(1) / d; mm.idi[i] = R(0); }
  }
  if (l == 0) {
    const R mr = to_r<R>(mt);
    mm.m = mr;
    spinor_u_from(ev.cht, ev.wpt, mr * ev.iwpt, mm.ut);
    spinor_v_from(ev.chb, ev.wptb, mr * ev.iwptb, mm.v);
  }
}

// colour-ordered gluon currents for one polarisation configuration (mass independent)
template <typename R>
__device__ __forceinline__ void gg_ttx_gluon_currents(const gg_ttx_event<R>& ev, const R (&eps)[2][4], gg_ttx_gluons<R>& J) {
#pragma unroll
  for (int m = 0; m < 4; ++m) J.J0[m] = eps[0][m];
#pragma unroll
  for (int m = 0; m < 4; ++m) J.J1[m] = eps[1][m];
  {  // J(0,1)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J0, ev.pg[0], J.J1, ev.pg[1], t);
    const R f = ev.fg[0];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J01[m] = f * t[m];
  }
}

// sum over top helicities and antitop helicities hb in [hb_lo, hb_hi) (0: -, 1: +) of
// sum_{s,s'} conj(A_s) Cint_{ss'} A_s' (Cint = C * COLOUR_DEN).  The antitop-side
// currents psi(Y) are emitted depth-first over suffixes Y, so only one per depth is live.
// The colour form of one helicity is evaluated in CS, the helicity sum in ACC.
// FORM, if given, replaces the scalar colour form: form(A) returns this lane's
// contribution for both top helicities (e.g. the tensor-core form).
template <typename R, typename ACC, bool WIDTH, typename CS = ACC, typename FORM = NoColourForm>
__device__ __forceinline__ ACC gg_ttx_quark_line(const gg_ttx_event<R>& ev, const gg_ttx_mass<R>& mm, const gg_ttx_gluons<R>& J, int hb_lo = 0, int hb_hi = 2, const FORM& form = FORM()) {
  ACC total = ACC(0);
#pragma unroll 1
  for (int hb = hb_lo; hb < hb_hi; ++hb) {
    const cx<R>* v = mm.v[hb];
    cx<R> A[2][2];
    {
      cx<R> psi0[4];
      {
        cx<R> t[4] = {};
        slash_acc(R(1), J.J0, v, t);
        if (WIDTH) fermion_prop(ev.q[0], mm.m, cx<R>{mm.idr[0], mm.idi[0]}, t, psi0);
        else fermion_prop_real(ev.q[0], mm.m, mm.idr[0], t, psi0);
      }
      {  // flow 1 = (1, 0)
        cx<R> x[4] = {};
        slash_acc(R(1), J.J1, psi0, x);
        slash_acc(R(-1), J.J01, v, x);
        A[0][1] = ubar_dot(mm.ut[0], x);
        A[1][1] = ubar_dot(mm.ut[1], x);
      }
    }
    {
      cx<R> psi1[4];
      {
        cx<R> t[4] = {};
        slash_acc(R(1), J.J1, v, t);
        if (WIDTH) fermion_prop(ev.q[1], mm.m, cx<R>{mm.idr[1], mm.idi[1]}, t, psi1);
        else fermion_prop_real(ev.q[1], mm.m, mm.idr[1], t, psi1);
      }
      {  // flow 0 = (0, 1)
        cx<R> x[4] = {};
        slash_acc(R(1), J.J0, psi1, x);
        slash_acc(R(1), J.J01, v, x);
        A[0][0] = ubar_dot(mm.ut[0], x);
        A[1][0] = ubar_dot(mm.ut[1], x);
      }
    }
    if constexpr (!std::is_same<FORM, NoColourForm>::value) {
      total += ACC(form(A));
    } else {
#pragma unroll
    for (int ht = 0; ht < 2; ++ht) {
      CS s = CS(0);
      s += CS(16) * (CS(A[ht][0].re) * CS(A[ht][0].re) + CS(A[ht][0].im) * CS(A[ht][0].im));
      s += CS(16) * (CS(A[ht][1].re) * CS(A[ht][1].re) + CS(A[ht][1].im) * CS(A[ht][1].im));
      s += CS(-4) * (CS(A[ht][0].re) * CS(A[ht][1].re) + CS(A[ht][0].im) * CS(A[ht][1].im));
      total += ACC(s);
    }
    }
  }
  return total;
}

// ---- gg_ttxg: g g -> t t~ + 1 g, 3 gluons, 6 colour flows
struct gg_ttxg_info {
  static constexpr int NGLUON = 3;
  static constexpr int NFLOW = 6;
  static constexpr int NGHEL = 8;
  static constexpr int COLOUR_DEN = 9;
  static constexpr int NSUFFIX = 6;   // gluon sets absorbed on the antitop side
  static constexpr int NGSET = 4;      // gluon sets of two or more (internal gluons)
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
#if defined(__CUDACC__)
// device copy for lane-indexed reads (tensor-core colour form)
__constant__ int gg_ttxg_colour_dev[6][6] = {
  {64, -8, -8, 1, 1, 10},
  {-8, 64, 1, 10, -8, 1},
  {-8, 1, 64, -8, 10, 1},
  {1, 10, -8, 64, 1, -8},
  {1, -8, 10, 1, 64, -8},
  {10, 1, 1, -8, -8, 64},
};
#endif

// gluon sets (internal gluon lines): 0={01}, 1={02}, 2={12}, 3={012}
// suffix sets (off-shell antitop lines): 0={0}, 1={1}, 2={2}, 3={01}, 4={02}, 5={12}
template <typename R>
struct gg_ttxg_event {
  R praw[20];     // particle momenta converted to R
  double dd[10];  // FP64 dot products of (pg_0..pg_2, p_tbar)
  R pg[3][4];          // outgoing-convention gluon momenta (incoming: -k)
  R pt[4], ptb[4];       // top, antitop
  R ps[4][4];        // momentum sum of each gluon set
  R fg[4];           // -1 / P^2 of each gluon set (P^2 in FP64)
  R q[6][4];        // -(p_tbar + P) of each suffix set
  double q2[6];     // q^2 in FP64 (the exact mode's mass slot subtracts m^2 in FP64)
  R qm[6];          // q^2 - m0^2 (FP64, then R): the mixed mode's slot adds m0^2 - m^2 in R
  cx<R> cht[2][2], chb[2][2];   // helicity 2-spinors chi-, chi+ of top / antitop
  R wpt, iwpt, wptb, iwptb;     // omega_+ and 1/omega_+ of top / antitop
};

template <typename R>
struct gg_ttxg_mass {   // one (event, mass slot), shared memory
  cx<R> ut[2][4];        // u(p_t) for top helicity -, +
  cx<R> v[2][4];         // v(p_tbar) for antitop helicity -, +
  R idr[6], idi[6];   // 1/(q^2 - m^2 + i m Gamma), real and imaginary parts
  R m;
};

template <typename R>
struct gg_ttxg_gluons {   // colour-ordered gluon currents of one polarisation configuration
  R J0[4];
  R J1[4];
  R J2[4];
  R J01[4];
  R J02[4];
  R J12[4];
  R J012[4];
  R J021[4];
  R J102[4];
};

// Event setup, phase 1, run by every lane l of nl lanes of the event: convert the
// FP64 momenta p (global, [npart][4], rows g g t t~ g..) to R and form the FP64
// dot products of the outgoing-convention vectors.  The invariants that cancel for
// soft or collinear gluons are built from these FP64 products.
template <typename R>
__device__ __forceinline__ void gg_ttxg_event_phase1(const double* __restrict__ p, gg_ttxg_event<R>& ev, int l, int nl) {
  for (int i = l; i < 20; i += nl) ev.praw[i] = to_r<R>(__ldg(p + i));
  for (int k = l; k < 10; k += nl) {
    int a = 0, b = 0;
    switch (k) {
      case 0: a = 0; b = 0; break;
      case 1: a = 0; b = 1; break;
      case 2: a = 0; b = 2; break;
      case 3: a = 0; b = 3; break;
      case 4: a = 1; b = 1; break;
      case 5: a = 1; b = 2; break;
      case 6: a = 1; b = 3; break;
      case 7: a = 2; b = 2; break;
      case 8: a = 2; b = 3; break;
      case 9: a = 3; b = 3; break;
    }
    // vector index -> (row, sign): gluons 0, 1 are incoming (-k), the antitop is row 3
    const int ra = a == 3 ? 3 : (a < 2 ? a : a + 2), rb = b == 3 ? 3 : (b < 2 ? b : b + 2);
    const double sa = (a < 2) ? -1.0 : 1.0, sb = (b < 2) ? -1.0 : 1.0;
    const double* x = p + 4 * ra;
    const double* y = p + 4 * rb;
    ev.dd[k] = sa * sb * (__ldg(x) * __ldg(y) - __ldg(x + 1) * __ldg(y + 1) - __ldg(x + 2) * __ldg(y + 2) - __ldg(x + 3) * __ldg(y + 3));
  }
}

// Event setup, phase 2 (after a barrier): lanes form the FP64 invariants (q^2 also
// less m02, the square of the launch's reference mass); lane 0 builds the R-typed
// vectors and the top/antitop spinor bases.
template <typename R>
__device__ __forceinline__ void gg_ttxg_event_phase2(gg_ttxg_event<R>& ev, double m02, int l, int nl) {
  for (int k = l; k < 10; k += nl) {
    switch (k) {
      case 0: ev.fg[0] = R(-1) / to_r<R>(ev.dd[0] + ev.dd[4] + 2.0 * ev.dd[1]); break;
      case 1: ev.fg[1] = R(-1) / to_r<R>(ev.dd[0] + ev.dd[7] + 2.0 * ev.dd[2]); break;
      case 2: ev.fg[2] = R(-1) / to_r<R>(ev.dd[4] + ev.dd[7] + 2.0 * ev.dd[5]); break;
      case 3: ev.fg[3] = R(-1) / to_r<R>(ev.dd[0] + ev.dd[4] + ev.dd[7] + 2.0 * ev.dd[1] + 2.0 * ev.dd[2] + 2.0 * ev.dd[5]); break;
      case 4: ev.q2[0] = ev.dd[0] + ev.dd[9] + 2.0 * ev.dd[3]; ev.qm[0] = to_r<R>(ev.q2[0] - m02); break;
      case 5: ev.q2[1] = ev.dd[4] + ev.dd[9] + 2.0 * ev.dd[6]; ev.qm[1] = to_r<R>(ev.q2[1] - m02); break;
      case 6: ev.q2[2] = ev.dd[7] + ev.dd[9] + 2.0 * ev.dd[8]; ev.qm[2] = to_r<R>(ev.q2[2] - m02); break;
      case 7: ev.q2[3] = ev.dd[0] + ev.dd[4] + ev.dd[9] + 2.0 * ev.dd[1] + 2.0 * ev.dd[3] + 2.0 * ev.dd[6]; ev.qm[3] = to_r<R>(ev.q2[3] - m02); break;
      case 8: ev.q2[4] = ev.dd[0] + ev.dd[7] + ev.dd[9] + 2.0 * ev.dd[2] + 2.0 * ev.dd[3] + 2.0 * ev.dd[8]; ev.qm[4] = to_r<R>(ev.q2[4] - m02); break;
      case 9: ev.q2[5] = ev.dd[4] + ev.dd[7] + ev.dd[9] + 2.0 * ev.dd[5] + 2.0 * ev.dd[6] + 2.0 * ev.dd[8]; ev.qm[5] = to_r<R>(ev.q2[5] - m02); break;
    }
  }
  if (l == 0) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      ev.pg[0][m] = -ev.praw[0 + m];
      ev.pg[1][m] = -ev.praw[4 + m];
      ev.pg[2][m] = ev.praw[16 + m];
      ev.pt[m] = ev.praw[8 + m];
      ev.ptb[m] = ev.praw[12 + m];
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.ps[0][m] = ev.pg[0][m] + ev.pg[1][m];
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.ps[1][m] = ev.pg[0][m] + ev.pg[2][m];
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.ps[2][m] = ev.pg[1][m] + ev.pg[2][m];
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.ps[3][m] = ev.pg[0][m] + ev.pg[1][m] + ev.pg[2][m];
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.q[0][m] = -(ev.ptb[m] + ev.pg[0][m]);
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.q[1][m] = -(ev.ptb[m] + ev.pg[1][m]);
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.q[2][m] = -(ev.ptb[m] + ev.pg[2][m]);
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.q[3][m] = -(ev.ptb[m] + ev.pg[0][m] + ev.pg[1][m]);
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.q[4][m] = -(ev.ptb[m] + ev.pg[0][m] + ev.pg[2][m]);
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.q[5][m] = -(ev.ptb[m] + ev.pg[1][m] + ev.pg[2][m]);
    R pabs;
    omegas(ev.pt, R(0), &pabs, &ev.wpt, &ev.iwpt);
    ev.iwpt = R(1) / ev.wpt;
    chi_pair(ev.pt, pabs, ev.cht[1], ev.cht[0]);
    omegas(ev.ptb, R(0), &pabs, &ev.wptb, &ev.iwptb);
    ev.iwptb = R(1) / ev.wptb;
    chi_pair(ev.ptb, pabs, ev.chb[1], ev.chb[0]);
  }
}

// Per (event, mass), run by every lane l of nl: inverse propagator denominators,
// q^2 - m^2 in FP64 in the exact mode; in the mixed mode (R = float) (q^2 - m0^2) +
// (m0^2 - m^2) in R with dm2 = m0^2 - m^2 from the launch's slot table, so the slot
// loop issues no FP64 instruction (exact at the reference mass, where dm2 = 0, and
// free of cancellation elsewhere); lane 0 builds the top spinors.
template <typename R, bool WIDTH>
__device__ __forceinline__ void gg_ttxg_mass_setup(const gg_ttxg_event<R>& ev, double mt, double wt, R dm2, gg_ttxg_mass<R>& mm, int l, int nl) {
  constexpr bool F32 = std::is_same<R, float>::value;
  const double m2 = mt * mt;
  const R mw = F32 ? to_r<R>(mt) * to_r<R>(wt) : R(mt * wt);
  for (int i = l; i < 6; i += nl) {
    const R d = F32 ? ev.qm[i] + dm2 : R(ev.q2[i] - m2);
    if (WIDTH) { const R nn = R(1) / (d * d + mw * mw); mm.idr[i] = d * nn; mm.idi[i] = -mw * nn; }
    else { mm.idr[i] = R(1) / d; mm.idi[i] = R(0); }
  }
  if (l == 0) {
    const R mr = to_r<R>(mt);
    mm.m = mr;
    spinor_u_from(ev.cht, ev.wpt, mr * ev.iwpt, mm.ut);
    spinor_v_from(ev.chb, ev.wptb, mr * ev.iwptb, mm.v);
  }
}

// colour-ordered gluon currents for one polarisation configuration (mass independent)
template <typename R>
__device__ __forceinline__ void gg_ttxg_gluon_currents(const gg_ttxg_event<R>& ev, const R (&eps)[3][4], gg_ttxg_gluons<R>& J) {
#pragma unroll
  for (int m = 0; m < 4; ++m) J.J0[m] = eps[0][m];
#pragma unroll
  for (int m = 0; m < 4; ++m) J.J1[m] = eps[1][m];
#pragma unroll
  for (int m = 0; m < 4; ++m) J.J2[m] = eps[2][m];
  {  // J(0,1)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J0, ev.pg[0], J.J1, ev.pg[1], t);
    const R f = ev.fg[0];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J01[m] = f * t[m];
  }
  {  // J(0,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J0, ev.pg[0], J.J2, ev.pg[2], t);
    const R f = ev.fg[1];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J02[m] = f * t[m];
  }
  {  // J(1,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J1, ev.pg[1], J.J2, ev.pg[2], t);
    const R f = ev.fg[2];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J12[m] = f * t[m];
  }
  {  // J(0,1,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J0, ev.pg[0], J.J12, ev.ps[2], t);
    vvv_acc(R(1), J.J01, ev.ps[0], J.J2, ev.pg[2], t);
    vvvv_acc(R(1), J.J0, J.J1, J.J2, t);
    const R f = ev.fg[3];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J012[m] = f * t[m];
  }
  {  // J(0,2,1)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(-1), J.J0, ev.pg[0], J.J12, ev.ps[2], t);
    vvv_acc(R(1), J.J02, ev.ps[1], J.J1, ev.pg[1], t);
    vvvv_acc(R(1), J.J0, J.J2, J.J1, t);
    const R f = ev.fg[3];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J021[m] = f * t[m];
  }
  {  // J(1,0,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J1, ev.pg[1], J.J02, ev.ps[1], t);
    vvv_acc(R(-1), J.J01, ev.ps[0], J.J2, ev.pg[2], t);
    vvvv_acc(R(1), J.J1, J.J0, J.J2, t);
    const R f = ev.fg[3];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J102[m] = f * t[m];
  }
}

// sum over top helicities and antitop helicities hb in [hb_lo, hb_hi) (0: -, 1: +) of
// sum_{s,s'} conj(A_s) Cint_{ss'} A_s' (Cint = C * COLOUR_DEN).  The antitop-side
// currents psi(Y) are emitted depth-first over suffixes Y, so only one per depth is live.
// The colour form of one helicity is evaluated in CS, the helicity sum in ACC.
// FORM, if given, replaces the scalar colour form: form(A) returns this lane's
// contribution for both top helicities (e.g. the tensor-core form).
template <typename R, typename ACC, bool WIDTH, typename CS = ACC, typename FORM = NoColourForm>
__device__ __forceinline__ ACC gg_ttxg_quark_line(const gg_ttxg_event<R>& ev, const gg_ttxg_mass<R>& mm, const gg_ttxg_gluons<R>& J, int hb_lo = 0, int hb_hi = 2, const FORM& form = FORM()) {
  ACC total = ACC(0);
#pragma unroll 1
  for (int hb = hb_lo; hb < hb_hi; ++hb) {
    const cx<R>* v = mm.v[hb];
    cx<R> A[2][6];
    {
      cx<R> psi0[4];
      {
        cx<R> t[4] = {};
        slash_acc(R(1), J.J0, v, t);
        if (WIDTH) fermion_prop(ev.q[0], mm.m, cx<R>{mm.idr[0], mm.idi[0]}, t, psi0);
        else fermion_prop_real(ev.q[0], mm.m, mm.idr[0], t, psi0);
      }
      {
        cx<R> psi10[4];
        {
          cx<R> t[4] = {};
          slash_acc(R(1), J.J1, psi0, t);
          slash_acc(R(-1), J.J01, v, t);
          if (WIDTH) fermion_prop(ev.q[3], mm.m, cx<R>{mm.idr[3], mm.idi[3]}, t, psi10);
          else fermion_prop_real(ev.q[3], mm.m, mm.idr[3], t, psi10);
        }
        {  // flow 5 = (2, 1, 0)
          cx<R> x[4] = {};
          slash_acc(R(1), J.J2, psi10, x);
          slash_acc(R(-1), J.J12, psi0, x);
          slash_acc(R(1), J.J012, v, x);
          A[0][5] = ubar_dot(mm.ut[0], x);
          A[1][5] = ubar_dot(mm.ut[1], x);
        }
      }
      {
        cx<R> psi20[4];
        {
          cx<R> t[4] = {};
          slash_acc(R(1), J.J2, psi0, t);
          slash_acc(R(-1), J.J02, v, t);
          if (WIDTH) fermion_prop(ev.q[4], mm.m, cx<R>{mm.idr[4], mm.idi[4]}, t, psi20);
          else fermion_prop_real(ev.q[4], mm.m, mm.idr[4], t, psi20);
        }
        {  // flow 3 = (1, 2, 0)
          cx<R> x[4] = {};
          slash_acc(R(1), J.J1, psi20, x);
          slash_acc(R(1), J.J12, psi0, x);
          slash_acc(R(1), J.J021, v, x);
          A[0][3] = ubar_dot(mm.ut[0], x);
          A[1][3] = ubar_dot(mm.ut[1], x);
        }
      }
    }
    {
      cx<R> psi1[4];
      {
        cx<R> t[4] = {};
        slash_acc(R(1), J.J1, v, t);
        if (WIDTH) fermion_prop(ev.q[1], mm.m, cx<R>{mm.idr[1], mm.idi[1]}, t, psi1);
        else fermion_prop_real(ev.q[1], mm.m, mm.idr[1], t, psi1);
      }
      {
        cx<R> psi01[4];
        {
          cx<R> t[4] = {};
          slash_acc(R(1), J.J0, psi1, t);
          slash_acc(R(1), J.J01, v, t);
          if (WIDTH) fermion_prop(ev.q[3], mm.m, cx<R>{mm.idr[3], mm.idi[3]}, t, psi01);
          else fermion_prop_real(ev.q[3], mm.m, mm.idr[3], t, psi01);
        }
        {  // flow 4 = (2, 0, 1)
          cx<R> x[4] = {};
          slash_acc(R(1), J.J2, psi01, x);
          slash_acc(R(-1), J.J02, psi1, x);
          slash_acc(R(1), J.J102, v, x);
          A[0][4] = ubar_dot(mm.ut[0], x);
          A[1][4] = ubar_dot(mm.ut[1], x);
        }
      }
      {
        cx<R> psi21[4];
        {
          cx<R> t[4] = {};
          slash_acc(R(1), J.J2, psi1, t);
          slash_acc(R(-1), J.J12, v, t);
          if (WIDTH) fermion_prop(ev.q[5], mm.m, cx<R>{mm.idr[5], mm.idi[5]}, t, psi21);
          else fermion_prop_real(ev.q[5], mm.m, mm.idr[5], t, psi21);
        }
        {  // flow 1 = (0, 2, 1)
          cx<R> x[4] = {};
          slash_acc(R(1), J.J0, psi21, x);
          slash_acc(R(1), J.J02, psi1, x);
          slash_acc(R(1), J.J021, v, x);
          A[0][1] = ubar_dot(mm.ut[0], x);
          A[1][1] = ubar_dot(mm.ut[1], x);
        }
      }
    }
    {
      cx<R> psi2[4];
      {
        cx<R> t[4] = {};
        slash_acc(R(1), J.J2, v, t);
        if (WIDTH) fermion_prop(ev.q[2], mm.m, cx<R>{mm.idr[2], mm.idi[2]}, t, psi2);
        else fermion_prop_real(ev.q[2], mm.m, mm.idr[2], t, psi2);
      }
      {
        cx<R> psi02[4];
        {
          cx<R> t[4] = {};
          slash_acc(R(1), J.J0, psi2, t);
          slash_acc(R(1), J.J02, v, t);
          if (WIDTH) fermion_prop(ev.q[4], mm.m, cx<R>{mm.idr[4], mm.idi[4]}, t, psi02);
          else fermion_prop_real(ev.q[4], mm.m, mm.idr[4], t, psi02);
        }
        {  // flow 2 = (1, 0, 2)
          cx<R> x[4] = {};
          slash_acc(R(1), J.J1, psi02, x);
          slash_acc(R(-1), J.J01, psi2, x);
          slash_acc(R(1), J.J102, v, x);
          A[0][2] = ubar_dot(mm.ut[0], x);
          A[1][2] = ubar_dot(mm.ut[1], x);
        }
      }
      {
        cx<R> psi12[4];
        {
          cx<R> t[4] = {};
          slash_acc(R(1), J.J1, psi2, t);
          slash_acc(R(1), J.J12, v, t);
          if (WIDTH) fermion_prop(ev.q[5], mm.m, cx<R>{mm.idr[5], mm.idi[5]}, t, psi12);
          else fermion_prop_real(ev.q[5], mm.m, mm.idr[5], t, psi12);
        }
        {  // flow 0 = (0, 1, 2)
          cx<R> x[4] = {};
          slash_acc(R(1), J.J0, psi12, x);
          slash_acc(R(1), J.J01, psi2, x);
          slash_acc(R(1), J.J012, v, x);
          A[0][0] = ubar_dot(mm.ut[0], x);
          A[1][0] = ubar_dot(mm.ut[1], x);
        }
      }
    }
    if constexpr (!std::is_same<FORM, NoColourForm>::value) {
      total += ACC(form(A));
    } else {
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
  }
  return total;
}

// ---- gg_ttxgg: g g -> t t~ + 2 g, 4 gluons, 24 colour flows
struct gg_ttxgg_info {
  static constexpr int NGLUON = 4;
  static constexpr int NFLOW = 24;
  static constexpr int NGHEL = 16;
  static constexpr int COLOUR_DEN = 54;
  static constexpr int NSUFFIX = 14;   // gluon sets absorbed on the antitop side
  static constexpr int NGSET = 11;      // gluon sets of two or more (internal gluons)
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
#if defined(__CUDACC__)
// device copy for lane-indexed reads (tensor-core colour form)
__constant__ int gg_ttxgg_colour_dev[24][24] = {
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
#endif

// gluon sets (internal gluon lines): 0={01}, 1={02}, 2={03}, 3={12}, 4={13}, 5={23}, 6={012}, 7={013}, 8={023}, 9={123}, 10={0123}
// suffix sets (off-shell antitop lines): 0={0}, 1={1}, 2={2}, 3={3}, 4={01}, 5={02}, 6={03}, 7={12}, 8={13}, 9={23}, 10={012}, 11={013}, 12={023}, 13={123}
template <typename R>
struct gg_ttxgg_event {
  R praw[24];     // particle momenta converted to R
  double dd[15];  // FP64 dot products of (pg_0..pg_3, p_tbar)
  R pg[4][4];          // outgoing-convention gluon momenta (incoming: -k)
  R pt[4], ptb[4];       // top, antitop
  R ps[11][4];        // momentum sum of each gluon set
  R fg[11];           // -1 / P^2 of each gluon set (P^2 in FP64)
  R q[14][4];        // -(p_tbar + P) of each suffix set
  double q2[14];     // q^2 in FP64 (the exact mode's mass slot subtracts m^2 in FP64)
  R qm[14];          // q^2 - m0^2 (FP64, then R): the mixed mode's slot adds m0^2 - m^2 in R
  cx<R> cht[2][2], chb[2][2];   // helicity 2-spinors chi-, chi+ of top / antitop
  R wpt, iwpt, wptb, iwptb;     // omega_+ and 1/omega_+ of top / antitop
};

template <typename R>
struct gg_ttxgg_mass {   // one (event, mass slot), shared memory
  cx<R> ut[2][4];        // u(p_t) for top helicity -, +
  cx<R> v[2][4];         // v(p_tbar) for antitop helicity -, +
  R idr[14], idi[14];   // 1/(q^2 - m^2 + i m Gamma), real and imaginary parts
  R m;
};

template <typename R>
struct gg_ttxgg_gluons {   // colour-ordered gluon currents of one polarisation configuration
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
};

// Event setup, phase 1, run by every lane l of nl lanes of the event: convert the
// FP64 momenta p (global, [npart][4], rows g g t t~ g..) to R and form the FP64
// dot products of the outgoing-convention vectors.  The invariants that cancel for
// soft or collinear gluons are built from these FP64 products.
template <typename R>
__device__ __forceinline__ void gg_ttxgg_event_phase1(const double* __restrict__ p, gg_ttxgg_event<R>& ev, int l, int nl) {
  for (int i = l; i < 24; i += nl) ev.praw[i] = to_r<R>(__ldg(p + i));
  for (int k = l; k < 15; k += nl) {
    int a = 0, b = 0;
    switch (k) {
      case 0: a = 0; b = 0; break;
      case 1: a = 0; b = 1; break;
      case 2: a = 0; b = 2; break;
      case 3: a = 0; b = 3; break;
      case 4: a = 0; b = 4; break;
      case 5: a = 1; b = 1; break;
      case 6: a = 1; b = 2; break;
      case 7: a = 1; b = 3; break;
      case 8: a = 1; b = 4; break;
      case 9: a = 2; b = 2; break;
      case 10: a = 2; b = 3; break;
      case 11: a = 2; b = 4; break;
      case 12: a = 3; b = 3; break;
      case 13: a = 3; b = 4; break;
      case 14: a = 4; b = 4; break;
    }
    // vector index -> (row, sign): gluons 0, 1 are incoming (-k), the antitop is row 3
    const int ra = a == 4 ? 3 : (a < 2 ? a : a + 2), rb = b == 4 ? 3 : (b < 2 ? b : b + 2);
    const double sa = (a < 2) ? -1.0 : 1.0, sb = (b < 2) ? -1.0 : 1.0;
    const double* x = p + 4 * ra;
    const double* y = p + 4 * rb;
    ev.dd[k] = sa * sb * (__ldg(x) * __ldg(y) - __ldg(x + 1) * __ldg(y + 1) - __ldg(x + 2) * __ldg(y + 2) - __ldg(x + 3) * __ldg(y + 3));
  }
}

// Event setup, phase 2 (after a barrier): lanes form the FP64 invariants (q^2 also
// less m02, the square of the launch's reference mass); lane 0 builds the R-typed
// vectors and the top/antitop spinor bases.
template <typename R>
__device__ __forceinline__ void gg_ttxgg_event_phase2(gg_ttxgg_event<R>& ev, double m02, int l, int nl) {
  for (int k = l; k < 25; k += nl) {
    switch (k) {
      case 0: ev.fg[0] = R(-1) / to_r<R>(ev.dd[0] + ev.dd[5] + 2.0 * ev.dd[1]); break;
      case 1: ev.fg[1] = R(-1) / to_r<R>(ev.dd[0] + ev.dd[9] + 2.0 * ev.dd[2]); break;
      case 2: ev.fg[2] = R(-1) / to_r<R>(ev.dd[0] + ev.dd[12] + 2.0 * ev.dd[3]); break;
      case 3: ev.fg[3] = R(-1) / to_r<R>(ev.dd[5] + ev.dd[9] + 2.0 * ev.dd[6]); break;
      case 4: ev.fg[4] = R(-1) / to_r<R>(ev.dd[5] + ev.dd[12] + 2.0 * ev.dd[7]); break;
      case 5: ev.fg[5] = R(-1) / to_r<R>(ev.dd[9] + ev.dd[12] + 2.0 * ev.dd[10]); break;
      case 6: ev.fg[6] = R(-1) / to_r<R>(ev.dd[0] + ev.dd[5] + ev.dd[9] + 2.0 * ev.dd[1] + 2.0 * ev.dd[2] + 2.0 * ev.dd[6]); break;
      case 7: ev.fg[7] = R(-1) / to_r<R>(ev.dd[0] + ev.dd[5] + ev.dd[12] + 2.0 * ev.dd[1] + 2.0 * ev.dd[3] + 2.0 * ev.dd[7]); break;
      case 8: ev.fg[8] = R(-1) / to_r<R>(ev.dd[0] + ev.dd[9] + ev.dd[12] + 2.0 * ev.dd[2] + 2.0 * ev.dd[3] + 2.0 * ev.dd[10]); break;
      case 9: ev.fg[9] = R(-1) / to_r<R>(ev.dd[5] + ev.dd[9] + ev.dd[12] + 2.0 * ev.dd[6] + 2.0 * ev.dd[7] + 2.0 * ev.dd[10]); break;
      case 10: ev.fg[10] = R(-1) / to_r<R>(ev.dd[0] + ev.dd[5] + ev.dd[9] + ev.dd[12] + 2.0 * ev.dd[1] + 2.0 * ev.dd[2] + 2.0 * ev.dd[3] + 2.0 * ev.dd[6] + 2.0 * ev.dd[7] + 2.0 * ev.dd[10]); break;
      case 11: ev.q2[0] = ev.dd[0] + ev.dd[14] + 2.0 * ev.dd[4]; ev.qm[0] = to_r<R>(ev.q2[0] - m02); break;
      case 12: ev.q2[1] = ev.dd[5] + ev.dd[14] + 2.0 * ev.dd[8]; ev.qm[1] = to_r<R>(ev.q2[1] - m02); break;
      case 13: ev.q2[2] = ev.dd[9] + ev.dd[14] + 2.0 * ev.dd[11]; ev.qm[2] = to_r<R>(ev.q2[2] - m02); break;
      case 14: ev.q2[3] = ev.dd[12] + ev.dd[14] + 2.0 * ev.dd[13]; ev.qm[3] = to_r<R>(ev.q2[3] - m02); break;
      case 15: ev.q2[4] = ev.dd[0] + ev.dd[5] + ev.dd[14] + 2.0 * ev.dd[1] + 2.0 * ev.dd[4] + 2.0 * ev.dd[8]; ev.qm[4] = to_r<R>(ev.q2[4] - m02); break;
      case 16: ev.q2[5] = ev.dd[0] + ev.dd[9] + ev.dd[14] + 2.0 * ev.dd[2] + 2.0 * ev.dd[4] + 2.0 * ev.dd[11]; ev.qm[5] = to_r<R>(ev.q2[5] - m02); break;
      case 17: ev.q2[6] = ev.dd[0] + ev.dd[12] + ev.dd[14] + 2.0 * ev.dd[3] + 2.0 * ev.dd[4] + 2.0 * ev.dd[13]; ev.qm[6] = to_r<R>(ev.q2[6] - m02); break;
      case 18: ev.q2[7] = ev.dd[5] + ev.dd[9] + ev.dd[14] + 2.0 * ev.dd[6] + 2.0 * ev.dd[8] + 2.0 * ev.dd[11]; ev.qm[7] = to_r<R>(ev.q2[7] - m02); break;
      case 19: ev.q2[8] = ev.dd[5] + ev.dd[12] + ev.dd[14] + 2.0 * ev.dd[7] + 2.0 * ev.dd[8] + 2.0 * ev.dd[13]; ev.qm[8] = to_r<R>(ev.q2[8] - m02); break;
      case 20: ev.q2[9] = ev.dd[9] + ev.dd[12] + ev.dd[14] + 2.0 * ev.dd[10] + 2.0 * ev.dd[11] + 2.0 * ev.dd[13]; ev.qm[9] = to_r<R>(ev.q2[9] - m02); break;
      case 21: ev.q2[10] = ev.dd[0] + ev.dd[5] + ev.dd[9] + ev.dd[14] + 2.0 * ev.dd[1] + 2.0 * ev.dd[2] + 2.0 * ev.dd[4] + 2.0 * ev.dd[6] + 2.0 * ev.dd[8] + 2.0 * ev.dd[11]; ev.qm[10] = to_r<R>(ev.q2[10] - m02); break;
      case 22: ev.q2[11] = ev.dd[0] + ev.dd[5] + ev.dd[12] + ev.dd[14] + 2.0 * ev.dd[1] + 2.0 * ev.dd[3] + 2.0 * ev.dd[4] + 2.0 * ev.dd[7] + 2.0 * ev.dd[8] + 2.0 * ev.dd[13]; ev.qm[11] = to_r<R>(ev.q2[11] - m02); break;
      case 23: ev.q2[12] = ev.dd[0] + ev.dd[9] + ev.dd[12] + ev.dd[14] + 2.0 * ev.dd[2] + 2.0 * ev.dd[3] + 2.0 * ev.dd[4] + 2.0 * ev.dd[10] + 2.0 * ev.dd[11] + 2.0 * ev.dd[13]; ev.qm[12] = to_r<R>(ev.q2[12] - m02); break;
      case 24: ev.q2[13] = ev.dd[5] + ev.dd[9] + ev.dd[12] + ev.dd[14] + 2.0 * ev.dd[6] + 2.0 * ev.dd[7] + 2.0 * ev.dd[8] + 2.0 * ev.dd[10] + 2.0 * ev.dd[11] + 2.0 * ev.dd[13]; ev.qm[13] = to_r<R>(ev.q2[13] - m02); break;
    }
  }
  if (l == 0) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      ev.pg[0][m] = -ev.praw[0 + m];
      ev.pg[1][m] = -ev.praw[4 + m];
      ev.pg[2][m] = ev.praw[16 + m];
      ev.pg[3][m] = ev.praw[20 + m];
      ev.pt[m] = ev.praw[8 + m];
      ev.ptb[m] = ev.praw[12 + m];
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.ps[0][m] = ev.pg[0][m] + ev.pg[1][m];
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.ps[1][m] = ev.pg[0][m] + ev.pg[2][m];
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.ps[2][m] = ev.pg[0][m] + ev.pg[3][m];
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.ps[3][m] = ev.pg[1][m] + ev.pg[2][m];
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.ps[4][m] = ev.pg[1][m] + ev.pg[3][m];
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.ps[5][m] = ev.pg[2][m] + ev.pg[3][m];
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.ps[6][m] = ev.pg[0][m] + ev.pg[1][m] + ev.pg[2][m];
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.ps[7][m] = ev.pg[0][m] + ev.pg[1][m] + ev.pg[3][m];
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.ps[8][m] = ev.pg[0][m] + ev.pg[2][m] + ev.pg[3][m];
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.ps[9][m] = ev.pg[1][m] + ev.pg[2][m] + ev.pg[3][m];
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.ps[10][m] = ev.pg[0][m] + ev.pg[1][m] + ev.pg[2][m] + ev.pg[3][m];
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.q[0][m] = -(ev.ptb[m] + ev.pg[0][m]);
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.q[1][m] = -(ev.ptb[m] + ev.pg[1][m]);
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.q[2][m] = -(ev.ptb[m] + ev.pg[2][m]);
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.q[3][m] = -(ev.ptb[m] + ev.pg[3][m]);
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.q[4][m] = -(ev.ptb[m] + ev.pg[0][m] + ev.pg[1][m]);
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.q[5][m] = -(ev.ptb[m] + ev.pg[0][m] + ev.pg[2][m]);
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.q[6][m] = -(ev.ptb[m] + ev.pg[0][m] + ev.pg[3][m]);
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.q[7][m] = -(ev.ptb[m] + ev.pg[1][m] + ev.pg[2][m]);
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.q[8][m] = -(ev.ptb[m] + ev.pg[1][m] + ev.pg[3][m]);
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.q[9][m] = -(ev.ptb[m] + ev.pg[2][m] + ev.pg[3][m]);
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.q[10][m] = -(ev.ptb[m] + ev.pg[0][m] + ev.pg[1][m] + ev.pg[2][m]);
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.q[11][m] = -(ev.ptb[m] + ev.pg[0][m] + ev.pg[1][m] + ev.pg[3][m]);
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.q[12][m] = -(ev.ptb[m] + ev.pg[0][m] + ev.pg[2][m] + ev.pg[3][m]);
#pragma unroll
    for (int m = 0; m < 4; ++m) ev.q[13][m] = -(ev.ptb[m] + ev.pg[1][m] + ev.pg[2][m] + ev.pg[3][m]);
    R pabs;
    omegas(ev.pt, R(0), &pabs, &ev.wpt, &ev.iwpt);
    ev.iwpt = R(1) / ev.wpt;
    chi_pair(ev.pt, pabs, ev.cht[1], ev.cht[0]);
    omegas(ev.ptb, R(0), &pabs, &ev.wptb, &ev.iwptb);
    ev.iwptb = R(1) / ev.wptb;
    chi_pair(ev.ptb, pabs, ev.chb[1], ev.chb[0]);
  }
}

// Per (event, mass), run by every lane l of nl: inverse propagator denominators,
// q^2 - m^2 in FP64 in the exact mode; in the mixed mode (R = float) (q^2 - m0^2) +
// (m0^2 - m^2) in R with dm2 = m0^2 - m^2 from the launch's slot table, so the slot
// loop issues no FP64 instruction (exact at the reference mass, where dm2 = 0, and
// free of cancellation elsewhere); lane 0 builds the top spinors.
template <typename R, bool WIDTH>
__device__ __forceinline__ void gg_ttxgg_mass_setup(const gg_ttxgg_event<R>& ev, double mt, double wt, R dm2, gg_ttxgg_mass<R>& mm, int l, int nl) {
  constexpr bool F32 = std::is_same<R, float>::value;
  const double m2 = mt * mt;
  const R mw = F32 ? to_r<R>(mt) * to_r<R>(wt) : R(mt * wt);
  for (int i = l; i < 14; i += nl) {
    const R d = F32 ? ev.qm[i] + dm2 : R(ev.q2[i] - m2);
    if (WIDTH) { const R nn = R(1) / (d * d + mw * mw); mm.idr[i] = d * nn; mm.idi[i] = -mw * nn; }
    else { mm.idr[i] = R(1) / d; mm.idi[i] = R(0); }
  }
  if (l == 0) {
    const R mr = to_r<R>(mt);
    mm.m = mr;
    spinor_u_from(ev.cht, ev.wpt, mr * ev.iwpt, mm.ut);
    spinor_v_from(ev.chb, ev.wptb, mr * ev.iwptb, mm.v);
  }
}

// colour-ordered gluon currents for one polarisation configuration (mass independent)
template <typename R>
__device__ __forceinline__ void gg_ttxgg_gluon_currents(const gg_ttxgg_event<R>& ev, const R (&eps)[4][4], gg_ttxgg_gluons<R>& J) {
#pragma unroll
  for (int m = 0; m < 4; ++m) J.J0[m] = eps[0][m];
#pragma unroll
  for (int m = 0; m < 4; ++m) J.J1[m] = eps[1][m];
#pragma unroll
  for (int m = 0; m < 4; ++m) J.J2[m] = eps[2][m];
#pragma unroll
  for (int m = 0; m < 4; ++m) J.J3[m] = eps[3][m];
  {  // J(0,1)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J0, ev.pg[0], J.J1, ev.pg[1], t);
    const R f = ev.fg[0];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J01[m] = f * t[m];
  }
  {  // J(0,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J0, ev.pg[0], J.J2, ev.pg[2], t);
    const R f = ev.fg[1];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J02[m] = f * t[m];
  }
  {  // J(0,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J0, ev.pg[0], J.J3, ev.pg[3], t);
    const R f = ev.fg[2];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J03[m] = f * t[m];
  }
  {  // J(1,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J1, ev.pg[1], J.J2, ev.pg[2], t);
    const R f = ev.fg[3];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J12[m] = f * t[m];
  }
  {  // J(1,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J1, ev.pg[1], J.J3, ev.pg[3], t);
    const R f = ev.fg[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J13[m] = f * t[m];
  }
  {  // J(2,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J2, ev.pg[2], J.J3, ev.pg[3], t);
    const R f = ev.fg[5];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J23[m] = f * t[m];
  }
  {  // J(0,1,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J0, ev.pg[0], J.J12, ev.ps[3], t);
    vvv_acc(R(1), J.J01, ev.ps[0], J.J2, ev.pg[2], t);
    vvvv_acc(R(1), J.J0, J.J1, J.J2, t);
    const R f = ev.fg[6];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J012[m] = f * t[m];
  }
  {  // J(0,1,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J0, ev.pg[0], J.J13, ev.ps[4], t);
    vvv_acc(R(1), J.J01, ev.ps[0], J.J3, ev.pg[3], t);
    vvvv_acc(R(1), J.J0, J.J1, J.J3, t);
    const R f = ev.fg[7];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J013[m] = f * t[m];
  }
  {  // J(0,2,1)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(-1), J.J0, ev.pg[0], J.J12, ev.ps[3], t);
    vvv_acc(R(1), J.J02, ev.ps[1], J.J1, ev.pg[1], t);
    vvvv_acc(R(1), J.J0, J.J2, J.J1, t);
    const R f = ev.fg[6];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J021[m] = f * t[m];
  }
  {  // J(0,2,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J0, ev.pg[0], J.J23, ev.ps[5], t);
    vvv_acc(R(1), J.J02, ev.ps[1], J.J3, ev.pg[3], t);
    vvvv_acc(R(1), J.J0, J.J2, J.J3, t);
    const R f = ev.fg[8];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J023[m] = f * t[m];
  }
  {  // J(0,3,1)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(-1), J.J0, ev.pg[0], J.J13, ev.ps[4], t);
    vvv_acc(R(1), J.J03, ev.ps[2], J.J1, ev.pg[1], t);
    vvvv_acc(R(1), J.J0, J.J3, J.J1, t);
    const R f = ev.fg[7];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J031[m] = f * t[m];
  }
  {  // J(0,3,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(-1), J.J0, ev.pg[0], J.J23, ev.ps[5], t);
    vvv_acc(R(1), J.J03, ev.ps[2], J.J2, ev.pg[2], t);
    vvvv_acc(R(1), J.J0, J.J3, J.J2, t);
    const R f = ev.fg[8];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J032[m] = f * t[m];
  }
  {  // J(1,0,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J1, ev.pg[1], J.J02, ev.ps[1], t);
    vvv_acc(R(-1), J.J01, ev.ps[0], J.J2, ev.pg[2], t);
    vvvv_acc(R(1), J.J1, J.J0, J.J2, t);
    const R f = ev.fg[6];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J102[m] = f * t[m];
  }
  {  // J(1,0,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J1, ev.pg[1], J.J03, ev.ps[2], t);
    vvv_acc(R(-1), J.J01, ev.ps[0], J.J3, ev.pg[3], t);
    vvvv_acc(R(1), J.J1, J.J0, J.J3, t);
    const R f = ev.fg[7];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J103[m] = f * t[m];
  }
  {  // J(1,2,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J1, ev.pg[1], J.J23, ev.ps[5], t);
    vvv_acc(R(1), J.J12, ev.ps[3], J.J3, ev.pg[3], t);
    vvvv_acc(R(1), J.J1, J.J2, J.J3, t);
    const R f = ev.fg[9];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J123[m] = f * t[m];
  }
  {  // J(1,3,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(-1), J.J1, ev.pg[1], J.J23, ev.ps[5], t);
    vvv_acc(R(1), J.J13, ev.ps[4], J.J2, ev.pg[2], t);
    vvvv_acc(R(1), J.J1, J.J3, J.J2, t);
    const R f = ev.fg[9];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J132[m] = f * t[m];
  }
  {  // J(2,0,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J2, ev.pg[2], J.J03, ev.ps[2], t);
    vvv_acc(R(-1), J.J02, ev.ps[1], J.J3, ev.pg[3], t);
    vvvv_acc(R(1), J.J2, J.J0, J.J3, t);
    const R f = ev.fg[8];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J203[m] = f * t[m];
  }
  {  // J(2,1,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J2, ev.pg[2], J.J13, ev.ps[4], t);
    vvv_acc(R(-1), J.J12, ev.ps[3], J.J3, ev.pg[3], t);
    vvvv_acc(R(1), J.J2, J.J1, J.J3, t);
    const R f = ev.fg[9];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J213[m] = f * t[m];
  }
  {  // J(0,1,2,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J0, ev.pg[0], J.J123, ev.ps[9], t);
    vvv_acc(R(1), J.J01, ev.ps[0], J.J23, ev.ps[5], t);
    vvv_acc(R(1), J.J012, ev.ps[6], J.J3, ev.pg[3], t);
    vvvv_acc(R(1), J.J0, J.J1, J.J23, t);
    vvvv_acc(R(1), J.J0, J.J12, J.J3, t);
    vvvv_acc(R(1), J.J01, J.J2, J.J3, t);
    const R f = ev.fg[10];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J0123[m] = f * t[m];
  }
  {  // J(0,1,3,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J0, ev.pg[0], J.J132, ev.ps[9], t);
    vvv_acc(R(-1), J.J01, ev.ps[0], J.J23, ev.ps[5], t);
    vvv_acc(R(1), J.J013, ev.ps[7], J.J2, ev.pg[2], t);
    vvvv_acc(R(-1), J.J0, J.J1, J.J23, t);
    vvvv_acc(R(1), J.J0, J.J13, J.J2, t);
    vvvv_acc(R(1), J.J01, J.J3, J.J2, t);
    const R f = ev.fg[10];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J0132[m] = f * t[m];
  }
  {  // J(0,2,1,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J0, ev.pg[0], J.J213, ev.ps[9], t);
    vvv_acc(R(1), J.J02, ev.ps[1], J.J13, ev.ps[4], t);
    vvv_acc(R(1), J.J021, ev.ps[6], J.J3, ev.pg[3], t);
    vvvv_acc(R(1), J.J0, J.J2, J.J13, t);
    vvvv_acc(R(-1), J.J0, J.J12, J.J3, t);
    vvvv_acc(R(1), J.J02, J.J1, J.J3, t);
    const R f = ev.fg[10];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J0213[m] = f * t[m];
  }
  {  // J(0,2,3,1)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J0, ev.pg[0], J.J132, ev.ps[9], t);
    vvv_acc(R(-1), J.J02, ev.ps[1], J.J13, ev.ps[4], t);
    vvv_acc(R(1), J.J023, ev.ps[8], J.J1, ev.pg[1], t);
    vvvv_acc(R(-1), J.J0, J.J2, J.J13, t);
    vvvv_acc(R(1), J.J0, J.J23, J.J1, t);
    vvvv_acc(R(1), J.J02, J.J3, J.J1, t);
    const R f = ev.fg[10];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J0231[m] = f * t[m];
  }
  {  // J(0,3,1,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J0, ev.pg[0], J.J213, ev.ps[9], t);
    vvv_acc(R(1), J.J03, ev.ps[2], J.J12, ev.ps[3], t);
    vvv_acc(R(1), J.J031, ev.ps[7], J.J2, ev.pg[2], t);
    vvvv_acc(R(1), J.J0, J.J3, J.J12, t);
    vvvv_acc(R(-1), J.J0, J.J13, J.J2, t);
    vvvv_acc(R(1), J.J03, J.J1, J.J2, t);
    const R f = ev.fg[10];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J0312[m] = f * t[m];
  }
  {  // J(0,3,2,1)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J0, ev.pg[0], J.J123, ev.ps[9], t);
    vvv_acc(R(-1), J.J03, ev.ps[2], J.J12, ev.ps[3], t);
    vvv_acc(R(1), J.J032, ev.ps[8], J.J1, ev.pg[1], t);
    vvvv_acc(R(-1), J.J0, J.J3, J.J12, t);
    vvvv_acc(R(-1), J.J0, J.J23, J.J1, t);
    vvvv_acc(R(1), J.J03, J.J2, J.J1, t);
    const R f = ev.fg[10];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J0321[m] = f * t[m];
  }
  {  // J(1,0,2,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J1, ev.pg[1], J.J023, ev.ps[8], t);
    vvv_acc(R(-1), J.J01, ev.ps[0], J.J23, ev.ps[5], t);
    vvv_acc(R(1), J.J102, ev.ps[6], J.J3, ev.pg[3], t);
    vvvv_acc(R(1), J.J1, J.J0, J.J23, t);
    vvvv_acc(R(1), J.J1, J.J02, J.J3, t);
    vvvv_acc(R(-1), J.J01, J.J2, J.J3, t);
    const R f = ev.fg[10];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J1023[m] = f * t[m];
  }
  {  // J(1,0,3,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J1, ev.pg[1], J.J032, ev.ps[8], t);
    vvv_acc(R(1), J.J01, ev.ps[0], J.J23, ev.ps[5], t);
    vvv_acc(R(1), J.J103, ev.ps[7], J.J2, ev.pg[2], t);
    vvvv_acc(R(-1), J.J1, J.J0, J.J23, t);
    vvvv_acc(R(1), J.J1, J.J03, J.J2, t);
    vvvv_acc(R(-1), J.J01, J.J3, J.J2, t);
    const R f = ev.fg[10];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J1032[m] = f * t[m];
  }
  {  // J(1,2,0,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J1, ev.pg[1], J.J203, ev.ps[8], t);
    vvv_acc(R(1), J.J12, ev.ps[3], J.J03, ev.ps[2], t);
    vvv_acc(R(1), J.J021, ev.ps[6], J.J3, ev.pg[3], t);
    vvvv_acc(R(1), J.J1, J.J2, J.J03, t);
    vvvv_acc(R(-1), J.J1, J.J02, J.J3, t);
    vvvv_acc(R(1), J.J12, J.J0, J.J3, t);
    const R f = ev.fg[10];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J1203[m] = f * t[m];
  }
  {  // J(1,3,0,2)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J1, ev.pg[1], J.J203, ev.ps[8], t);
    vvv_acc(R(1), J.J13, ev.ps[4], J.J02, ev.ps[1], t);
    vvv_acc(R(1), J.J031, ev.ps[7], J.J2, ev.pg[2], t);
    vvvv_acc(R(1), J.J1, J.J3, J.J02, t);
    vvvv_acc(R(-1), J.J1, J.J03, J.J2, t);
    vvvv_acc(R(1), J.J13, J.J0, J.J2, t);
    const R f = ev.fg[10];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J1302[m] = f * t[m];
  }
  {  // J(2,0,1,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J2, ev.pg[2], J.J013, ev.ps[7], t);
    vvv_acc(R(-1), J.J02, ev.ps[1], J.J13, ev.ps[4], t);
    vvv_acc(R(1), J.J102, ev.ps[6], J.J3, ev.pg[3], t);
    vvvv_acc(R(1), J.J2, J.J0, J.J13, t);
    vvvv_acc(R(1), J.J2, J.J01, J.J3, t);
    vvvv_acc(R(-1), J.J02, J.J1, J.J3, t);
    const R f = ev.fg[10];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J2013[m] = f * t[m];
  }
  {  // J(2,1,0,3)
    R t[4] = {R(0), R(0), R(0), R(0)};
    vvv_acc(R(1), J.J2, ev.pg[2], J.J103, ev.ps[7], t);
    vvv_acc(R(-1), J.J12, ev.ps[3], J.J03, ev.ps[2], t);
    vvv_acc(R(1), J.J012, ev.ps[6], J.J3, ev.pg[3], t);
    vvvv_acc(R(1), J.J2, J.J1, J.J03, t);
    vvvv_acc(R(-1), J.J2, J.J01, J.J3, t);
    vvvv_acc(R(-1), J.J12, J.J0, J.J3, t);
    const R f = ev.fg[10];
#pragma unroll
    for (int m = 0; m < 4; ++m) J.J2103[m] = f * t[m];
  }
}

// sum over top helicities and antitop helicities hb in [hb_lo, hb_hi) (0: -, 1: +) of
// sum_{s,s'} conj(A_s) Cint_{ss'} A_s' (Cint = C * COLOUR_DEN).  The antitop-side
// currents psi(Y) are emitted depth-first over suffixes Y, so only one per depth is live.
// The colour form of one helicity is evaluated in CS, the helicity sum in ACC.
// FORM, if given, replaces the scalar colour form: form(A) returns this lane's
// contribution for both top helicities (e.g. the tensor-core form).
template <typename R, typename ACC, bool WIDTH, typename CS = ACC, typename FORM = NoColourForm>
__device__ __forceinline__ ACC gg_ttxgg_quark_line(const gg_ttxgg_event<R>& ev, const gg_ttxgg_mass<R>& mm, const gg_ttxgg_gluons<R>& J, int hb_lo = 0, int hb_hi = 2, const FORM& form = FORM()) {
  ACC total = ACC(0);
#pragma unroll 1
  for (int hb = hb_lo; hb < hb_hi; ++hb) {
    const cx<R>* v = mm.v[hb];
    cx<R> A[2][24];
    {
      cx<R> psi0[4];
      {
        cx<R> t[4] = {};
        slash_acc(R(1), J.J0, v, t);
        if (WIDTH) fermion_prop(ev.q[0], mm.m, cx<R>{mm.idr[0], mm.idi[0]}, t, psi0);
        else fermion_prop_real(ev.q[0], mm.m, mm.idr[0], t, psi0);
      }
      {
        cx<R> psi10[4];
        {
          cx<R> t[4] = {};
          slash_acc(R(1), J.J1, psi0, t);
          slash_acc(R(-1), J.J01, v, t);
          if (WIDTH) fermion_prop(ev.q[4], mm.m, cx<R>{mm.idr[4], mm.idi[4]}, t, psi10);
          else fermion_prop_real(ev.q[4], mm.m, mm.idr[4], t, psi10);
        }
        {
          cx<R> psi210[4];
          {
            cx<R> t[4] = {};
            slash_acc(R(1), J.J2, psi10, t);
            slash_acc(R(-1), J.J12, psi0, t);
            slash_acc(R(1), J.J012, v, t);
            if (WIDTH) fermion_prop(ev.q[10], mm.m, cx<R>{mm.idr[10], mm.idi[10]}, t, psi210);
            else fermion_prop_real(ev.q[10], mm.m, mm.idr[10], t, psi210);
          }
          {  // flow 23 = (3, 2, 1, 0)
            cx<R> x[4] = {};
            slash_acc(R(1), J.J3, psi210, x);
            slash_acc(R(-1), J.J23, psi10, x);
            slash_acc(R(1), J.J123, psi0, x);
            slash_acc(R(-1), J.J0123, v, x);
            A[0][23] = ubar_dot(mm.ut[0], x);
            A[1][23] = ubar_dot(mm.ut[1], x);
          }
        }
        {
          cx<R> psi310[4];
          {
            cx<R> t[4] = {};
            slash_acc(R(1), J.J3, psi10, t);
            slash_acc(R(-1), J.J13, psi0, t);
            slash_acc(R(1), J.J013, v, t);
            if (WIDTH) fermion_prop(ev.q[11], mm.m, cx<R>{mm.idr[11], mm.idi[11]}, t, psi310);
            else fermion_prop_real(ev.q[11], mm.m, mm.idr[11], t, psi310);
          }
          {  // flow 17 = (2, 3, 1, 0)
            cx<R> x[4] = {};
            slash_acc(R(1), J.J2, psi310, x);
            slash_acc(R(1), J.J23, psi10, x);
            slash_acc(R(1), J.J132, psi0, x);
            slash_acc(R(-1), J.J0132, v, x);
            A[0][17] = ubar_dot(mm.ut[0], x);
            A[1][17] = ubar_dot(mm.ut[1], x);
          }
        }
      }
      {
        cx<R> psi20[4];
        {
          cx<R> t[4] = {};
          slash_acc(R(1), J.J2, psi0, t);
          slash_acc(R(-1), J.J02, v, t);
          if (WIDTH) fermion_prop(ev.q[5], mm.m, cx<R>{mm.idr[5], mm.idi[5]}, t, psi20);
          else fermion_prop_real(ev.q[5], mm.m, mm.idr[5], t, psi20);
        }
        {
          cx<R> psi120[4];
          {
            cx<R> t[4] = {};
            slash_acc(R(1), J.J1, psi20, t);
            slash_acc(R(1), J.J12, psi0, t);
            slash_acc(R(1), J.J021, v, t);
            if (WIDTH) fermion_prop(ev.q[10], mm.m, cx<R>{mm.idr[10], mm.idi[10]}, t, psi120);
            else fermion_prop_real(ev.q[10], mm.m, mm.idr[10], t, psi120);
          }
          {  // flow 21 = (3, 1, 2, 0)
            cx<R> x[4] = {};
            slash_acc(R(1), J.J3, psi120, x);
            slash_acc(R(-1), J.J13, psi20, x);
            slash_acc(R(1), J.J213, psi0, x);
            slash_acc(R(-1), J.J0213, v, x);
            A[0][21] = ubar_dot(mm.ut[0], x);
            A[1][21] = ubar_dot(mm.ut[1], x);
          }
        }
        {
          cx<R> psi320[4];
          {
            cx<R> t[4] = {};
            slash_acc(R(1), J.J3, psi20, t);
            slash_acc(R(-1), J.J23, psi0, t);
            slash_acc(R(1), J.J023, v, t);
            if (WIDTH) fermion_prop(ev.q[12], mm.m, cx<R>{mm.idr[12], mm.idi[12]}, t, psi320);
            else fermion_prop_real(ev.q[12], mm.m, mm.idr[12], t, psi320);
          }
          {  // flow 11 = (1, 3, 2, 0)
            cx<R> x[4] = {};
            slash_acc(R(1), J.J1, psi320, x);
            slash_acc(R(1), J.J13, psi20, x);
            slash_acc(R(1), J.J132, psi0, x);
            slash_acc(R(-1), J.J0231, v, x);
            A[0][11] = ubar_dot(mm.ut[0], x);
            A[1][11] = ubar_dot(mm.ut[1], x);
          }
        }
      }
      {
        cx<R> psi30[4];
        {
          cx<R> t[4] = {};
          slash_acc(R(1), J.J3, psi0, t);
          slash_acc(R(-1), J.J03, v, t);
          if (WIDTH) fermion_prop(ev.q[6], mm.m, cx<R>{mm.idr[6], mm.idi[6]}, t, psi30);
          else fermion_prop_real(ev.q[6], mm.m, mm.idr[6], t, psi30);
        }
        {
          cx<R> psi130[4];
          {
            cx<R> t[4] = {};
            slash_acc(R(1), J.J1, psi30, t);
            slash_acc(R(1), J.J13, psi0, t);
            slash_acc(R(1), J.J031, v, t);
            if (WIDTH) fermion_prop(ev.q[11], mm.m, cx<R>{mm.idr[11], mm.idi[11]}, t, psi130);
            else fermion_prop_real(ev.q[11], mm.m, mm.idr[11], t, psi130);
          }
          {  // flow 15 = (2, 1, 3, 0)
            cx<R> x[4] = {};
            slash_acc(R(1), J.J2, psi130, x);
            slash_acc(R(-1), J.J12, psi30, x);
            slash_acc(R(1), J.J213, psi0, x);
            slash_acc(R(-1), J.J0312, v, x);
            A[0][15] = ubar_dot(mm.ut[0], x);
            A[1][15] = ubar_dot(mm.ut[1], x);
          }
        }
        {
          cx<R> psi230[4];
          {
            cx<R> t[4] = {};
            slash_acc(R(1), J.J2, psi30, t);
            slash_acc(R(1), J.J23, psi0, t);
            slash_acc(R(1), J.J032, v, t);
            if (WIDTH) fermion_prop(ev.q[12], mm.m, cx<R>{mm.idr[12], mm.idi[12]}, t, psi230);
            else fermion_prop_real(ev.q[12], mm.m, mm.idr[12], t, psi230);
          }
          {  // flow 9 = (1, 2, 3, 0)
            cx<R> x[4] = {};
            slash_acc(R(1), J.J1, psi230, x);
            slash_acc(R(1), J.J12, psi30, x);
            slash_acc(R(1), J.J123, psi0, x);
            slash_acc(R(-1), J.J0321, v, x);
            A[0][9] = ubar_dot(mm.ut[0], x);
            A[1][9] = ubar_dot(mm.ut[1], x);
          }
        }
      }
    }
    {
      cx<R> psi1[4];
      {
        cx<R> t[4] = {};
        slash_acc(R(1), J.J1, v, t);
        if (WIDTH) fermion_prop(ev.q[1], mm.m, cx<R>{mm.idr[1], mm.idi[1]}, t, psi1);
        else fermion_prop_real(ev.q[1], mm.m, mm.idr[1], t, psi1);
      }
      {
        cx<R> psi01[4];
        {
          cx<R> t[4] = {};
          slash_acc(R(1), J.J0, psi1, t);
          slash_acc(R(1), J.J01, v, t);
          if (WIDTH) fermion_prop(ev.q[4], mm.m, cx<R>{mm.idr[4], mm.idi[4]}, t, psi01);
          else fermion_prop_real(ev.q[4], mm.m, mm.idr[4], t, psi01);
        }
        {
          cx<R> psi201[4];
          {
            cx<R> t[4] = {};
            slash_acc(R(1), J.J2, psi01, t);
            slash_acc(R(-1), J.J02, psi1, t);
            slash_acc(R(1), J.J102, v, t);
            if (WIDTH) fermion_prop(ev.q[10], mm.m, cx<R>{mm.idr[10], mm.idi[10]}, t, psi201);
            else fermion_prop_real(ev.q[10], mm.m, mm.idr[10], t, psi201);
          }
          {  // flow 22 = (3, 2, 0, 1)
            cx<R> x[4] = {};
            slash_acc(R(1), J.J3, psi201, x);
            slash_acc(R(-1), J.J23, psi01, x);
            slash_acc(R(1), J.J023, psi1, x);
            slash_acc(R(-1), J.J1023, v, x);
            A[0][22] = ubar_dot(mm.ut[0], x);
            A[1][22] = ubar_dot(mm.ut[1], x);
          }
        }
        {
          cx<R> psi301[4];
          {
            cx<R> t[4] = {};
            slash_acc(R(1), J.J3, psi01, t);
            slash_acc(R(-1), J.J03, psi1, t);
            slash_acc(R(1), J.J103, v, t);
            if (WIDTH) fermion_prop(ev.q[11], mm.m, cx<R>{mm.idr[11], mm.idi[11]}, t, psi301);
            else fermion_prop_real(ev.q[11], mm.m, mm.idr[11], t, psi301);
          }
          {  // flow 16 = (2, 3, 0, 1)
            cx<R> x[4] = {};
            slash_acc(R(1), J.J2, psi301, x);
            slash_acc(R(1), J.J23, psi01, x);
            slash_acc(R(1), J.J032, psi1, x);
            slash_acc(R(-1), J.J1032, v, x);
            A[0][16] = ubar_dot(mm.ut[0], x);
            A[1][16] = ubar_dot(mm.ut[1], x);
          }
        }
      }
      {
        cx<R> psi21[4];
        {
          cx<R> t[4] = {};
          slash_acc(R(1), J.J2, psi1, t);
          slash_acc(R(-1), J.J12, v, t);
          if (WIDTH) fermion_prop(ev.q[7], mm.m, cx<R>{mm.idr[7], mm.idi[7]}, t, psi21);
          else fermion_prop_real(ev.q[7], mm.m, mm.idr[7], t, psi21);
        }
        {
          cx<R> psi021[4];
          {
            cx<R> t[4] = {};
            slash_acc(R(1), J.J0, psi21, t);
            slash_acc(R(1), J.J02, psi1, t);
            slash_acc(R(1), J.J021, v, t);
            if (WIDTH) fermion_prop(ev.q[10], mm.m, cx<R>{mm.idr[10], mm.idi[10]}, t, psi021);
            else fermion_prop_real(ev.q[10], mm.m, mm.idr[10], t, psi021);
          }
          {  // flow 19 = (3, 0, 2, 1)
            cx<R> x[4] = {};
            slash_acc(R(1), J.J3, psi021, x);
            slash_acc(R(-1), J.J03, psi21, x);
            slash_acc(R(1), J.J203, psi1, x);
            slash_acc(R(-1), J.J1203, v, x);
            A[0][19] = ubar_dot(mm.ut[0], x);
            A[1][19] = ubar_dot(mm.ut[1], x);
          }
        }
        {
          cx<R> psi321[4];
          {
            cx<R> t[4] = {};
            slash_acc(R(1), J.J3, psi21, t);
            slash_acc(R(-1), J.J23, psi1, t);
            slash_acc(R(1), J.J123, v, t);
            if (WIDTH) fermion_prop(ev.q[13], mm.m, cx<R>{mm.idr[13], mm.idi[13]}, t, psi321);
            else fermion_prop_real(ev.q[13], mm.m, mm.idr[13], t, psi321);
          }
          {  // flow 5 = (0, 3, 2, 1)
            cx<R> x[4] = {};
            slash_acc(R(1), J.J0, psi321, x);
            slash_acc(R(1), J.J03, psi21, x);
            slash_acc(R(1), J.J032, psi1, x);
            slash_acc(R(1), J.J0321, v, x);
            A[0][5] = ubar_dot(mm.ut[0], x);
            A[1][5] = ubar_dot(mm.ut[1], x);
          }
        }
      }
      {
        cx<R> psi31[4];
        {
          cx<R> t[4] = {};
          slash_acc(R(1), J.J3, psi1, t);
          slash_acc(R(-1), J.J13, v, t);
          if (WIDTH) fermion_prop(ev.q[8], mm.m, cx<R>{mm.idr[8], mm.idi[8]}, t, psi31);
          else fermion_prop_real(ev.q[8], mm.m, mm.idr[8], t, psi31);
        }
        {
          cx<R> psi031[4];
          {
            cx<R> t[4] = {};
            slash_acc(R(1), J.J0, psi31, t);
            slash_acc(R(1), J.J03, psi1, t);
            slash_acc(R(1), J.J031, v, t);
            if (WIDTH) fermion_prop(ev.q[11], mm.m, cx<R>{mm.idr[11], mm.idi[11]}, t, psi031);
            else fermion_prop_real(ev.q[11], mm.m, mm.idr[11], t, psi031);
          }
          {  // flow 13 = (2, 0, 3, 1)
            cx<R> x[4] = {};
            slash_acc(R(1), J.J2, psi031, x);
            slash_acc(R(-1), J.J02, psi31, x);
            slash_acc(R(1), J.J203, psi1, x);
            slash_acc(R(-1), J.J1302, v, x);
            A[0][13] = ubar_dot(mm.ut[0], x);
            A[1][13] = ubar_dot(mm.ut[1], x);
          }
        }
        {
          cx<R> psi231[4];
          {
            cx<R> t[4] = {};
            slash_acc(R(1), J.J2, psi31, t);
            slash_acc(R(1), J.J23, psi1, t);
            slash_acc(R(1), J.J132, v, t);
            if (WIDTH) fermion_prop(ev.q[13], mm.m, cx<R>{mm.idr[13], mm.idi[13]}, t, psi231);
            else fermion_prop_real(ev.q[13], mm.m, mm.idr[13], t, psi231);
          }
          {  // flow 3 = (0, 2, 3, 1)
            cx<R> x[4] = {};
            slash_acc(R(1), J.J0, psi231, x);
            slash_acc(R(1), J.J02, psi31, x);
            slash_acc(R(1), J.J023, psi1, x);
            slash_acc(R(1), J.J0231, v, x);
            A[0][3] = ubar_dot(mm.ut[0], x);
            A[1][3] = ubar_dot(mm.ut[1], x);
          }
        }
      }
    }
    {
      cx<R> psi2[4];
      {
        cx<R> t[4] = {};
        slash_acc(R(1), J.J2, v, t);
        if (WIDTH) fermion_prop(ev.q[2], mm.m, cx<R>{mm.idr[2], mm.idi[2]}, t, psi2);
        else fermion_prop_real(ev.q[2], mm.m, mm.idr[2], t, psi2);
      }
      {
        cx<R> psi02[4];
        {
          cx<R> t[4] = {};
          slash_acc(R(1), J.J0, psi2, t);
          slash_acc(R(1), J.J02, v, t);
          if (WIDTH) fermion_prop(ev.q[5], mm.m, cx<R>{mm.idr[5], mm.idi[5]}, t, psi02);
          else fermion_prop_real(ev.q[5], mm.m, mm.idr[5], t, psi02);
        }
        {
          cx<R> psi102[4];
          {
            cx<R> t[4] = {};
            slash_acc(R(1), J.J1, psi02, t);
            slash_acc(R(-1), J.J01, psi2, t);
            slash_acc(R(1), J.J102, v, t);
            if (WIDTH) fermion_prop(ev.q[10], mm.m, cx<R>{mm.idr[10], mm.idi[10]}, t, psi102);
            else fermion_prop_real(ev.q[10], mm.m, mm.idr[10], t, psi102);
          }
          {  // flow 20 = (3, 1, 0, 2)
            cx<R> x[4] = {};
            slash_acc(R(1), J.J3, psi102, x);
            slash_acc(R(-1), J.J13, psi02, x);
            slash_acc(R(1), J.J013, psi2, x);
            slash_acc(R(-1), J.J2013, v, x);
            A[0][20] = ubar_dot(mm.ut[0], x);
            A[1][20] = ubar_dot(mm.ut[1], x);
          }
        }
        {
          cx<R> psi302[4];
          {
            cx<R> t[4] = {};
            slash_acc(R(1), J.J3, psi02, t);
            slash_acc(R(-1), J.J03, psi2, t);
            slash_acc(R(1), J.J203, v, t);
            if (WIDTH) fermion_prop(ev.q[12], mm.m, cx<R>{mm.idr[12], mm.idi[12]}, t, psi302);
            else fermion_prop_real(ev.q[12], mm.m, mm.idr[12], t, psi302);
          }
          {  // flow 10 = (1, 3, 0, 2)
            cx<R> x[4] = {};
            slash_acc(R(1), J.J1, psi302, x);
            slash_acc(R(1), J.J13, psi02, x);
            slash_acc(R(1), J.J031, psi2, x);
            slash_acc(R(1), J.J1302, v, x);
            A[0][10] = ubar_dot(mm.ut[0], x);
            A[1][10] = ubar_dot(mm.ut[1], x);
          }
        }
      }
      {
        cx<R> psi12[4];
        {
          cx<R> t[4] = {};
          slash_acc(R(1), J.J1, psi2, t);
          slash_acc(R(1), J.J12, v, t);
          if (WIDTH) fermion_prop(ev.q[7], mm.m, cx<R>{mm.idr[7], mm.idi[7]}, t, psi12);
          else fermion_prop_real(ev.q[7], mm.m, mm.idr[7], t, psi12);
        }
        {
          cx<R> psi012[4];
          {
            cx<R> t[4] = {};
            slash_acc(R(1), J.J0, psi12, t);
            slash_acc(R(1), J.J01, psi2, t);
            slash_acc(R(1), J.J012, v, t);
            if (WIDTH) fermion_prop(ev.q[10], mm.m, cx<R>{mm.idr[10], mm.idi[10]}, t, psi012);
            else fermion_prop_real(ev.q[10], mm.m, mm.idr[10], t, psi012);
          }
          {  // flow 18 = (3, 0, 1, 2)
            cx<R> x[4] = {};
            slash_acc(R(1), J.J3, psi012, x);
            slash_acc(R(-1), J.J03, psi12, x);
            slash_acc(R(1), J.J103, psi2, x);
            slash_acc(R(-1), J.J2103, v, x);
            A[0][18] = ubar_dot(mm.ut[0], x);
            A[1][18] = ubar_dot(mm.ut[1], x);
          }
        }
        {
          cx<R> psi312[4];
          {
            cx<R> t[4] = {};
            slash_acc(R(1), J.J3, psi12, t);
            slash_acc(R(-1), J.J13, psi2, t);
            slash_acc(R(1), J.J213, v, t);
            if (WIDTH) fermion_prop(ev.q[13], mm.m, cx<R>{mm.idr[13], mm.idi[13]}, t, psi312);
            else fermion_prop_real(ev.q[13], mm.m, mm.idr[13], t, psi312);
          }
          {  // flow 4 = (0, 3, 1, 2)
            cx<R> x[4] = {};
            slash_acc(R(1), J.J0, psi312, x);
            slash_acc(R(1), J.J03, psi12, x);
            slash_acc(R(1), J.J031, psi2, x);
            slash_acc(R(1), J.J0312, v, x);
            A[0][4] = ubar_dot(mm.ut[0], x);
            A[1][4] = ubar_dot(mm.ut[1], x);
          }
        }
      }
      {
        cx<R> psi32[4];
        {
          cx<R> t[4] = {};
          slash_acc(R(1), J.J3, psi2, t);
          slash_acc(R(-1), J.J23, v, t);
          if (WIDTH) fermion_prop(ev.q[9], mm.m, cx<R>{mm.idr[9], mm.idi[9]}, t, psi32);
          else fermion_prop_real(ev.q[9], mm.m, mm.idr[9], t, psi32);
        }
        {
          cx<R> psi032[4];
          {
            cx<R> t[4] = {};
            slash_acc(R(1), J.J0, psi32, t);
            slash_acc(R(1), J.J03, psi2, t);
            slash_acc(R(1), J.J032, v, t);
            if (WIDTH) fermion_prop(ev.q[12], mm.m, cx<R>{mm.idr[12], mm.idi[12]}, t, psi032);
            else fermion_prop_real(ev.q[12], mm.m, mm.idr[12], t, psi032);
          }
          {  // flow 7 = (1, 0, 3, 2)
            cx<R> x[4] = {};
            slash_acc(R(1), J.J1, psi032, x);
            slash_acc(R(-1), J.J01, psi32, x);
            slash_acc(R(1), J.J103, psi2, x);
            slash_acc(R(1), J.J1032, v, x);
            A[0][7] = ubar_dot(mm.ut[0], x);
            A[1][7] = ubar_dot(mm.ut[1], x);
          }
        }
        {
          cx<R> psi132[4];
          {
            cx<R> t[4] = {};
            slash_acc(R(1), J.J1, psi32, t);
            slash_acc(R(1), J.J13, psi2, t);
            slash_acc(R(1), J.J132, v, t);
            if (WIDTH) fermion_prop(ev.q[13], mm.m, cx<R>{mm.idr[13], mm.idi[13]}, t, psi132);
            else fermion_prop_real(ev.q[13], mm.m, mm.idr[13], t, psi132);
          }
          {  // flow 1 = (0, 1, 3, 2)
            cx<R> x[4] = {};
            slash_acc(R(1), J.J0, psi132, x);
            slash_acc(R(1), J.J01, psi32, x);
            slash_acc(R(1), J.J013, psi2, x);
            slash_acc(R(1), J.J0132, v, x);
            A[0][1] = ubar_dot(mm.ut[0], x);
            A[1][1] = ubar_dot(mm.ut[1], x);
          }
        }
      }
    }
    {
      cx<R> psi3[4];
      {
        cx<R> t[4] = {};
        slash_acc(R(1), J.J3, v, t);
        if (WIDTH) fermion_prop(ev.q[3], mm.m, cx<R>{mm.idr[3], mm.idi[3]}, t, psi3);
        else fermion_prop_real(ev.q[3], mm.m, mm.idr[3], t, psi3);
      }
      {
        cx<R> psi03[4];
        {
          cx<R> t[4] = {};
          slash_acc(R(1), J.J0, psi3, t);
          slash_acc(R(1), J.J03, v, t);
          if (WIDTH) fermion_prop(ev.q[6], mm.m, cx<R>{mm.idr[6], mm.idi[6]}, t, psi03);
          else fermion_prop_real(ev.q[6], mm.m, mm.idr[6], t, psi03);
        }
        {
          cx<R> psi103[4];
          {
            cx<R> t[4] = {};
            slash_acc(R(1), J.J1, psi03, t);
            slash_acc(R(-1), J.J01, psi3, t);
            slash_acc(R(1), J.J103, v, t);
            if (WIDTH) fermion_prop(ev.q[11], mm.m, cx<R>{mm.idr[11], mm.idi[11]}, t, psi103);
            else fermion_prop_real(ev.q[11], mm.m, mm.idr[11], t, psi103);
          }
          {  // flow 14 = (2, 1, 0, 3)
            cx<R> x[4] = {};
            slash_acc(R(1), J.J2, psi103, x);
            slash_acc(R(-1), J.J12, psi03, x);
            slash_acc(R(1), J.J012, psi3, x);
            slash_acc(R(1), J.J2103, v, x);
            A[0][14] = ubar_dot(mm.ut[0], x);
            A[1][14] = ubar_dot(mm.ut[1], x);
          }
        }
        {
          cx<R> psi203[4];
          {
            cx<R> t[4] = {};
            slash_acc(R(1), J.J2, psi03, t);
            slash_acc(R(-1), J.J02, psi3, t);
            slash_acc(R(1), J.J203, v, t);
            if (WIDTH) fermion_prop(ev.q[12], mm.m, cx<R>{mm.idr[12], mm.idi[12]}, t, psi203);
            else fermion_prop_real(ev.q[12], mm.m, mm.idr[12], t, psi203);
          }
          {  // flow 8 = (1, 2, 0, 3)
            cx<R> x[4] = {};
            slash_acc(R(1), J.J1, psi203, x);
            slash_acc(R(1), J.J12, psi03, x);
            slash_acc(R(1), J.J021, psi3, x);
            slash_acc(R(1), J.J1203, v, x);
            A[0][8] = ubar_dot(mm.ut[0], x);
            A[1][8] = ubar_dot(mm.ut[1], x);
          }
        }
      }
      {
        cx<R> psi13[4];
        {
          cx<R> t[4] = {};
          slash_acc(R(1), J.J1, psi3, t);
          slash_acc(R(1), J.J13, v, t);
          if (WIDTH) fermion_prop(ev.q[8], mm.m, cx<R>{mm.idr[8], mm.idi[8]}, t, psi13);
          else fermion_prop_real(ev.q[8], mm.m, mm.idr[8], t, psi13);
        }
        {
          cx<R> psi013[4];
          {
            cx<R> t[4] = {};
            slash_acc(R(1), J.J0, psi13, t);
            slash_acc(R(1), J.J01, psi3, t);
            slash_acc(R(1), J.J013, v, t);
            if (WIDTH) fermion_prop(ev.q[11], mm.m, cx<R>{mm.idr[11], mm.idi[11]}, t, psi013);
            else fermion_prop_real(ev.q[11], mm.m, mm.idr[11], t, psi013);
          }
          {  // flow 12 = (2, 0, 1, 3)
            cx<R> x[4] = {};
            slash_acc(R(1), J.J2, psi013, x);
            slash_acc(R(-1), J.J02, psi13, x);
            slash_acc(R(1), J.J102, psi3, x);
            slash_acc(R(1), J.J2013, v, x);
            A[0][12] = ubar_dot(mm.ut[0], x);
            A[1][12] = ubar_dot(mm.ut[1], x);
          }
        }
        {
          cx<R> psi213[4];
          {
            cx<R> t[4] = {};
            slash_acc(R(1), J.J2, psi13, t);
            slash_acc(R(-1), J.J12, psi3, t);
            slash_acc(R(1), J.J213, v, t);
            if (WIDTH) fermion_prop(ev.q[13], mm.m, cx<R>{mm.idr[13], mm.idi[13]}, t, psi213);
            else fermion_prop_real(ev.q[13], mm.m, mm.idr[13], t, psi213);
          }
          {  // flow 2 = (0, 2, 1, 3)
            cx<R> x[4] = {};
            slash_acc(R(1), J.J0, psi213, x);
            slash_acc(R(1), J.J02, psi13, x);
            slash_acc(R(1), J.J021, psi3, x);
            slash_acc(R(1), J.J0213, v, x);
            A[0][2] = ubar_dot(mm.ut[0], x);
            A[1][2] = ubar_dot(mm.ut[1], x);
          }
        }
      }
      {
        cx<R> psi23[4];
        {
          cx<R> t[4] = {};
          slash_acc(R(1), J.J2, psi3, t);
          slash_acc(R(1), J.J23, v, t);
          if (WIDTH) fermion_prop(ev.q[9], mm.m, cx<R>{mm.idr[9], mm.idi[9]}, t, psi23);
          else fermion_prop_real(ev.q[9], mm.m, mm.idr[9], t, psi23);
        }
        {
          cx<R> psi023[4];
          {
            cx<R> t[4] = {};
            slash_acc(R(1), J.J0, psi23, t);
            slash_acc(R(1), J.J02, psi3, t);
            slash_acc(R(1), J.J023, v, t);
            if (WIDTH) fermion_prop(ev.q[12], mm.m, cx<R>{mm.idr[12], mm.idi[12]}, t, psi023);
            else fermion_prop_real(ev.q[12], mm.m, mm.idr[12], t, psi023);
          }
          {  // flow 6 = (1, 0, 2, 3)
            cx<R> x[4] = {};
            slash_acc(R(1), J.J1, psi023, x);
            slash_acc(R(-1), J.J01, psi23, x);
            slash_acc(R(1), J.J102, psi3, x);
            slash_acc(R(1), J.J1023, v, x);
            A[0][6] = ubar_dot(mm.ut[0], x);
            A[1][6] = ubar_dot(mm.ut[1], x);
          }
        }
        {
          cx<R> psi123[4];
          {
            cx<R> t[4] = {};
            slash_acc(R(1), J.J1, psi23, t);
            slash_acc(R(1), J.J12, psi3, t);
            slash_acc(R(1), J.J123, v, t);
            if (WIDTH) fermion_prop(ev.q[13], mm.m, cx<R>{mm.idr[13], mm.idi[13]}, t, psi123);
            else fermion_prop_real(ev.q[13], mm.m, mm.idr[13], t, psi123);
          }
          {  // flow 0 = (0, 1, 2, 3)
            cx<R> x[4] = {};
            slash_acc(R(1), J.J0, psi123, x);
            slash_acc(R(1), J.J01, psi23, x);
            slash_acc(R(1), J.J012, psi3, x);
            slash_acc(R(1), J.J0123, v, x);
            A[0][0] = ubar_dot(mm.ut[0], x);
            A[1][0] = ubar_dot(mm.ut[1], x);
          }
        }
      }
    }
    if constexpr (!std::is_same<FORM, NoColourForm>::value) {
      total += ACC(form(A));
    } else {
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
  }
  return total;
}

}  // namespace rex
