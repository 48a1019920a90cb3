// The g g -> t t~ g quark line in double-float, written as loops (sm_103a).
//
// The generated quark line (generated/qcd_amplitudes.cuh) expands the six colour-
// ordered flows into straight-line code.  In double-float every operation is 7 to 15
// FP32 instructions, and that straight-line code outgrows the instruction caches: the
// kernel then waits on instruction fetch.  This form computes the same currents in the
// same order, but as a loop over the gluon attached first to the top line (a = 0, 1, 2)
// with a loop over the two choices of the second gluon inside it, reading its operands
// through index tables:
//   psi_a  = P(q_a)  (J_a  v)
//   psi_ab = P(q_ab) (J_b psi_a  + s1 J_ab v)
//   x_f    =          J_c psi_ab + s2 J_bc psi_a + J_abc v,   A_f(h) = ubar_h(p_t) x_f
// where J_... are the colour-ordered gluon currents of the lane's polarisation
// configuration (in shared memory, indexable), P(q) the top propagator
// -(q-slash + m)/(q^2 - m^2 + i m Gamma), v the antitop spinor and ubar_h the top
// spinors of both helicities.  The colour sum is the generated one:
// sum_h sum_{f,f'} C_ff' Re(conj(A_f(h)) A_f'(h)), C the integer flow matrix.
#pragma once
#include <cuda_runtime.h>

#include "df64.cuh"
#include "generated/qcd_amplitudes.cuh"

namespace rex {

// One (a, b) branch: current indices into the gluon currents {J0, J1, J2, J01, J02,
// J12, J012, J021, J102}, propagator index of q_ab, signs and the flow it closes.
struct GgTtxgDfRow {
  signed char jb, jab, s1, qab, jc, jbc, s2, jabc, flow;
};

__constant__ GgTtxgDfRow kGgTtxgDfRows[6] = {
    {1, 3, -1, 3, 2, 5, -1, 6, 5},   // a = 0, b = 1: flow (2, 1, 0)
    {2, 4, -1, 4, 1, 5, 1, 7, 3},    // a = 0, b = 2: flow (1, 2, 0)
    {0, 3, 1, 3, 2, 4, -1, 8, 4},    // a = 1, b = 0: flow (2, 0, 1)
    {2, 5, -1, 5, 0, 4, 1, 7, 1},    // a = 1, b = 2: flow (0, 2, 1)
    {0, 4, 1, 4, 1, 3, -1, 8, 2},    // a = 2, b = 0: flow (1, 0, 2)
    {1, 5, 1, 5, 0, 3, 1, 6, 0},     // a = 2, b = 1: flow (0, 1, 2)
};

template <bool WIDTH>
__device__ __forceinline__ void gg_ttxg_df_prop(const gg_ttxg_event<df64>& ev, const gg_ttxg_mass<df64>& mm,
                                                int k, const cx<df64>* t, cx<df64>* out) {
  if (WIDTH) fermion_prop(ev.q[k], mm.m, cx<df64>{mm.idr[k], mm.idi[k]}, t, out);
  else fermion_prop_real(ev.q[k], mm.m, mm.idr[k], t, out);
}

// J: the lane's nine gluon currents, [9][4], in shared memory.  FORM: the colour form
// of a helicity-exclusive tile (qcd_kernel.cuh), or NoColourForm for the helicity sum.
template <bool WIDTH, typename FORM = NoColourForm>
__device__ __forceinline__ df64 gg_ttxg_quark_line_df64(const gg_ttxg_event<df64>& ev,
                                                        const gg_ttxg_mass<df64>& mm, const df64 (*J)[4],
                                                        int hb_lo, int hb_hi, const FORM& form = FORM()) {
  df64 total = df64(0);
#pragma unroll 1
  for (int hb = hb_lo; hb < hb_hi; ++hb) {
    const cx<df64>* v = mm.v[hb];
    cx<df64> A[2][6];
#pragma unroll 1
    for (int a = 0; a < 3; ++a) {
      cx<df64> psia[4];
      {
        cx<df64> t[4] = {};
        slash_acc(df64(1), J[a], v, t);
        gg_ttxg_df_prop<WIDTH>(ev, mm, a, t, psia);
      }
      // Rolled as well: the unrolled pair of branches doubled the loop's code and left
      // the kernel 17 % slower (instruction fetch again), for no saving in registers.
#pragma unroll 1
      for (int bi = 0; bi < 2; ++bi) {
        const GgTtxgDfRow r = kGgTtxgDfRows[2 * a + bi];
        cx<df64> psiab[4];
        {
          cx<df64> t[4] = {};
          slash_acc(df64(1), J[r.jb], psia, t);
          slash_acc(df64((int)r.s1), J[r.jab], v, t);
          gg_ttxg_df_prop<WIDTH>(ev, mm, r.qab, t, psiab);
        }
        cx<df64> x[4] = {};
        slash_acc(df64(1), J[r.jc], psiab, x);
        slash_acc(df64((int)r.s2), J[r.jbc], psia, x);
        slash_acc(df64(1), J[r.jabc], v, x);
        A[0][r.flow] = ubar_dot(mm.ut[0], x);
        A[1][r.flow] = ubar_dot(mm.ut[1], x);
      }
    }
    if constexpr (!std::is_same<FORM, NoColourForm>::value) {
      total = total + form(A);
    } else {
#pragma unroll 1
      for (int ht = 0; ht < 2; ++ht) {
        float s = 0.f, c = 0.f;
#pragma unroll
        for (int f = 0; f < 6; ++f)
#pragma unroll
          for (int g = f; g < 6; ++g) {
            const df64 w = df64(gg_ttxg_colour_dev[f][g] * (f == g ? 1 : 2));
            df64_acc_term(s, c, w * A[ht][f].re, A[ht][g].re);
            df64_acc_term(s, c, w * A[ht][f].im, A[ht][g].im);
          }
        total = total + df64_renorm(s, c);
      }
    }
  }
  return total;
}

}  // namespace rex
