// q(1) q~(2) -> t(3) t~(4) through one s-channel gluon: device code shared by the
// standalone kernel and the persistent multi-process kernel (sm_103a).
//
// Amplitude of helicity configuration h = (l1, l2, l3, l4):
//     A_h = J_in . J_out,   J_in = vbar(p2) gamma^mu u(p1),   J_out = ubar(p3) gamma_mu v(p4),
// times g^2 / s and the colour structure t^a_{ji} t^a_{kl}, whose sum over colours is
// (N^2 - 1)/4 = 2 (folded into the per-point factor with the 1/36 average and g^4).
//
// Steps (a1 .. a8 of the hot path) for a tile of 128 events, thread per event:
//   a1  the tile's momenta are staged in shared memory by coalesced loads;
//   a3  the light quarks are massless, so J_in is parameter independent and
//       non-zero only for opposite q, q~ helicities (chirality conservation):
//       two currents per event.  The top spinors are u(+) = (w- chi+, w+ chi+),
//       u(-) = (w+ chi-, w- chi-), v(+) = (w+ chi-, -w- chi-), v(-) = (w- chi+, -w+ chi+)
//       with w+ = sqrt(E + |p|) kept and w- = m / w+, so for each top-helicity pair
//       J_out = aL(m) BL + aR(m) BR with mass-independent chiral bilinears
//       BR = xi^dag sigma^mu eta, BL = xi^dag sigmabar^mu eta and real aL, aR;
//   a5  D_X = J_in . B_X per (q helicity, top-helicity pair, chirality X);
//   a7  sum_h |aL DL + aR DR|^2 = aL^2 sum|DL|^2 + aR^2 sum|DR|^2 + 2 aL aR sum Re(DL* DR);
//       with aL aR = -m^2 for every pair and aL^2, aR^2 in {m^2 r^+-2, m^4 / W^2, W^2}
//       (r = w+(4)/w+(3), W = w+(3) w+(4)) the helicity sum is exactly
//           C0 + C2 m^2 + C4 m^4,
//       three per-event constants: every parameter point then costs two FMAs;
//   a8  ratio epilogue w_out = w_in |M_j|^2 / |M_0|^2 (0 if |M_0|^2 == 0): s, the
//       incoming scale and the coupling factor of the original point cancel, so
//       the event keeps q = C / P(m0^2) and point j, with a = f_j / f_0, gives
//           w_out = w (q0 a + q2 a m_j^2 + q4 a m_j^4);
//       points at the original top mass (any width or alpha_s) give w a exactly.
//       Consecutive threads write consecutive outputs.
// The top width enters no propagator of this diagram and is ignored.
//
// Precision.  FP64 mode: everything in FP64.  Mixed mode: B300 issues FP64 at 1/64
// of the FP32 rate (2 FMA per SM per clock), so the mixed tile runs no FP64
// instruction per output or per event: momenta and weights are converted
// FP64 <-> FP32 on the integer ALUs (IEEE-754 bit fields, round to nearest even),
// the constants, q and the per-point polynomial are FP32, and only points at the
// original mass take the FP64 product w a.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "fpconv.cuh"
#include "qq_amplitude.cuh"
#include "rex_internal.cuh"

namespace rex {

constexpr int QQ_BLOCK = 128;

template <typename R>
struct QqTile {
  static constexpr int EPB = QQ_BLOCK;
  static constexpr int ROW = 17;   // padded row of 16 momenta (conflict-free row reads)
  static constexpr bool MIXED = std::is_same<R, float>::value;

  struct Smem {
    double mom[EPB * ROW];
    alignas(16) R qw[EPB][4];    // C / P(m0^2) (0 if |M_0|^2 == 0) and w, per event
    double w[EPB];               // w_in in FP64 (0 if |M_0|^2 == 0, NaN if it is NaN)
    R pa[MAX_POINTS][3];         // a_j, a_j m_j^2, a_j m_j^4 with a_j = f_j / f_0
    double r[MAX_POINTS];        // a_j in FP64
    int same[MAX_POINTS];        // point j at the original top mass
    int any_same;
    R m0sq;
  };

  // w_out of event e (tile row) at point j
  template <bool SAME>
  static __device__ __forceinline__ double weight(const Smem& sm, int e, R a0, R a2, R a4, bool same, double r) {
    if (SAME && same) return sm.w[e] * r;
    R q[4];
    if constexpr (MIXED) {
      const float4 v = *reinterpret_cast<const float4*>(sm.qw[e]);
      q[0] = v.x; q[1] = v.y; q[2] = v.z; q[3] = v.w;
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) q[i] = sm.qw[e][i];
    }
    const R rho = fma(q[2], a4, fma(q[1], a2, q[0] * a0));
    if constexpr (MIXED) return f32_to_f64_alu(q[3] * rho);
    else return q[3] * rho;
  }

  // a8: every output of the tile; a thread keeps one point's constants in registers
  // and walks events, so consecutive threads write consecutive outputs of a row
  template <bool SAME>
  static __device__ __forceinline__ void write_outputs(const Smem& sm, int nblk, int k, int64_t ev0,
                                                       int64_t stride, double* __restrict__ out) {
    const int tid = threadIdx.x;
    if (k <= QQ_BLOCK) {
      const int ne = QQ_BLOCK / k;             // events per pass
      if (tid >= ne * k) return;
      const int e0 = tid / k, j = tid - e0 * k;
      const R a0 = sm.pa[j][0], a2 = sm.pa[j][1], a4 = sm.pa[j][2];
      const bool same = SAME && sm.same[j];
      const double r = SAME ? sm.r[j] : 0.0;
      double* o = out + (ev0 + e0) * stride + j;
      const int64_t step = (int64_t)ne * stride;
      for (int e = e0; e < nblk; e += ne, o += step) *o = weight<SAME>(sm, e, a0, a2, a4, same, r);
    } else {
      for (int j = tid; j < k; j += QQ_BLOCK) {
        const R a0 = sm.pa[j][0], a2 = sm.pa[j][1], a4 = sm.pa[j][2];
        const bool same = SAME && sm.same[j];
        const double r = SAME ? sm.r[j] : 0.0;
        double* o = out + ev0 * stride + j;
        for (int e = 0; e < nblk; ++e, o += stride) *o = weight<SAME>(sm, e, a0, a2, a4, same, r);
      }
    }
  }

  // EXCL: helicity-exclusive, hel[ev][0..3] = the event's (l1, l2, l3, l4)
  template <bool EXCL = false, class TABLE>
  static __device__ __forceinline__ void run(Smem& sm, const double* __restrict__ mom,
                                             const double* __restrict__ w_in, int64_t nev, int64_t tile,
                                             const TABLE& lp, double* __restrict__ out,
                                             const signed char* __restrict__ hel = nullptr) {
    const int tid = threadIdx.x;
    const int64_t ev0 = tile * EPB;
    const int nblk = (int)((nev - ev0) < EPB ? (nev - ev0) : EPB);
    // a1: coalesced 16-byte loads of the tile's [nblk][4][4] momenta
    const double2* src = reinterpret_cast<const double2*>(mom + ev0 * 16);
    for (int i = tid; i < nblk * 8; i += QQ_BLOCK) {
      const double2 v = __ldg(src + i);
      const int row = i >> 3, col = (i & 7) * 2;
      sm.mom[row * ROW + col] = v.x;
      sm.mom[row * ROW + col + 1] = v.y;
    }
    // a2: the launch's points
    const int k = lp.mode == OUT_RATIO ? lp.k : 0;
    if (tid == 0) {
      if constexpr (MIXED) {
        const float m0 = f64_to_f32_alu(lp.mass[0]);
        sm.m0sq = m0 * m0;
      } else {
        sm.m0sq = lp.mass[0] * lp.mass[0];
      }
      sm.any_same = 0;
    }
    __syncthreads();
    for (int j = tid; j < k; j += QQ_BLOCK) {
      const double m = lp.mass[lp.slot[j]];
      // the original mass (bitwise; masses are positive and finite)
      const int same = __double_as_longlong(m) == __double_as_longlong(lp.mass[0]);
      if constexpr (MIXED) {
        // FP32 without FP64 instructions (FP64 issues at 1/64 of the FP32 rate)
        const float mf = f64_to_f32_alu(m);
        const float a = f64_to_f32_alu(lp.factor[j]) / f64_to_f32_alu(lp.factor0);
        const float am2 = a * (mf * mf);
        sm.pa[j][0] = a;
        sm.pa[j][1] = am2;
        sm.pa[j][2] = am2 * (mf * mf);
        if (same) sm.r[j] = lp.factor[j] / lp.factor0;
      } else {
        const double a = lp.factor[j] / lp.factor0;
        const double am2 = a * (m * m);
        sm.pa[j][0] = a;
        sm.pa[j][1] = am2;
        sm.pa[j][2] = am2 * (m * m);
        sm.r[j] = a;
      }
      sm.same[j] = same;
      if (same) sm.any_same = 1;
    }
    if (tid < nblk) {
      R p[4][4];
      unsigned ahi_max = 0u;   // mixed: largest |momentum| high word
      double fin = 0.0;        // FP64: sum of 0 * momentum, NaN iff one is not finite
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const double v = sm.mom[tid * ROW + i];
        if constexpr (MIXED) {
          p[i >> 2][i & 3] = f64_to_f32_alu_finite(v, ahi_max);
        } else {
          p[i >> 2][i & 3] = v;
          fin = fma(v, 0.0, fin);
        }
      }
      R c[3], e12;
      if constexpr (EXCL) {
        const signed char* he = hel + (ev0 + tid) * 4;
        qq_ttx_coefficients_h<R>(p, he[0], he[1], he[2], he[3], c, &e12);
      } else {
        qq_ttx_coefficients<R>(p, c, &e12);
      }
      const R m0sq = sm.m0sq;
      R p0 = (c[2] * m0sq + c[1]) * m0sq + c[0];
      // a non-finite momentum (in the mixed mode also one beyond the FP32 range) makes
      // the event NaN; checked on the bit patterns (the energies of the massless
      // quarks cancel from the ratio, so arithmetic alone would not always show it)
      if constexpr (MIXED) {
        if (ahi_max >= (1151u << 20)) p0 = __int_as_float(0x7fc00000);
      } else {
        p0 += fin;
      }
      if (lp.mode == OUT_ME2) {
        // |M|^2 itself: times the incoming scale, 1/s^2 and the coupling factor (FP64)
        double q[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) q[m] = sm.mom[tid * ROW + m] + sm.mom[tid * ROW + 4 + m];
        const double s = q[0] * q[0] - q[1] * q[1] - q[2] * q[2] - q[3] * q[3];
        out[ev0 + tid] = double(p0) * double(e12) / (s * s) * lp.factor0;
        return;
      }
      const double w = w_in[ev0 + tid];
      const bool zero = p0 == R(0), bad = !(p0 == p0);
      const R inv = (zero || bad) ? R(0) : R(1) / p0;
      const double wz = zero ? 0.0 : (bad ? __longlong_as_double(0x7ff8000000000000LL) : w);
#pragma unroll
      for (int i = 0; i < 3; ++i) sm.qw[tid][i] = bad ? p0 : c[i] * inv;
      if constexpr (MIXED) sm.qw[tid][3] = f64_to_f32_alu(wz);
      else sm.qw[tid][3] = wz;
      sm.w[tid] = wz;
    }
    if (lp.mode != OUT_RATIO || k == 0) return;
    __syncthreads();
    if (sm.any_same) write_outputs<true>(sm, nblk, k, ev0, lp.out_stride, out);
    else write_outputs<false>(sm, nblk, k, ev0, lp.out_stride, out);
  }
};

}  // namespace rex
