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
//   a8  ratio epilogue w_out = w_in |M_j|^2 / |M_0|^2 (0 if |M_0|^2 == 0), one
//       FP64 reciprocal per event, consecutive threads writing consecutive outputs.
// The top width enters no propagator of this diagram and is ignored.  FP64 in
// the exact mode; in the mixed mode the per-event constants are built in FP32
// from FP32 momenta, and s, the polynomial and the epilogue stay FP64.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "qq_amplitude.cuh"
#include "rex_internal.cuh"

namespace rex {

constexpr int QQ_BLOCK = 128;

template <typename R>
struct QqTile {
  static constexpr int EPB = QQ_BLOCK;
  static constexpr int ROW = 17;   // padded row of 16 momenta (conflict-free row reads)

  struct Smem {
    double mom[EPB * ROW];
    double c[3][EPB];
    double m0[EPB];
    double inv0[EPB];
    double w[EPB];
    double pt[MAX_POINTS][2];    // (m^2, factor) per point of the launch
  };

  template <class TABLE>
  static __device__ __forceinline__ void run(Smem& sm, const double* __restrict__ mom,
                                             const double* __restrict__ w_in, int64_t nev, int64_t tile,
                                             const TABLE& lp, double* __restrict__ out) {
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
    // a2: the launch's points (m^2, factor)
    const int k = lp.mode == OUT_RATIO ? lp.k : 0;
    for (int j = tid; j < k; j += QQ_BLOCK) {
      const double m = lp.mass[lp.slot[j]];
      sm.pt[j][0] = m * m;
      sm.pt[j][1] = lp.factor[j];
    }
    __syncthreads();
    if (tid < nblk) {
      double p[4][4];
#pragma unroll
      for (int i = 0; i < 16; ++i) p[i >> 2][i & 3] = sm.mom[tid * ROW + i];
      double c[3];
      qq_ttx_coefficients<R>(p, c);
      const double m2 = lp.mass[0] * lp.mass[0];
      const double m0 = ((c[2] * m2 + c[1]) * m2 + c[0]) * lp.factor0;
      sm.c[0][tid] = c[0];
      sm.c[1][tid] = c[1];
      sm.c[2][tid] = c[2];
      sm.m0[tid] = m0;
      sm.inv0[tid] = m0 == 0.0 ? 0.0 : 1.0 / m0;
      if (lp.mode == OUT_ME2) out[ev0 + tid] = m0;
      else sm.w[tid] = w_in[ev0 + tid];
    }
    if (lp.mode != OUT_RATIO) return;
    __syncthreads();
    for (int idx = tid; idx < nblk * k; idx += QQ_BLOCK) {
      const int e = idx / k;
      const int j = idx - e * k;
      const double m2 = sm.pt[j][0];
      const double mj = ((sm.c[2][e] * m2 + sm.c[1][e]) * m2 + sm.c[0][e]) * sm.pt[j][1];
      const double m0 = sm.m0[e], w = sm.w[e];
      out[(ev0 + e) * lp.out_stride + j] = (m0 == 0.0) ? 0.0 : (mj == m0 ? w : w * (mj * sm.inv0[e]));
    }
  }
};

}  // namespace rex
