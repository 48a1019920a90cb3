// e+(1) e-(2) -> mu+(3) mu-(4) through photon and Z: device code shared by the
// standalone kernel and the persistent multi-process kernel.
//
// Thread per event.  For each of the 16 helicity configurations the chiral
// lepton currents  Je_X = vbar(p1) gamma^mu P_X u(p2),  Jm_Y = ubar(p4) gamma^mu P_Y v(p3)
// are parameter independent; a parameter point only changes the coefficients
//     amp = e^2 Q^2 / s (Je . Jm) + sum_{X,Y} gZ^2 g_X g_Y / (s - mZ^2 + i mZ GZ) (JeX . JmY),
// (FFV1P0_3-style vector/chiral currents closed FFV1_0-style).
#pragma once
#include <cuda_runtime.h>

#include "helas.cuh"
#include "rex_internal.cuh"

namespace rex {

// b^dag sigmabar^mu a (left, sign -1 on the spatial part) or b^dag sigma^mu a (right)
__device__ __forceinline__ void chiral_current(const cx<double>* b, const cx<double>* a, double sgn,
                                               cx<double>* j) {
  const cx<double> b0a0 = cdot1(b[0], a[0]), b0a1 = cdot1(b[0], a[1]);
  const cx<double> b1a0 = cdot1(b[1], a[0]), b1a1 = cdot1(b[1], a[1]);
  j[0] = b0a0 + b1a1;
  const cx<double> sx = b0a1 + b1a0;
  // b^dag sigma_y a = -i b0* a1 + i b1* a0
  const cx<double> d = b1a0 - b0a1;
  const cx<double> sy = cx<double>{-d.im, d.re};
  const cx<double> sz = b0a0 - b1a1;
  j[1] = sgn * sx;
  j[2] = sgn * sy;
  j[3] = sgn * sz;
}

__device__ __forceinline__ cx<double> cmdot(const cx<double>* a, const cx<double>* b) {
  return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}

// One tile of 128 events, thread per event.  TABLE: k, mode, out_stride, pt[0..k].
//
// With d_a(h) = JeX(h).JmY(h) for the four chirality pairs a = (X, Y) and the
// point's coefficients c_a, the helicity sum is a Hermitian form
//     sum_h |sum_a c_a d_a(h)|^2 = c^dag H c,   H_ab = sum_h conj(d_a(h)) d_b(h),
// so H (parameter independent) is built once per event and every point costs one
// 4x4 form.
//
// Helicity filtering: the leptons are massless, so a vector or axial current of a
// fermion-antifermion pair vanishes unless their helicities are opposite.  Of the
// 16 configurations only (l1, l2, l3, l4) = (+,-,+,-), (-,+,+,-), (+,-,-,+), (-,+,-,+)
// (h = 5, 6, 9, 10) reach H; the other 12 contribute exact zeros (their spinor halves
// are w- chi with w- = 0/w+ = 0), so summing the 4 gives the same H bit for bit.
//
// Helicity-exclusive form (EXCL): H is built from the event's own configuration
// hel[ev][0..3] = (l1, l2, l3, l4) (positive: +1, otherwise -1) alone; a configuration
// the chirality rule forbids gives H = 0, hence |M_0|^2 = 0 and new weights 0.
template <class TABLE, bool EXCL = false, int TPB = 128>
__device__ __forceinline__ void ee_tile(const double* __restrict__ mom, const double* __restrict__ w_in,
                                        int64_t nev, int64_t tile, const TABLE& lp, double* __restrict__ out,
                                        const signed char* __restrict__ hel = nullptr) {
  const int64_t ev = tile * TPB + threadIdx.x;
  if (ev >= nev) return;
  double p[4][4];
  const double2* src = reinterpret_cast<const double2*>(mom + ev * 16);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const double2 v = __ldg(src + i);
    p[i / 2][(i % 2) * 2] = v.x;
    p[i / 2][(i % 2) * 2 + 1] = v.y;
  }
  double q[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) q[m] = p[0][m] + p[1][m];
  const double s = mdot(q, q);

  // H: diagonal (real) and upper triangle (complex) of the 4x4 Hermitian form
  double hd[4] = {0.0, 0.0, 0.0, 0.0};
  cx<double> ho[6] = {};
  int hev = 0;
  if constexpr (EXCL) {
    const signed char* he = hel + ev * 4;
    hev = (he[0] > 0 ? 1 : 0) | (he[1] > 0 ? 2 : 0) | (he[2] > 0 ? 4 : 0) | (he[3] > 0 ? 8 : 0);
  }
  // both helicity spinors of every lepton from one helicity basis and one omega_+
  // per lepton (massless: omega_- = 0); index 0: helicity -, 1: +.  FP64 square roots
  // are the expensive part of this thread's work on B300, so they are not repeated
  // per configuration.
  cx<double> v1[2][4], u2[2][4], v3[2][4], u4[2][4];
  {
    cx<double> chi[2][2];
    double pabs, wp, wm;
    omegas(p[0], 0.0, &pabs, &wp, &wm);
    chi_pair(p[0], pabs, chi[1], chi[0]);
    spinor_v_from(chi, wp, wm, v1);
    omegas(p[1], 0.0, &pabs, &wp, &wm);
    chi_pair(p[1], pabs, chi[1], chi[0]);
    spinor_u_from(chi, wp, wm, u2);
    omegas(p[2], 0.0, &pabs, &wp, &wm);
    chi_pair(p[2], pabs, chi[1], chi[0]);
    spinor_v_from(chi, wp, wm, v3);
    omegas(p[3], 0.0, &pabs, &wp, &wm);
    chi_pair(p[3], pabs, chi[1], chi[0]);
    spinor_u_from(chi, wp, wm, u4);
  }
#pragma unroll 1
  for (int hi = 0; hi < (EXCL ? 1 : 4); ++hi) {
    const int h = EXCL ? hev : ((hi & 1) ? 6 : 5) + ((hi & 2) ? 4 : 0);   // 5, 6, 9, 10
    const int i1 = h & 1, i2 = (h >> 1) & 1, i3 = (h >> 2) & 1, i4 = (h >> 3) & 1;
    cx<double> je[2][4], jm[2][4];
    chiral_current(v1[i1], u2[i2], -1.0, je[0]);          // vbar1 gamma P_L u2
    chiral_current(v1[i1] + 2, u2[i2] + 2, 1.0, je[1]);   // vbar1 gamma P_R u2
    chiral_current(u4[i4], v3[i3], -1.0, jm[0]);          // ubar4 gamma P_L v3
    chiral_current(u4[i4] + 2, v3[i3] + 2, 1.0, jm[1]);   // ubar4 gamma P_R v3
    cx<double> d[4];
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
      for (int y = 0; y < 2; ++y) d[2 * x + y] = cmdot(je[x], jm[y]);
    int o = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      hd[a] += d[a].re * d[a].re + d[a].im * d[a].im;
#pragma unroll
      for (int b2 = a + 1; b2 < 4; ++b2) {
        ho[o] = ho[o] + cdot1(d[a], d[b2]);   // conj(d_a) d_b
        ++o;
      }
    }
  }

  double me2_0 = 0.0;
  for (int j = 0; j <= lp.k; ++j) {
    const EwPoint& c = lp.pt[j];
    const double den_re = s - c.mz2, den_im = c.mzwz;
    const double nn = 1.0 / (den_re * den_re + den_im * den_im);
    const cx<double> dz = cx<double>{den_re * nn, -den_im * nn};   // 1/(s - mZ^2 + i mZ GZ)
    const double ca = c.e2qq / s;
    cx<double> coef[4];
#pragma unroll
    for (int xy = 0; xy < 4; ++xy) coef[xy] = cx<double>{ca, 0.0} + c.gzz[xy] * dz;
    // sum_h |sum_a c_a d_a|^2 = sum_ab conj(c_a) c_b H_ab
    //                        = sum_a |c_a|^2 H_aa + 2 Re sum_{a<b} conj(c_a) c_b H_ab
    double sum = 0.0;
    int o = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      sum += (coef[a].re * coef[a].re + coef[a].im * coef[a].im) * hd[a];
#pragma unroll
      for (int b2 = a + 1; b2 < 4; ++b2) {
        const cx<double> cc = cdot1(coef[a], coef[b2]);   // conj(c_a) c_b
        const cx<double> t = cc * ho[o++];
        sum += 2.0 * t.re;
      }
    }
    const double me2 = sum * c.avg;
    if (lp.mode == OUT_ME2) {
      out[ev] = me2;
      return;
    }
    if (j == 0) {
      me2_0 = me2;
    } else {
      out[ev * lp.out_stride + (j - 1)] = (me2_0 == 0.0) ? 0.0 : w_in[ev] * (me2 / me2_0);
    }
  }
}

// The helicity sum with four lanes per event (standalone kernel, blocks of 128 =
// 32 events): lane q evaluates configuration h = 5, 6, 9, 10 for q = 0..3.  Lane q
// builds lepton q's helicity basis and omega_+ (the FP64 square roots, once per
// lepton), the lanes exchange the parts their configuration needs, each forms its d_a
// and H contribution, and a butterfly over the four lanes sums H.  Every lane then
// evaluates the original point and every fourth new point.  B300 issues FP64 at 2
// FMA per clock per SM, so for a sample of a few thousand events the chain a thread
// carries, not the pipe, sets the time: a quarter of the thread-per-event chain.
template <class TABLE>
__device__ __forceinline__ void ee_tile_split(const double* __restrict__ mom, const double* __restrict__ w_in,
                                              int64_t nev, int64_t tile, const TABLE& lp, double* __restrict__ out) {
  const int q = threadIdx.x & 3;
  const int64_t ev = tile * 32 + (threadIdx.x >> 2);
  const bool valid = ev < nev;
  const int64_t evc = valid ? ev : nev - 1;
  double p[4][4];
  const double2* src = reinterpret_cast<const double2*>(mom + evc * 16);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const double2 v = __ldg(src + i);
    p[i / 2][(i % 2) * 2] = v.x;
    p[i / 2][(i % 2) * 2 + 1] = v.y;
  }
  double qs[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) qs[m] = p[0][m] + p[1][m];
  const double s = mdot(qs, qs);
  // lepton q: helicity 2-spinors chi-, chi+ and omega_+ (massless: omega_- = 0)
  cx<double> chi[2][2];
  double wp;
  {
    double pabs, wm;
    const double* pq = q == 0 ? p[0] : (q == 1 ? p[1] : (q == 2 ? p[2] : p[3]));
    omegas(pq, 0.0, &pabs, &wp, &wm);
    chi_pair(pq, pabs, chi[1], chi[0]);
  }
  // this lane's configuration: helicity index (0: -, 1: +) of each lepton
  const int h = (q & 1 ? 6 : 5) + (q & 2 ? 4 : 0);
  const int base = threadIdx.x & 28;   // lane 0 of the event within the warp
  cx<double> sp[4][4];                 // v1, u2, v3, u4 of the configuration
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    // lepton t's 2-spinor for this lane's helicity, and its omega_+, from lane t
    const int it = (h >> t) & 1;
    const unsigned src_lane = (unsigned)(base + t);
    cx<double> c[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        c[a][b].re = __shfl_sync(0xffffffffu, chi[a][b].re, src_lane);
        c[a][b].im = __shfl_sync(0xffffffffu, chi[a][b].im, src_lane);
      }
    const double w = __shfl_sync(0xffffffffu, wp, src_lane);
    cx<double> both[2][4];
    if (t == 0 || t == 2) spinor_v_from(c, w, 0.0, both);
    else spinor_u_from(c, w, 0.0, both);
#pragma unroll
    for (int i = 0; i < 4; ++i) sp[t][i] = both[it][i];
  }
  cx<double> je[2][4], jm[2][4];
  chiral_current(sp[0], sp[1], -1.0, je[0]);          // vbar1 gamma P_L u2
  chiral_current(sp[0] + 2, sp[1] + 2, 1.0, je[1]);   // vbar1 gamma P_R u2
  chiral_current(sp[3], sp[2], -1.0, jm[0]);          // ubar4 gamma P_L v3
  chiral_current(sp[3] + 2, sp[2] + 2, 1.0, jm[1]);   // ubar4 gamma P_R v3
  cx<double> d[4];
#pragma unroll
  for (int x = 0; x < 2; ++x)
#pragma unroll
    for (int y = 0; y < 2; ++y) d[2 * x + y] = cmdot(je[x], jm[y]);
  double hd[4];
  cx<double> ho[6];
  {
    int o = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      hd[a] = d[a].re * d[a].re + d[a].im * d[a].im;
#pragma unroll
      for (int b2 = a + 1; b2 < 4; ++b2) ho[o++] = cdot1(d[a], d[b2]);   // conj(d_a) d_b
    }
  }
#pragma unroll
  for (int off = 1; off < 4; off <<= 1) {
#pragma unroll
    for (int a = 0; a < 4; ++a) hd[a] += __shfl_xor_sync(0xffffffffu, hd[a], off);
#pragma unroll
    for (int o = 0; o < 6; ++o) {
      ho[o].re += __shfl_xor_sync(0xffffffffu, ho[o].re, off);
      ho[o].im += __shfl_xor_sync(0xffffffffu, ho[o].im, off);
    }
  }
  if (!valid) return;
  auto me2_at = [&](const EwPoint& c) {
    const double den_re = s - c.mz2, den_im = c.mzwz;
    const double nn = 1.0 / (den_re * den_re + den_im * den_im);
    const cx<double> dz = cx<double>{den_re * nn, -den_im * nn};   // 1/(s - mZ^2 + i mZ GZ)
    const double ca = c.e2qq / s;
    cx<double> coef[4];
#pragma unroll
    for (int xy = 0; xy < 4; ++xy) coef[xy] = cx<double>{ca, 0.0} + c.gzz[xy] * dz;
    double sum = 0.0;
    int o = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      sum += (coef[a].re * coef[a].re + coef[a].im * coef[a].im) * hd[a];
#pragma unroll
      for (int b2 = a + 1; b2 < 4; ++b2) {
        const cx<double> t = cdot1(coef[a], coef[b2]) * ho[o++];
        sum += 2.0 * t.re;
      }
    }
    return sum * c.avg;
  };
  const double me2_0 = me2_at(lp.pt[0]);
  if (lp.mode == OUT_ME2) {
    if (q == 0) out[ev] = me2_0;
    return;
  }
  for (int j = 1 + q; j <= lp.k; j += 4) {
    const double me2 = me2_at(lp.pt[j]);
    out[ev * lp.out_stride + (j - 1)] = (me2_0 == 0.0) ? 0.0 : w_in[ev] * (me2 / me2_0);
  }
}

static __global__ void __launch_bounds__(128)
    ee_reweight_split_kernel(const double* __restrict__ mom, const double* __restrict__ w_in, int64_t nev,
                             const __grid_constant__ EwLaunch lp, double* __restrict__ out) {
  ee_tile_split<EwLaunch>(mom, w_in, nev, (int64_t)blockIdx.x, lp, out);
}

template <bool EXCL, int TPB>
static __global__ void __launch_bounds__(TPB)
    ee_reweight_kernel(const double* __restrict__ mom, const double* __restrict__ w_in, int64_t nev,
                       const __grid_constant__ EwLaunch lp, double* __restrict__ out,
                       const signed char* __restrict__ hel) {
  ee_tile<EwLaunch, EXCL, TPB>(mom, w_in, nev, (int64_t)blockIdx.x, lp, out, hel);
}

}  // namespace rex
