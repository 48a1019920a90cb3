// q(1) q~(2) -> t(3) t~(4) g(5): the reweighting tile (sm_103a), shared by the
// standalone kernel and the persistent multi-process kernel.
//
// Blocks of 128 threads, 4 lanes per event (light-quark helicity pair x gluon
// polarisation), 32 events per tile.
//   a1     each lane loads its event's FP64 momenta (the 4 lanes read the same 160 B);
//          the six FP64 invariants of the tile's 32 events are computed once, warp w
//          taking invariant w (warps 0, 1 also 4, 5) for every event, so no lane
//          diverges; in the mixed mode these are the only FP64 instructions per
//          event (B300 issues FP64 at 1/64 of the FP32 rate): momenta and invariants
//          are converted on the integer ALUs, reciprocals and every per-slot
//          quantity (m, m0^2 - m^2, m Gamma from a per-block table) are FP32;
//   a3-a5  the lane builds its parameter-independent currents once
//          (qqg_lane_setup), then per distinct (m_t, Gamma_t) slot its 4 top-helicity
//          pairs' 5 amplitudes (qqg_slot);
//   a6-a7  integer colour form, helicity sum over the lane's 4 pairs and across the 4
//          lanes (warp shuffles): FP64 in the exact mode, FP32 in the mixed mode
//          (non-negative terms);
//   a8     ratio epilogue w_out = w_in |M_j|^2 / |M_0|^2 (0 if |M_0|^2 == 0) in FP64,
//          consecutive threads writing consecutive outputs.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "df64.cuh"
#include "fpconv.cuh"
#include "qqg_amplitude.cuh"
#include "rex_internal.cuh"

namespace rex {

// qqg_form for double-float amplitudes: the fifteen colour-weighted products as one
// sum, each added with one TwoSum, one renormalisation at the end
__device__ __forceinline__ df64 qqg_form(const cx<df64> (&a)[5]) {
  float s = 0.f, c = 0.f;
#pragma unroll
  for (int d = 0; d < 5; ++d)
#pragma unroll
    for (int d2 = d; d2 < 5; ++d2) {
      const df64 w = df64(qqg_colour(d, d2) * (d == d2 ? 1 : 2));
      df64_acc_term(s, c, w * a[d].re, a[d2].re);
      df64_acc_term(s, c, w * a[d].im, a[d2].im);
    }
  return df64_renorm(s, c);
}

}  // namespace rex

namespace rex {

constexpr int QQG_BLOCK = 128;
constexpr int QQG_LANES = 4;

constexpr QqgCrossing kQqgDirect = {{0, 1, 2, 3, 4}, {0, 0, 0, 0, 0}};

// x with its sign flipped where neg (an integer XOR on the high word: no FP64 issue)
__device__ __forceinline__ double qqg_flip(double x, bool neg) {
  return __hiloint2double(__double2hiint(x) ^ (neg ? (int)0x80000000 : 0), __double2loint(x));
}

// Invariant t of an event (FP64 because (p1 - k)^2 and the top denominators cancel
// for collinear or soft gluons), over the slot momenta of the channel cr:
// t = 0 s, 1 s', 2 (p1 - k)^2, 3 (k - p2)^2, 4 (p3 + k)^2 - m0^2, 5 (p4 + k)^2 - m0^2;
// p: the event's [5][4] FP64 record.
__device__ __forceinline__ double qqg_invariant_fp64(const double* __restrict__ p, int t, double m0,
                                                     const QqgCrossing& cr) {
  // the two slots and the sign: t -> (a, b, minus) with x = p_a -/+ p_b
  const int a = t == 0 ? 0 : (t == 1 ? 2 : (t == 2 ? 0 : (t == 3 ? 4 : (t == 4 ? 2 : 3))));
  const int b = t == 0 ? 1 : (t == 1 ? 3 : (t == 2 ? 4 : (t == 3 ? 1 : 4)));
  const bool minus = t == 2 || t == 3;
  const double* pa = p + 4 * cr.src[a];
  const double* pb = p + 4 * cr.src[b];
  const bool na = cr.neg[a] != 0, nb = (cr.neg[b] != 0) != minus;
  double x[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) x[m] = qqg_flip(pa[m], na) + qqg_flip(pb[m], nb);
  const double v = mdot(x, x);
  return t >= 4 ? v - m0 * m0 : v;
}

// T_CHANNEL: the channel's light line is crossed (q g, q~ g and their beam swaps), so
// the gluon on it is a t-channel one and the lanes take the gauge split of their
// current when it is forward (qqg_lane_gauge_split); the direct q q~ channel and q~ q
// run the plain tile.
template <typename R, bool T_CHANNEL = false>
struct QqgTile {
  static constexpr int EPB = QQG_BLOCK / QQG_LANES;

  struct Smem {
    double me2s[EPB][MAX_MASS + 1];
    double mult[MAX_POINTS];   // mixed mode: per point, f_j / f_0 (slot 0) or f_j
    int slotj[MAX_POINTS];     // mixed mode: per point, its mass slot
    R mr[MAX_MASS], dm2[MAX_MASS], mw[MAX_MASS];   // per slot: m, m0^2 - m^2, m Gamma
    R inv[T_CHANNEL ? 8 : 6][EPB];                 // per event: the invariants (1/x for 0..3)
    QqgSplit<R> split[T_CHANNEL ? QQG_BLOCK : 1];  // per lane: current, vertex vector, gauge split
  };

  static __device__ __forceinline__ R to_r(double x) {
    if constexpr (std::is_same<R, float>::value) return f64_to_f32_alu(x);
    else return x;
  }

  // EXCL: helicity-exclusive, hel[ev][0..4] = the event's (l1, l2, l3, l4, lg); the
  // event's one configuration is evaluated by each of its 4 lanes for every 4th slot.
  // cr: the channel (the direct one for EXCL).
  template <bool EXCL = false, class TABLE>
  static __device__ __forceinline__ void run(Smem& sm, const double* __restrict__ mom,
                                             const double* __restrict__ w_in, int64_t nev, int64_t tile,
                                             const TABLE& lp, double* __restrict__ out,
                                             const signed char* __restrict__ hel = nullptr,
                                             const QqgCrossing& cr = kQqgDirect) {
    const int tid = threadIdx.x;
    const int el = tid / QQG_LANES, lane = tid % QQG_LANES;
    const int64_t ev0 = tile * EPB;
    const int64_t ev = ev0 + el;
    const bool valid = ev < nev;
    const int64_t evc = valid ? ev : nev - 1;
    // per-slot table (slot 0 is the reference mass m0)
    for (int s = tid; s < lp.nmass; s += QQG_BLOCK) {
      const double m = lp.mass[s], m0 = lp.mass[0];
      sm.mr[s] = to_r(m);
      sm.dm2[s] = to_r((m0 - m) * (m0 + m));
      sm.mw[s] = to_r(m * lp.width[s]);
    }
    double pd[5][4];
    R p[5][4];
    static_assert(EPB == 32 && QQG_BLOCK == 128, "one warp per invariant type over the tile's 32 events");
    // slot i <- the channel's particle cr.src[i], its sign flipped where crossed
    const double2* src = reinterpret_cast<const double2*>(mom + evc * 20);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const double2* q = src + 2 * cr.src[i];
      const double2 v0 = __ldg(q), v1 = __ldg(q + 1);
      const bool ng = cr.neg[i] != 0;
      pd[i][0] = qqg_flip(v0.x, ng);
      pd[i][1] = qqg_flip(v0.y, ng);
      pd[i][2] = qqg_flip(v1.x, ng);
      pd[i][3] = qqg_flip(v1.y, ng);
    }
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
      for (int m = 0; m < 4; ++m) p[i][m] = to_r(pd[i][m]);
    // the tile's invariants: warp w, lane e -> invariant w and 4 + w of event e
    // (6, 7: p3^2 - m0^2 and p4^2 - m0^2 of the top and antitop, for the gauge split)
    {
      const int w = tid >> 5, e = tid & 31;
      const int64_t ei = ev0 + e < nev ? ev0 + e : nev - 1;
      const double* pe = mom + ei * 20;
      const double m0 = lp.mass[0];
      const double v = qqg_invariant_fp64(pe, w, m0, cr);
      sm.inv[w][e] = R(1) / to_r(v);
      if (w < 2) {
        sm.inv[4 + w][e] = to_r(qqg_invariant_fp64(pe, 4 + w, m0, cr));
      } else if constexpr (T_CHANNEL) {
        const double* pt = pe + 4 * cr.src[w];   // slots 2, 3: the top and antitop, never crossed
        sm.inv[4 + w][e] = to_r(mdot(pt, pt) - m0 * m0);
      }
    }
    if constexpr (EXCL) {
      QqgLaneH<R> L;
      qqg_lane_setup_h<R>(p, hel + evc * 5, L);
      __syncthreads();
      QqgInvariants<R> inv;
      inv.is = sm.inv[0][el];
      inv.isp = sm.inv[1][el];
      inv.ia1 = sm.inv[2][el];
      inv.ia2 = sm.inv[3][el];
      inv.d3 = sm.inv[4][el];
      inv.d4 = sm.inv[5][el];
      qqg_lane_scale_h(inv, L);
      for (int s = lane; s < lp.nmass; s += QQG_LANES)
        sm.me2s[el][s] = valid ? double(qqg_slot_h<R>(L, sm.mr[s], sm.dm2[s], sm.mw[s])) : 0.0;
    } else {
      QqgLane<R> L;
      qqg_lane_setup<R>(p, lane & 1, lane >> 1, L, (cr.neg[0] ? 1 : 0) | (cr.neg[1] ? 2 : 0) | (cr.neg[4] ? 4 : 0));
      __syncthreads();
      QqgInvariants<R> inv;
      inv.is = sm.inv[0][el];
      inv.isp = sm.inv[1][el];
      inv.ia1 = sm.inv[2][el];
      inv.ia2 = sm.inv[3][el];
      inv.d3 = sm.inv[4][el];
      inv.d4 = sm.inv[5][el];
      qqg_lane_scale(inv, L);
      // a gluon of small virtuality on the light line (a forward light quark of a
      // crossed channel, |s| < s' / 256): the gauge split keeps its cancellation out of
      // the arithmetic
      if constexpr (T_CHANNEL) {
        // a forward light quark (|t| < s' / 256): the gauge split keeps the cancellation of
        // the t-channel gluon's diagrams out of the arithmetic
        QqgSplit<R>& sp = sm.split[tid];
        qqg_split_clear(sp);
        if (abs(inv.is) > R(256) * abs(inv.isp))
          qqg_lane_gauge_split<R>(pd, lane & 1, (cr.neg[0] ? 1 : 0) | (cr.neg[1] ? 2 : 0), sm.inv[6][el],
                                  sm.inv[7][el], L, sp);
        for (int s = 0; s < lp.nmass; ++s) {
          R part = valid ? qqg_slot_split<R>(L, sm.mr[s], sm.dm2[s], sm.mw[s], &sp) : R(0);
          part += shfl_xor(part, 1);
          part += shfl_xor(part, 2);
          if (lane == 0) sm.me2s[el][s] = double(part);
        }
      } else {
      for (int s = 0; s < lp.nmass; ++s) {
        R part = valid ? qqg_slot<R>(L, sm.mr[s], sm.dm2[s], sm.mw[s]) : R(0);
        part += shfl_xor(part, 1);
        part += shfl_xor(part, 2);
        if (lane == 0) sm.me2s[el][s] = double(part);
      }
      }
    }
    __syncthreads();
    const int nblk = (int)((nev - ev0) < EPB ? (nev - ev0) : EPB);
    if (lp.mode == OUT_RATIO) {
      const int k = lp.k;
      if constexpr (!std::is_same<R, float>::value) {   // FP64 and double-float
        for (int idx = tid; idx < nblk * k; idx += QQG_BLOCK) {
          const int e = idx / k;
          const int j = idx - e * k;
          const double m0 = sm.me2s[e][0] * lp.factor0;
          const double mj = sm.me2s[e][lp.slot[j]] * lp.factor[j];
          const double w = w_in[ev0 + e];
          out[(ev0 + e) * lp.out_stride + j] = (m0 == 0.0) ? 0.0 : w * (mj / m0);
        }
      } else {
        // mixed mode: per event the slot sums become w |M_s|^2 / |M_0|^2 with one FP64
        // division and slot 0 holds w itself (0 if |M_0|^2 == 0, NaN if it is NaN); each
        // output is one FP64 product with the point's multiplier (f_j / f_0 on the
        // original slot, so an unchanged point keeps its weight exactly, f_j elsewhere)
        for (int j = tid; j < k; j += QQG_BLOCK) {
          sm.slotj[j] = lp.slot[j];
          sm.mult[j] = lp.slot[j] == 0 ? lp.factor[j] / lp.factor0 : lp.factor[j];
        }
        for (int e = tid; e < nblk; e += QQG_BLOCK) {
          const double m0 = sm.me2s[e][0] * lp.factor0;
          const double w = w_in[ev0 + e];
          const double wi = m0 == 0.0 ? 0.0 : w / m0;
          for (int sl = 1; sl < lp.nmass; ++sl) sm.me2s[e][sl] *= wi;
          sm.me2s[e][0] = m0 == 0.0 ? 0.0 : (m0 == m0 ? w : m0);
        }
        __syncthreads();
        const int kk = k > 0 ? k : 1;
        int e = tid / kk, j = tid - (tid / kk) * kk;
        const int de = QQG_BLOCK / kk, dj = QQG_BLOCK - (QQG_BLOCK / kk) * kk;
        for (int idx = tid; idx < nblk * k; idx += QQG_BLOCK) {
          out[(ev0 + e) * lp.out_stride + j] = sm.me2s[e][sm.slotj[j]] * sm.mult[j];
          e += de;
          j += dj;
          if (j >= k) {
            j -= k;
            ++e;
          }
        }
      }
    } else {
      for (int e = tid; e < nblk; e += QQG_BLOCK) out[ev0 + e] = sm.me2s[e][0] * lp.factor0;
    }
  }
};

}  // namespace rex
