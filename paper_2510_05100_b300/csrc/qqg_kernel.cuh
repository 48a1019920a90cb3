// q(1) q~(2) -> t(3) t~(4) g(5): the reweighting tile (sm_103a), shared by the
// standalone kernel and the persistent multi-process kernel.
//
// Blocks of 128 threads, 4 lanes per event (light-quark helicity pair x gluon
// polarisation), 32 events per tile.
//   a1     each lane loads its event's FP64 momenta (the 4 lanes read the same 160 B);
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

#include "qqg_amplitude.cuh"
#include "rex_internal.cuh"

namespace rex {

constexpr int QQG_BLOCK = 128;
constexpr int QQG_LANES = 4;

template <typename R>
struct QqgTile {
  static constexpr int EPB = QQG_BLOCK / QQG_LANES;

  struct Smem {
    double me2s[EPB][MAX_MASS + 1];
    double inv0[EPB];
  };

  template <class TABLE>
  static __device__ __forceinline__ void run(Smem& sm, const double* __restrict__ mom,
                                             const double* __restrict__ w_in, int64_t nev, int64_t tile,
                                             const TABLE& lp, double* __restrict__ out) {
    const int tid = threadIdx.x;
    const int el = tid / QQG_LANES, lane = tid % QQG_LANES;
    const int64_t ev0 = tile * EPB;
    const int64_t ev = ev0 + el;
    const bool valid = ev < nev;
    const int64_t evc = valid ? ev : nev - 1;
    double pd[5][4];
    R p[5][4];
    const double2* src = reinterpret_cast<const double2*>(mom + evc * 20);
#pragma unroll
    for (int i = 0; i < 10; ++i) {
      const double2 v = __ldg(src + i);
      pd[(2 * i) >> 2][(2 * i) & 3] = v.x;
      pd[(2 * i + 1) >> 2][(2 * i + 1) & 3] = v.y;
    }
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
      for (int m = 0; m < 4; ++m) p[i][m] = R(pd[i][m]);
    QqgLane<R> L;
    qqg_lane_setup<R>(pd, p, lane & 1, lane >> 1, L);
    for (int s = 0; s < lp.nmass; ++s) {
      R part = valid ? qqg_slot<R>(L, lp.mass[s], lp.width[s]) : R(0);
      part += __shfl_xor_sync(0xffffffffu, part, 1);
      part += __shfl_xor_sync(0xffffffffu, part, 2);
      if (lane == 0) sm.me2s[el][s] = double(part);
    }
    __syncthreads();
    const int nblk = (int)((nev - ev0) < EPB ? (nev - ev0) : EPB);
    if (lp.mode == OUT_RATIO) {
      const int k = lp.k;
      if constexpr (std::is_same<R, double>::value) {
        for (int idx = tid; idx < nblk * k; idx += QQG_BLOCK) {
          const int e = idx / k;
          const int j = idx - e * k;
          const double m0 = sm.me2s[e][0] * lp.factor0;
          const double mj = sm.me2s[e][lp.slot[j]] * lp.factor[j];
          const double w = w_in[ev0 + e];
          out[(ev0 + e) * lp.out_stride + j] = (m0 == 0.0) ? 0.0 : w * (mj / m0);
        }
      } else {
        for (int e = tid; e < nblk; e += QQG_BLOCK) {
          const double m0 = sm.me2s[e][0] * lp.factor0;
          sm.inv0[e] = m0 == 0.0 ? 0.0 : 1.0 / m0;
        }
        __syncthreads();
        for (int idx = tid; idx < nblk * k; idx += QQG_BLOCK) {
          const int e = idx / k;
          const int j = idx - e * k;
          const double m0 = sm.me2s[e][0] * lp.factor0;
          const double mj = sm.me2s[e][lp.slot[j]] * lp.factor[j];
          const double w = w_in[ev0 + e];
          out[(ev0 + e) * lp.out_stride + j] = (m0 == 0.0) ? 0.0 : (mj == m0 ? w : w * (mj * sm.inv0[e]));
        }
      }
    } else {
      for (int e = tid; e < nblk; e += QQG_BLOCK) out[ev0 + e] = sm.me2s[e][0] * lp.factor0;
    }
  }
};

}  // namespace rex
