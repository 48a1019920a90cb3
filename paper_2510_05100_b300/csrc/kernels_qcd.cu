// Fused reweighting kernels for g g -> t t~ + k g on sm_103a.
//
// One launch runs every step of the hot path for a tile of events:
//   a1  FP64 momenta [nev][npart][4] -> registers (outgoing-momentum convention)
//   a3  external wavefunctions (linear gluon polarisations; top spinors per mass)
//   a4  colour-ordered gluon currents (once per event and gluon polarisation,
//       shared by every parameter point) and off-shell top currents (per mass)
//   a5  colour-flow amplitudes A(s) (jamps)
//   a6  colour sum  sum_{s,s'} conj(A_s) C_ss' A_s'  with the exact integer matrix
//   a7  helicity sum: top/antitop helicities inside the thread, gluon
//       polarisations across the NGHEL lanes of the event (warp shuffles), FP64
//   a8  ratio epilogue  w_out = w_in * |M_j|^2 / |M_0|^2  (0 if |M_0|^2 == 0)
//
// Thread mapping: NGHEL = 2^n lanes per event (one gluon polarisation
// configuration each), 128 threads per block, 128/NGHEL events per block.
// The amplitude is evaluated once per distinct (mt, Gamma_t) slot; alpha_s
// enters only through the exact overall factor (4 pi alpha_s)^n of a
// tree amplitude with n external gluons and no other coupling.
#include <cuda_runtime.h>

#include "generated/qcd_amplitudes.cuh"
#include "rex_internal.cuh"

namespace rex {

template <int PROC>
struct QcdProc;

#define REX_QCD_PROC(KIND, NAME)                                                              \
  template <>                                                                                 \
  struct QcdProc<KIND> {                                                                      \
    using info = NAME##_info;                                                                 \
    template <typename R>                                                                     \
    using gluons = NAME##_gluons<R>;                                                          \
    template <typename R>                                                                     \
    static __device__ __forceinline__ void gluon_state(const R (&pg)[info::NGLUON][4],        \
                                                       const R (&eps)[info::NGLUON][4],       \
                                                       const R (&ptb)[4], gluons<R>& st) {    \
      NAME##_gluon_state(pg, eps, ptb, st);                                                   \
    }                                                                                         \
    template <typename R, typename ACC, bool W>                                               \
    static __device__ __forceinline__ ACC quark_line(const gluons<R>& st, const R (&pt)[4],   \
                                                     const R (&ptb)[4], R m, R w) {           \
      return NAME##_quark_line<R, ACC, W, R>(st, pt, ptb, m, w);                              \
    }                                                                                         \
  };

REX_QCD_PROC(PROC_GG_TTX, gg_ttx)
REX_QCD_PROC(PROC_GG_TTXG, gg_ttxg)
REX_QCD_PROC(PROC_GG_TTXGG, gg_ttxgg)
#undef REX_QCD_PROC

constexpr int QCD_BLOCK = 128;

template <int PROC, typename R, bool WIDTH>
__global__ void __launch_bounds__(QCD_BLOCK)
    qcd_reweight_kernel(const double* __restrict__ mom, const double* __restrict__ w_in,
                        int64_t nev, const __grid_constant__ QcdLaunch lp,
                        double* __restrict__ out) {
  using P = QcdProc<PROC>;
  constexpr int NG = P::info::NGLUON;
  constexpr int NPART = NG + 2;
  constexpr int NH = P::info::NGHEL;
  constexpr int EPB = QCD_BLOCK / NH;
  static_assert(32 % NH == 0 || NH % 32 == 0, "gluon-polarisation lanes must tile a warp");
  static_assert(NH <= 32, "one event per warp at most");
  __shared__ double me2s[EPB][MAX_MASS + 1];

  const int tid = threadIdx.x;
  const int el = tid / NH;
  const int gh = tid - el * NH;
  const int64_t ev0 = (int64_t)blockIdx.x * EPB;
  const int64_t ev = ev0 + el;
  const bool valid = ev < nev;
  const int64_t evc = valid ? ev : nev - 1;

  // a1: momenta of this event (NH lanes read the same 32*NPART bytes; L1 broadcast)
  R p[NPART][4];
  {
    const double2* src = reinterpret_cast<const double2*>(mom + evc * (NPART * 4));
#pragma unroll
    for (int i = 0; i < NPART * 2; ++i) {
      const double2 v = __ldg(src + i);
      p[i / 2][(i % 2) * 2 + 0] = R(v.x);
      p[i / 2][(i % 2) * 2 + 1] = R(v.y);
    }
  }
  R pg[NG][4], eps[NG][4], pt[4], ptb[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    pg[0][m] = -p[0][m];
    pg[1][m] = -p[1][m];
#pragma unroll
    for (int g = 2; g < NG; ++g) pg[g][m] = p[g + 2][m];
    pt[m] = p[2][m];
    ptb[m] = p[3][m];
  }
  // a3: linear polarisation of each gluon from this lane's bit
  pol_linear(p[0], (gh >> 0) & 1, eps[0]);
  pol_linear(p[1], (gh >> 1) & 1, eps[1]);
#pragma unroll
  for (int g = 2; g < NG; ++g) pol_linear(p[g + 2], (gh >> g) & 1, eps[g]);

  // a4: mass-independent gluon currents
  typename P::template gluons<R> st;
  P::gluon_state(pg, eps, ptb, st);

  // a4-a7 per distinct mass slot
  for (int m = 0; m < lp.nmass; ++m) {
    double s = 0.0;
    if (valid) s = P::template quark_line<R, double, WIDTH>(st, pt, ptb, R(lp.mass[m]), R(lp.width[m]));
#pragma unroll
    for (int off = NH / 2; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (gh == 0) me2s[el][m] = s;
  }
  __syncthreads();

  // a8: epilogue, consecutive threads write consecutive outputs of the block's rows
  const int nblk = (int)((nev - ev0) < EPB ? (nev - ev0) : EPB);
  if (lp.mode == OUT_RATIO) {
    const int k = lp.k;
    for (int idx = tid; idx < nblk * k; idx += QCD_BLOCK) {
      const int e = idx / k;
      const int j = idx - e * k;
      const double m0 = me2s[e][0] * lp.factor0;
      const double mj = me2s[e][lp.slot[j]] * lp.factor[j];
      const double w = w_in[ev0 + e];
      out[(ev0 + e) * lp.out_stride + j] = (m0 == 0.0) ? 0.0 : w * (mj / m0);
    }
  } else {
    for (int e = tid; e < nblk; e += QCD_BLOCK) out[ev0 + e] = me2s[e][0] * lp.factor0;
  }
}

template <int PROC, typename R>
static int launch_one(const double* mom, const double* w_in, int64_t nev, const QcdLaunch& lp,
                      double* out, cudaStream_t st) {
  constexpr int EPB = QCD_BLOCK / QcdProc<PROC>::info::NGHEL;
  const int64_t blocks = (nev + EPB - 1) / EPB;
  if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
  if (lp.has_width)
    qcd_reweight_kernel<PROC, R, true><<<(unsigned)blocks, QCD_BLOCK, 0, st>>>(mom, w_in, nev, lp, out);
  else
    qcd_reweight_kernel<PROC, R, false><<<(unsigned)blocks, QCD_BLOCK, 0, st>>>(mom, w_in, nev, lp, out);
  return (int)cudaGetLastError();
}

int launch_qcd(int proc, int mixed, const double* mom, const double* w_in, int64_t nev,
               const QcdLaunch& lp, double* out, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (proc) {
    case PROC_GG_TTX:
      return mixed ? launch_one<PROC_GG_TTX, float>(mom, w_in, nev, lp, out, st)
                   : launch_one<PROC_GG_TTX, double>(mom, w_in, nev, lp, out, st);
    case PROC_GG_TTXG:
      return mixed ? launch_one<PROC_GG_TTXG, float>(mom, w_in, nev, lp, out, st)
                   : launch_one<PROC_GG_TTXG, double>(mom, w_in, nev, lp, out, st);
    case PROC_GG_TTXGG:
      return mixed ? launch_one<PROC_GG_TTXGG, float>(mom, w_in, nev, lp, out, st)
                   : launch_one<PROC_GG_TTXGG, double>(mom, w_in, nev, lp, out, st);
    default:
      return (int)cudaErrorInvalidValue;
  }
}

}  // namespace rex
