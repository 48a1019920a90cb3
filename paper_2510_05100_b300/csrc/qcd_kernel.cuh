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
//       polarisations across the NGHEL lanes of the event (warp shuffles); FP64
//       in the exact mode, FP32 in the mixed mode (non-negative terms)
//   a8  ratio epilogue  w_out = w_in * |M_j|^2 / |M_0|^2  (0 if |M_0|^2 == 0), FP64
//
// Thread mapping (kernel variants, chosen per process and precision):
//   SPLIT = 0: NGHEL = 2^n lanes per event, one gluon polarisation configuration
//              each, both antitop helicities inside the lane;
//   SPLIT = 1: 2 NGHEL lanes per event, the antitop helicity split across lanes
//              (half the live state per lane, gluon currents computed twice);
//   MINB: minimum resident blocks per SM requested from the register allocator.
// Blocks of 128 threads, 128 / lanes-per-event events per block.
// The amplitude is evaluated once per distinct (mt, Gamma_t) slot; alpha_s
// enters only through the exact overall factor (4 pi alpha_s)^n of a
// tree amplitude with n external gluons and no other coupling.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "colour_tc.cuh"
#include "df64.cuh"
#include "generated/qcd_amplitudes.cuh"
#include "gg_ttxg_df64.cuh"
#include "rex_internal.cuh"

namespace rex {


template <int PROC>
struct QcdProc;

#define REX_QCD_PROC(KIND, NAME)                                                              \
  template <>                                                                                 \
  struct QcdProc<KIND> {                                                                      \
    using info = NAME##_info;                                                                 \
    template <typename R>                                                                     \
    using event = NAME##_event<R>;                                                            \
    template <typename R>                                                                     \
    using mass = NAME##_mass<R>;                                                              \
    template <typename R>                                                                     \
    using gluons = NAME##_gluons<R>;                                                          \
    template <typename R>                                                                     \
    static __device__ __forceinline__ void event_phase1(const double* p, event<R>& ev, int l, \
                                                        int nl) {                             \
      NAME##_event_phase1(p, ev, l, nl);                                                      \
    }                                                                                         \
    template <typename R>                                                                     \
    static __device__ __forceinline__ void event_phase2(event<R>& ev, double m02, int l,      \
                                                        int nl) {                             \
      NAME##_event_phase2(ev, m02, l, nl);                                                    \
    }                                                                                         \
    template <typename R, bool W>                                                             \
    static __device__ __forceinline__ void mass_setup(const event<R>& ev, double m, double w, \
                                                      R dm2, mass<R>& mm, int l, int nl) {    \
      NAME##_mass_setup<R, W>(ev, m, w, dm2, mm, l, nl);                                      \
    }                                                                                         \
    template <typename R>                                                                     \
    static __device__ __forceinline__ void gluon_currents(const event<R>& ev,                 \
                                                          const R (&eps)[info::NGLUON][4],    \
                                                          gluons<R>& J) {                     \
      NAME##_gluon_currents(ev, eps, J);                                                      \
    }                                                                                         \
    template <typename R, typename ACC, bool W, typename FORM = NoColourForm>                 \
    static __device__ __forceinline__ ACC quark_line(const event<R>& ev, const mass<R>& mm,   \
                                                     const gluons<R>& J, int lo, int hi,      \
                                                     const FORM& form = FORM()) {             \
      return NAME##_quark_line<R, ACC, W, R, FORM>(ev, mm, J, lo, hi, form);                  \
    }                                                                                         \
    static __device__ __forceinline__ const int (&colour())[info::NFLOW][info::NFLOW] {       \
      return NAME##_colour_dev;                                                               \
    }                                                                                         \
  };

REX_QCD_PROC(PROC_GG_TTX, gg_ttx)
REX_QCD_PROC(PROC_GG_TTXG, gg_ttxg)
REX_QCD_PROC(PROC_GG_TTXGG, gg_ttxgg)
#undef REX_QCD_PROC

constexpr int QCD_BLOCK = 128;

// One tile of events (EPB = 128 / lanes-per-event) through the whole path.
// TABLE is the launch's parameter table (QcdLaunch, or a batch table of the
// persistent multi-process kernel): nmass, mass[], width[], k, mode,
// out_stride, slot[], factor[], factor0.
// Helicity-exclusive colour form: each lane holds the jamps of one real linear
// polarisation configuration of the gluons (its bits gh); an amplitude is linear in
// every polarisation vector, so the jamps of the event's helicity configuration are
// J_h = sum over the event's lanes of c_lane * A_lane with
//     c_lane = prod over gluons with bit 1 of (-i lambda_g sigma_g),
// where e_lambda ~ (e1 - i lambda sigma e2)/sqrt(2) (incoming: eps, outgoing: eps*)
// and sigma_g = -1 only where the linear basis is left-handed about the vector it
// was built from (a momentum exactly along -z).  The event's lanes add their terms
// with warp shuffles; lane 0 of the event returns
//     2^-NG sum_{f,f'} Cint_{ff'} Re(conj(J_f) J_f'),
// the others 0, so the lane sum of the helicity loop is |M_h|^2 (times COLOUR_DEN).
// A configuration that a selection rule forbids (angular momentum in on-shell
// g g -> t t~, four of the sixteen) is zero only to the rounding of its inputs: on
// momenta rounded to FP64 it comes out at or below 1e-14 of the sum over the gluon
// configurations at the same top helicities (the lanes' own colour forms, basis
// independent).  A term below ZERO_TERM of that sum is returned as 0, so that its
// weight follows the 1/0 -> 0 rule instead of a ratio of rounding residues: 1e-13 in
// FP64, 1e-11 in FP32; the smallest physical term seen is 1.2e-11 of it (g g -> t t~ g).
template <typename R, int NF, int NGH, int NG>
struct ExclusiveColourForm {
  static constexpr double ZERO_TERM = std::is_same<R, float>::value ? 1e-11 : 1e-13;
  cx<R> c;        // this lane's coefficient
  int ht;         // the event's top helicity (0: -, 1: +)
  bool lead;      // lane 0 of the event
  const int (*col)[NF];
  __device__ __forceinline__ R operator()(const cx<R> (&A)[2][NF]) const {
    cx<R> J[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) J[f] = A[ht][f];
    R scale = form(J);   // this lane's own linear configuration
#pragma unroll
    for (int f = 0; f < NF; ++f) J[f] = c * J[f];
#pragma unroll
    for (int off = 1; off < NGH; off <<= 1) {
      scale += shfl_xor(scale, off);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        J[f].re += shfl_xor(J[f].re, off);
        J[f].im += shfl_xor(J[f].im, off);
      }
    }
    const R s = form(J) * (R(1) / R(1 << NG));
    return (lead && !(s < R(ZERO_TERM) * scale)) ? s : R(0);
  }
  // sum_{f,f'} Cint_{ff'} Re(conj(J_f) J_f')
  __device__ __forceinline__ R form(const cx<R> (&J)[NF]) const {
    R s = R(0);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      R t = R(col[f][f]) * (J[f].re * J[f].re + J[f].im * J[f].im);
#pragma unroll
      for (int g = f + 1; g < NF; ++g) t += R(2 * col[f][g]) * (J[f].re * J[g].re + J[f].im * J[g].im);
      s += t;
    }
    return s;
  }
};

template <int PROC, typename R, bool WIDTH, int SPLIT, bool TC_REQ = false, bool EXCL = false>
struct QcdTile {
  using P = QcdProc<PROC>;
  static constexpr int NG = P::info::NGLUON;
  static constexpr int NF = P::info::NFLOW;
  static constexpr int NPART = NG + 2;
  static constexpr int NGH = P::info::NGHEL;
  static constexpr int NH = NGH << SPLIT;
  static constexpr int EPB = QCD_BLOCK / NH;
  // tensor-core colour form: FP32 amplitudes and events of >= 8 lanes only
  static constexpr bool TC = TC_REQ && std::is_same<R, float>::value && NH >= 8;
  static_assert(32 % NH == 0 || NH % 32 == 0, "gluon-polarisation lanes must tile a warp");
  static_assert(NH <= 32, "one event per warp at most");
  static_assert(!EXCL || (SPLIT == 0 && !TC), "helicity-exclusive tiles: one lane per gluon configuration");

  static constexpr bool F32 = std::is_same<R, float>::value;
  // double-float g g -> t t~ g: the quark line as loops (gg_ttxg_df64.cuh), reading the
  // lane's gluon currents from shared memory
  static constexpr bool DF_LOOP = std::is_same<R, df64>::value && PROC == PROC_GG_TTXG && !TC_REQ;
  struct Smem {
    double me2s[EPB][F32 ? 1 : MAX_MASS + 1];   // exact mode: the slot sums; mixed mode: w
    float me2f[F32 ? EPB : 1][MAX_MASS + 1];   // mixed mode: the FP32 slot sums
    double mult[MAX_POINTS];   // mixed mode: per point, f_j / f_0
    float multf[MAX_POINTS];   // mixed mode: the same in FP32
    int slotj[MAX_POINTS];     // mixed mode: per point, its mass slot
    R dm2[MAX_MASS];           // per slot: m0^2 - m^2 (the mixed mode's propagators)
    typename P::template event<R> evs[EPB];
    typename P::template mass<R> mss[EPB];
    alignas(16) __half tc[TC ? QCD_BLOCK / 32 : 1][TC ? ColourTc<NF>::WARP_HALVES : 1];
    typename P::template gluons<R> js[DF_LOOP ? EPB : 1][DF_LOOP ? NGH : 1];
  };

  // Slot group [s_lo, s_hi) (the persistent kernel's split of a tile's mass slots over
  // several work items, for batches too small to fill the GPU): the tile evaluates slot
  // 0 (the original point, every ratio's denominator) and the slots of its group, and
  // writes the outputs at those slots, the ones at slot 0 only if own0.  The defaults
  // take every slot.
  template <class TABLE>
  static __device__ __forceinline__ void run(Smem& sm, const double* __restrict__ mom,
                                             const double* __restrict__ w_in, int64_t nev, int64_t tile,
                                             const TABLE& lp, double* __restrict__ out,
                                             const signed char* __restrict__ hel = nullptr, int s_lo = 1,
                                             int s_hi = MAX_MASS + 1, bool own0 = true) {
    const int tid = threadIdx.x;
    const int el = tid / NH;
    const int lane_ev = tid - el * NH;
    const int gh = lane_ev % NGH;
    const int hb_lo = SPLIT ? lane_ev / NGH : 0;
    const int hb_hi = SPLIT ? hb_lo + 1 : 2;
    const bool leader = lane_ev == 0;
    const int64_t ev0 = tile * EPB;
    const int64_t ev = ev0 + el;
    const bool valid = ev < nev;
    const int64_t evc = valid ? ev : nev - 1;

    // a1/a2: the event's lanes load its FP64 momenta, convert them and form the
    // FP64 invariants cooperatively (two phases, block barriers between them); the
    // slot table of m0^2 - m^2 (m0 = slot 0's mass) for the mixed mode's propagators
    const double m0 = lp.mass[0];
    for (int m = tid; m < lp.nmass; m += QCD_BLOCK) sm.dm2[m] = to_r<R>((m0 - lp.mass[m]) * (m0 + lp.mass[m]));
    P::event_phase1(mom + evc * (NPART * 4), sm.evs[el], lane_ev, NH);
    __syncthreads();
    P::event_phase2(sm.evs[el], m0 * m0, lane_ev, NH);
    __syncthreads();
    const auto& evd = sm.evs[el];

    // a3: linear polarisation of each gluon from this lane's bits; a4: gluon currents
    R eps[NG][4];
#pragma unroll
    for (int g = 0; g < NG; ++g) pol_linear(evd.pg[g], (gh >> g) & 1, eps[g]);
    typename P::template gluons<R> J;
    P::gluon_currents(evd, eps, J);
    if constexpr (DF_LOOP) {
      if (hb_lo == 0) sm.js[el][gh] = J;   // read after the slot loop's first barrier
    }

    // a6 on tensor cores: the colour matrix as MMA B fragments in this warp's smem
    if constexpr (TC) ColourTc<NF>::load(P::colour(), sm.tc[tid >> 5]);

    // helicity-exclusive: the event's configuration (process order g g t t~ g..) and
    // this lane's coefficient in its amplitude
    ExclusiveColourForm<R, NF, NGH, NG> xform{cx<R>{R(1), R(0)}, 0, gh == 0, P::colour()};
    int hb_x = 0;
    if constexpr (EXCL) {
      const signed char* h = hel + evc * NPART;
      xform.ht = h[2] > 0 ? 1 : 0;
      hb_x = h[3] > 0 ? 1 : 0;
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        if (!((gh >> g) & 1)) continue;
        const int lam = h[g < 2 ? g : g + 2] > 0 ? 1 : -1;
        const R* d = evd.pg[g];
        // the same test as pol_linear's branch: the fixed (x, y) basis is left-handed
        // about a vector along -z
        const bool left = !(d[1] * d[1] + d[2] * d[2] > R(0)) && d[3] < R(0);
        const R f = R(left ? lam : -lam);   // factor -i lambda sigma = i f
        xform.c = cx<R>{-f * xform.c.im, f * xform.c.re};
      }
    }

    // a3-a7 per distinct mass slot (of the group)
    for (int m = 0; m < lp.nmass; ++m) {
      if (m != 0 && (m < s_lo || m >= s_hi)) continue;
      P::template mass_setup<R, WIDTH>(evd, lp.mass[m], lp.width[m], sm.dm2[m], sm.mss[el], lane_ev, NH);
      __syncthreads();
      // a7: the helicity sum adds non-negative terms (no cancellation): FP64 in the
      // exact mode, FP32 in the mixed mode (relative error <= 64 * 2^-24)
      R s = R(0);
      if constexpr (EXCL && DF_LOOP) {
        s = gg_ttxg_quark_line_df64<WIDTH>(evd, sm.mss[el], reinterpret_cast<const df64(*)[4]>(&sm.js[el][gh]),
                                           hb_x, hb_x + 1, xform);
        if (!valid) s = R(0);
      } else if constexpr (EXCL) {
        // every lane takes part in the event's shuffles; only the event's own antitop
        // helicity is evaluated
        s = P::template quark_line<R, R, WIDTH>(evd, sm.mss[el], J, hb_x, hb_x + 1, xform);
        if (!valid) s = R(0);
      } else if constexpr (TC) {
        // every lane takes part in the warp-wide MMA form; lane 8t of the warp
        // receives the colour sum of m16 tile t (part of its event), the others 0
        __half* tcs = sm.tc[tid >> 5];
        auto form = [&](const cx<float> (&A)[2][NF]) { return ColourTc<NF>::template form<NH>(A, tcs); };
        s = P::template quark_line<R, R, WIDTH>(evd, sm.mss[el], J, hb_lo, hb_hi, form);
        if (!valid) s = R(0);
      } else if constexpr (DF_LOOP) {
        if (valid)
          s = gg_ttxg_quark_line_df64<WIDTH>(evd, sm.mss[el],
                                             reinterpret_cast<const df64(*)[4]>(&sm.js[el][gh]), hb_lo, hb_hi);
      } else {
        if (valid) s = P::template quark_line<R, R, WIDTH>(evd, sm.mss[el], J, hb_lo, hb_hi);
      }
#pragma unroll
      for (int off = NH / 2; off > 0; off >>= 1) s += shfl_xor(s, off);
      if (leader) {
        if constexpr (F32) sm.me2f[el][m] = s;
        else sm.me2s[el][m] = double(s);
      }
      __syncthreads();
    }

    // a8: epilogue, consecutive threads write consecutive outputs of the tile's rows
    const int nblk = (int)((nev - ev0) < EPB ? (nev - ev0) : EPB);
    if (lp.mode == OUT_RATIO) {
      const int k = lp.k;
      if constexpr (!F32) {   // FP64 and double-float: the FP64 slot sums and ratio
        for (int idx = tid; idx < nblk * k; idx += QCD_BLOCK) {
          const int e = idx / k;
          const int j = idx - e * k;
          const int sl = lp.slot[j];
          if (sl == 0 ? !own0 : (sl < s_lo || sl >= s_hi)) continue;
          const double m0 = sm.me2s[e][0] * lp.factor0;
          const double mj = sm.me2s[e][sl] * lp.factor[j];
          const double w = w_in[ev0 + e];
          out[(ev0 + e) * lp.out_stride + j] = (m0 == 0.0) ? 0.0 : w * (mj / m0);
        }
      } else {
        // mixed mode (B300 issues FP64 at 1/64 of the FP32 rate): the ratio in FP32.
        // Per event the FP32 slot sums become w |M_s|^2 / |M_0|^2 (one FP32 division),
        // and an output at slot s > 0 is that times f_j / f_0 in FP32, converted to FP64
        // on the integer ALUs.  An output at the original slot is w (f_j / f_0) in FP64,
        // so an unchanged point keeps its weight exactly; slot 0 holds w (0 if
        // |M_0|^2 == 0, NaN if it is NaN).
        for (int j = tid; j < k; j += QCD_BLOCK) {
          sm.slotj[j] = lp.slot[j];
          sm.mult[j] = lp.factor[j] / lp.factor0;
          sm.multf[j] = to_r<float>(sm.mult[j]);
        }
        for (int e = tid; e < nblk; e += QCD_BLOCK) {
          const float m0 = sm.me2f[e][0];
          const double w = w_in[ev0 + e];
          const float wi = m0 == 0.f ? 0.f : to_r<float>(w) / m0;
          const int lo = s_lo > 1 ? s_lo : 1, hi = s_hi < lp.nmass ? s_hi : lp.nmass;
          for (int sl = lo; sl < hi; ++sl) sm.me2f[e][sl] *= wi;
          sm.me2s[e][0] = m0 == 0.f ? 0.0 : (m0 == m0 ? w : (double)m0);
        }
        __syncthreads();
        // output idx = e * k + j; (e, j) advance without an integer division per output
        const int kk = k > 0 ? k : 1;
        int e = tid / kk, j = tid - (tid / kk) * kk;
        const int de = QCD_BLOCK / kk, dj = QCD_BLOCK - (QCD_BLOCK / kk) * kk;
        for (int idx = tid; idx < nblk * k; idx += QCD_BLOCK) {
          const int sl = sm.slotj[j];
          if (sl == 0 ? own0 : (sl >= s_lo && sl < s_hi))
            out[(ev0 + e) * lp.out_stride + j] =
                sl == 0 ? sm.me2s[e][0] * sm.mult[j] : f32_to_f64_alu(sm.me2f[e][sl] * sm.multf[j]);
          e += de;
          j += dj;
          if (j >= k) {
            j -= k;
            ++e;
          }
        }
      }
    } else {
      if (own0)
        for (int e = tid; e < nblk; e += QCD_BLOCK)
          out[ev0 + e] = (F32 ? (double)sm.me2f[e][0] : sm.me2s[e][0]) * lp.factor0;
    }
  }
};

template <int PROC, typename R, bool WIDTH, int SPLIT, int MINB, bool TC = false>
__global__ void __launch_bounds__(QCD_BLOCK, MINB)
    qcd_reweight_kernel(const double* __restrict__ mom, const double* __restrict__ w_in,
                        int64_t nev, const __grid_constant__ QcdLaunch lp,
                        double* __restrict__ out) {
  using T = QcdTile<PROC, R, WIDTH, SPLIT, TC>;
  __shared__ typename T::Smem sm;
  T::run(sm, mom, w_in, nev, (int64_t)blockIdx.x, lp, out);
}

// Variant table (SPLIT, MINB, TC) shared by every process.  TC selects the
// tensor-core colour form (mixed precision, >= 8 lanes per event; the scalar
// form otherwise).
struct QcdVariant {
  int split, minb, tc;
};
constexpr QcdVariant kQcdVariants[QCD_NVARIANT] = {{0, 1, 0}, {1, 1, 0}, {0, 3, 0}, {1, 3, 0}, {0, 4, 0},
                                                   {0, 3, 1}, {1, 3, 1}, {0, 1, 1}, {1, 1, 1}};

template <int PROC, typename R, int V>
static int launch_v(const double* mom, const double* w_in, int64_t nev, const QcdLaunch& lp,
                    double* out, cudaStream_t st) {
  constexpr int SPLIT = kQcdVariants[V].split;
  constexpr int MINB = kQcdVariants[V].minb;
  constexpr bool TC = kQcdVariants[V].tc != 0 && std::is_same<R, float>::value;
  constexpr int EPB = QCD_BLOCK / (QcdProc<PROC>::info::NGHEL << SPLIT);
  const int64_t blocks = (nev + EPB - 1) / EPB;
  if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
  if (lp.has_width)   // rare: one (SPLIT = 0) variant carries complex propagators
    qcd_reweight_kernel<PROC, R, true, 0, 1>
        <<<(unsigned)((nev + QCD_BLOCK / QcdProc<PROC>::info::NGHEL - 1) /
                      (QCD_BLOCK / QcdProc<PROC>::info::NGHEL)),
           QCD_BLOCK, 0, st>>>(mom, w_in, nev, lp, out);
  else
    qcd_reweight_kernel<PROC, R, false, SPLIT, MINB, TC><<<(unsigned)blocks, QCD_BLOCK, 0, st>>>(mom, w_in, nev,
                                                                                                lp, out);
  return (int)cudaGetLastError();
}

template <int PROC, typename R>
static int launch_variant(int variant, const double* mom, const double* w_in, int64_t nev, const QcdLaunch& lp,
                          double* out, cudaStream_t st) {
  switch (variant) {
    case 0: return launch_v<PROC, R, 0>(mom, w_in, nev, lp, out, st);
    case 1: return launch_v<PROC, R, 1>(mom, w_in, nev, lp, out, st);
    case 2: return launch_v<PROC, R, 2>(mom, w_in, nev, lp, out, st);
    case 3: return launch_v<PROC, R, 3>(mom, w_in, nev, lp, out, st);
    case 4: return launch_v<PROC, R, 4>(mom, w_in, nev, lp, out, st);
    case 5: return launch_v<PROC, R, 5>(mom, w_in, nev, lp, out, st);
    case 6: return launch_v<PROC, R, 6>(mom, w_in, nev, lp, out, st);
    case 7: return launch_v<PROC, R, 7>(mom, w_in, nev, lp, out, st);
    case 8: return launch_v<PROC, R, 8>(mom, w_in, nev, lp, out, st);
    default: return (int)cudaErrorInvalidValue;
  }
}

// resident blocks per SM the register allocator must allow in the helicity-exclusive
// kernels: 4 in mixed precision (16 warps per SM; g g -> t t~ g 2^20 x 16 in 3.73 ms
// against 4.79 ms at the 245 registers of 1 block), except g g -> t t~ g g, whose
// lanes would spill 3 KB at 128 registers; 1 in FP64
template <int PROC, typename R>
constexpr int exclusive_minb() {
  return (std::is_same<R, float>::value && PROC != PROC_GG_TTXGG) ? 4 : 1;
}

template <int PROC, typename R, bool WIDTH>
__global__ void __launch_bounds__(QCD_BLOCK, exclusive_minb<PROC, R>())
    qcd_exclusive_kernel(const double* __restrict__ mom, const double* __restrict__ w_in, int64_t nev,
                         const __grid_constant__ QcdLaunch lp, double* __restrict__ out,
                         const signed char* __restrict__ hel) {
  using T = QcdTile<PROC, R, WIDTH, 0, false, true>;
  __shared__ typename T::Smem sm;
  T::run(sm, mom, w_in, nev, (int64_t)blockIdx.x, lp, out, hel);
}

template <int PROC, typename R>
static int launch_exclusive(const double* mom, const double* w_in, int64_t nev, const QcdLaunch& lp, double* out,
                            const signed char* hel, cudaStream_t st) {
  constexpr int EPB = QCD_BLOCK / QcdProc<PROC>::info::NGHEL;
  const int64_t blocks = (nev + EPB - 1) / EPB;
  if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
  if (lp.has_width)
    qcd_exclusive_kernel<PROC, R, true><<<(unsigned)blocks, QCD_BLOCK, 0, st>>>(mom, w_in, nev, lp, out, hel);
  else
    qcd_exclusive_kernel<PROC, R, false><<<(unsigned)blocks, QCD_BLOCK, 0, st>>>(mom, w_in, nev, lp, out, hel);
  return (int)cudaGetLastError();
}

// helicity-exclusive launcher of one g g process (rex_reweight_helicity)
#define REX_DEFINE_QCD_EXCLUSIVE_LAUNCHER(KIND, NAME)                                                  \
  int launch_##NAME##_exclusive(int mixed, const double* mom, const double* w_in, int64_t nev,          \
                                const QcdLaunch& lp, double* out, void* stream, const signed char* hel) { \
    cudaStream_t st = static_cast<cudaStream_t>(stream);                                                \
    return mixed ? launch_exclusive<KIND, float>(mom, w_in, nev, lp, out, hel, st)                      \
                 : launch_exclusive<KIND, double>(mom, w_in, nev, lp, out, hel, st);                    \
  }

// double-float amplitudes (REX_DF64, df64.cuh): one mapping, split 0 (one lane per
// gluon configuration), at the register allocator's own occupancy (255 registers,
// 8 warps per SM).  g g -> t t~ g runs the looped quark line (gg_ttxg_df64.cuh): 2^20 x
// 16 in 72.9 ms unsplit, 83.2 ms with the antitop helicity split over two lanes (which
// helped the straight-line form: 162.7 against 167.3 ms), 89.5 ms split at 3 blocks per
// SM (168 registers), 106.4 ms at 4 (128 registers, 344 B of spill).
template <int PROC>
constexpr int df64_split() {
  return 0;
}

template <int PROC>
static int launch_df64_t(const double* mom, const double* w_in, int64_t nev, const QcdLaunch& lp, double* out,
                         cudaStream_t st) {
  constexpr int SPLIT = df64_split<PROC>();
  constexpr int EPB = QCD_BLOCK / (QcdProc<PROC>::info::NGHEL << SPLIT);
  const int64_t blocks = (nev + EPB - 1) / EPB;
  if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
  if (lp.has_width)
    qcd_reweight_kernel<PROC, df64, true, SPLIT, 1><<<(unsigned)blocks, QCD_BLOCK, 0, st>>>(mom, w_in, nev, lp, out);
  else
    qcd_reweight_kernel<PROC, df64, false, SPLIT, 1><<<(unsigned)blocks, QCD_BLOCK, 0, st>>>(mom, w_in, nev, lp, out);
  return (int)cudaGetLastError();
}

// helicity-exclusive double-float tile (g g -> t t~ g: the looped quark line)
template <int PROC>
static int launch_df64_exclusive_t(const double* mom, const double* w_in, int64_t nev, const QcdLaunch& lp,
                                   double* out, const signed char* hel, cudaStream_t st) {
  constexpr int EPB = QCD_BLOCK / QcdProc<PROC>::info::NGHEL;
  const int64_t blocks = (nev + EPB - 1) / EPB;
  if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
  if (lp.has_width)
    qcd_exclusive_kernel<PROC, df64, true><<<(unsigned)blocks, QCD_BLOCK, 0, st>>>(mom, w_in, nev, lp, out, hel);
  else
    qcd_exclusive_kernel<PROC, df64, false><<<(unsigned)blocks, QCD_BLOCK, 0, st>>>(mom, w_in, nev, lp, out, hel);
  return (int)cudaGetLastError();
}

#define REX_DEFINE_QCD_DF64_LAUNCHER(KIND, NAME)                                                       \
  int launch_##NAME##_df64(const double* mom, const double* w_in, int64_t nev, const QcdLaunch& lp,   \
                           double* out, void* stream) {                                               \
    return launch_df64_t<KIND>(mom, w_in, nev, lp, out, static_cast<cudaStream_t>(stream));          \
  }

#define REX_DEFINE_QCD_LAUNCHER(KIND, NAME)                                                          \
  int launch_##NAME(int mixed, int variant, const double* mom, const double* w_in, int64_t nev,     \
                    const QcdLaunch& lp, double* out, void* stream) {                              \
    cudaStream_t st = static_cast<cudaStream_t>(stream);                                           \
    return mixed ? launch_variant<KIND, float>(variant, mom, w_in, nev, lp, out, st)               \
                 : launch_variant<KIND, double>(variant, mom, w_in, nev, lp, out, st);             \
  }

}  // namespace rex
