// Host-side flop counter for the generated amplitude code (measurement tool).
//
// Instantiates the device routines of helas.cuh and generated/qcd_amplitudes.cuh
// with a scalar type that carries no value and only tallies arithmetic
// operations (+, -, *, / and sqrt count one flop each; a fused multiply-add is
// therefore two, as on the FMA pipe).  Amplitude arithmetic (type R) and the
// colour/helicity accumulation (type ACC) are tallied separately, so the FP64
// and FP32 work of each precision mode can be read off.  Prints JSON.
#include <cmath>
#include <cstdio>

#define __device__
#define __host__
#define __forceinline__ inline

template <int TAG>
struct Cnt {
  static long long flops;
  double v;  // never read for counting; keeps comparisons well-formed
  Cnt() : v(0) {}
  Cnt(double x) : v(x) {}
  template <int U>
  explicit Cnt(Cnt<U> o) : v(o.v) {}   // R -> ACC conversion is free
};
template <int TAG>
long long Cnt<TAG>::flops = 0;

#define REX_CNT_BIN(op)                                                  \
  template <int T>                                                       \
  inline Cnt<T> operator op(Cnt<T> a, Cnt<T> b) {                        \
    ++Cnt<T>::flops;                                                     \
    return Cnt<T>(a.v op b.v);                                           \
  }                                                                      \
  template <int T>                                                       \
  inline Cnt<T>& operator op##=(Cnt<T>& a, Cnt<T> b) {                   \
    ++Cnt<T>::flops;                                                     \
    a.v = a.v op b.v;                                                    \
    return a;                                                            \
  }
REX_CNT_BIN(+)
REX_CNT_BIN(-)
REX_CNT_BIN(*)
REX_CNT_BIN(/)
#undef REX_CNT_BIN
template <int T>
inline Cnt<T> operator-(Cnt<T> a) { return Cnt<T>(-a.v); }   // sign flips are free
template <int T>
inline bool operator>(Cnt<T> a, Cnt<T> b) { return a.v > b.v; }
template <int T>
inline bool operator>=(Cnt<T> a, Cnt<T> b) { return a.v >= b.v; }
template <int T>
inline bool operator<=(Cnt<T> a, Cnt<T> b) { return a.v <= b.v; }
template <int T>
inline Cnt<T> sqrt(Cnt<T> a) { ++Cnt<T>::flops; return Cnt<T>(std::sqrt(a.v)); }
template <int T>
inline Cnt<T> rsqrt(Cnt<T> a) { ++Cnt<T>::flops; return Cnt<T>(1.0 / std::sqrt(a.v)); }

using RC = Cnt<0>;    // amplitude arithmetic
using AC = Cnt<1>;    // colour / helicity accumulation

#include "../generated/qcd_amplitudes.cuh"

using namespace rex;

template <int NG, class ST, class GS, class QL>
void count(const char* name, int nghel, GS gs, QL ql, bool last) {
  const int ngluon = NG;
  RC pg[NG][4], eps[NG][4], pt[4], ptb[4];
  for (int i = 0; i < NG; ++i)
    for (int m = 0; m < 4; ++m) {
      pg[i][m] = RC(1.0 + i + 0.1 * m);
      eps[i][m] = RC(0.5);
    }
  for (int m = 0; m < 4; ++m) {
    pt[m] = RC(2.0 + m);
    ptb[m] = RC(3.0 + m);
  }
  ST st;
  RC::flops = 0;
  AC::flops = 0;
  gs(pg, eps, ptb, st);
  const long long f_state = RC::flops;
  // external polarisation vectors (pol_linear) are counted with the state
  RC e[4];
  RC::flops = 0;
  for (int g = 0; g < ngluon; ++g) pol_linear(pg[g], 0, e);
  const long long f_pol = RC::flops;
  RC::flops = 0;
  AC::flops = 0;
  ql(st, pt, ptb, RC(173.0), RC(0.0));
  const long long f_line_r = RC::flops, f_line_a = AC::flops;
  std::printf("  \"%s\": {\"nghel\": %d, \"gluon_state\": %lld, \"polarisations\": %lld, "
              "\"quark_line_amp\": %lld, \"quark_line_acc\": %lld}%s\n",
              name, nghel, f_state, f_pol, f_line_r, f_line_a, last ? "" : ",");
}

int main() {
  std::printf("{\n");
  count<2, gg_ttx_gluons<RC>>(
      "gg_ttx", 4, [](auto& a, auto& b, auto& c, auto& d) { gg_ttx_gluon_state(a, b, c, d); },
      [](auto& s, auto& a, auto& b, RC m, RC w) { return gg_ttx_quark_line<RC, AC, false>(s, a, b, m, w); },
      false);
  count<3, gg_ttxg_gluons<RC>>(
      "gg_ttxg", 8, [](auto& a, auto& b, auto& c, auto& d) { gg_ttxg_gluon_state(a, b, c, d); },
      [](auto& s, auto& a, auto& b, RC m, RC w) { return gg_ttxg_quark_line<RC, AC, false>(s, a, b, m, w); },
      false);
  count<4, gg_ttxgg_gluons<RC>>(
      "gg_ttxgg", 16, [](auto& a, auto& b, auto& c, auto& d) { gg_ttxgg_gluon_state(a, b, c, d); },
      [](auto& s, auto& a, auto& b, RC m, RC w) { return gg_ttxgg_quark_line<RC, AC, false>(s, a, b, m, w); },
      true);
  std::printf("}\n");
  return 0;
}
