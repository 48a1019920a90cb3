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
#define __restrict__
template <typename T>
inline T __ldg(const T* p) { return *p; }

template <int TAG>
struct Cnt {
  static long long flops;
  double v;  // never read for counting; keeps comparisons well-formed
  Cnt() : v(0) {}
  Cnt(double x) : v(x) {}
  template <int U>
  explicit Cnt(Cnt<U> o) : v(o.v) {}   // R -> ACC conversion is free
  explicit operator double() const { return v; }   // R -> FP64 conversion is free
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
inline Cnt<T> fma(Cnt<T> a, Cnt<T> b, Cnt<T> c) { Cnt<T>::flops += 2; return Cnt<T>(a.v * b.v + c.v); }
template <int T>
inline Cnt<T> sqrt(Cnt<T> a) { ++Cnt<T>::flops; return Cnt<T>(std::sqrt(a.v)); }
template <int T>
inline Cnt<T> rsqrt(Cnt<T> a) { ++Cnt<T>::flops; return Cnt<T>(1.0 / std::sqrt(a.v)); }

using RC = Cnt<0>;    // amplitude arithmetic
using AC = Cnt<1>;    // colour / helicity accumulation

// Double-float (REX_DF64) cost of each operation in FP32 flops as df64.cuh performs
// them (an FMA counts two, a division or square root one): sum 10, product 10,
// fused multiply-add 18, quotient 25, square root 12, reciprocal square root 37, and
// slash_acc 404, ubar_dot 246, vvv_acc 501, vvvv_acc 381, cdotm 246 and qqg_form 753
// (below); sign flips, comparisons and
// FP64 -> double-float conversions cost none.
struct DC {
  static long long flops;
  double v;
  DC() : v(0) {}
  DC(double x) : v(x) {}
  explicit operator double() const { return v; }
};
long long DC::flops = 0;
inline DC operator+(DC a, DC b) { DC::flops += 10; return DC(a.v + b.v); }
inline DC operator-(DC a, DC b) { DC::flops += 10; return DC(a.v - b.v); }
inline DC operator*(DC a, DC b) { DC::flops += 10; return DC(a.v * b.v); }
inline DC operator/(DC a, DC b) { DC::flops += 25; return DC(a.v / b.v); }
inline DC& operator+=(DC& a, DC b) { a = a + b; return a; }
inline DC& operator-=(DC& a, DC b) { a = a - b; return a; }
inline DC& operator*=(DC& a, DC b) { a = a * b; return a; }
inline DC operator-(DC a) { return DC(-a.v); }
inline bool operator>(DC a, DC b) { return a.v > b.v; }
inline bool operator>=(DC a, DC b) { return a.v >= b.v; }
inline bool operator<=(DC a, DC b) { return a.v <= b.v; }
inline DC fma(DC a, DC b, DC c) { DC::flops += 18; return DC(a.v * b.v + c.v); }
inline DC sqrt(DC a) { DC::flops += 12; return DC(std::sqrt(a.v)); }
inline DC rsqrt(DC a) { DC::flops += 37; return DC(1.0 / std::sqrt(a.v)); }

#include "../helas.cuh"

// df64.cuh's slash_acc for double-float values (s = +-1 as a sign, three products per
// output component each added with one TwoSum, one renormalisation per component):
// two double-float sums (20) + 24 products x 15 + 8 renormalisations x 3 = 404 FP32 flops
inline void slash_acc(DC s, const DC* a, const rex::cx<DC>* psi, rex::cx<DC>* out) {
  const long long keep = DC::flops;
  const double am = s.v * (a[0].v - a[3].v), ap = s.v * (a[0].v + a[3].v), a1 = s.v * a[1].v, a2 = s.v * a[2].v;
  out[0].re.v += am * psi[2].re.v - a1 * psi[3].re.v - a2 * psi[3].im.v;
  out[0].im.v += am * psi[2].im.v - a1 * psi[3].im.v + a2 * psi[3].re.v;
  out[1].re.v += ap * psi[3].re.v - a1 * psi[2].re.v + a2 * psi[2].im.v;
  out[1].im.v += ap * psi[3].im.v - a1 * psi[2].im.v - a2 * psi[2].re.v;
  out[2].re.v += ap * psi[0].re.v + a1 * psi[1].re.v + a2 * psi[1].im.v;
  out[2].im.v += ap * psi[0].im.v + a1 * psi[1].im.v - a2 * psi[1].re.v;
  out[3].re.v += am * psi[1].re.v + a1 * psi[0].re.v - a2 * psi[0].im.v;
  out[3].im.v += am * psi[1].im.v + a1 * psi[0].im.v + a2 * psi[0].re.v;
  DC::flops = keep + 404;
}

// df64.cuh's closure and vertex helpers for double-float values (products summed with
// one TwoSum each and one renormalisation per sum; s = +-1 as a sign; 2x exact):
// ubar_dot two eight-product sums = 246; vvv_acc 8 sums (80) + 3 Minkowski products
// (3 x 63) + 4 differences (40) + 4 three-product accumulations (4 x 48) = 501;
// vvvv_acc 3 x 63 + 4 x 48 = 381.
inline rex::cx<DC> ubar_dot(const rex::cx<DC>* u, const rex::cx<DC>* x) {
  const long long keep = DC::flops;
  const rex::cx<DC> r = rex::cdot1(u[0], x[2]) + rex::cdot1(u[1], x[3]) + rex::cdot1(u[2], x[0]) + rex::cdot1(u[3], x[1]);
  DC::flops = keep + 246;
  return r;
}
inline void vvv_acc(DC s, const DC* jx, const DC* px, const DC* jy, const DC* py, DC* out) {
  const long long keep = DC::flops;
  DC a[4], b[4];
  for (int m = 0; m < 4; ++m) {
    a[m] = px[m] + DC(2.0) * py[m];
    b[m] = DC(2.0) * px[m] + py[m];
  }
  const DC xy = s * rex::mdot(jx, jy), xa = s * rex::mdot(jx, a), yb = s * rex::mdot(jy, b);
  for (int m = 0; m < 4; ++m) out[m] = out[m] + xy * (py[m] - px[m]) - xa * jy[m] + yb * jx[m];
  DC::flops = keep + 501;
}
inline void vvvv_acc(DC s, const DC* jx, const DC* jy, const DC* jz, DC* out) {
  const long long keep = DC::flops;
  const DC xy = s * rex::mdot(jx, jy), yz = s * rex::mdot(jy, jz), xz2 = DC(-2.0) * s * rex::mdot(jx, jz);
  for (int m = 0; m < 4; ++m) out[m] = out[m] + xy * jz[m] + yz * jx[m] + xz2 * jy[m];
  DC::flops = keep + 381;
}

#include "../generated/qcd_amplitudes.cuh"
#include "../qq_amplitude.cuh"
#include "../qqg_amplitude.cuh"

// df64.cuh's cdotm (two eight-product sums = 246) and qqg_kernel.cuh's qqg_form for
// double-float values (30 colour-weighted products: 30 x (10 + 15) + one
// renormalisation 3 = 753)
inline rex::cx<DC> cdotm(const rex::cx<DC>* a, const rex::cx<DC>* b) {
  const long long keep = DC::flops;
  const rex::cx<DC> r = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  DC::flops = keep + 246;
  return r;
}
inline DC qqg_form(const rex::cx<DC> (&a)[5]) {
  double f = 0;
  for (int d = 0; d < 5; ++d)
    for (int d2 = d; d2 < 5; ++d2)
      f += rex::qqg_colour(d, d2) * (d == d2 ? 1 : 2) * (a[d].re.v * a[d2].re.v + a[d].im.v * a[d2].im.v);
  DC::flops += 753;
  return DC(f);
}

using namespace rex;

// FP64 invariants in the event and mass setup are plain doubles and are not
// counted (a few tens of operations per event).
// Counts per call: event setup (once per event), mass setup (once per event and
// mass slot), gluon currents (once per event and polarisation configuration),
// polarisation vectors (idem), quark line (once per event, polarisation
// configuration and mass slot; and its amplitude arithmetic for one antitop
// helicity, what a helicity-exclusive tile evaluates).
template <int NG, class EV, class MS, class GL, class ES, class MSF, class GC, class QL, class QLX>
void count(const char* name, int nghel, ES es, MSF msf, GC gc, QL ql, QLX qlx, bool last) {
  double p[NG + 2][4];
  RC eps[NG][4], pr[NG + 2][4];
  for (int i = 0; i < NG + 2; ++i)
    for (int m = 0; m < 4; ++m) {
      p[i][m] = 1.0 + i + 0.1 * m;
      pr[i][m] = RC(p[i][m]);
    }
  for (int i = 0; i < NG; ++i)
    for (int m = 0; m < 4; ++m) eps[i][m] = RC(0.5);
  EV ev;
  MS mm;
  GL J;
  RC::flops = 0;
  es(&p[0][0], ev);
  const long long f_event = RC::flops;
  RC::flops = 0;
  msf(ev, 173.0, 0.0, mm);
  const long long f_mass = RC::flops;
  RC::flops = 0;
  RC e[4];
  for (int g = 0; g < NG; ++g) pol_linear(pr[g], 0, e);
  const long long f_pol = RC::flops;
  RC::flops = 0;
  gc(ev, eps, J);
  const long long f_gluon = RC::flops;
  RC::flops = 0;
  AC::flops = 0;
  ql(ev, mm, J);
  const long long f_line_r = RC::flops, f_line_a = AC::flops;
  RC::flops = 0;
  qlx(ev, mm, J);
  const long long f_line_x = RC::flops;
  std::printf("  \"%s\": {\"nghel\": %d, \"event_setup\": %lld, \"mass_setup\": %lld, "
              "\"polarisations\": %lld, \"gluon_currents\": %lld, \"quark_line_amp\": %lld, "
              "\"quark_line_acc\": %lld, \"quark_line_amp_one_antitop\": %lld}%s\n",
              name, nghel, f_event, f_mass, f_pol, f_gluon, f_line_r, f_line_a, f_line_x, last ? "" : ",");
}

#define REX_COUNT(NAME, NG, LAST)                                                                   \
  count<NG, NAME##_event<RC>, NAME##_mass<RC>, NAME##_gluons<RC>>(                                  \
      #NAME, 1 << NG,                                                                               \
      [](const double* p, auto& ev) { NAME##_event_phase1(p, ev, 0, 1); NAME##_event_phase2(ev, 173.0 * 173.0, 0, 1); }, \
      [](auto& ev, double m, double w, auto& mm) { NAME##_mass_setup<RC, false>(ev, m, w, RC(0.0), mm, 0, 1); }, \
      [](auto& ev, auto& eps, auto& J) { NAME##_gluon_currents(ev, eps, J); },                       \
      [](auto& ev, auto& mm, auto& J) { return NAME##_quark_line<RC, AC, false, RC>(ev, mm, J); },      \
      [](auto& ev, auto& mm, auto& J) { return NAME##_quark_line<RC, AC, false, RC>(ev, mm, J, 0, 1); }, LAST)

// The same routines in double-float: FP32 flops per call (split 0 accounting: both
// antitop helicities per quark-line call).
template <int NG, class EV, class MS, class GL, class ES, class MSF, class GC, class QL, class QLX>
void count_df(const char* name, int nghel, ES es, MSF msf, GC gc, QL ql, QLX qlx) {
  double p[NG + 2][4];
  DC eps[NG][4], pr[NG + 2][4];
  for (int i = 0; i < NG + 2; ++i)
    for (int m = 0; m < 4; ++m) {
      p[i][m] = 1.0 + i + 0.1 * m;
      pr[i][m] = DC(p[i][m]);
    }
  for (int i = 0; i < NG; ++i)
    for (int m = 0; m < 4; ++m) eps[i][m] = DC(0.5);
  EV ev;
  MS mm;
  GL J;
  DC::flops = 0;
  es(&p[0][0], ev);
  const long long f_event = DC::flops;
  DC::flops = 0;
  msf(ev, 173.0, 0.0, mm);
  const long long f_mass = DC::flops;
  DC::flops = 0;
  DC e[4];
  for (int g = 0; g < NG; ++g) pol_linear(pr[g], 0, e);
  const long long f_pol = DC::flops;
  DC::flops = 0;
  gc(ev, eps, J);
  const long long f_gluon = DC::flops;
  DC::flops = 0;
  ql(ev, mm, J);
  const long long f_line = DC::flops;
  DC::flops = 0;
  qlx(ev, mm, J);
  const long long f_line_x = DC::flops;
  std::printf("  \"%s_df64\": {\"nghel\": %d, \"event_setup\": %lld, \"mass_setup\": %lld, "
              "\"polarisations\": %lld, \"gluon_currents\": %lld, \"quark_line_amp\": %lld, "
              "\"quark_line_acc\": 0, \"quark_line_amp_one_antitop\": %lld},\n",
              name, nghel, f_event, f_mass, f_pol, f_gluon, f_line, f_line_x);
}

#define REX_COUNT_DF(NAME, NG)                                                                      \
  count_df<NG, NAME##_event<DC>, NAME##_mass<DC>, NAME##_gluons<DC>>(                                \
      #NAME, 1 << NG,                                                                               \
      [](const double* p, auto& ev) { NAME##_event_phase1(p, ev, 0, 1); NAME##_event_phase2(ev, 173.0 * 173.0, 0, 1); }, \
      [](auto& ev, double m, double w, auto& mm) { NAME##_mass_setup<DC, false>(ev, m, w, DC(0.0), mm, 0, 1); }, \
      [](auto& ev, auto& eps, auto& J) { NAME##_gluon_currents(ev, eps, J); },                       \
      [](auto& ev, auto& mm, auto& J) { return NAME##_quark_line<DC, DC, false, DC>(ev, mm, J); },      \
      [](auto& ev, auto& mm, auto& J) { return NAME##_quark_line<DC, DC, false, DC>(ev, mm, J, 0, 1); })

int main() {
  std::printf("{\n");
  REX_COUNT_DF(gg_ttx, 2);
  REX_COUNT_DF(gg_ttxg, 3);
  REX_COUNT(gg_ttx, 2, false);
  REX_COUNT(gg_ttxg, 3, false);
  REX_COUNT(gg_ttxgg, 4, false);
  {
    // q q~ -> t t~: the per-event constants; the caller adds the normalisation by
    // the original point (a division and three products) and the per-point
    // polynomial and weight product
    RC p[4][4];
    for (int i = 0; i < 4; ++i)
      for (int m = 0; m < 4; ++m) p[i][m] = RC(1.0 + i + 0.1 * m);
    RC c[3], e12;
    RC::flops = 0;
    qq_ttx_coefficients<RC>(p, c, &e12);
    std::printf("  \"qq_ttx\": {\"nghel\": 1, \"event_setup\": %lld, \"mass_setup\": 0, "
                "\"polarisations\": 0, \"gluon_currents\": 0, \"quark_line_amp\": 0, "
                "\"quark_line_acc\": 0},\n", RC::flops);
  }
  {
    // q q~ -> t t~ g: 4 lanes per event; lane set-up once per event, the slot routine
    // once per mass slot (the six FP64 invariants and the reciprocals not counted)
    double pd[5][4];
    RC p[5][4];
    for (int i = 0; i < 5; ++i)
      for (int m = 0; m < 4; ++m) {
        pd[i][m] = 1.0 + i + 0.1 * m;
        p[i][m] = RC(pd[i][m]);
      }
    QqgInvariants<RC> inv{RC(1e-6), RC(1e-6), RC(-1e-4), RC(-1e-4), RC(100.0), RC(120.0)};
    QqgLane<RC> L;
    RC::flops = 0;
    qqg_lane_setup<RC>(p, 0, 0, L);
    qqg_lane_scale<RC>(inv, L);
    const long long f_setup = RC::flops;
    RC::flops = 0;
    qqg_slot<RC>(L, RC(171.0), RC(700.0), RC(0.0));
    const long long f_slot = RC::flops;
    std::printf("  \"qq_ttxg\": {\"nghel\": 1, \"event_setup\": %lld, \"mass_setup\": %lld, "
                "\"polarisations\": 0, \"gluon_currents\": 0, \"quark_line_amp\": 0, "
                "\"quark_line_acc\": 0},\n", 4 * f_setup, 4 * f_slot);
    // the same lanes in double-float (FP32 flops)
    DC pdc[5][4];
    for (int i = 0; i < 5; ++i)
      for (int m = 0; m < 4; ++m) pdc[i][m] = DC(pd[i][m]);
    QqgInvariants<DC> invd{DC(1e-6), DC(1e-6), DC(-1e-4), DC(-1e-4), DC(100.0), DC(120.0)};
    QqgLane<DC> Ld;
    DC::flops = 0;
    qqg_lane_setup<DC>(pdc, 0, 0, Ld);
    qqg_lane_scale<DC>(invd, Ld);
    const long long d_setup = DC::flops;
    DC::flops = 0;
    qqg_slot<DC>(Ld, DC(171.0), DC(700.0), DC(0.0));
    const long long d_slot = DC::flops;
    std::printf("  \"qq_ttxg_df64\": {\"nghel\": 1, \"event_setup\": %lld, \"mass_setup\": %lld, "
                "\"polarisations\": 0, \"gluon_currents\": 0, \"quark_line_amp\": 0, "
                "\"quark_line_acc\": 0}\n", 4 * d_setup, 4 * d_slot);
  }
  std::printf("}\n");
  return 0;
}
