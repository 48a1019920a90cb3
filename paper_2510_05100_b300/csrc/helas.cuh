// Device building blocks for tree-level helicity amplitudes (sm_103a).
//
// Written for this library from the chiral-basis definitions; the routine
// names echo the HELAS families they play the role of (external wavefunctions
// ixxxxx/oxxxxx/vxxxxx, vertex currents VVV1P0_1 / FFV1_1, closures FFV1_0).
//
// Conventions: metric (+,-,-,-); chiral basis, gamma^mu = [[0, sigma^mu],
// [sigmabar^mu, 0]], spinor components ordered (left-handed 0,1 | right-handed
// 2,3).  Lorentz vectors are upper-index (E, px, py, pz).
//
// Helicity sums are basis independent, so:
//  * gluons use REAL linear polarisation vectors e1, e2 (transverse, orthonormal);
//    every pure-gluon current built from them is a real 4-vector;
//  * fermions use helicity spinors in this file's own phase convention.
//
// Mass in external spinors when a parameter point changes a mass while the
// momentum is kept: omega_+ = sqrt(E + |p|), omega_- = m / omega_+ (equal to
// sqrt(E - |p|) on shell).  This is the spinor of the on-shell momentum with the
// same direction and the same E + |p| as p, with mass m.
#pragma once
#if defined(__CUDACC__)
#include <cuda_runtime.h>

#include "fpconv.cuh"
#endif

namespace rex {

// FP64 -> R.  In device code R = float converts on the integer ALUs (fpconv.cuh:
// round to nearest even, B300 issues FP64-pipe conversions at 1/64 of the FP32 rate);
// any other R is a plain conversion.
template <typename R>
__device__ __forceinline__ R to_r(double x) { return R(x); }
#if defined(__CUDACC__)
template <>
__device__ __forceinline__ float to_r<float>(double x) { return f64_to_f32_alu(x); }
#endif

template <typename R>
struct cx {
  R re, im;
};

// Amplitude types whose every operation expands to many instructions (double-float,
// df64.cuh, specialises it): loops that are unrolled for FP32 and FP64 stay rolled for
// them, so that the code fits the instruction caches.
template <typename R>
struct expensive_arith {
  static constexpr bool value = false;
};

template <typename R>
__device__ __forceinline__ cx<R> cmk(R a, R b) { return cx<R>{a, b}; }
template <typename R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return cx<R>{a.re + b.re, a.im + b.im}; }
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return cx<R>{a.re - b.re, a.im - b.im}; }
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a) { return cx<R>{-a.re, -a.im}; }
template <typename R>
__device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return cx<R>{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return cx<R>{s * a.re, s * a.im}; }
template <typename R>
__device__ __forceinline__ cx<R> conjg(cx<R> a) { return cx<R>{a.re, -a.im}; }
// conj(a) * b
template <typename R>
__device__ __forceinline__ cx<R> cdot1(cx<R> a, cx<R> b) {
  return cx<R>{a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}

template <typename R>
__device__ __forceinline__ R mdot(const R* a, const R* b) {
  return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}

// ---------------------------------------------------------------------------
// external wavefunctions
// ---------------------------------------------------------------------------

// Linear polarisation vector e_{which} (which = 0, 1) of a massless momentum k:
// e1 = (0, kx kz, ky kz, -kT^2)/(|k| kT), e2 = (0, -ky, kx, 0)/kT; along the
// beam axis e1 = x-hat, e2 = y-hat.  (vxxxxx role, linear basis.)
template <typename R>
__device__ __forceinline__ void pol_linear(const R* k, int which, R* eps) {
  const R kx = k[1], ky = k[2], kz = k[3];
  const R kt2 = kx * kx + ky * ky;
  eps[0] = R(0);
  if (kt2 > R(0)) {
    const R kt = sqrt(kt2);
    const R kabs = sqrt(kt2 + kz * kz);
    if (which == 0) {
      const R f = kz / (kabs * kt);
      eps[1] = kx * f;
      eps[2] = ky * f;
      eps[3] = -kt / kabs;
    } else {
      eps[1] = -ky / kt;
      eps[2] = kx / kt;
      eps[3] = R(0);
    }
  } else {
    eps[1] = which == 0 ? R(1) : R(0);
    eps[2] = which == 0 ? R(0) : R(1);
    eps[3] = R(0);
  }
}

// Two-component helicity eigenvectors chi_+, chi_- of (p-hat . sigma).
// chi_+ = (|p|+pz, px + i py)/N, chi_- = (-px + i py, |p|+pz)/N, N^2 = 2|p|(|p|+pz);
// |p|+pz is taken as pT^2/(|p|-pz) for pz < 0 to avoid cancellation.
template <typename R>
__device__ __forceinline__ void chi_pair(const R* p, R pabs, cx<R>* chip, cx<R>* chim) {
  const R px = p[1], py = p[2], pz = p[3];
  const R pt2 = px * px + py * py;
  if (pt2 > R(0)) {
    const R a = pz >= R(0) ? pabs + pz : pt2 / (pabs - pz);
    const R nrm = rsqrt(R(2) * pabs * a);
    const R an = a * nrm;
    chip[0] = cx<R>{an, R(0)};
    chip[1] = cx<R>{px * nrm, py * nrm};
    chim[0] = cx<R>{-px * nrm, py * nrm};
    chim[1] = cx<R>{an, R(0)};
  } else if (pz >= R(0)) {           // along +z, or at rest (take +z)
    chip[0] = cx<R>{R(1), R(0)};
    chip[1] = cx<R>{R(0), R(0)};
    chim[0] = cx<R>{R(0), R(0)};
    chim[1] = cx<R>{R(1), R(0)};
  } else {                           // along -z
    chip[0] = cx<R>{R(0), R(0)};
    chip[1] = cx<R>{R(1), R(0)};
    chim[0] = cx<R>{R(-1), R(0)};
    chim[1] = cx<R>{R(0), R(0)};
  }
}

// omega_+ = sqrt(E + |p|), omega_- = m / omega_+.
template <typename R>
__device__ __forceinline__ void omegas(const R* p, R m, R* pabs, R* wp, R* wm) {
  const R a = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
  *pabs = a;
  const R w = sqrt(p[0] + a);
  *wp = w;
  *wm = m / w;
}

// u(p, hel) of an outgoing fermion, to be closed as ubar (oxxxxx role):
// u(+) = (w- chi+, w+ chi+), u(-) = (w+ chi-, w- chi-).
template <typename R>
__device__ __forceinline__ void spinor_u(const R* p, R m, int hel, cx<R>* u) {
  R pabs, wp, wm;
  omegas(p, m, &pabs, &wp, &wm);
  cx<R> cp[2], cm[2];
  chi_pair(p, pabs, cp, cm);
  if (hel > 0) {
    u[0] = wm * cp[0]; u[1] = wm * cp[1]; u[2] = wp * cp[0]; u[3] = wp * cp[1];
  } else {
    u[0] = wp * cm[0]; u[1] = wp * cm[1]; u[2] = wm * cm[0]; u[3] = wm * cm[1];
  }
}

// v(p, hel) of an outgoing antifermion (ixxxxx role): eta = chi_{-hel},
// v(+) = (w+ chi-, -w- chi-), v(-) = (w- chi+, -w+ chi+).
template <typename R>
__device__ __forceinline__ void spinor_v(const R* p, R m, int hel, cx<R>* v) {
  R pabs, wp, wm;
  omegas(p, m, &pabs, &wp, &wm);
  cx<R> cp[2], cm[2];
  chi_pair(p, pabs, cp, cm);
  if (hel > 0) {
    v[0] = wp * cm[0]; v[1] = wp * cm[1]; v[2] = (-wm) * cm[0]; v[3] = (-wm) * cm[1];
  } else {
    v[0] = wm * cp[0]; v[1] = wm * cp[1]; v[2] = (-wp) * cp[0]; v[3] = (-wp) * cp[1];
  }
}

// Spinors from precomputed helicity 2-spinors chi[0] = chi-, chi[1] = chi+ and
// omega_+ = wp, omega_- = wm (= m / omega_+), for both helicities (index 0: -, 1: +).
template <typename R>
__device__ __forceinline__ void spinor_u_from(const cx<R> (&chi)[2][2], R wp, R wm, cx<R> (&u)[2][4]) {
  u[1][0] = wm * chi[1][0]; u[1][1] = wm * chi[1][1]; u[1][2] = wp * chi[1][0]; u[1][3] = wp * chi[1][1];
  u[0][0] = wp * chi[0][0]; u[0][1] = wp * chi[0][1]; u[0][2] = wm * chi[0][0]; u[0][3] = wm * chi[0][1];
}

template <typename R>
__device__ __forceinline__ void spinor_v_from(const cx<R> (&chi)[2][2], R wp, R wm, cx<R> (&v)[2][4]) {
  v[1][0] = wp * chi[0][0]; v[1][1] = wp * chi[0][1]; v[1][2] = (-wm) * chi[0][0]; v[1][3] = (-wm) * chi[0][1];
  v[0][0] = wm * chi[1][0]; v[0][1] = wm * chi[1][1]; v[0][2] = (-wp) * chi[1][0]; v[0][3] = (-wp) * chi[1][1];
}

// ---------------------------------------------------------------------------
// fermion-line operations
// ---------------------------------------------------------------------------

// out += s * (gamma . a) psi for a real 4-vector a, written as pure FMA chains:
//   out0 += (a0-a3) psi2 - (a1 - i a2) psi3      out1 += -(a1 + i a2) psi2 + (a0+a3) psi3
//   out2 += (a0+a3) psi0 + (a1 - i a2) psi1      out3 +=  (a1 + i a2) psi0 + (a0-a3) psi1
template <typename R>
__device__ __forceinline__ void slash_acc(R s, const R* a, const cx<R>* psi, cx<R>* out) {
  const R am = s * (a[0] - a[3]), ap = s * (a[0] + a[3]);
  const R a1 = s * a[1], a2 = s * a[2];
  out[0].re = fma(am, psi[2].re, fma(-a1, psi[3].re, fma(-a2, psi[3].im, out[0].re)));
  out[0].im = fma(am, psi[2].im, fma(-a1, psi[3].im, fma(a2, psi[3].re, out[0].im)));
  out[1].re = fma(ap, psi[3].re, fma(-a1, psi[2].re, fma(a2, psi[2].im, out[1].re)));
  out[1].im = fma(ap, psi[3].im, fma(-a1, psi[2].im, fma(-a2, psi[2].re, out[1].im)));
  out[2].re = fma(ap, psi[0].re, fma(a1, psi[1].re, fma(a2, psi[1].im, out[2].re)));
  out[2].im = fma(ap, psi[0].im, fma(a1, psi[1].im, fma(-a2, psi[1].re, out[2].im)));
  out[3].re = fma(am, psi[1].re, fma(a1, psi[0].re, fma(-a2, psi[0].im, out[3].re)));
  out[3].im = fma(am, psi[1].im, fma(a1, psi[0].im, fma(a2, psi[0].re, out[3].im)));
}

#if defined(__CUDACC__)
// FP32: the same FMA chains on (re, im) pairs with packed FP32x2 FMAs (one
// instruction per complex component); each lane rounds exactly as above.
template <>
__device__ __forceinline__ void slash_acc<float>(float s, const float* a, const cx<float>* psi, cx<float>* out) {
  const float am = s * (a[0] - a[3]), ap = s * (a[0] + a[3]);
  const float a1 = s * a[1], a2 = s * a[2];
  auto P = [](const cx<float>& z) { return make_float2(z.re, z.im); };
  auto X = [](const cx<float>& z) { return make_float2(z.im, z.re); };
  auto B = [](float x) { return make_float2(x, x); };
  float2 o;
  o = __ffma2_rn(make_float2(-a2, a2), X(psi[3]), P(out[0]));
  o = __ffma2_rn(B(-a1), P(psi[3]), o);
  o = __ffma2_rn(B(am), P(psi[2]), o);
  out[0] = cx<float>{o.x, o.y};
  o = __ffma2_rn(make_float2(a2, -a2), X(psi[2]), P(out[1]));
  o = __ffma2_rn(B(-a1), P(psi[2]), o);
  o = __ffma2_rn(B(ap), P(psi[3]), o);
  out[1] = cx<float>{o.x, o.y};
  o = __ffma2_rn(make_float2(a2, -a2), X(psi[1]), P(out[2]));
  o = __ffma2_rn(B(a1), P(psi[1]), o);
  o = __ffma2_rn(B(ap), P(psi[0]), o);
  out[2] = cx<float>{o.x, o.y};
  o = __ffma2_rn(make_float2(-a2, a2), X(psi[0]), P(out[3]));
  o = __ffma2_rn(B(a1), P(psi[0]), o);
  o = __ffma2_rn(B(am), P(psi[1]), o);
  out[3] = cx<float>{o.x, o.y};
}
#endif

// out = (gamma . a) psi + c psi for real a and real c (FMA chains).
template <typename R>
__device__ __forceinline__ void slash_plus_scalar(const R* a, R c, const cx<R>* psi, cx<R>* out) {
#pragma unroll
  for (int i = 0; i < 4; ++i) out[i] = cx<R>{c * psi[i].re, c * psi[i].im};
  slash_acc(R(1), a, psi, out);
}

#if defined(__CUDACC__)
// FP32 with packed FP32x2 arithmetic (mixed mode): the scaling by c on (re, im) pairs
template <>
__device__ __forceinline__ void slash_plus_scalar<float>(const float* a, float c, const cx<float>* psi,
                                                         cx<float>* out) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 o = __fmul2_rn(make_float2(c, c), make_float2(psi[i].re, psi[i].im));
    out[i] = cx<float>{o.x, o.y};
  }
  slash_acc(1.0f, a, psi, out);
}
#endif

// Fermion propagator (FFV1_1 role) with the vertex and propagator factors i*i = -1:
//   out = -(q-slash + m) in / (q^2 - m^2 + i m Gamma).
// Zero width: the real factor f = -1/(q^2 - m^2) is folded into q and m
// (qf = f q, mf = f m) so the whole operation is FMA chains.
template <typename R>
__device__ __forceinline__ void fermion_prop_real(const R* q, R m, R invden, const cx<R>* in, cx<R>* out) {
  const R f = -invden;
  const R qf[4] = {f * q[0], f * q[1], f * q[2], f * q[3]};
  slash_plus_scalar(qf, f * m, in, out);
}

// Complex inverse denominator (non-zero width).
template <typename R>
__device__ __forceinline__ void fermion_prop(const R* q, R m, cx<R> invden, const cx<R>* in, cx<R>* out) {
  cx<R> t[4];
  slash_plus_scalar(q, m, in, t);
#pragma unroll
  for (int i = 0; i < 4; ++i) out[i] = -(t[i] * invden);
}

// ubar(u) . x = u_L^dag x_R + u_R^dag x_L  (FFV1_0 closure role).
template <typename R>
__device__ __forceinline__ cx<R> ubar_dot(const cx<R>* u, const cx<R>* x) {
  return cdot1(u[0], x[2]) + cdot1(u[1], x[3]) + cdot1(u[2], x[0]) + cdot1(u[3], x[1]);
}

// ---------------------------------------------------------------------------
// colour-ordered gluon vertices (VVV1P0_1 / VVVV roles), real currents
// ---------------------------------------------------------------------------

#if defined(__CUDACC__)
// FP32: conj(u) . x summed as one chain of packed FP32x2 FMAs on (re, im)
template <>
__device__ __forceinline__ cx<float> ubar_dot<float>(const cx<float>* u, const cx<float>* x) {
  float2 acc = make_float2(0.f, 0.f);
  const int xi[4] = {2, 3, 0, 1};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const cx<float> a = u[i], b = x[xi[i]];
    acc = __ffma2_rn(make_float2(a.re, a.re), make_float2(b.re, b.im), acc);
    acc = __ffma2_rn(make_float2(a.im, -a.im), make_float2(b.im, b.re), acc);
  }
  return cx<float>{acc.x, acc.y};
}
#endif

// out += s * [ (X.Y)(PY - PX) - (X.(PX + 2 PY)) Y + (Y.(2 PX + PY)) X ]
template <typename R>
__device__ __forceinline__ void vvv_acc(R s, const R* jx, const R* px, const R* jy, const R* py, R* out) {
  R a[4], b[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    a[m] = px[m] + R(2) * py[m];
    b[m] = R(2) * px[m] + py[m];
  }
  const R xy = s * mdot(jx, jy);
  const R xa = s * mdot(jx, a);
  const R yb = s * mdot(jy, b);
#pragma unroll
  for (int m = 0; m < 4; ++m) out[m] += xy * (py[m] - px[m]) - xa * jy[m] + yb * jx[m];
}

// out += s * [ (X.Y) Z + (Y.Z) X - 2 (X.Z) Y ]
template <typename R>
__device__ __forceinline__ void vvvv_acc(R s, const R* jx, const R* jy, const R* jz, R* out) {
  const R xy = s * mdot(jx, jy);
  const R yz = s * mdot(jy, jz);
  const R xz2 = R(-2) * s * mdot(jx, jz);
#pragma unroll
  for (int m = 0; m < 4; ++m) out[m] += xy * jz[m] + yz * jx[m] + xz2 * jy[m];
}

}  // namespace rex
