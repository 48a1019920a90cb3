// Reweighted cross sections and their errors on the GPU (sm_103a).
//
// Sec. 3.1.2:  sigma'_j = C sum_i w'_ij  (C = sigma / sum_i w_i),
//              dsigma'_j = dsigma * mean_i(w'_ij / w_i) + sigma * std_i(w'_ij),
// falling back to dsigma * max(sigma'_j / sigma, sigma / sigma'_j) when the
// error is infinite, NaN or non-positive.  std is the population standard
// deviation; the mean of w'/w runs over events with w_i != 0.
//
// The statistics are accumulated over any number of calls (a sample split over
// several processes or batches) in a fixed order, so that the result does not
// depend on how the GPU schedules the blocks:
//   pass 1  block b of the grid reduces events [b E, (b+1) E): each thread keeps
//           shifted sums (first value K: S = sum (x - K), SS = sum (x - K)^2) of
//           its events for one point, in double-float (FP64 for a block whose values
//           leave its range), turned into (n, mean, M2, sum = n K + S) in FP64;
//           the threads of a point merge in a fixed order (Chan, Golub & LeVeque 1979);
//   pass 2  one block per point merges the blocks' partials with a fixed-shape
//           tree, then into the accumulator;
//   result  sigma', dsigma' and the fallback flag per point.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "../../include/rex.h"
#include "dev_alloc.h"
#include "df64.cuh"
#include "fpconv.cuh"

namespace {

constexpr int XS_TJ = 32;          // points per block (x)
constexpr int XS_TE = 8;           // event rows per block (y)
constexpr int XS_EB = 2048;        // events per block

struct Moments {                   // count, mean, sum of squared deviations, plain sum, ratio sum
  double n, mean, m2, s1, r;
};

__host__ __device__ inline Moments merge(const Moments& a, const Moments& b) {
  if (b.n == 0.0) return a;
  if (a.n == 0.0) return b;
  Moments c;
  c.n = a.n + b.n;
  const double d = b.mean - a.mean, fb = b.n / c.n;
  c.mean = a.mean + d * fb;
  c.m2 = a.m2 + b.m2 + d * d * (a.n * fb);
  c.s1 = a.s1 + b.s1;
  c.r = a.r + b.r;
  return c;
}

struct Scalars {                   // per block / accumulator: events, events with w != 0, sum of w
  double n, nr, sw;
};

thread_local std::string g_xerr;
int xfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_xerr = buf;
  return code;
}

// Per-thread sums of pass 1 for point j: the count, the first value K, S = sum (x - K),
// SS = sum (x - K)^2 and r = sum x / w over the events with w != 0; the block's
// scalars (events with w != 0, sum of w) come from the threads of column group 0.
struct ThreadSums {
  int cnt;
  bool wide;   // a value outside the double-float range (DF only)
  double K, S, SS, r, nr, sw;
};

// Bit-field helpers on the two 32-bit halves of an FP64 value (32-bit integer
// instructions only).
// The biased exponent (0 for zero and subnormals).
__device__ __forceinline__ int exponent_of(double x) { return (__double2hiint(x) >> 20) & 0x7ff; }

__device__ __forceinline__ bool is_zero(double x) {
  return (((unsigned)__double2hiint(x) << 1) | (unsigned)__double2loint(x)) == 0u;
}

// x / 2^e for a normal x whose result stays normal: the exponent field minus e.
__device__ __forceinline__ double scale_down(double x, int e) {
  return __hiloint2double(__double2hiint(x) - (e << 20), __double2loint(x));
}

// An integer |n| < 2^22 as FP32 without a conversion instruction (B300 runs those at
// the FP64 rate): n added to the bit pattern of 2^23 + 2^22, then that offset removed.
__device__ __forceinline__ float small_int_to_float(int n) {
  return __fsub_rn(__int_as_float(0x4B400000 + n), 12582912.0f);
}

// FP64 -> double-float without an FP64 or conversion instruction, for a normal x with a
// binary exponent in [-60, 60]: hi keeps the 24 leading significand bits (rounded half
// up), lo the remaining 29 as a signed integer, assembled in FP32 from its upper 22 and
// lower 7 bits and scaled by powers of two; hi + lo equals x to 2^-53 |x|.
__device__ __forceinline__ rex::df64 split_df(double x) {
  const unsigned h = (unsigned)__double2hiint(x), l = (unsigned)__double2loint(x);
  const unsigned sign = h & 0x80000000u;
  const int e = (int)((h >> 20) & 0x7ffu) - 1023;
  unsigned top = (((h & 0xfffffu) | 0x100000u) << 3) | (l >> 29);   // 2^23 <= top < 2^24
  int rem = (int)(l & 0x1fffffffu);                                  // the 29 bits below
  if (rem >= (1 << 28)) {
    ++top;
    rem -= 1 << 29;
  }
  const int eh = top == (1u << 24) ? e + 1 : e;        // rounding carried into the exponent
  const float hi = __uint_as_float(sign | ((unsigned)(eh + 127) << 23) | (top & 0x7fffffu));
  const float lo = __fmaf_rn(small_int_to_float(rem >> 7), __uint_as_float((unsigned)(e - 45 + 127) << 23),
                             __fmul_rn(small_int_to_float(rem & 127), __uint_as_float((unsigned)(e - 52 + 127) << 23)));
  return rex::df64_make(hi, sign ? -lo : lo);
}

__device__ __forceinline__ double df_to_double(rex::df64 v) {
  return rex::f32_to_f64_alu(v.hi) + rex::f32_to_f64_alu(v.lo);
}

// pass 1 of one thread.  A warp takes 32 events at a time: each lane loads one event's
// w and forms its reciprocal (one per event), then the warp walks the 32 events
// G = 32 / kw at a time, lane L on event L / kw and point by kw + L % kw (kw = lanes per
// event: the next power of two >= k, at most 32), so that every lane has work when
// k < 32.
// DF: the sums and the reciprocal in double-float on the FP32 pipe (B300 issues FP64,
// conversions included, at 1/64 of the FP32 rate), each value first scaled by 2^-e0
// (e0: the exponent of the thread's first value; an exact power-of-two scaling undone
// at the end) and split into two FP32 numbers with integer instructions.  A value
// further than 2^40 from that scale, a w outside [2^-60, 2^60], a subnormal, an
// infinity or a NaN is beyond what the FP32 exponent range carries for the sums and
// squares: the result is then flagged (wide), and the caller recomputes the whole block
// in FP64 (in the same order, so the result stays bitwise reproducible).
template <bool DF>
__device__ __forceinline__ ThreadSums thread_sums(const double* __restrict__ w_in, const double* __restrict__ w_out,
                                                  int64_t e_beg, int64_t e_end, int k, int kw, int j) {
  const int lane = threadIdx.x, te = threadIdx.y;
  const int G = XS_TJ / kw;                      // events per warp step
  const int sub = lane / kw;
  int cnt = 0;                                   // integer count: keeps the FP64 pipe for the sums
  double K = 0.0, S = 0.0, SS = 0.0, r = 0.0;
  int nnz = 0;                                   // events with w != 0 (column group 0)
  double sw = 0.0;
  rex::df64 Kd = rex::df64_make(0.f, 0.f), Sd = Kd, SSd = Kd, rd = Kd;
  int e0 = 0;                                    // DF: the scale exponent (unbiased)
  bool out_of_range = false;
  if constexpr (DF) {
    // the thread's first value (event e_beg + 32 te + sub): K, its scale and its split
    const int64_t e_first = e_beg + (int64_t)te * XS_TJ + sub;
    if (e_first < e_end && j < k) {
      K = w_out[e_first * k + j];
      const int ek = exponent_of(K);
      if (ek == 0x7ff || (ek == 0 && !is_zero(K))) out_of_range = true;
      else if (!is_zero(K)) {
        e0 = ek - 1023;
        Kd = split_df(scale_down(K, e0));
      }
    }
  }
  for (int64_t g0 = e_beg + (int64_t)te * XS_TJ; g0 < e_end; g0 += (int64_t)XS_TE * XS_TJ) {
    const int64_t el = g0 + lane;
    const double wl = el < e_end ? w_in[el] : 0.0;
    double il = 0.0;
    if constexpr (!DF) il = wl != 0.0 ? 1.0 / wl : 0.0;
    if (blockIdx.y == 0 && el < e_end) {
      nnz += is_zero(wl) ? 0 : 1;
      sw += wl;
    }
    rex::df64 ild = rex::df64_make(0.f, 0.f);
    if constexpr (DF) {
      // 1 / w in double-float (no FP64 division): w within [2^-60, 2^60] or zero
      const int ew = exponent_of(wl);
      if (!is_zero(wl)) {
        if (ew < 1023 - 60 || ew >= 1023 + 60) out_of_range = true;
        else ild = rex::df64(1) / split_df(wl);
      }
    }
    for (int s = 0; s < XS_TJ; s += G) {
      const int src = s + sub;                     // event of this lane within the 32
      const double w = __shfl_sync(0xffffffffu, wl, src);
      const int64_t e = g0 + src;
      if constexpr (DF) {
        const rex::df64 inv = rex::df64_make(__shfl_sync(0xffffffffu, ild.hi, src),
                                             __shfl_sync(0xffffffffu, ild.lo, src));
        if (e < e_end && j < k) {
          const double x = w_out[e * k + j];
          const int ex = exponent_of(x);
          rex::df64 xd = rex::df64_make(0.f, 0.f);
          if (!is_zero(x)) {
            if (ex == 0 || ex == 0x7ff || ex - 1023 - e0 < -40 || ex - 1023 - e0 >= 40) out_of_range = true;
            else xd = split_df(scale_down(x, e0));
          }
          const rex::df64 d = xd - Kd;
          Sd = Sd + d;
          SSd = fma(d, d, SSd);
          if (!is_zero(w)) rd = fma(xd, inv, rd);      // w != 0 (either sign of zero)
          ++cnt;
        }
      } else {
        const double inv = __shfl_sync(0xffffffffu, il, src);
        if (e < e_end && j < k) {
          const double x = w_out[e * k + j];
          if (cnt == 0) K = x;
          const double d = x - K;
          S += d;
          SS = fma(d, d, SS);
          if (__double_as_longlong(w) << 1) r = fma(x, inv, r);
          ++cnt;
        }
      }
    }
  }
  if constexpr (DF) {
    const double p2 = __longlong_as_double((long long)(e0 + 1023) << 52);   // 2^e0, e0 of a normal K
    S = df_to_double(Sd) * p2;
    SS = df_to_double(SSd) * p2 * p2;
    r = df_to_double(rd) * p2;
  }
  return ThreadSums{cnt, out_of_range, K, S, SS, r, (double)nnz, sw};
}

// pass 1: partial moments of events [bx E, bx E + E) for the points of column group
// by, from the threads' sums in double-float, or in FP64 for a block with a value
// outside the double-float range (see thread_sums).  The Chan-Golub-LeVeque merges of
// the threads' moments and everything after them stay FP64.
__global__ void __launch_bounds__(XS_TJ* XS_TE, 2) xsec_partials_kernel(const double* __restrict__ w_in,
                                                                     const double* __restrict__ w_out, int64_t nev,
                                                                     int k, int kw, Moments* __restrict__ part,
                                                                     Scalars* __restrict__ psc) {
  __shared__ Moments sm[XS_TE][XS_TJ];
  __shared__ Scalars ssc[XS_TE][XS_TJ];
  const int lane = threadIdx.x, te = threadIdx.y;
  const int G = XS_TJ / kw;
  const int sub = lane / kw, jl = lane - sub * kw;
  const int j = blockIdx.y * kw + jl;
  const int64_t e_beg = (int64_t)blockIdx.x * XS_EB;
  const int64_t e_end = (e_beg + XS_EB < nev) ? e_beg + XS_EB : nev;
  ThreadSums ts = thread_sums<true>(w_in, w_out, e_beg, e_end, k, kw, j);
  if (__syncthreads_or(ts.wide)) ts = thread_sums<false>(w_in, w_out, e_beg, e_end, k, kw, j);
  const int cnt = ts.cnt;
  const double K = ts.K, S = ts.S, SS = ts.SS, r = ts.r, nr = ts.nr, sw = ts.sw;
  Moments m;
  m.n = (double)cnt;
  m.mean = cnt > 0 ? K + S / m.n : 0.0;
  m.m2 = cnt > 0 ? SS - S * (S / m.n) : 0.0;
  m.s1 = m.n * K + S;
  m.r = r;
  sm[te][lane] = m;
  ssc[te][lane] = Scalars{0.0, nr, sw};
  __syncthreads();
  if (te == 0 && lane < kw) {
    // the G lanes of point j in each of the 8 warps, in a fixed order
    Moments acc = sm[0][lane];
    for (int t = 0; t < XS_TE; ++t)
      for (int g = 0; g < G; ++g)
        if (t | g) acc = merge(acc, sm[t][g * kw + lane]);
    if (j < k) part[(int64_t)blockIdx.x * k + j] = acc;
  }
  if (te == 0 && lane == 0 && blockIdx.y == 0) {
    Scalars sc{(double)(e_end - e_beg), 0.0, 0.0};
    for (int t = 0; t < XS_TE; ++t)
      for (int l = 0; l < XS_TJ; ++l) {
        sc.nr += ssc[t][l].nr;
        sc.sw += ssc[t][l].sw;
      }
    psc[blockIdx.x] = sc;
  }
}

// pass 2: one block per point merges the blocks' partials with a fixed-shape
// tree (thread t takes partials t, t + 256, ... in order, then a pairwise tree
// over the 256 threads), then into the accumulator; block 0 also sums the scalars.
constexpr int XS_MERGE = 256;
__global__ void __launch_bounds__(XS_MERGE) xsec_merge_kernel(const Moments* __restrict__ part,
                                                              const Scalars* __restrict__ psc, int nblk, int k,
                                                              Moments* __restrict__ acc, Scalars* __restrict__ asc) {
  __shared__ Moments sm[XS_MERGE];
  __shared__ Scalars ss[XS_MERGE];
  const int j = blockIdx.x, t = threadIdx.x;
  Moments m{0.0, 0.0, 0.0, 0.0, 0.0};
  Scalars sc{0.0, 0.0, 0.0};
  for (int b = t; b < nblk; b += XS_MERGE) {
    m = merge(m, part[(int64_t)b * k + j]);
    if (j == 0) {
      sc.n += psc[b].n;
      sc.nr += psc[b].nr;
      sc.sw += psc[b].sw;
    }
  }
  sm[t] = m;
  ss[t] = sc;
  __syncthreads();
  for (int stride = XS_MERGE / 2; stride > 0; stride >>= 1) {
    if (t < stride) {
      sm[t] = merge(sm[t], sm[t + stride]);
      ss[t].n += ss[t + stride].n;
      ss[t].nr += ss[t + stride].nr;
      ss[t].sw += ss[t + stride].sw;
    }
    __syncthreads();
  }
  if (t == 0) {
    acc[j] = merge(acc[j], sm[0]);
    if (j == 0) {
      Scalars a = asc[0];
      a.n += ss[0].n;
      a.nr += ss[0].nr;
      a.sw += ss[0].sw;
      asc[0] = a;
    }
  }
}

__global__ void xsec_result_kernel(const Moments* __restrict__ acc, const Scalars* __restrict__ asc, int k,
                                   double sigma, double dsigma, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  const Moments m = acc[j];
  const Scalars s = asc[0];
  const double c = sigma / s.sw;
  const double sig = c * m.s1;
  const double mean_ratio = s.nr > 0.0 ? m.r / s.nr : NAN;
  const double sd = sqrt(m.n > 0.0 ? (m.m2 > 0.0 ? m.m2 : 0.0) / m.n : NAN);
  double ds = dsigma * mean_ratio + sigma * sd;
  double fb = 0.0;
  if (!isfinite(ds) || ds <= 0.0) {
    const double r1 = sigma != 0.0 ? sig / sigma : INFINITY;
    const double r2 = sig != 0.0 ? sigma / sig : INFINITY;
    ds = dsigma * ((r2 > r1) ? r2 : r1);
    fb = 1.0;
  }
  out[j] = sig;
  out[k + j] = ds;
  out[2 * k + j] = fb;
}

}  // namespace

struct rex_xsec {
  int k;
  Moments* acc;        // [k]
  Scalars* asc;        // [1]
  Moments* part;       // [nblk][k], grown on demand
  Scalars* psc;        // [nblk]
  int64_t part_blocks;
  double* res;         // [3][k]
};

extern "C" {

const char* rex_xsec_last_error(void) { return g_xerr.c_str(); }

int rex_xsec_create(int k, rex_xsec** out) {
  if (!out) return xfail(REX_EINVAL, "null output handle pointer");
  *out = nullptr;
  if (k < 1 || k > (1 << 20)) return xfail(REX_EINVAL, "k must be in 1..2^20");
  rex_xsec* x = new (std::nothrow) rex_xsec();
  if (!x) return xfail(REX_ENOMEM, "out of host memory");
  x->k = k;
  cudaError_t e = rex::dev_malloc(&x->acc, sizeof(Moments) * k);
  if (e == cudaSuccess) e = rex::dev_malloc(&x->asc, sizeof(Scalars));
  if (e == cudaSuccess) e = rex::dev_malloc(&x->res, sizeof(double) * 3 * k);
  if (e == cudaSuccess) e = cudaMemset(x->acc, 0, sizeof(Moments) * k);
  if (e == cudaSuccess) e = cudaMemset(x->asc, 0, sizeof(Scalars));
  if (e != cudaSuccess) {
    cudaFree(x->acc);
    cudaFree(x->asc);
    cudaFree(x->res);
    delete x;
    return xfail(REX_ENOMEM, "accumulator allocation failed: %s", cudaGetErrorString(e));
  }
  *out = x;
  return REX_OK;
}

int rex_xsec_reset(rex_xsec* x, void* stream) {
  if (!x) return xfail(REX_EINVAL, "null handle");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(x->acc, 0, sizeof(Moments) * x->k, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(x->asc, 0, sizeof(Scalars), st);
  return e == cudaSuccess ? REX_OK : xfail(REX_ECUDA, "reset: %s", cudaGetErrorString(e));
}

int rex_xsec_accumulate(rex_xsec* x, const double* w_in, const double* w_out, int64_t nev, void* stream) {
  if (!x) return xfail(REX_EINVAL, "null handle");
  if (nev < 0) return xfail(REX_EINVAL, "nev < 0");
  if (nev == 0) return REX_OK;
  if (!w_in || !w_out) return xfail(REX_EINVAL, "null array");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t nblk = (nev + XS_EB - 1) / XS_EB;
  if (nblk > 0x7fffffffLL) return xfail(REX_EINVAL, "too many events for one call");
  if (nblk > x->part_blocks) {
    // growing the partials buffer: earlier calls on this handle must have finished with it
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(x->part);
    cudaFree(x->psc);
    x->part = nullptr;
    x->psc = nullptr;
    x->part_blocks = 0;
    if (e == cudaSuccess) e = rex::dev_malloc(&x->part, sizeof(Moments) * x->k * nblk);
    if (e == cudaSuccess) e = rex::dev_malloc(&x->psc, sizeof(Scalars) * nblk);
    if (e != cudaSuccess) {
      cudaFree(x->part);
      cudaFree(x->psc);
      x->part = nullptr;
      x->psc = nullptr;
      return xfail(REX_ENOMEM, "partials allocation failed: %s", cudaGetErrorString(e));
    }
    x->part_blocks = nblk;
  }
  int kw = 1;
  while (kw < x->k && kw < XS_TJ) kw <<= 1;   // lanes per event
  const dim3 grid((unsigned)nblk, (unsigned)((x->k + kw - 1) / kw));
  if (grid.y > 65535) return xfail(REX_EINVAL, "too many points");
  xsec_partials_kernel<<<grid, dim3(XS_TJ, XS_TE), 0, st>>>(w_in, w_out, nev, x->k, kw, x->part, x->psc);
  xsec_merge_kernel<<<x->k, XS_MERGE, 0, st>>>(x->part, x->psc, (int)nblk, x->k, x->acc, x->asc);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? REX_OK : xfail(REX_ECUDA, "accumulate: %s", cudaGetErrorString(e));
}

int rex_xsec_result(rex_xsec* x, double sigma, double dsigma, double* sigma_out, double* dsigma_out, int* fallback,
                    void* stream) {
  if (!x) return xfail(REX_EINVAL, "null handle");
  if (!sigma_out || !dsigma_out) return xfail(REX_EINVAL, "null output array");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int k = x->k;
  xsec_result_kernel<<<(k + 127) / 128, 128, 0, st>>>(x->acc, x->asc, k, sigma, dsigma, x->res);
  double* h = new (std::nothrow) double[3 * (size_t)k];
  if (!h) return xfail(REX_ENOMEM, "out of host memory");
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, x->res, sizeof(double) * 3 * k, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) {
    std::memcpy(sigma_out, h, sizeof(double) * k);
    std::memcpy(dsigma_out, h + k, sizeof(double) * k);
    if (fallback)
      for (int j = 0; j < k; ++j) fallback[j] = h[2 * k + j] != 0.0;
  }
  delete[] h;
  return e == cudaSuccess ? REX_OK : xfail(REX_ECUDA, "result: %s", cudaGetErrorString(e));
}

int rex_xsec_get_state(rex_xsec* x, double* state, void* stream) {
  if (!x || !state) return xfail(REX_EINVAL, "null argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  static_assert(sizeof(Moments) == 5 * sizeof(double) && sizeof(Scalars) == 3 * sizeof(double), "packed state");
  cudaError_t e = cudaMemcpyAsync(state, x->acc, sizeof(Moments) * x->k, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(state + 5 * (size_t)x->k, x->asc, sizeof(Scalars), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? REX_OK : xfail(REX_ECUDA, "get_state: %s", cudaGetErrorString(e));
}

int rex_xsec_set_state(rex_xsec* x, const double* state, void* stream) {
  if (!x || !state) return xfail(REX_EINVAL, "null argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(x->acc, state, sizeof(Moments) * x->k, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(x->asc, state + 5 * (size_t)x->k, sizeof(Scalars), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? REX_OK : xfail(REX_ECUDA, "set_state: %s", cudaGetErrorString(e));
}

int rex_xsec_merge_states(const double* a, const double* b, int k, double* out) {
  if (!a || !b || !out || k < 1) return xfail(REX_EINVAL, "bad arguments");
  for (int j = 0; j < k; ++j) {
    Moments ma, mb;
    std::memcpy(&ma, a + 5 * (size_t)j, sizeof ma);
    std::memcpy(&mb, b + 5 * (size_t)j, sizeof mb);
    const Moments m = merge(ma, mb);
    std::memcpy(out + 5 * (size_t)j, &m, sizeof m);
  }
  for (int i = 0; i < 3; ++i) out[5 * (size_t)k + i] = a[5 * (size_t)k + i] + b[5 * (size_t)k + i];
  return REX_OK;
}

void rex_xsec_free(rex_xsec* x) {
  if (!x) return;
  cudaFree(x->acc);
  cudaFree(x->asc);
  cudaFree(x->part);
  cudaFree(x->psc);
  cudaFree(x->res);
  delete x;
}

}  // extern "C"
