// Reweighted cross sections and their errors on the GPU (sm_103a).
//
// Sec. 3.1.2:  sigma'_j = C sum_i w'_ij  (C = sigma / sum_i w_i),
//              dsigma'_j = dsigma * mean_i(w'_ij / w_i) + sigma * std_i(w'_ij),
// falling back to dsigma * max(sigma'_j / sigma, sigma / sigma'_j) when the
// error is infinite, NaN or non-positive.  std is the population standard
// deviation; the mean of w'/w runs over events with w_i != 0.
//
// The statistics are accumulated over any number of calls (a sample split over
// several processes or batches) in FP64 and in a fixed order, so that the result
// does not depend on how the GPU schedules the blocks:
//   pass 1  block b of the grid reduces events [b E, (b+1) E): each thread keeps
//           shifted sums (first value K: S = sum (x - K), SS = sum (x - K)^2) of
//           its events for one point, turned into (n, mean, M2, sum = n K + S);
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

// pass 1: partial moments of events [bx E, bx E + E) for the points of column
// group by.  A warp takes 32 events at a time: each lane loads one event's w and
// forms its reciprocal (one warp-wide FP64 division per 32 events), then the
// warp walks the 32 events G = 32 / kw at a time, lane L on event L / kw and
// point by kw + L % kw (kw = lanes per event: the next power of two >= k, at
// most 32), so that every lane has work when k < 32.
__global__ void __launch_bounds__(XS_TJ* XS_TE) xsec_partials_kernel(const double* __restrict__ w_in,
                                                                     const double* __restrict__ w_out, int64_t nev,
                                                                     int k, int kw, Moments* __restrict__ part,
                                                                     Scalars* __restrict__ psc) {
  __shared__ Moments sm[XS_TE][XS_TJ];
  __shared__ Scalars ssc[XS_TE][XS_TJ];
  const int lane = threadIdx.x, te = threadIdx.y;
  const int G = XS_TJ / kw;                      // events per warp step
  const int sub = lane / kw, jl = lane - sub * kw;
  const int j = blockIdx.y * kw + jl;
  const int64_t e_beg = (int64_t)blockIdx.x * XS_EB;
  const int64_t e_end = (e_beg + XS_EB < nev) ? e_beg + XS_EB : nev;
  int cnt = 0;                                   // integer count: keeps the FP64 pipe for the sums
  double K = 0.0, S = 0.0, SS = 0.0, r = 0.0;
  double nr = 0.0, sw = 0.0;
  for (int64_t g0 = e_beg + (int64_t)te * XS_TJ; g0 < e_end; g0 += (int64_t)XS_TE * XS_TJ) {
    const int64_t el = g0 + lane;
    const double wl = el < e_end ? w_in[el] : 0.0;
    const double il = wl != 0.0 ? 1.0 / wl : 0.0;
    if (blockIdx.y == 0 && el < e_end) {
      nr += (wl != 0.0) ? 1.0 : 0.0;
      sw += wl;
    }
    for (int s = 0; s < XS_TJ; s += G) {
      const int src = s + sub;                     // event of this lane within the 32
      const double w = __shfl_sync(0xffffffffu, wl, src);
      const double inv = __shfl_sync(0xffffffffu, il, src);
      const int64_t e = g0 + src;
      if (e < e_end && j < k) {
        const double x = w_out[e * k + j];
        if (cnt == 0) K = x;
        const double d = x - K;
        S += d;
        SS = fma(d, d, SS);
        if (__double_as_longlong(w) << 1) r = fma(x, inv, r);   // w != 0 (either sign of zero)
        ++cnt;
      }
    }
  }
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
