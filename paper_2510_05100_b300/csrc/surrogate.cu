// MLP surrogate of the log weight ratio, trained and evaluated on the GPU (sm_103a).
//
// The network (22 -> 4 x 256 GELU -> 2) predicts r = log(|M(p;theta)|^2/|M(p;theta_0)|^2)
// and an estimate of its own absolute error.  Every step is a kernel of this file
// or of surrogate_gemm.cuh: input features, BF16 tensor-core GEMMs with FP32
// accumulation and fused bias/GELU epilogues, the output head with the loss and
// its gradient, split-K weight gradients, Adam, and for inference the split
// first layer, the weight epilogue and the exact fallback of flagged events.
//
// Parameter layout (FP32 master copy, one flat array, every matrix [in][out]):
//   W1 [32][256] (rows 22..31 zero), b1 [256], W2 [256][256], b2, W3, b3, W4, b4,
//   W5 [256][2], b5 [2].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <random>
#include <string>
#include <vector>

#include "../../include/rex.h"
#include "dev_alloc.h"
#include "surrogate_fused.cuh"
#include "surrogate_gemm.cuh"

using namespace rex;

namespace {

constexpr int NIN = 22, NINP = 32, WID = 256, NOUT = 2;
constexpr int64_t OFF_W1 = 0;
constexpr int64_t OFF_B1 = OFF_W1 + (int64_t)NINP * WID;
constexpr int64_t OFF_W2 = OFF_B1 + WID;
constexpr int64_t OFF_B2 = OFF_W2 + (int64_t)WID * WID;
constexpr int64_t OFF_W3 = OFF_B2 + WID;
constexpr int64_t OFF_B3 = OFF_W3 + (int64_t)WID * WID;
constexpr int64_t OFF_W4 = OFF_B3 + WID;
constexpr int64_t OFF_B4 = OFF_W4 + (int64_t)WID * WID;
constexpr int64_t OFF_W5 = OFF_B4 + WID;
constexpr int64_t OFF_B5 = OFF_W5 + (int64_t)WID * NOUT;
constexpr int64_t NPARAM = OFF_B5 + NOUT;
const int64_t OFF_W[4] = {OFF_W1, OFF_W2, OFF_W3, OFF_W4};
const int64_t OFF_B[4] = {OFF_B1, OFF_B2, OFF_B3, OFF_B4};
const int KIN[4] = {NINP, WID, WID, WID};

// feature scales: momenta in TeV, (mt - 173)/3, (alphas - 0.118)/0.008
constexpr double MOM_SCALE = 1.0e-3, MT_REF = 173.0, MT_SCALE = 1.0 / 3.0, AS_REF = 0.118, AS_SCALE = 1.0 / 0.008;

thread_local std::string g_err;
int sfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}
int scuda(cudaError_t e, const char* what) {
  return sfail(REX_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): counter-based index draws
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
// Training features for n samples.
//   explicit_order = 1: sample i is event i with its own point (pmt[i], pas[i])
//                       and ratio[i] (gradient checks);
//   explicit_order = 0: sample i is the pair idx = SplitMix64(seed, step, i) mod (nev k),
//                       event idx / k, point idx % k, ratio[e][j] (training).
// Features: momenta in TeV, (mt - 173)/3, (alphas - 0.118)/0.008, zero padding to 32;
// target log(ratio) - apow * log(alphas / as0) (the exact coupling part removed).
__global__ void features_kernel(const double* __restrict__ mom, const double* __restrict__ ratio,
                                const double* __restrict__ pmt, const double* __restrict__ pas, int64_t nev, int k,
                                int n, int explicit_order, uint64_t seed, uint64_t step, double as0, int apow,
                                __nv_bfloat16* __restrict__ X, float* __restrict__ T) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t e, j, r;
  if (explicit_order) {
    e = i;
    j = i;
    r = i;
  } else {
    const int64_t idx =
        (int64_t)(splitmix64(seed ^ (step * 0x100000001B3ull) ^ ((uint64_t)i << 20)) % (uint64_t)(nev * k));
    e = idx / k;
    j = idx - e * k;
    r = idx;
  }
  const double* p = mom + e * 20;
  __nv_bfloat16* x = X + (int64_t)i * NINP;
#pragma unroll
  for (int c = 0; c < 20; ++c) x[c] = __float2bfloat16((float)(p[c] * MOM_SCALE));
  x[20] = __float2bfloat16((float)((pmt[j] - MT_REF) * MT_SCALE));
  x[21] = __float2bfloat16((float)((pas[j] - AS_REF) * AS_SCALE));
#pragma unroll
  for (int c = NIN; c < NINP; ++c) x[c] = __float2bfloat16(0.f);
  T[i] = (float)(log(ratio[r]) - (apow ? apow * log(pas[j] / as0) : 0.0));
}

// Output head, loss and their gradients.  One warp per sample.
//   [y, e] = a4 W5 + b5; loss = (y - t)^2 + (e - |y - t|)^2 (the error head's
//   target |y - t| held constant); dOut = 2 (y - t)/n, 2 (e - |y - t|)/n;
//   dz4 = (dOut W5^T) * gelu'(z4).  Per-block partial sums of dW5, db5, loss.
__global__ void __launch_bounds__(256) head_train_kernel(const __nv_bfloat16* __restrict__ A4, const float* __restrict__ Z4,
                                                          const float* __restrict__ P, const float* __restrict__ T, int n,
                                                          __nv_bfloat16* __restrict__ dZ4, float* __restrict__ part) {
  __shared__ float w5[WID][NOUT];
  __shared__ float acc[WID * NOUT + NOUT + 1];
  for (int t = threadIdx.x; t < WID * NOUT; t += blockDim.x) w5[t / NOUT][t % NOUT] = P[OFF_W5 + t];
  for (int t = threadIdx.x; t < WID * NOUT + NOUT + 1; t += blockDim.x) acc[t] = 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * 8 + warp;
  if (i < n) {
    float a[8], y = 0.f, e = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int c = lane + 32 * q;
      a[q] = __bfloat162float(A4[(int64_t)i * WID + c]);
      y += a[q] * w5[c][0];
      e += a[q] * w5[c][1];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      y += __shfl_xor_sync(0xffffffffu, y, off);
      e += __shfl_xor_sync(0xffffffffu, e, off);
    }
    y += P[OFF_B5];
    e += P[OFF_B5 + 1];
    const float res = y - T[i];
    const float tgt = fabsf(res);
    const float d0 = 2.f * res / n, d1 = 2.f * (e - tgt) / n;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int c = lane + 32 * q;
      const float da = d0 * w5[c][0] + d1 * w5[c][1];
      dZ4[(int64_t)i * WID + c] = __float2bfloat16(da * gelu_grad_f(Z4[(int64_t)i * WID + c]));
      atomicAdd(&acc[c * NOUT + 0], a[q] * d0);    // shared-memory atomics: per-block partials
      atomicAdd(&acc[c * NOUT + 1], a[q] * d1);
    }
    if (lane == 0) {
      atomicAdd(&acc[WID * NOUT + 0], d0);
      atomicAdd(&acc[WID * NOUT + 1], d1);
      atomicAdd(&acc[WID * NOUT + 2], (res * res + (e - tgt) * (e - tgt)) / n);
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < WID * NOUT + NOUT + 1; t += blockDim.x)
    part[(int64_t)blockIdx.x * (WID * NOUT + NOUT + 1) + t] = acc[t];
}

// Column sums of a BF16 matrix [rows][cols] over row chunks of 128: part[chunk][col].
__global__ void colsum_kernel(const __nv_bfloat16* __restrict__ D, int rows, int cols, float* __restrict__ part) {
  const int c = threadIdx.x + blockIdx.y * blockDim.x;
  if (c >= cols) return;
  const int r0 = blockIdx.x * 128, r1 = min(rows, r0 + 128);
  float s = 0.f;
  for (int r = r0; r < r1; ++r) s += __bfloat162float(D[(int64_t)r * cols + c]);
  part[(int64_t)blockIdx.x * cols + c] = s;
}

// out[i] = sum_s part[s][i]  (deterministic order)
__global__ void reduce_parts_kernel(const float* __restrict__ part, int nsplit, int64_t len, int64_t stride,
                                    float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  float s = 0.f;
  for (int q = 0; q < nsplit; ++q) s += part[q * stride + i];
  out[i] = s;
}

// Adam on the flat FP32 parameters; refreshes the BF16 copies of W1..W4.
__global__ void adam_kernel(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M,
                            float* __restrict__ V, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2, __nv_bfloat16* __restrict__ W1b, __nv_bfloat16* __restrict__ W2b,
                            __nv_bfloat16* __restrict__ W3b, __nv_bfloat16* __restrict__ W4b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = G[i];
  const float m = b1 * M[i] + (1.f - b1) * g;
  const float v = b2 * V[i] + (1.f - b2) * g * g;
  M[i] = m;
  V[i] = v;
  const float w = P[i] - lr * (m / c1) / (sqrtf(v / c2) + eps);
  P[i] = w;
  if (i >= OFF_W1 && i < OFF_B1) W1b[i - OFF_W1] = __float2bfloat16(w);
  else if (i >= OFF_W2 && i < OFF_B2) W2b[i - OFF_W2] = __float2bfloat16(w);
  else if (i >= OFF_W3 && i < OFF_B3) W3b[i - OFF_W3] = __float2bfloat16(w);
  else if (i >= OFF_W4 && i < OFF_B4) W4b[i - OFF_W4] = __float2bfloat16(w);
}

__global__ void to_bf16_kernel(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __float2bfloat16(src[i]);
}

// Inference: per-event part of layer 1 uses the GEMM on event features (the
// two parameter columns zero); per-point part: P1[j] = x_pt(j) W1[20:22] + b1.
__global__ void event_features_kernel(const double* __restrict__ mom, int64_t nev, __nv_bfloat16* __restrict__ X) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nev) return;
  __nv_bfloat16* x = X + i * NINP;
#pragma unroll
  for (int c = 0; c < 20; ++c) x[c] = __float2bfloat16((float)(mom[i * 20 + c] * MOM_SCALE));
#pragma unroll
  for (int c = 20; c < NINP; ++c) x[c] = __float2bfloat16(0.f);
}

__global__ void point_part_kernel(const float* __restrict__ P, const double* __restrict__ pmt,
                                  const double* __restrict__ pas, int k, double as0, int apow,
                                  float* __restrict__ P1, float* __restrict__ OFF) {
  const int j = blockIdx.x, c = threadIdx.x;
  if (j >= k || c >= WID) return;
  // exact coupling part of the log ratio, added back to the network's output
  if (c == 0) OFF[j] = apow ? (float)(apow * log(pas[j] / as0)) : 0.f;
  // the point features round to BF16 exactly as in training
  const float f0 = __bfloat162float(__float2bfloat16((float)((pmt[j] - MT_REF) * MT_SCALE)));
  const float f1 = __bfloat162float(__float2bfloat16((float)((pas[j] - AS_REF) * AS_SCALE)));
  const float w0 = __bfloat162float(__float2bfloat16(P[OFF_W1 + 20 * WID + c]));
  const float w1 = __bfloat162float(__float2bfloat16(P[OFF_W1 + 21 * WID + c]));
  P1[j * WID + c] = f0 * w0 + f1 * w1 + P[OFF_B1 + c];
}

// Per-point table of the fused kernel: the two point features rounded to BF16
// (as in training) and the exact coupling part.
__global__ void point_table_kernel(const double* __restrict__ pmt, const double* __restrict__ pas, int k,
                                   double as0, int apow, float4* __restrict__ ptab) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  const float f0 = __bfloat162float(__float2bfloat16((float)((pmt[j] - MT_REF) * MT_SCALE)));
  const float f1 = __bfloat162float(__float2bfloat16((float)((pas[j] - AS_REF) * AS_SCALE)));
  ptab[j] = make_float4(f0, f1, apow ? (float)(apow * log(pas[j] / as0)) : 0.f, 0.f);
}

// A1[(e, j)] = gelu(E1[e] + P1[j]) for the pairs of an event chunk (pair = e * k + j)
__global__ void expand_kernel(const float* __restrict__ E1, const float* __restrict__ P1, int64_t nev, int k,
                              __nv_bfloat16* __restrict__ A1) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t pairs = nev * k;
  if (t >= pairs * (WID / 2)) return;
  const int64_t pr = t / (WID / 2);
  const int c = (int)(t - pr * (WID / 2)) * 2;
  const int64_t e = pr / k;
  const int j = (int)(pr - e * k);
  const float z0 = E1[e * WID + c] + P1[j * WID + c];
  const float z1 = E1[e * WID + c + 1] + P1[j * WID + c + 1];
  reinterpret_cast<__nv_bfloat162*>(A1)[t] = __floats2bfloat162_rn(gelu_f(z0), gelu_f(z1));
}

// Inference head: pred = network output + exact coupling part OFF[j], err per
// pair; new weight w_in * exp(pred); flag events whose predicted error exceeds
// tau.  One warp per pair.
__global__ void __launch_bounds__(256) head_infer_kernel(const __nv_bfloat16* __restrict__ A4, const float* __restrict__ P,
                                                          const float* __restrict__ OFF, int64_t pairs, int k,
                                                          int64_t ev_base,
                                                          const double* __restrict__ w_in, float tau,
                                                          float* __restrict__ pred, float* __restrict__ err,
                                                          double* __restrict__ w_out, int* __restrict__ flag) {
  __shared__ float w5[WID][NOUT];
  for (int t = threadIdx.x; t < WID * NOUT; t += blockDim.x) w5[t / NOUT][t % NOUT] = P[OFF_W5 + t];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t pr = (int64_t)blockIdx.x * 8 + warp;
  if (pr >= pairs) return;
  float y = 0.f, e = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int c = lane + 32 * q;
    const float a = __bfloat162float(A4[pr * WID + c]);
    y += a * w5[c][0];
    e += a * w5[c][1];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    y += __shfl_xor_sync(0xffffffffu, y, off);
    e += __shfl_xor_sync(0xffffffffu, e, off);
  }
  if (lane == 0) {
    const int64_t ev = ev_base + pr / k;
    y += P[OFF_B5] + OFF[pr - (pr / k) * k];
    e += P[OFF_B5 + 1];
    if (pred) pred[ev_base * k + pr] = y;
    if (err) err[ev_base * k + pr] = e;
    if (w_out) w_out[ev_base * k + pr] = w_in[ev] * (double)expf(y);
    if (flag && !(e <= tau)) flag[ev] = 1;   // NaN errors fall back too
  }
}

// Fallback plumbing: list the flagged events, gather their momenta and weights,
// and scatter the exact rows back.
__global__ void compact_kernel(const int* __restrict__ flag, int64_t nev, int* __restrict__ count,
                               int64_t* __restrict__ list) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nev || !flag[i]) return;
  const int pos = atomicAdd(count, 1);
  list[pos] = i;
}

__global__ void gather_kernel(const int64_t* __restrict__ list, int n, const double* __restrict__ mom,
                              const double* __restrict__ w_in, double* __restrict__ gm, double* __restrict__ gw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t e = list[i];
#pragma unroll
  for (int c = 0; c < 20; ++c) gm[(int64_t)i * 20 + c] = mom[e * 20 + c];
  gw[i] = w_in[e];
}

__global__ void scatter_kernel(const int64_t* __restrict__ list, int n, int k, const double* __restrict__ src,
                               double* __restrict__ w_out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * k) return;
  const int64_t i = t / k;
  const int j = (int)(t - i * k);
  w_out[list[i] * k + j] = src[t];
}

// Input-domain guard of the fallback.  For g g -> t t~ g the network's largest
// errors sit where the final gluon is soft or collinear: there |M|^2 is singular and
// the ratio varies fastest with the top mass.  y = min over the other four partons i
// of 2 k.p_i / s_hat (k the final gluon, s_hat = (p_1 + p_2)^2) measures both
// limits; events with y below the guard (or a NaN y) fall back.
__device__ __forceinline__ double soft_collinear_y(const double* __restrict__ p) {
  auto dot = [&](int a, int b) {
    return p[4 * a] * p[4 * b] - p[4 * a + 1] * p[4 * b + 1] - p[4 * a + 2] * p[4 * b + 2] - p[4 * a + 3] * p[4 * b + 3];
  };
  const double shat = dot(0, 0) + 2.0 * dot(0, 1) + dot(1, 1);
  double y = dot(4, 0);
#pragma unroll
  for (int i = 1; i < 4; ++i) y = fmin(y, dot(4, i));
  return 2.0 * y / shat;
}

__global__ void guard_kernel(const double* __restrict__ mom, int64_t nev, double y0, int* __restrict__ flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nev) return;
  const double y = soft_collinear_y(mom + i * 20);
  if (!(y >= y0)) flag[i] = 1;
}

// Per-event calibration statistics over k points: the largest predicted error
// (+inf if any is NaN), the number of points whose |pred - log(ratio)| exceeds the
// bound (a non-positive or NaN ratio counts as exceeding it), and y.
__global__ void calib_stats_kernel(const double* __restrict__ mom, const float* __restrict__ pred,
                                   const float* __restrict__ err, const double* __restrict__ ratio, int64_t nev,
                                   int k, double bound, float* __restrict__ emax, int* __restrict__ nbad,
                                   double* __restrict__ yout) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nev) return;
  float em = -INFINITY;
  int bad = 0;
  for (int j = 0; j < k; ++j) {
    const float e = err[i * k + j];
    em = (e == e) ? fmaxf(em, e) : INFINITY;
    const double r = ratio[i * k + j];
    const double d = r > 0.0 ? fabs((double)pred[i * k + j] - log(r)) : INFINITY;
    bad += !(d <= bound);
  }
  emax[i] = em;
  nbad[i] = bad;
  yout[i] = soft_collinear_y(mom + i * 20);
}

__global__ void fill_kernel(double* __restrict__ x, int64_t n, double v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <bool A_T, bool B_T, int EPI>
cudaError_t gemm(const GemmArgs& g, int splits, cudaStream_t st) {
  dim3 grid((g.N + GBN - 1) / GBN, (g.M + GBM - 1) / GBM, splits);
  gemm_bf16_kernel<A_T, B_T, EPI><<<grid, GTHREADS, 0, st>>>(g);
  return cudaGetLastError();
}

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (cap >= bytes) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    const cudaError_t e = rex::dev_malloc(&p, bytes);
    if (e == cudaSuccess) cap = bytes;
    return e;
  }
  template <typename T>
  T* as() const {
    return static_cast<T*>(p);
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

}  // namespace

struct rex_surrogate {
  float *params, *grads, *m, *v;
  __nv_bfloat16* wb[4];
  int step;
  double as0 = 0.118;   // exact coupling part: apow * log(alphas / as0)
  int apow = 0;
  int kernel = REX_SURROGATE_FUSED;   // inference kernel
  double guard_y = 0.0;   // events with soft_collinear_y < guard_y fall back (0: off)
  // work buffers, grown on demand
  DevBuf X, T, Z[4], A[4], dZa, dZb, part, pmt, pas, E1, P1, OFFS, flag, cnt, list, gmom, gw, gout;
  DevBuf PK, PTAB, STATUS;   // fused inference: packed weight images, point table, wait status
  DevBuf CP, CE, CR, CW, CS1, CS2, CS3;   // calibration: pred, err, exact ratio, unit weights, per-event stats
};

namespace {

void release(rex_surrogate* s) {
  cudaFree(s->params);
  cudaFree(s->grads);
  cudaFree(s->m);
  cudaFree(s->v);
  for (auto& w : s->wb) cudaFree(w);
  for (DevBuf* b : {&s->X, &s->T, &s->dZa, &s->dZb, &s->part, &s->pmt, &s->pas, &s->E1, &s->P1, &s->OFFS, &s->flag, &s->cnt,
                    &s->list, &s->gmom, &s->gw, &s->gout, &s->PK, &s->PTAB, &s->STATUS, &s->CP, &s->CE, &s->CR,
                    &s->CW, &s->CS1, &s->CS2, &s->CS3})
    b->release();
  for (int l = 0; l < 4; ++l) {
    s->Z[l].release();
    s->A[l].release();
  }
}

cudaError_t refresh_bf16(rex_surrogate* s, cudaStream_t st) {
  for (int l = 0; l < 4; ++l) {
    const int64_t n = (int64_t)KIN[l] * WID;
    to_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s->params + OFF_W[l], s->wb[l], n);
  }
  return cudaGetLastError();
}

cudaError_t ensure_batch(rex_surrogate* s, int64_t n) {
  cudaError_t e = s->X.ensure(n * NINP * 2);
  if (e == cudaSuccess) e = s->T.ensure(n * 4);
  for (int l = 0; l < 4 && e == cudaSuccess; ++l) {
    e = s->Z[l].ensure(n * WID * 4);
    if (e == cudaSuccess) e = s->A[l].ensure(n * WID * 2);
  }
  if (e == cudaSuccess) e = s->dZa.ensure(n * WID * 2);
  if (e == cudaSuccess) e = s->dZb.ensure(n * WID * 2);
  const int64_t head_parts = (n + 7) / 8 * (WID * NOUT + NOUT + 1);
  const int64_t wsplit = 16 * (int64_t)WID * WID, col_parts = (n + 127) / 128 * WID;
  const int64_t pmax = head_parts > wsplit ? head_parts : wsplit;
  if (e == cudaSuccess) e = s->part.ensure((pmax > col_parts ? pmax : col_parts) * 4);
  return e;
}

// Forward + backward of one batch of n samples already in s->X / s->T; fills
// s->grads and (if loss_dev) writes the mean loss to loss_dev.
int forward_backward(rex_surrogate* s, int n, float* loss_dev, cudaStream_t st) {
  cudaError_t e;
  // forward: Z_l = A_{l-1} W_l + b_l, A_l = gelu(Z_l)
  for (int l = 0; l < 4; ++l) {
    GemmArgs g{};
    g.M = n;
    g.N = WID;
    g.K = KIN[l];
    g.A = l == 0 ? s->X.as<__nv_bfloat16>() : s->A[l - 1].as<__nv_bfloat16>();
    g.lda = KIN[l];
    g.B = s->wb[l];
    g.ldb = WID;
    g.C32 = s->Z[l].as<float>();
    g.ldc = WID;
    g.C16 = s->A[l].as<__nv_bfloat16>();
    g.ldc16 = WID;
    g.bias = s->params + OFF_B[l];
    g.k_per_split = g.K;
    if ((e = gemm<false, false, EPI_FWD>(g, 1, st)) != cudaSuccess) return scuda(e, "forward gemm");
  }
  // head + loss + dZ4
  const int hblocks = (n + 7) / 8;
  float* part = s->part.as<float>();
  head_train_kernel<<<hblocks, 256, 0, st>>>(s->A[3].as<__nv_bfloat16>(), s->Z[3].as<float>(), s->params,
                                              s->T.as<float>(), n, s->dZa.as<__nv_bfloat16>(), part);
  const int hlen = WID * NOUT + NOUT + 1;
  // head partials -> grads[W5], grads[b5] (contiguous), loss
  reduce_parts_kernel<<<(WID * NOUT + NOUT + 255) / 256, 256, 0, st>>>(part, hblocks, WID * NOUT + NOUT, hlen,
                                                                       s->grads + OFF_W5);
  if (loss_dev) reduce_parts_kernel<<<1, 1, 0, st>>>(part + WID * NOUT + NOUT, hblocks, 1, hlen, loss_dev);
  if ((e = cudaGetLastError()) != cudaSuccess) return scuda(e, "head");
  // backward through layers 4..1
  __nv_bfloat16* dz = s->dZa.as<__nv_bfloat16>();
  __nv_bfloat16* dz_next = s->dZb.as<__nv_bfloat16>();
  for (int l = 3; l >= 0; --l) {
    // dW_l = A_{l-1}^T dZ_l  (split-K over the batch; deterministic partial sums)
    const int splits = n >= 4096 ? 16 : 1;
    int kps = (n + splits - 1) / splits;
    kps = (kps + GBK - 1) / GBK * GBK;
    GemmArgs g{};
    g.M = KIN[l];
    g.N = WID;
    g.K = n;
    g.A = l == 0 ? s->X.as<__nv_bfloat16>() : s->A[l - 1].as<__nv_bfloat16>();
    g.lda = KIN[l];
    g.B = dz;
    g.ldb = WID;
    g.C32 = part;
    g.ldc = WID;
    g.k_per_split = kps;
    g.split_stride = (int64_t)KIN[l] * WID;
    const int nsplit = (n + kps - 1) / kps;
    if ((e = gemm<true, false, EPI_F32>(g, nsplit, st)) != cudaSuccess) return scuda(e, "weight-gradient gemm");
    const int64_t wl = (int64_t)KIN[l] * WID;
    reduce_parts_kernel<<<(unsigned)((wl + 255) / 256), 256, 0, st>>>(part, nsplit, wl, g.split_stride,
                                                                       s->grads + OFF_W[l]);
    // db_l = column sums of dZ_l
    const int chunks = (n + 127) / 128;
    colsum_kernel<<<dim3(chunks, 1), WID, 0, st>>>(dz, n, WID, part);
    reduce_parts_kernel<<<1, WID, 0, st>>>(part, chunks, WID, WID, s->grads + OFF_B[l]);
    if (l > 0) {
      // dZ_{l-1} = (dZ_l W_l^T) * gelu'(Z_{l-1})
      GemmArgs b{};
      b.M = n;
      b.N = KIN[l];
      b.K = WID;
      b.A = dz;
      b.lda = WID;
      b.B = s->wb[l];
      b.ldb = WID;
      b.C16 = dz_next;
      b.ldc16 = KIN[l];
      b.zprev = s->Z[l - 1].as<float>();
      b.ldz = WID;
      b.k_per_split = WID;
      if ((e = gemm<false, true, EPI_BWD>(b, 1, st)) != cudaSuccess) return scuda(e, "backward gemm");
      std::swap(dz, dz_next);
    }
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return scuda(e, "backward");
  return REX_OK;
}

// Layer-by-layer inference: per event chunk, the layer-1 GEMM on event features
// plus the per-point part, then three mma.sync GEMMs with fused bias/GELU and
// the head kernel (activations round-trip through global memory).
int infer_layered(rex_surrogate* s, const double* momenta, const double* w_in, int64_t nev, const rex_params* pts,
                  int k, float tau, double* w_out, float* pred, float* err, cudaStream_t st) {
  // events per chunk: at most 8192 events and 2^19 (event, point) pairs
  int64_t chunk = ((int64_t)1 << 19) / k;
  if (chunk > 8192) chunk = 8192;
  if (chunk < 1) chunk = 1;
  const int64_t cev = nev < chunk ? nev : chunk;
  const int64_t cpairs = cev * k;
  cudaError_t e = s->X.ensure(cev * NINP * 2);
  if (e == cudaSuccess) e = s->E1.ensure(cev * WID * 4);
  if (e == cudaSuccess) e = s->P1.ensure((size_t)k * WID * 4);
  if (e == cudaSuccess) e = s->OFFS.ensure((size_t)k * 4);
  if (e == cudaSuccess) e = s->pmt.ensure((size_t)k * 8);
  if (e == cudaSuccess) e = s->pas.ensure((size_t)k * 8);
  if (e == cudaSuccess) e = s->A[0].ensure(cpairs * WID * 2);
  if (e == cudaSuccess) e = s->A[1].ensure(cpairs * WID * 2);
  if (e == cudaSuccess && w_out) e = s->flag.ensure(nev * 4);
  if (e != cudaSuccess) return sfail(REX_ENOMEM, "inference buffers: %s", cudaGetErrorString(e));
  std::vector<double> hm(k), ha(k);
  for (int j = 0; j < k; ++j) {
    hm[j] = pts[j].mt;
    ha[j] = pts[j].alphas;
  }
  e = cudaMemcpyAsync(s->pmt.p, hm.data(), k * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->pas.p, ha.data(), k * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && w_out) e = cudaMemsetAsync(s->flag.p, 0, nev * 4, st);
  if (e != cudaSuccess) return scuda(e, "inference set-up");
  point_part_kernel<<<k, WID, 0, st>>>(s->params, s->pmt.as<double>(), s->pas.as<double>(), k, s->as0, s->apow,
                                       s->P1.as<float>(), s->OFFS.as<float>());
  for (int64_t e0 = 0; e0 < nev; e0 += chunk) {
    const int64_t ne = (nev - e0) < chunk ? (nev - e0) : chunk;
    const int64_t np = ne * k;
    event_features_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(momenta + e0 * 20, ne,
                                                                        s->X.as<__nv_bfloat16>());
    // per-event part of layer 1: E1 = x_ev W1 (parameter columns of x_ev are zero)
    GemmArgs g{};
    g.M = (int)ne;
    g.N = WID;
    g.K = NINP;
    g.A = s->X.as<__nv_bfloat16>();
    g.lda = NINP;
    g.B = s->wb[0];
    g.ldb = WID;
    g.C32 = s->E1.as<float>();
    g.ldc = WID;
    g.k_per_split = NINP;
    if ((e = gemm<false, false, EPI_F32>(g, 1, st)) != cudaSuccess) return scuda(e, "layer-1 gemm");
    expand_kernel<<<(unsigned)((np * (WID / 2) + 255) / 256), 256, 0, st>>>(s->E1.as<float>(), s->P1.as<float>(), ne,
                                                                            k, s->A[0].as<__nv_bfloat16>());
    // layers 2..4 on the chunk's pairs (no pre-activations kept)
    __nv_bfloat16* cur = s->A[0].as<__nv_bfloat16>();
    __nv_bfloat16* nxt = s->A[1].as<__nv_bfloat16>();
    for (int l = 1; l < 4; ++l) {
      GemmArgs f{};
      f.M = (int)np;
      f.N = WID;
      f.K = WID;
      f.A = cur;
      f.lda = WID;
      f.B = s->wb[l];
      f.ldb = WID;
      f.C32 = nullptr;
      f.C16 = nxt;
      f.ldc16 = WID;
      f.bias = s->params + OFF_B[l];
      f.k_per_split = WID;
      if ((e = gemm<false, false, EPI_FWD>(f, 1, st)) != cudaSuccess) return scuda(e, "hidden gemm");
      std::swap(cur, nxt);
    }
    head_infer_kernel<<<(unsigned)((np + 7) / 8), 256, 0, st>>>(cur, s->params, s->OFFS.as<float>(), np, k, e0,
                                                                 w_in, tau, pred, err,
                                                                 w_out, w_out ? s->flag.as<int>() : nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return scuda(e, "inference head");
  }
  return REX_OK;
}

// Fused inference (surrogate_fused.cuh): one persistent tcgen05 kernel.
int infer_fused(rex_surrogate* s, const double* momenta, const double* w_in, int64_t nev, const rex_params* pts,
                int k, float tau, double* w_out, float* pred, float* err, cudaStream_t st) {
  const size_t img1 = (size_t)FW * FK1, img = (size_t)FW * FW;
  cudaError_t e = s->PK.ensure((img1 + 3 * img) * 2);
  if (e == cudaSuccess) e = s->X.ensure((size_t)nev * NINP * 2);
  if (e == cudaSuccess) e = s->PTAB.ensure((size_t)k * sizeof(float4));
  if (e == cudaSuccess) e = s->STATUS.ensure(4);
  if (e == cudaSuccess) e = s->pmt.ensure((size_t)k * 8);
  if (e == cudaSuccess) e = s->pas.ensure((size_t)k * 8);
  if (e == cudaSuccess && w_out) e = s->flag.ensure(nev * 4);
  if (e != cudaSuccess) return sfail(REX_ENOMEM, "inference buffers: %s", cudaGetErrorString(e));
  std::vector<double> hm(k), ha(k);
  for (int j = 0; j < k; ++j) {
    hm[j] = pts[j].mt;
    ha[j] = pts[j].alphas;
  }
  e = cudaMemcpyAsync(s->pmt.p, hm.data(), k * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->pas.p, ha.data(), k * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && w_out) e = cudaMemsetAsync(s->flag.p, 0, nev * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->STATUS.p, 0, 4, st);
  if (e != cudaSuccess) return scuda(e, "inference set-up");
  __nv_bfloat16* pk = s->PK.as<__nv_bfloat16>();
  pack_kmajor_kernel<<<(unsigned)((img1 + 255) / 256), 256, 0, st>>>(s->params + OFF_W1, FK1, 1.0f, pk);
  for (int l = 1; l < 4; ++l)
    pack_kmajor_kernel<<<(unsigned)((img + 255) / 256), 256, 0, st>>>(s->params + OFF_W[l], FW, FWSCALE,
                                                                      pk + img1 + (l - 1) * img);
  point_table_kernel<<<(k + 127) / 128, 128, 0, st>>>(s->pmt.as<double>(), s->pas.as<double>(), k, s->as0, s->apow,
                                                      s->PTAB.as<float4>());
  // per-event features (momenta in TeV, BF16), read by every pair of the event
  event_features_kernel<<<(unsigned)((nev + 255) / 256), 256, 0, st>>>(momenta, nev, s->X.as<__nv_bfloat16>());
  if ((e = cudaGetLastError()) != cudaSuccess) return scuda(e, "weight packing");
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(fused_mlp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(FusedSmem))) != cudaSuccess)
    return scuda(e, "fused kernel set-up");
  FusedArgs fa{};
  fa.xev = s->X.as<__nv_bfloat16>();
  fa.w_in = w_in;
  fa.nev = nev;
  fa.k = k;
  fa.ptab = s->PTAB.as<float4>();
  fa.w1 = pk;
  fa.w234 = pk + img1;
  for (int l = 0; l < 4; ++l) fa.bias[l] = s->params + OFF_B[l];
  fa.w5 = s->params + OFF_W5;
  fa.b5 = s->params + OFF_B5;
  fa.tau = tau;
  fa.pred = pred;
  fa.err = err;
  fa.w_out = w_out;
  fa.flag = w_out ? s->flag.as<int>() : nullptr;
  fa.status = s->STATUS.as<int>();
  // two tiles per CTA at a time: no more CTAs than tile pairs
  const int64_t pairs = ((nev * k + FM - 1) / FM + 1) / 2;
  const int grid = (int)(pairs < sms ? pairs : sms);
  fused_mlp_kernel<<<grid, FTHREADS, sizeof(FusedSmem), st>>>(fa);
  e = cudaGetLastError();
  return e == cudaSuccess ? REX_OK : scuda(e, "fused inference kernel");
}

int check_handle(const rex_surrogate* s) { return s ? REX_OK : sfail(REX_EINVAL, "null surrogate handle"); }

}  // namespace

extern "C" {

int64_t rex_surrogate_num_params(void) { return NPARAM; }

const char* rex_surrogate_last_error(void) { return g_err.c_str(); }

int rex_surrogate_create(unsigned long long seed, rex_surrogate** out) {
  if (!out) return sfail(REX_EINVAL, "null output handle pointer");
  *out = nullptr;
  rex_surrogate* s = new (std::nothrow) rex_surrogate();
  if (!s) return sfail(REX_ENOMEM, "out of host memory");
  cudaError_t e = rex::dev_malloc(&s->params, NPARAM * 4);
  if (e == cudaSuccess) e = rex::dev_malloc(&s->grads, NPARAM * 4);
  if (e == cudaSuccess) e = rex::dev_malloc(&s->m, NPARAM * 4);
  if (e == cudaSuccess) e = rex::dev_malloc(&s->v, NPARAM * 4);
  for (int l = 0; l < 4 && e == cudaSuccess; ++l) e = rex::dev_malloc(&s->wb[l], (size_t)KIN[l] * WID * 2);
  if (e != cudaSuccess) {
    release(s);
    delete s;
    return sfail(REX_ENOMEM, "surrogate allocation failed: %s", cudaGetErrorString(e));
  }
  // He-normal initialisation on the host (std::mt19937_64, Box-Muller by std::normal_distribution)
  std::vector<float> h(NPARAM, 0.f);
  std::mt19937_64 rng(seed);
  const int kin_true[5] = {NIN, WID, WID, WID, WID};
  const int64_t offw[5] = {OFF_W1, OFF_W2, OFF_W3, OFF_W4, OFF_W5};
  const int nout[5] = {WID, WID, WID, WID, NOUT};
  for (int l = 0; l < 5; ++l) {
    std::normal_distribution<float> nd(0.f, std::sqrt(2.f / kin_true[l]));
    for (int r = 0; r < kin_true[l]; ++r)
      for (int c = 0; c < nout[l]; ++c) h[offw[l] + (int64_t)r * nout[l] + c] = nd(rng);
  }
  e = cudaMemcpy(s->params, h.data(), NPARAM * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(s->m, 0, NPARAM * 4);
  if (e == cudaSuccess) e = cudaMemset(s->v, 0, NPARAM * 4);
  if (e == cudaSuccess) e = refresh_bf16(s, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    release(s);
    delete s;
    return scuda(e, "surrogate initialisation");
  }
  *out = s;
  return REX_OK;
}

int rex_surrogate_set_weights(rex_surrogate* s, const float* host, int64_t n) {
  int rc = check_handle(s);
  if (rc) return rc;
  if (!host || n != NPARAM) return sfail(REX_EINVAL, "expected %lld parameters", (long long)NPARAM);
  cudaError_t e = cudaMemcpy(s->params, host, NPARAM * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(s->m, 0, NPARAM * 4);
  if (e == cudaSuccess) e = cudaMemset(s->v, 0, NPARAM * 4);
  if (e == cudaSuccess) e = refresh_bf16(s, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  s->step = 0;
  return e == cudaSuccess ? REX_OK : scuda(e, "set weights");
}

int rex_surrogate_get_weights(rex_surrogate* s, float* host, int64_t n) {
  int rc = check_handle(s);
  if (rc) return rc;
  if (!host || n != NPARAM) return sfail(REX_EINVAL, "expected %lld parameters", (long long)NPARAM);
  const cudaError_t e = cudaMemcpy(host, s->params, NPARAM * 4, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? REX_OK : scuda(e, "get weights");
}

int rex_surrogate_loss_grad(rex_surrogate* s, const double* momenta, const double* ratio, const double* mt,
                            const double* alphas, int64_t n, float* loss_host, float* grad_host, void* stream) {
  int rc = check_handle(s);
  if (rc) return rc;
  if (n <= 0 || n > (1 << 22) || n % 32 || !momenta || !ratio || !mt || !alphas)
    return sfail(REX_EINVAL, "loss_grad needs 0 < n <= 2^22 samples, n a multiple of 32, non-null arrays");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = ensure_batch(s, n);
  if (e != cudaSuccess) return sfail(REX_ENOMEM, "batch buffers: %s", cudaGetErrorString(e));
  // sample i = event i with its own point (mt[i], alphas[i]) and ratio[i]
  features_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(momenta, ratio, mt, alphas, n, 1, (int)n, 1, 0, 0,
                                                               s->as0, s->apow, s->X.as<__nv_bfloat16>(),
                                                               s->T.as<float>());
  DevBuf& loss = s->gout;
  if ((e = loss.ensure(8)) != cudaSuccess) return sfail(REX_ENOMEM, "loss buffer");
  rc = forward_backward(s, (int)n, loss.as<float>(), st);
  if (rc) return rc;
  if (grad_host) {
    e = cudaMemcpyAsync(grad_host, s->grads, NPARAM * 4, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return scuda(e, "copy gradients");
  }
  if (loss_host) {
    e = cudaMemcpyAsync(loss_host, loss.as<float>(), 4, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return scuda(e, "copy loss");
  }
  e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? REX_OK : scuda(e, "loss_grad");
}

int rex_surrogate_train(rex_surrogate* s, const double* momenta, const double* ratio, int64_t nev,
                        const rex_params* pts, int k, int steps, int batch, float lr, unsigned long long seed,
                        float* loss_host, void* stream) {
  int rc = check_handle(s);
  if (rc) return rc;
  if (nev <= 0 || k <= 0 || steps < 0 || batch <= 0 || batch > (1 << 20) || batch % 128 || !momenta || !ratio || !pts)
    return sfail(REX_EINVAL, "train needs nev > 0, k > 0, steps >= 0, batch a multiple of 128 up to 2^20");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = ensure_batch(s, batch);
  if (e == cudaSuccess) e = s->pmt.ensure((size_t)k * 8);
  if (e == cudaSuccess) e = s->pas.ensure((size_t)k * 8);
  if (e == cudaSuccess) e = s->gout.ensure((size_t)(steps > 0 ? steps : 1) * 4);
  if (e != cudaSuccess) return sfail(REX_ENOMEM, "training buffers: %s", cudaGetErrorString(e));
  std::vector<double> hm(k), ha(k);
  for (int j = 0; j < k; ++j) {
    hm[j] = pts[j].mt;
    ha[j] = pts[j].alphas;
  }
  e = cudaMemcpyAsync(s->pmt.p, hm.data(), k * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->pas.p, ha.data(), k * 8, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return scuda(e, "copy points");
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int it = 0; it < steps; ++it) {
    features_kernel<<<(unsigned)((batch + 255) / 256), 256, 0, st>>>(
        momenta, ratio, s->pmt.as<double>(), s->pas.as<double>(), nev, k, batch, 0, seed, (uint64_t)s->step,
        s->as0, s->apow, s->X.as<__nv_bfloat16>(), s->T.as<float>());
    rc = forward_backward(s, batch, s->gout.as<float>() + it, st);
    if (rc) return rc;
    s->step += 1;
    const float c1 = 1.f - std::pow(b1, (float)s->step), c2 = 1.f - std::pow(b2, (float)s->step);
    adam_kernel<<<(unsigned)((NPARAM + 255) / 256), 256, 0, st>>>(s->params, s->grads, s->m, s->v, NPARAM, lr, b1,
                                                                   b2, eps, c1, c2, s->wb[0], s->wb[1], s->wb[2],
                                                                   s->wb[3]);
    if ((e = cudaGetLastError()) != cudaSuccess) return scuda(e, "adam");
  }
  if (loss_host && steps > 0) {
    e = cudaMemcpyAsync(loss_host, s->gout.p, (size_t)steps * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return scuda(e, "copy losses");
  }
  return REX_OK;
}

int rex_surrogate_reweight(rex_surrogate* s, rex_proc* exact, const double* momenta, const double* w_in, int64_t nev,
                           const rex_params* pts, int k, float tau, double* w_out, float* pred, float* err,
                           int64_t* n_fallback, void* stream) {
  int rc = check_handle(s);
  if (rc) return rc;
  if (nev < 0 || k < 0) return sfail(REX_EINVAL, "nev < 0 or k < 0");
  if (n_fallback) *n_fallback = 0;
  if (nev == 0 || k == 0) return REX_OK;
  if (!momenta || !pts || (w_out && !w_in)) return sfail(REX_EINVAL, "null array");
  if (k > 4096) return sfail(REX_EINVAL, "at most 4096 points per call");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  rc = s->kernel == REX_SURROGATE_FUSED ? infer_fused(s, momenta, w_in, nev, pts, k, tau, w_out, pred, err, st)
                                        : infer_layered(s, momenta, w_in, nev, pts, k, tau, w_out, pred, err, st);
  if (rc) return rc;
  if (!w_out || !exact) return REX_OK;
  // exact fallback of the flagged events (predicted error above tau, or outside the guard)
  if ((e = s->cnt.ensure(8)) != cudaSuccess || (e = s->list.ensure(nev * 8)) != cudaSuccess)
    return sfail(REX_ENOMEM, "fallback buffers");
  if (s->guard_y > 0.0) {
    guard_kernel<<<(unsigned)((nev + 255) / 256), 256, 0, st>>>(momenta, nev, s->guard_y, s->flag.as<int>());
    if ((e = cudaGetLastError()) != cudaSuccess) return scuda(e, "fallback guard");
  }
  if ((e = cudaMemsetAsync(s->cnt.p, 0, 4, st)) != cudaSuccess) return scuda(e, "fallback counter");
  compact_kernel<<<(unsigned)((nev + 255) / 256), 256, 0, st>>>(s->flag.as<int>(), nev, s->cnt.as<int>(),
                                                                s->list.as<int64_t>());
  int nflag = 0, status = 0;
  e = cudaMemcpyAsync(&nflag, s->cnt.p, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && s->kernel == REX_SURROGATE_FUSED)
    e = cudaMemcpyAsync(&status, s->STATUS.p, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return scuda(e, "fallback count");
  if (status) return sfail(REX_ECUDA, "fused inference kernel: a bounded wait gave up");
  if (n_fallback) *n_fallback = nflag;
  if (nflag == 0) return REX_OK;
  if ((e = s->gmom.ensure((size_t)nflag * 20 * 8)) != cudaSuccess || (e = s->gw.ensure((size_t)nflag * 8)) != cudaSuccess ||
      (e = s->gout.ensure((size_t)nflag * k * 8)) != cudaSuccess)
    return sfail(REX_ENOMEM, "fallback buffers");
  gather_kernel<<<(nflag + 255) / 256, 256, 0, st>>>(s->list.as<int64_t>(), nflag, momenta, w_in,
                                                     s->gmom.as<double>(), s->gw.as<double>());
  rc = rex_reweight(exact, s->gmom.as<double>(), s->gw.as<double>(), nflag, pts, k, s->gout.as<double>(), stream);
  if (rc) return sfail(rc, "exact fallback: %s", rex_last_error());
  scatter_kernel<<<(unsigned)(((int64_t)nflag * k + 255) / 256), 256, 0, st>>>(s->list.as<int64_t>(), nflag, k,
                                                                              s->gout.as<double>(), w_out);
  e = cudaGetLastError();
  return e == cudaSuccess ? REX_OK : scuda(e, "fallback scatter");
}

int rex_surrogate_set_guard(rex_surrogate* s, double y_min) {
  const int rc = check_handle(s);
  if (rc) return rc;
  if (!(y_min >= 0.0 && y_min < 1.0)) return sfail(REX_EINVAL, "guard y_min must be in [0, 1) (got %g)", y_min);
  s->guard_y = y_min;
  return REX_OK;
}

int rex_surrogate_calibrate(rex_surrogate* s, rex_proc* exact, const double* momenta, int64_t nev,
                            const rex_params* pts, int k, double bound, double max_escape, float* tau_out,
                            double* guard_out, double* fallback_out, double* escape_out, void* stream) {
  int rc = check_handle(s);
  if (rc) return rc;
  if (!exact || !momenta || !pts || !tau_out || !guard_out) return sfail(REX_EINVAL, "null argument");
  if (nev < 1 || k < 1 || k > 4096) return sfail(REX_EINVAL, "need nev >= 1 and 1 <= k <= 4096");
  if (!(bound > 0.0) || !(max_escape >= 0.0 && max_escape < 1.0))
    return sfail(REX_EINVAL, "bound must be > 0 and max_escape in [0, 1)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t pairs = (size_t)nev * k;
  cudaError_t e = s->CP.ensure(pairs * 4);
  if (e == cudaSuccess) e = s->CE.ensure(pairs * 4);
  if (e == cudaSuccess) e = s->CR.ensure(pairs * 8);
  if (e == cudaSuccess) e = s->CW.ensure((size_t)nev * 8);
  if (e == cudaSuccess) e = s->CS1.ensure((size_t)nev * 4);
  if (e == cudaSuccess) e = s->CS2.ensure((size_t)nev * 4);
  if (e == cudaSuccess) e = s->CS3.ensure((size_t)nev * 8);
  if (e != cudaSuccess) return sfail(REX_ENOMEM, "calibration buffers: %s", cudaGetErrorString(e));
  // the network's prediction and error estimate, and the exact ratio (unit weights)
  rc = s->kernel == REX_SURROGATE_FUSED
           ? infer_fused(s, momenta, nullptr, nev, pts, k, 0.f, nullptr, s->CP.as<float>(), s->CE.as<float>(), st)
           : infer_layered(s, momenta, nullptr, nev, pts, k, 0.f, nullptr, s->CP.as<float>(), s->CE.as<float>(), st);
  if (rc) return rc;
  fill_kernel<<<(unsigned)((nev + 255) / 256), 256, 0, st>>>(s->CW.as<double>(), nev, 1.0);
  rc = rex_reweight(exact, momenta, s->CW.as<double>(), nev, pts, k, s->CR.as<double>(), stream);
  if (rc) return sfail(rc, "exact ratios: %s", rex_last_error());
  calib_stats_kernel<<<(unsigned)((nev + 255) / 256), 256, 0, st>>>(
      momenta, s->CP.as<float>(), s->CE.as<float>(), s->CR.as<double>(), nev, k, bound, s->CS1.as<float>(),
      s->CS2.as<int>(), s->CS3.as<double>());
  if ((e = cudaGetLastError()) != cudaSuccess) return scuda(e, "calibration statistics");
  std::vector<float> emax(nev);
  std::vector<int> nbad(nev);
  std::vector<double> y(nev);
  int status = 0;
  e = cudaMemcpyAsync(emax.data(), s->CS1.p, nev * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(nbad.data(), s->CS2.p, nev * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(y.data(), s->CS3.p, nev * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && s->kernel == REX_SURROGATE_FUSED)
    e = cudaMemcpyAsync(&status, s->STATUS.p, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return scuda(e, "calibration copy");
  if (status) return sfail(REX_ECUDA, "fused inference kernel: a bounded wait gave up");
  // candidate guards: off, and the y below which a given share of the events lies
  std::vector<double> ys;
  for (double v : y)
    if (v == v) ys.push_back(v);
  std::sort(ys.begin(), ys.end());
  std::vector<double> guards{0.0};
  for (double q : {0.0025, 0.005, 0.01, 0.02, 0.03, 0.05, 0.075, 0.1, 0.15, 0.2, 0.25, 0.3, 0.4, 0.5})
    if (!ys.empty()) guards.push_back(ys[(size_t)(q * (ys.size() - 1))]);
  // for each guard: keep the events inside it in order of their largest predicted
  // error, as far as the kept pairs' share above the bound stays within max_escape
  double best_fb = 2.0, best_guard = 0.0, best_esc = 0.0;
  float best_tau = -INFINITY;
  std::vector<int64_t> order;
  for (double g : guards) {
    order.clear();
    for (int64_t i = 0; i < nev; ++i)
      if (g == 0.0 || y[i] >= g) order.push_back(i);
    std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return emax[a] < emax[b]; });
    int64_t bad = 0, keep = 0, cbad = 0;
    for (size_t r = 0; r < order.size(); ++r) {
      const float t = emax[order[r]];
      if (!(t < INFINITY)) break;
      cbad += nbad[order[r]];
      // a threshold keeps every event with the same largest error: decide at the last of a tie
      if (r + 1 < order.size() && emax[order[r + 1]] == t) continue;
      if ((double)cbad > max_escape * (double)(r + 1) * k) continue;
      keep = (int64_t)r + 1;
      bad = cbad;
    }
    const double fb = 1.0 - (double)keep / (double)nev;
    if (fb < best_fb) {
      best_fb = fb;
      best_guard = g;
      best_tau = keep ? emax[order[keep - 1]] : -INFINITY;
      best_esc = keep ? (double)bad / ((double)keep * k) : 0.0;
    }
  }
  s->guard_y = best_guard;
  *tau_out = best_tau;
  *guard_out = best_guard;
  if (fallback_out) *fallback_out = best_fb;
  if (escape_out) *escape_out = best_esc;
  return REX_OK;
}

// File format (native endianness): "REXSURR1", int64 parameter count, double
// alphas0, int32 power, int32 step, then params, Adam m and v (FP32 each).
int rex_surrogate_save(rex_surrogate* s, const char* path) {
  int rc = check_handle(s);
  if (rc) return rc;
  if (!path) return sfail(REX_EINVAL, "null path");
  std::vector<float> buf(3 * (size_t)NPARAM);
  cudaError_t e = cudaMemcpy(buf.data(), s->params, NPARAM * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(buf.data() + NPARAM, s->m, NPARAM * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(buf.data() + 2 * NPARAM, s->v, NPARAM * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return scuda(e, "save: copy parameters");
  FILE* f = std::fopen(path, "wb");
  if (!f) return sfail(REX_EINVAL, "cannot open %s for writing", path);
  const int64_t n = NPARAM;
  const int32_t pw = s->apow, st = s->step;
  bool ok = std::fwrite("REXSURR1", 1, 8, f) == 8 && std::fwrite(&n, 8, 1, f) == 1 &&
            std::fwrite(&s->as0, 8, 1, f) == 1 && std::fwrite(&pw, 4, 1, f) == 1 && std::fwrite(&st, 4, 1, f) == 1 &&
            std::fwrite(buf.data(), 4, buf.size(), f) == buf.size();
  ok = (std::fclose(f) == 0) && ok;
  return ok ? REX_OK : sfail(REX_EINVAL, "short write to %s", path);
}

int rex_surrogate_load(rex_surrogate* s, const char* path) {
  int rc = check_handle(s);
  if (rc) return rc;
  if (!path) return sfail(REX_EINVAL, "null path");
  FILE* f = std::fopen(path, "rb");
  if (!f) return sfail(REX_EINVAL, "cannot open %s", path);
  char magic[8];
  int64_t n = 0;
  double as0 = 0.0;
  int32_t pw = 0, st = 0;
  std::vector<float> buf(3 * (size_t)NPARAM);
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "REXSURR1", 8) == 0 && std::fread(&n, 8, 1, f) == 1 &&
            n == NPARAM && std::fread(&as0, 8, 1, f) == 1 && std::fread(&pw, 4, 1, f) == 1 &&
            std::fread(&st, 4, 1, f) == 1 && std::fread(buf.data(), 4, buf.size(), f) == buf.size();
  std::fclose(f);
  if (!ok || !(as0 > 0.0) || pw < 0 || pw > 8 || st < 0)
    return sfail(REX_EINVAL, "%s is not a surrogate file of this network", path);
  cudaError_t e = cudaMemcpy(s->params, buf.data(), NPARAM * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->m, buf.data() + NPARAM, NPARAM * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->v, buf.data() + 2 * NPARAM, NPARAM * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = refresh_bf16(s, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return scuda(e, "load: copy parameters");
  s->as0 = as0;
  s->apow = pw;
  s->step = st;
  return REX_OK;
}

int rex_surrogate_set_kernel(rex_surrogate* s, int kind) {
  const int rc = check_handle(s);
  if (rc) return rc;
  if (kind != REX_SURROGATE_FUSED && kind != REX_SURROGATE_LAYERED) return sfail(REX_EINVAL, "unknown kernel kind");
  s->kernel = kind;
  return REX_OK;
}

int rex_surrogate_set_exact_alphas(rex_surrogate* s, double alphas0, int power) {
  const int rc = check_handle(s);
  if (rc) return rc;
  if (power < 0 || power > 8 || !(alphas0 > 0.0)) return sfail(REX_EINVAL, "need 0 <= power <= 8 and alphas0 > 0");
  s->as0 = alphas0;
  s->apow = power;
  return REX_OK;
}

void rex_surrogate_free(rex_surrogate* s) {
  if (!s) return;
  release(s);
  delete s;
}

}  // extern "C"
