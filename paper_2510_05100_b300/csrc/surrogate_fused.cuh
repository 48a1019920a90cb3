// Fused surrogate inference on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// One persistent CTA per SM walks tiles of 128 (event, point) pairs.  A tile
// goes through the whole network without leaving the SM:
//   x (32 BF16 features: 20 momentum components in TeV, the point's two
//   features, zero padding) -> [tcgen05.mma, K = 32] -> +b1, GELU ->
//   [tcgen05.mma, K = 256] x 3 with +b, GELU epilogues -> output head
//   (two FP32 dot products over the 256 BF16 activations) -> pred, err, w_out.
// The accumulator (128 x 256 FP32) lives in tensor memory (256 columns); the
// activations (128 x 256 BF16) stay in shared memory between layers; the
// weights (BF16 images of W^T in the MMA's K-major core-matrix layout,
// prepared by pack_kmajor_kernel) are streamed from L2 into a 128 KB buffer
// with the bulk-copy engine, the next layer's load overlapping the current
// epilogue.  Numerics match the layer-by-layer path: BF16 operands and
// activations, FP32 accumulation, bias and GELU in FP32, FP32 head.
//
// Thread roles: 8 warps; warp w reads TMEM lanes 32 (w % 4) .. + 31 (its tile
// rows) and columns [128 (w / 4), + 128); thread 0 issues the MMAs and copies.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "surrogate_gemm.cuh"
#include "tc05.cuh"

namespace rex {

constexpr int FM = 128;          // pairs per tile = TMEM lanes = MMA M
constexpr int FW = 256;          // hidden width = MMA N = TMEM columns
constexpr int FK1 = 32;          // padded input features
constexpr int FTHREADS = 256;

// Element (r, k) of a K-major BF16 operand image with K columns: core matrices
// of 8 rows x 8 elements (128 B, rows 16 B apart); the K/8 core matrices of a
// row group are contiguous (LBO = 128 B); row groups are K * 16 B apart (SBO).
__host__ __device__ constexpr int kmajor_index(int r, int k, int K) {
  return (r >> 3) * (K / 8) * 64 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

struct FusedArgs {
  const double* mom;           // [nev][20] FP64
  const double* w_in;          // [nev] (may be null when w_out is)
  int64_t nev;
  int k;
  const float4* ptab;          // [k]: (mt feature, alphas feature) rounded to BF16, coupling part, 0
  const __nv_bfloat16* w1;     // image of W1^T: [256][32]
  const __nv_bfloat16* w234;   // images of W2^T, W3^T, W4^T: [3][256][256]
  const float* bias[4];        // b1..b4 [256] each
  const float* w5;             // [256][2]
  const float* b5;             // [2]
  float tau;
  float* pred;                 // [nev][k] or null
  float* err;                  // [nev][k] or null
  double* w_out;               // [nev][k] or null
  int* flag;                   // [nev] or null: set to 1 where some err > tau (or NaN)
  int* status;                 // set to 1 if a bounded wait gave up
};

struct FusedSmem {
  __nv_bfloat16 act[FM * FW];   // A operand: input features, then activations
  __nv_bfloat16 w[FW * FW];     // B operand of layers 2-4
  __nv_bfloat16 w1[FW * FK1];   // B operand of layer 1 (resident)
  float bias[4][FW];
  float w5[FW][2];
  float red[FM][2];
  uint64_t bar_w, bar_mma;
  uint32_t tmem_base;
  int abort;
};

__global__ void pack_kmajor_kernel(const float* __restrict__ W, int K, __nv_bfloat16* __restrict__ dst) {
  // W: [K][256] row-major FP32 -> BF16 image of W^T ([256 rows n][K columns k])
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= FW * K) return;
  const int n = i / K, kk = i - (i / K) * K;
  dst[kmajor_index(n, kk, K)] = __float2bfloat16(W[(int64_t)kk * FW + n]);
}

namespace fused_detail {

constexpr uint64_t kTimeoutNs = 2000000000ull;   // 2 s per wait

// wait for an MMA group; gives up early when another thread has aborted
__device__ __forceinline__ bool wait_mma(FusedSmem& sm, uint32_t parity) {
  if (tc05::mbar_test(&sm.bar_mma, parity)) return true;
  const uint64_t t0 = tc05::globaltimer_ns();
  for (;;) {
    if (tc05::mbar_test(&sm.bar_mma, parity)) return true;
    if (*reinterpret_cast<volatile int*>(&sm.abort)) return false;
    if (tc05::globaltimer_ns() - t0 > kTimeoutNs) return false;
  }
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

}  // namespace fused_detail

__global__ void __launch_bounds__(FTHREADS, 1) fused_mlp_kernel(const __grid_constant__ FusedArgs a) {
  using namespace fused_detail;
  extern __shared__ __align__(1024) unsigned char fused_smem_raw[];
  FusedSmem& sm = *reinterpret_cast<FusedSmem*>(fused_smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = warp & 3, hcol = warp >> 2;
  const int row = q * 32 + lane;   // tile row of this thread in the epilogues
  constexpr uint32_t IDESC = tc05::idesc_bf16_f32(FM, FW);
  constexpr uint64_t D256 = tc05::smem_desc_bits(128, (FW / 8) * 128);
  constexpr uint64_t D32 = tc05::smem_desc_bits(128, (FK1 / 8) * 128);
  const int64_t npairs = a.nev * (int64_t)a.k;
  const int64_t ntiles = (npairs + FM - 1) / FM;

  if (tid == 0) {
    tc05::mbar_init(&sm.bar_w, 1);
    tc05::mbar_init(&sm.bar_mma, 1);
    sm.abort = 0;
    tc05::fence_mbar_init();
  }
  if (warp == 0) {
    tc05::tmem_alloc(&sm.tmem_base, FW);
    tc05::tmem_relinquish();
  }
  for (int i = tid; i < 4 * FW; i += FTHREADS) sm.bias[i / FW][i % FW] = a.bias[i / FW][i % FW];
  for (int i = tid; i < FW * 2; i += FTHREADS) (&sm.w5[0][0])[i] = a.w5[i];
  tc05::fence_before_sync();
  __syncthreads();
  tc05::fence_after_sync();
  const uint32_t tmem = sm.tmem_base;
  const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);

  uint32_t ph_w = 0, ph_mma = 0;   // parities of the next phase to complete
  bool w_pending = false;          // thread 0: a weight copy is in flight
  bool mma_pending = false;        // thread 0: an MMA group was committed and not yet waited for

  // thread 0: start the copy of a weight image into sm.w (or sm.w1)
  auto load_w = [&](void* dst, const void* src, uint32_t bytes) {
    tc05::mbar_expect_tx(&sm.bar_w, bytes);
    tc05::bulk_g2s(dst, src, bytes, &sm.bar_w);
    w_pending = true;
  };
  auto wait_w = [&]() -> bool {
    const bool ok = tc05::mbar_wait(&sm.bar_w, ph_w, kTimeoutNs);
    if (ok) {
      ph_w ^= 1;
      w_pending = false;
    }
    return ok;
  };
  // thread 0: one layer's MMAs (K = 16 per instruction) and their commit
  auto issue_layer = [&](const __nv_bfloat16* B, uint64_t bdesc_bits, int ksteps) {
    tc05::fence_after_sync();
#pragma unroll 1
    for (int s = 0; s < ksteps; ++s)
      tc05::mma_bf16(tmem, tc05::smem_desc(sm.act + 128 * s, D256), tc05::smem_desc(B + 128 * s, bdesc_bits), IDESC,
                     s > 0);
    tc05::mma_commit(&sm.bar_mma);
    mma_pending = true;
  };

  if (tid == 0) {
    load_w(sm.w1, a.w1, FW * FK1 * 2);
    if (!wait_w()) sm.abort = 1;
  }
  __syncthreads();

  for (int64_t tile = blockIdx.x; tile < ntiles && !sm.abort; tile += gridDim.x) {
    const int64_t p0 = tile * FM;
    // ---- stage the tile's input features (16 per thread) --------------------------
    {
      const int r = tid & (FM - 1), hx = tid >> 7;
      const int64_t p = p0 + r;
      float f[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) f[c] = 0.f;
      if (p < npairs) {
        const int64_t e = p / a.k;
        const int j = (int)(p - e * a.k);
        const double* m = a.mom + e * 20;
        if (hx == 0) {
#pragma unroll
          for (int c = 0; c < 16; ++c) f[c] = (float)(m[c] * 1.0e-3);
        } else {
#pragma unroll
          for (int c = 0; c < 4; ++c) f[c] = (float)(m[16 + c] * 1.0e-3);
          const float4 pt = a.ptab[j];
          f[4] = pt.x;
          f[5] = pt.y;
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint4 v = make_uint4(pack_bf16(f[8 * h], f[8 * h + 1]), pack_bf16(f[8 * h + 2], f[8 * h + 3]),
                             pack_bf16(f[8 * h + 4], f[8 * h + 5]), pack_bf16(f[8 * h + 6], f[8 * h + 7]));
        *reinterpret_cast<uint4*>(&sm.act[kmajor_index(r, hx * 16 + 8 * h, FW)]) = v;
      }
    }
    tc05::fence_proxy_async();
    tc05::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      issue_layer(sm.w1, D32, FK1 / 16);                 // layer 1
      load_w(sm.w, a.w234, FW * FW * 2);                 // W2 (the buffer is free)
    }

    // ---- layers: epilogue of layer l + 1 then the MMAs of layer l + 2 -------------
#pragma unroll 1
    for (int l = 0; l < 4; ++l) {
      // every thread waits for the layer's MMAs; the block leaves together on failure
      const bool ok = wait_mma(sm, ph_mma);
      if (__syncthreads_or(!ok)) {
        if (tid == 0) sm.abort = 1;
        break;
      }
      ph_mma ^= 1;
      mma_pending = false;
      tc05::fence_after_sync();
      // the MMAs of layer l + 1 have finished reading sm.w: start the next image
      if (tid == 0 && l >= 1 && l <= 2) load_w(sm.w, a.w234 + (size_t)l * FW * FW, FW * FW * 2);
      if (l < 3) {
        // z = acc + b, a = gelu(z) -> BF16 activations for the next layer
#pragma unroll 1
        for (int cc = 0; cc < 4; ++cc) {
          const int c0 = hcol * 128 + cc * 32;
          float v[32];
          tc05::tmem_ld32(trow + (uint32_t)c0, v);
          uint32_t pk[16];
#pragma unroll
          for (int i = 0; i < 32; i += 2)
            pk[i / 2] = pack_bf16(gelu_f(v[i] + sm.bias[l][c0 + i]), gelu_f(v[i + 1] + sm.bias[l][c0 + i + 1]));
#pragma unroll
          for (int j = 0; j < 4; ++j)
            *reinterpret_cast<uint4*>(&sm.act[kmajor_index(row, c0 + 8 * j, FW)]) =
                make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
        }
        tc05::fence_proxy_async();
        tc05::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
          if (!wait_w())
            sm.abort = 1;   // the others see it in wait_mma and leave at the vote
          else
            issue_layer(sm.w, D256, FW / 16);
        }
      } else {
        // output head on the BF16 activations of layer 4
        float y = 0.f, er = 0.f;
#pragma unroll 1
        for (int cc = 0; cc < 4; ++cc) {
          const int c0 = hcol * 128 + cc * 32;
          float v[32];
          tc05::tmem_ld32(trow + (uint32_t)c0, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const float act = __bfloat162float(__float2bfloat16(gelu_f(v[i] + sm.bias[3][c0 + i])));
            y = fmaf(act, sm.w5[c0 + i][0], y);
            er = fmaf(act, sm.w5[c0 + i][1], er);
          }
        }
        if (hcol == 1) {
          sm.red[row][0] = y;
          sm.red[row][1] = er;
        }
        tc05::fence_before_sync();
        __syncthreads();
        if (hcol == 0) {
          const int64_t p = p0 + row;
          if (p < npairs) {
            const int64_t e = p / a.k;
            const int j = (int)(p - e * a.k);
            y += sm.red[row][0] + a.b5[0] + a.ptab[j].z;
            er += sm.red[row][1] + a.b5[1];
            if (a.pred) a.pred[p] = y;
            if (a.err) a.err[p] = er;
            if (a.w_out) a.w_out[p] = a.w_in[e] * exp((double)y);
            if (a.flag && !(er <= a.tau)) a.flag[e] = 1;   // NaN errors fall back too
          }
        }
        __syncthreads();
      }
    }
  }

  // ---- drain: no copy or MMA may still be writing when TMEM is released ---------
  if (tid == 0) {
    if (w_pending && !tc05::mbar_wait(&sm.bar_w, ph_w, kTimeoutNs)) sm.abort = 1;
    if (mma_pending && !tc05::mbar_wait(&sm.bar_mma, ph_mma, kTimeoutNs)) sm.abort = 1;
  }
  tc05::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc05::fence_after_sync();
    tc05::tmem_dealloc(tmem, FW);
  }
  if (tid == 0 && sm.abort) atomicExch(a.status, 1);
}

}  // namespace rex
