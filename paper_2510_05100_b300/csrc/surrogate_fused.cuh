// Fused surrogate inference on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// One persistent CTA per SM walks tiles of 128 (event, point) pairs.  A tile
// goes through the whole network without leaving the SM:
//   x (32 BF16 features: the event's 20 momentum components in TeV from a
//   per-event table, the point's two features, zero padding) -> [tcgen05.mma, K = 32] -> +b1, GELU ->
//   [tcgen05.mma, K = 256] x 3 with +b, GELU epilogues -> output head
//   (two FP32 dot products over the 256 BF16 activations) -> pred, err, w_out.
//
// Warp roles (288 threads):
//   warps 0-7  epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its tile
//              rows) and the 128 columns of group g = w / 4; it turns the FP32
//              accumulator into BF16 activations (bias + GELU, packed FP32x2
//              arithmetic, one hardware tanh per element) written to shared
//              memory in 32-column chunks, and computes the output head;
//   warp 8     MMA issue (one lane): the layer MMAs and the weight copies.
// Overlap: the accumulator is double-buffered in TMEM (2 x 256 columns; the
// layers of a tile alternate between them), and each 32-column chunk of
// activations is handed to the MMA warp through an mbarrier as soon as it is
// written, so the MMAs of layer l+1 run while the epilogue of layer l is
// still producing its later chunks; the next tile's layer-1 MMAs overlap the
// current tile's output head.
// Weights: BF16 images of W^T cut into 8 K-chunks of 32 (16 KB each) stream
// from L2 with the bulk-copy engine through an 8-slot ring; slot c is refilled
// with the next layer's chunk c once the MMAs reading it have completed.
// Numerics equal the layer-by-layer path: BF16 operands and activations, FP32
// accumulation, bias and GELU in FP32 (same operation sequence), FP32 head and
// FP32 exp in w_out = w_in exp(pred).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "surrogate_gemm.cuh"
#include "tc05.cuh"

namespace rex {

constexpr int FM = 128;                  // pairs per tile = TMEM lanes = MMA M
constexpr int FW = 256;                  // hidden width = MMA N
constexpr int FK1 = 32;                  // padded input features
constexpr int FCH = 32;                  // K columns per weight / activation chunk
constexpr int FNCH = FW / FCH;           // 8 chunks per hidden layer
constexpr int FCHUNK = FW * FCH;         // BF16 elements of one weight chunk (16 KB)
constexpr int FEPI_WARPS = 8;                  // epilogue warps: 4 lane quarters x column groups
constexpr int FGROUPS = FEPI_WARPS / 4;          // column groups
constexpr int FGCOLS = FW / FGROUPS;             // columns per group
constexpr int FGCH = FNCH / FGROUPS;             // 32-column chunks per group
constexpr int FEPI_THREADS = 32 * FEPI_WARPS;
#ifndef REX_FUSED_FENCE
#define REX_FUSED_FENCE 1
#endif
constexpr int FFENCE = REX_FUSED_FENCE;          // activation chunks per proxy fence and hand-off
static_assert(FGCH % FFENCE == 0, "hand-off groups must tile a column group");
constexpr int FTHREADS = FEPI_THREADS + 32;
constexpr int FTMEM_COLS = 512;          // two accumulators of 256 columns

// Element (r, k) of a K-major BF16 operand with K columns: core matrices of 8
// rows x 8 elements (128 B, rows 16 B apart); the K/8 core matrices of a row
// group are contiguous (LBO = 128 B); row groups are K * 16 B apart (SBO).
__host__ __device__ constexpr int kmajor_index(int r, int k, int K) {
  return (r >> 3) * (K / 8) * 64 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}
// Element (n, k) of a weight image: chunk k / 32, a [256][32] K-major block each.
__host__ __device__ constexpr int wimage_index(int n, int k) {
  return (k / FCH) * FCHUNK + kmajor_index(n, k % FCH, FCH);
}

struct FusedArgs {
  const __nv_bfloat16* xev;    // [nev][32] event features (momenta in TeV, zeros from column 20)
  const double* w_in;          // [nev] (may be null when w_out is)
  int64_t nev;
  int k;
  const float4* ptab;          // [k]: (mt feature, alphas feature) rounded to BF16, coupling part, 0
  const __nv_bfloat16* w1;     // image of W1^T: one chunk [256][32]
  const __nv_bfloat16* w234;   // images of W2^T, W3^T, W4^T: [3][8 chunks][256][32]
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
  __nv_bfloat16 act[FM * FW];           // A operand: input features, then activations
  __nv_bfloat16 wring[FNCH][FCHUNK];    // B operand of layers 2-4, one K-chunk per slot
  __nv_bfloat16 w1[FCHUNK];             // B operand of layer 1 (resident)
  float bias[4][FW];
  float w5[FW][2];
  float red[2][FGROUPS - 1][FM][2];     // output-head partial sums of column groups 1.., by tile parity
  float b5[2];
  uint64_t w_full[FNCH], w_empty[FNCH], chunk_ready[FNCH];
  uint64_t acc_full[2], acc_empty[2];
  uint64_t x_ready, w1_full, head_ready, drain;
  uint32_t tmem_base;
  int abort;
};

// W: [K][256] row-major FP32 -> BF16 weight image of W^T
__global__ void pack_kmajor_kernel(const float* __restrict__ W, int K, __nv_bfloat16* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= FW * K) return;
  const int n = i / K, kk = i - (i / K) * K;
  dst[wimage_index(n, kk)] = __float2bfloat16(W[(int64_t)kk * FW + n]);
}

namespace fused_detail {

constexpr uint64_t kTimeoutNs = 2000000000ull;   // 2 s per wait

// Wait for the phase of `bar` with the given parity; false on timeout or when
// another warp has aborted.
__device__ __forceinline__ bool wait_bar(FusedSmem& sm, uint64_t* bar, uint32_t parity) {
  if (tc05::mbar_test(bar, parity)) return true;
  const uint64_t t0 = tc05::globaltimer_ns();
  for (;;) {
    if (tc05::mbar_test(bar, parity)) return true;
    if (*reinterpret_cast<volatile int*>(&sm.abort)) return false;
    if (tc05::globaltimer_ns() - t0 > kTimeoutNs) return false;
  }
}

__device__ __forceinline__ void arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc05::saddr(bar)) : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// gelu (tanh form) of two values, the same operation sequence as gelu_f
__device__ __forceinline__ float2 gelu2(float2 z) {
  const float2 C0 = make_float2(GELU_C0, GELU_C0), C1 = make_float2(GELU_C1, GELU_C1);
  const float2 u = __fmul2_rn(z, __ffma2_rn(__fmul2_rn(z, z), C1, C0));
  const float2 h = __fmul2_rn(z, make_float2(0.5f, 0.5f));
  return __ffma2_rn(h, make_float2(tanh_hw(u.x), tanh_hw(u.y)), h);
}

// First pair of a tile: event e0 and point j0 (one 64-bit division per tile).
struct TileOrigin {
  int64_t e0;
  uint32_t j0;
};
__device__ __forceinline__ TileOrigin tile_origin(int64_t tile, int k) {
  const int64_t p0 = tile * FM;
  const int64_t e0 = p0 / k;
  return {e0, (uint32_t)(p0 - e0 * k)};
}
// event and point of row r of a tile (32-bit arithmetic)
__device__ __forceinline__ void pair_of(const TileOrigin& o, int r, uint32_t k, int64_t& e, int& j) {
  const uint32_t n = o.j0 + (uint32_t)r;
  const uint32_t de = n / k;
  e = o.e0 + de;
  j = (int)(n - de * k);
}

// Stage the input features of one tile into act (K columns 0..31), by the
// epilogue threads: row tid % 128, features FPP (tid / 128) .. + FPP - 1, copied
// from the event's table row with the point's two features put in columns 20, 21.
__device__ __forceinline__ void stage_x(FusedSmem& sm, const FusedArgs& a, int64_t tile, int64_t npairs, int tid) {
  constexpr int FPP = FK1 * FM / FEPI_THREADS;   // features per thread (16 or 8)
  const int r = tid & (FM - 1), part = tid >> 7;
  uint4 v[FPP / 8];
#pragma unroll
  for (int u = 0; u < FPP / 8; ++u) v[u] = make_uint4(0u, 0u, 0u, 0u);
  if (tile * FM + r < npairs) {
    int64_t e;
    int j;
    pair_of(tile_origin(tile, a.k), r, (uint32_t)a.k, e, j);
    const uint4* xe = reinterpret_cast<const uint4*>(a.xev + e * FK1);
#pragma unroll
    for (int u = 0; u < FPP / 8; ++u) {
      const int q8 = part * (FPP / 8) + u;          // 8-feature group: 0, 1 momenta; 2 momenta + point; 3 zero
      if (q8 < 3) v[u] = xe[q8];
      if (q8 == 2) {
        const float4 pt = a.ptab[j];
        v[u].z = pack_bf16(pt.x, pt.y);             // features 20, 21
      }
    }
  }
#pragma unroll
  for (int u = 0; u < FPP / 8; ++u)
    *reinterpret_cast<uint4*>(&sm.act[kmajor_index(r, part * FPP + 8 * u, FW)]) = v[u];
}

}  // namespace fused_detail

__global__ void __launch_bounds__(FTHREADS, 1) fused_mlp_kernel(const __grid_constant__ FusedArgs a) {
  using namespace fused_detail;
  extern __shared__ __align__(1024) unsigned char fused_smem_raw[];
  FusedSmem& sm = *reinterpret_cast<FusedSmem*>(fused_smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t npairs = a.nev * (int64_t)a.k;
  const int64_t ntiles = (npairs + FM - 1) / FM;

  if (tid == 0) {
    for (int c = 0; c < FNCH; ++c) {
      tc05::mbar_init(&sm.w_full[c], 1);
      tc05::mbar_init(&sm.w_empty[c], 1);
      tc05::mbar_init(&sm.chunk_ready[c], 4);          // the 4 warps (lane quarters) of a column group
    }
    for (int b = 0; b < 2; ++b) {
      tc05::mbar_init(&sm.acc_full[b], 1);
      tc05::mbar_init(&sm.acc_empty[b], FEPI_WARPS);
    }
    tc05::mbar_init(&sm.x_ready, FEPI_WARPS);
    tc05::mbar_init(&sm.w1_full, 1);
    tc05::mbar_init(&sm.head_ready, 4 * (FGROUPS - 1));   // the warps of column groups 1..
    tc05::mbar_init(&sm.drain, 1);
    sm.abort = 0;
    tc05::fence_mbar_init();
  }
  if (warp == 0) {
    tc05::tmem_alloc(&sm.tmem_base, FTMEM_COLS);
    tc05::tmem_relinquish();
  }
  for (int i = tid; i < 4 * FW; i += FTHREADS) sm.bias[i / FW][i % FW] = a.bias[i / FW][i % FW];
  for (int i = tid; i < FW * 2; i += FTHREADS) (&sm.w5[0][0])[i] = a.w5[i];
  if (tid < 2) sm.b5[tid] = a.b5[tid];
  tc05::fence_before_sync();
  __syncthreads();
  tc05::fence_after_sync();
  const uint32_t tmem = sm.tmem_base;

  if (warp == FEPI_WARPS) {
    // ============================ MMA warp ============================
    if (lane == 0) {
      constexpr uint32_t IDESC = tc05::idesc_bf16_f32(FM, FW);
      constexpr uint64_t DACT = tc05::smem_desc_bits(128, (FW / 8) * 128);   // act: 256 columns
      constexpr uint64_t DCH = tc05::smem_desc_bits(128, (FCH / 8) * 128);   // weight chunk: 32 columns
      // per-slot phase parities and in-flight copies, one bit per slot
      uint32_t ph_wfull = 0, ph_wempty = 0, ph_ready = 0, pending = 0;
      uint32_t ph_empty[2] = {0, 0}, ph_x = 0;
      auto load_chunk = [&](int c, const __nv_bfloat16* src) {
        tc05::mbar_expect_tx(&sm.w_full[c], FCHUNK * 2);
        tc05::bulk_g2s(sm.wring[c], src, FCHUNK * 2, &sm.w_full[c]);
        pending |= 1u << c;
      };
      tc05::mbar_expect_tx(&sm.w1_full, FCHUNK * 2);
      tc05::bulk_g2s(sm.w1, a.w1, FCHUNK * 2, &sm.w1_full);
      for (int c = 0; c < FNCH; ++c) load_chunk(c, a.w234 + (size_t)c * FCHUNK);
      bool ok = wait_bar(sm, &sm.w1_full, 0);
      for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
        // layer 1 -> accumulator 0
        ok = wait_bar(sm, &sm.acc_empty[0], ph_empty[0]) && wait_bar(sm, &sm.x_ready, ph_x);
        if (!ok) break;
        ph_empty[0] ^= 1;
        ph_x ^= 1;
        tc05::fence_after_sync();
        for (int s = 0; s < FK1 / 16; ++s)
          tc05::mma_bf16(tmem, tc05::smem_desc(sm.act + 128 * s, DACT), tc05::smem_desc(sm.w1 + 128 * s, DCH),
                         IDESC, s > 0);
        tc05::mma_commit(&sm.acc_full[0]);
        // layers 2-4 -> accumulators 1, 0, 1
        for (int l = 1; ok && l < 4; ++l) {
          const int b = l & 1;
          const uint32_t dst = tmem + (uint32_t)(b * FW);
          if (!(ok = wait_bar(sm, &sm.acc_empty[b], ph_empty[b]))) break;
          ph_empty[b] ^= 1;
          bool first = true;
          for (int i = 0; i < FNCH; ++i) {
            const int c = (i % FGROUPS) * FGCH + i / FGROUPS;   // the column groups advance together
            if (!(ok = wait_bar(sm, &sm.chunk_ready[c], (ph_ready >> c) & 1u) &&
                       wait_bar(sm, &sm.w_full[c], (ph_wfull >> c) & 1u)))
              break;
            ph_ready ^= 1u << c;
            ph_wfull ^= 1u << c;
            pending &= ~(1u << c);
            tc05::fence_after_sync();
#pragma unroll
            for (int j = 0; j < FCH / 16; ++j) {
              tc05::mma_bf16(dst, tc05::smem_desc(sm.act + 128 * (2 * c + j), DACT),
                             tc05::smem_desc(sm.wring[c] + 128 * j, DCH), IDESC, first ? 0u : 1u);
              first = false;
            }
            tc05::mma_commit(&sm.w_empty[c]);
          }
          if (!ok) break;
          tc05::mma_commit(&sm.acc_full[b]);
          // refill the ring with the next layer's chunks as this layer's MMAs release them
          if (l < 3 || tile + gridDim.x < ntiles) {
            const __nv_bfloat16* src = a.w234 + (size_t)(l < 3 ? l : 0) * FNCH * FCHUNK;
            for (int c = 0; ok && c < FNCH; ++c) {
              if (!(ok = wait_bar(sm, &sm.w_empty[c], (ph_wempty >> c) & 1u))) break;
              ph_wempty ^= 1u << c;
              load_chunk(c, src + (size_t)c * FCHUNK);
            }
          }
        }
      }
      if (!ok) sm.abort = 1;
      // drain: every MMA issued by this thread, and every weight copy in flight
      tc05::mma_commit(&sm.drain);
      if (!tc05::mbar_wait(&sm.drain, 0, kTimeoutNs)) sm.abort = 1;
      for (int c = 0; c < FNCH; ++c)
        if (((pending >> c) & 1u) && !tc05::mbar_wait(&sm.w_full[c], (ph_wfull >> c) & 1u, kTimeoutNs)) sm.abort = 1;
    }
    __syncwarp();
  } else {
    // ========================== epilogue warps ==========================
    const int q = warp & 3, g = warp >> 2;
    const int row = q * 32 + lane;   // tile row = TMEM lane
    const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
    uint32_t ph_full[2] = {0, 0}, ph_head = 0;
    bool ok = true;
    // both accumulators start empty
    if (lane == 0) {
      arrive(&sm.acc_empty[0]);
      arrive(&sm.acc_empty[1]);
    }
    if (blockIdx.x < ntiles) {
      stage_x(sm, a, blockIdx.x, npairs, tid);
      tc05::fence_proxy_async();
      __syncwarp();
      if (lane == 0) arrive(&sm.x_ready);
    }
    int parity = 0;
    for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, parity ^= 1) {
      for (int l = 0; l < 4; ++l) {
        const int b = l & 1;
        if (!(ok = wait_bar(sm, &sm.acc_full[b], ph_full[b]))) break;
        ph_full[b] ^= 1;
        tc05::fence_after_sync();
        const uint32_t tacc = trow + (uint32_t)(b * FW);
        if (l < 3) {
          // z = acc + b, a = gelu(z) -> BF16 activation chunks for the next layer;
          // the TMEM load of chunk cc + 1 runs while chunk cc is computed
          // the TMEM load of chunk cc + 1 runs while chunk cc is computed
          uint32_t ra[32], rb[32];
          tc05::tmem_ld32_async(tacc + (uint32_t)(g * FGCOLS), ra);
#pragma unroll
          for (int cc = 0; cc < FGCH; ++cc) {
            uint32_t(&cur)[32] = (cc & 1) ? rb : ra;
            uint32_t(&nxt)[32] = (cc & 1) ? ra : rb;
            tc05::tmem_wait_ld(cur);
            if (cc + 1 < FGCH) tc05::tmem_ld32_async(tacc + (uint32_t)(g * FGCOLS + (cc + 1) * FCH), nxt);
            const int c = g * FGCH + cc, c0 = c * FCH;
            const float2* bb = reinterpret_cast<const float2*>(&sm.bias[l][c0]);
            uint32_t pk[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const float2 y = gelu2(__fadd2_rn(make_float2(__uint_as_float(cur[2 * i]), __uint_as_float(cur[2 * i + 1])), bb[i]));
              pk[i] = pack_bf16(y.x, y.y);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
              *reinterpret_cast<uint4*>(&sm.act[kmajor_index(row, c0 + 8 * j, FW)]) =
                  make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
            // hand the chunks to the MMA warp FFENCE at a time (one proxy fence each)
            if ((cc + 1) % FFENCE == 0) {
              tc05::fence_proxy_async();
              __syncwarp();
              if (lane == 0)
                for (int u = 0; u < FFENCE; ++u) arrive(&sm.chunk_ready[c - u]);
            }
          }
          tc05::fence_before_sync();
          __syncwarp();
          if (lane == 0) arrive(&sm.acc_empty[b]);
        } else {
          // layer 4 has finished reading act: stage the next tile's features first,
          // so that its layer-1 MMAs run during this output head
          const int64_t next = tile + gridDim.x;
          if (next < ntiles) {
            stage_x(sm, a, next, npairs, tid);
            tc05::fence_proxy_async();
            __syncwarp();
            if (lane == 0) arrive(&sm.x_ready);
          }
          float2 ye = make_float2(0.f, 0.f);   // (y, e) partial sums over this warp's columns
          const float2* w5 = reinterpret_cast<const float2*>(&sm.w5[0][0]);
          uint32_t ra[32], rb[32];
          tc05::tmem_ld32_async(tacc + (uint32_t)(g * FGCOLS), ra);
#pragma unroll
          for (int cc = 0; cc < FGCH; ++cc) {
            uint32_t(&cur)[32] = (cc & 1) ? rb : ra;
            uint32_t(&nxt)[32] = (cc & 1) ? ra : rb;
            tc05::tmem_wait_ld(cur);
            if (cc + 1 < FGCH) tc05::tmem_ld32_async(tacc + (uint32_t)(g * FGCOLS + (cc + 1) * FCH), nxt);
            const int c0 = g * FGCOLS + cc * FCH;
            const float2* bb = reinterpret_cast<const float2*>(&sm.bias[3][c0]);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const float2 y = gelu2(__fadd2_rn(make_float2(__uint_as_float(cur[2 * i]), __uint_as_float(cur[2 * i + 1])), bb[i]));
              const float a0 = __bfloat162float(__float2bfloat16(y.x));
              const float a1 = __bfloat162float(__float2bfloat16(y.y));
              ye = __ffma2_rn(make_float2(a0, a0), w5[c0 + 2 * i], ye);
              ye = __ffma2_rn(make_float2(a1, a1), w5[c0 + 2 * i + 1], ye);
            }
          }
          tc05::fence_before_sync();
          __syncwarp();
          if (lane == 0) arrive(&sm.acc_empty[b]);
          if (g > 0) {
            sm.red[parity][g - 1][row][0] = ye.x;
            sm.red[parity][g - 1][row][1] = ye.y;
            __syncwarp();
            if (lane == 0) arrive(&sm.head_ready);
          } else {
            if (!(ok = wait_bar(sm, &sm.head_ready, ph_head))) break;
            ph_head ^= 1;
            const int64_t p = tile * FM + row;
            if (p < npairs) {
              int64_t e;
              int j;
              pair_of(tile_origin(tile, a.k), row, (uint32_t)a.k, e, j);
              float y = ye.x, er = ye.y;
#pragma unroll
              for (int h = 0; h < FGROUPS - 1; ++h) {
                y += sm.red[parity][h][row][0];
                er += sm.red[parity][h][row][1];
              }
              y += sm.b5[0] + a.ptab[j].z;
              er += sm.b5[1];
              if (a.pred) a.pred[p] = y;
              if (a.err) a.err[p] = er;
              if (a.w_out) a.w_out[p] = a.w_in[e] * (double)expf(y);
              if (a.flag && !(er <= a.tau)) a.flag[e] = 1;   // NaN errors fall back too
            }
          }
        }
      }
    }
    if (!ok) sm.abort = 1;
  }

  // ---- release TMEM once no MMA, copy or TMEM load of this CTA is in flight ----
  tc05::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc05::fence_after_sync();
    tc05::tmem_dealloc(tmem, FTMEM_COLS);
  }
  if (tid == 0 && sm.abort) atomicExch(a.status, 1);
}

}  // namespace rex
