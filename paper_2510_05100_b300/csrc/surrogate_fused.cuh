// Fused surrogate inference on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// One persistent CTA per SM takes tiles of 128 (event, point) pairs two at a
// time (tile slots 0 and 1).  A tile goes through the whole network without
// leaving the SM:
//   x (32 BF16 features: the event's 20 momentum components in TeV from a
//   per-event table, the point's two features, zero padding) -> [tcgen05.mma, K = 32] -> GELU ->
//   [tcgen05.mma, K = 256] x 3 with GELU epilogues -> output head
//   (two FP32 dot products over the 256 BF16 activations) -> pred, err, w_out.
//
// Warp roles (576 threads):
//   warps 0-15 epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its tile
//              rows) and the 64 columns of group g = w / 4; it turns the FP32
//              accumulator into BF16 activations (GELU in packed FP32x2
//              arithmetic, one hardware tanh per element) written to shared
//              memory in 32-column chunks, and computes the output head;
//   warp 16    MMA issue (one lane);
//   warp 17    weight producer (the copy for ring slot r issued by lane r).
// Ping-pong: each tile slot has its own accumulator (TMEM columns 256 s ..
// 256 s + 255) and its own activation buffer, and the MMAs alternate between
// the slots layer by layer, slot 1 two layers behind slot 0 (step k: slot 0
// layer k % 4, then slot 1 layer (k - 2) % 4), so the epilogue of one slot's
// layer runs while the tensor cores work on the other slot, and the short
// layer-1 MMAs of the two slots are never adjacent.  A slot's epilogue hands a
// whole layer to the MMA warp with one mbarrier (activations in shared memory,
// accumulator read, next bias stored).
// Bias: right after reading a chunk of its accumulator, the epilogue writes the
// bias of the layer that accumulates there next into the same TMEM columns, so
// every MMA of a layer accumulates onto its bias and the epilogue adds nothing.
// Weights: BF16 images of W^T cut into 8 K-chunks of 32 (16 KB each) stream
// from L2 through a ring of FNSLOT slots, in the order the MMAs read them (each
// chunk once per tile); the producer warp refills a slot as soon as the MMAs
// reading it have completed, the copy issued by the slot's own lane (bulk copies
// issued by one thread complete one after another, copies of different threads
// overlap) while the warp stays converged (lanes spinning on different barriers
// in one warp delayed the refills).  W1 stays resident.  The images of W2, W3, W4 and the head weights are scaled by
// 1/2 (exact in BF16 and FP32) and the epilogues produce 2 gelu(z) = z (1 + tanh
// u), which saves the multiplication by 1/2: the products entering every
// accumulation are the same as with unscaled weights and gelu(z).
// Numerics: BF16 operands and activations, FP32 accumulation starting from the
// FP32 bias, GELU in FP32 (tanh form, hardware tanh), FP32 head and FP32 exp in
// w_out = w_in exp(pred).
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
constexpr int FEPI_WARPS = 16;                 // epilogue warps: 4 lane quarters x column groups
constexpr int FGROUPS = FEPI_WARPS / 4;          // column groups
constexpr int FGCOLS = FW / FGROUPS;             // columns per group
constexpr int FGCH = FNCH / FGROUPS;             // 32-column chunks per group
constexpr int FEPI_THREADS = 32 * FEPI_WARPS;
constexpr int FMMA_WARP = FEPI_WARPS;            // issues the MMAs
constexpr int FPROD_WARP = FEPI_WARPS + 1;       // issues the weight copies
constexpr int FTHREADS = FEPI_THREADS + 64;
constexpr int FTMEM_COLS = 512;          // two accumulators (tile slots) of 256 columns
constexpr int FNSLOT = 4;                // weight ring slots

constexpr float FWSCALE = 0.5f;          // scale of the W2..W4 images and of the head weights

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
  const __nv_bfloat16* w234;   // images of W2^T, W3^T, W4^T scaled by FWSCALE: [3][8 chunks][256][32]
  const float* bias[4];        // b1..b4 [256] each
  const float* w5;             // [256][2] (unscaled)
  const float* b5;             // [2]
  float tau;
  float* pred;                 // [nev][k] or null
  float* err;                  // [nev][k] or null
  double* w_out;               // [nev][k] or null
  int* flag;                   // [nev] or null: set to 1 where some err > tau (or NaN)
  int* status;                 // set to 1 if a bounded wait gave up
};

struct FusedSmem {
  __nv_bfloat16 act[2][FM * FW];        // per tile slot, A operand: input features, then activations
  __nv_bfloat16 wring[FNSLOT][FCHUNK];  // B operand of layers 2-4, one K-chunk per slot
  __nv_bfloat16 w1[FCHUNK];             // B operand of layer 1 (resident)
  float bias[4][FW];
  float w5[FW][2];                      // head weights times FWSCALE
  float red[2][FGROUPS - 1][FM][2];     // output-head partial sums of column groups 1.., by tile slot
  float b5[2];
  uint64_t w_full[FNSLOT], w_empty[FNSLOT];
  uint64_t acc_full[2], acc_ready[2];   // per tile slot: accumulated / read and holding the next bias
  uint64_t x_ready[2], head_ready[2];
  uint64_t w1_full, drain;
  uint32_t tmem_base;
  int abort;
};

// W: [K][256] row-major FP32 -> BF16 weight image of (scale W)^T; scale is a
// power of two, so the image is scale times the image of W.
__global__ void pack_kmajor_kernel(const float* __restrict__ W, int K, float scale, __nv_bfloat16* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= FW * K) return;
  const int n = i / K, kk = i - (i / K) * K;
  dst[wimage_index(n, kk)] = __float2bfloat16(scale * W[(int64_t)kk * FW + n]);
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

// 2 gelu(z) (tanh form) of two values: z (1 + tanh u), u = z (C0 + C1 z^2).
// With h = z / 2, fma(z, t, z) = 2 fma(h, t, h) exactly, the sequence of gelu_f.
__device__ __forceinline__ float2 gelu2_twice(float2 z) {
  const float2 C0 = make_float2(GELU_C0, GELU_C0), C1 = make_float2(GELU_C1, GELU_C1);
  const float2 u = __fmul2_rn(z, __ffma2_rn(__fmul2_rn(z, z), C1, C0));
  return __ffma2_rn(z, make_float2(tanh_hw(u.x), tanh_hw(u.y)), z);
}

// Write the 32 bias values b[c0 .. c0 + 31] into every lane of the warp's TMEM
// columns taddr .. taddr + 31 (asynchronous; tmem_wait_st completes it).
__device__ __forceinline__ void store_bias(uint32_t taddr, const float* b) {
  uint32_t v[32];
  const uint4* src = reinterpret_cast<const uint4*>(b);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const uint4 q = src[i];
    v[4 * i] = q.x;
    v[4 * i + 1] = q.y;
    v[4 * i + 2] = q.z;
    v[4 * i + 3] = q.w;
  }
  tc05::tmem_st32(taddr, v);
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

// Input features of one tile, by the epilogue threads: row tid % 128, features
// 8 (tid / 128) .. + 7 (one 16-byte group), from the event's table row with the
// point's two features put in columns 20, 21.  load_x issues the global loads
// (zeros past the last pair); store_x writes the group into K columns 0..31 of a
// tile slot's activation buffer once the slot's previous layer 4 has completed.
static_assert(FK1 * FM == 8 * FEPI_THREADS, "one 8-feature group per epilogue thread");
__device__ __forceinline__ uint4 load_x(const FusedArgs& a, int64_t tile, int64_t npairs, int tid) {
  const int r = tid & (FM - 1), q8 = tid >> 7;    // 8-feature group: 0, 1 momenta; 2 momenta + point; 3 zero
  uint4 v = make_uint4(0u, 0u, 0u, 0u);
  if (q8 < 3 && tile * FM + r < npairs) {
    int64_t e;
    int j;
    pair_of(tile_origin(tile, a.k), r, (uint32_t)a.k, e, j);
    v = reinterpret_cast<const uint4*>(a.xev + e * FK1)[q8];
    if (q8 == 2) {
      const float4 pt = a.ptab[j];
      v.z = pack_bf16(pt.x, pt.y);                 // features 20, 21
    }
  }
  return v;
}
__device__ __forceinline__ void store_x(__nv_bfloat16* act, uint4 v, int tid) {
  *reinterpret_cast<uint4*>(&act[kmajor_index(tid & (FM - 1), 8 * (tid >> 7), FW)]) = v;
}

// MMA order of the chunks of a layer: the column groups advance together.
__device__ __forceinline__ int chunk_at(int i) { return (i % FGROUPS) * FGCH + i / FGROUPS; }
// Schedule: step k runs one layer of each tile slot, slot 0 first; slot s runs
// layer (k - FLAG s) % 4 of its tile (k - FLAG s) / 4, so slot 1 trails slot 0 by
// FLAG layers and a slot's short layer 1 is never next to the other slot's (an
// epilogue always overlaps a K = 256 layer of the other slot, but one per tile).
constexpr int FLAG = 2;
__device__ __forceinline__ bool step_work(int64_t k, int s, int64_t per_slot, int& layer, int64_t& t) {
  const int64_t kk = k - FLAG * s;
  if (kk < 0 || kk >= 4 * per_slot) return false;
  layer = (int)(kk & 3);
  t = kk >> 2;
  return true;
}

}  // namespace fused_detail

__global__ void __launch_bounds__(FTHREADS, 1) fused_mlp_kernel(const __grid_constant__ FusedArgs a) {
  using namespace fused_detail;
  extern __shared__ __align__(1024) unsigned char fused_smem_raw[];
  FusedSmem& sm = *reinterpret_cast<FusedSmem*>(fused_smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t npairs = a.nev * (int64_t)a.k;
  const int64_t ntiles = (npairs + FM - 1) / FM;
  // this CTA's tiles blockIdx.x + u gridDim.x, u < nmine; tile slot s takes u = 2 t + s
  // for t < per_slot (past nmine a phantom tile: zero inputs, no outputs)
  const int64_t nmine = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t per_slot = (nmine + 1) / 2;
  const int64_t nsteps = per_slot > 0 ? 4 * per_slot + FLAG : 0;
  auto tile_of = [&](int64_t t, int s) { return (int64_t)blockIdx.x + (2 * t + s) * (int64_t)gridDim.x; };

  if (tid == 0) {
    for (int r = 0; r < FNSLOT; ++r) {
      tc05::mbar_init(&sm.w_full[r], 1);
      tc05::mbar_init(&sm.w_empty[r], 1);
    }
    for (int s = 0; s < 2; ++s) {
      tc05::mbar_init(&sm.acc_full[s], 1);
      tc05::mbar_init(&sm.acc_ready[s], FEPI_WARPS);
      tc05::mbar_init(&sm.x_ready[s], FEPI_WARPS);
      tc05::mbar_init(&sm.head_ready[s], 4 * (FGROUPS - 1));   // the warps of column groups 1..
    }
    tc05::mbar_init(&sm.w1_full, 1);
    tc05::mbar_init(&sm.drain, 1);
    sm.abort = 0;
    tc05::fence_mbar_init();
  }
  if (warp == 0) {
    tc05::tmem_alloc(&sm.tmem_base, FTMEM_COLS);
    tc05::tmem_relinquish();
  }
  for (int i = tid; i < 4 * FW; i += FTHREADS) sm.bias[i / FW][i % FW] = a.bias[i / FW][i % FW];
  for (int i = tid; i < FW * 2; i += FTHREADS) (&sm.w5[0][0])[i] = FWSCALE * a.w5[i];
  if (tid < 2) sm.b5[tid] = a.b5[tid];
  tc05::fence_before_sync();
  __syncthreads();
  tc05::fence_after_sync();
  const uint32_t tmem = sm.tmem_base;

  if (warp == FPROD_WARP) {
    // ========================= weight producer =========================
    // The warp walks the ring uses in the MMAs' order (per step and slot with a
    // layer >= 2, its 8 chunks); use f goes to ring slot r = f % FNSLOT and its copy
    // is issued by lane r (bulk copies issued by one thread complete one after
    // another, copies of different threads overlap), after the whole warp has seen
    // the slot's previous chunk read by its MMAs.
    {
      bool ok = true;
      uint32_t f = 0;
      if (lane == 0) {
        tc05::mbar_expect_tx(&sm.w1_full, FCHUNK * 2);
        tc05::bulk_g2s(sm.w1, a.w1, FCHUNK * 2, &sm.w1_full);
      }
      for (int64_t k = 0; ok && k < nsteps; ++k)
        for (int ts = 0; ok && ts < 2; ++ts) {
          int l;
          int64_t t;
          if (!step_work(k, ts, per_slot, l, t) || l == 0) continue;
          for (int i = 0; i < FNCH; ++i, ++f) {
            const uint32_t r = f % FNSLOT, use = f / FNSLOT;
            if (use > 0 && !(ok = wait_bar(sm, &sm.w_empty[r], (use - 1) & 1u))) break;
            if (lane == (int)r) {
              tc05::mbar_expect_tx(&sm.w_full[r], FCHUNK * 2);
              tc05::bulk_g2s(sm.wring[r], a.w234 + ((size_t)(l - 1) * FNCH + chunk_at(i)) * FCHUNK, FCHUNK * 2,
                             &sm.w_full[r]);
            }
            __syncwarp();
          }
        }
      if (!ok && lane == 0) sm.abort = 1;
      // drain: every copy issued has landed (normally consumed already)
      if (lane == 0 && !tc05::mbar_wait(&sm.w1_full, 0, kTimeoutNs)) sm.abort = 1;
      if (lane < FNSLOT && (uint32_t)lane < f) {
        const uint32_t last = (f - 1 - (uint32_t)lane) / FNSLOT;   // the slot's last use
        if (!tc05::mbar_wait(&sm.w_full[lane], last & 1u, kTimeoutNs)) sm.abort = 1;
      }
    }
    __syncwarp();
  } else if (warp == FMMA_WARP) {
    // ============================ MMA warp ============================
    if (lane == 0) {
      constexpr uint32_t IDESC = tc05::idesc_bf16_f32(FM, FW);
      constexpr uint64_t DACT = tc05::smem_desc_bits(128, (FW / 8) * 128);   // act: 256 columns
      constexpr uint64_t DCH = tc05::smem_desc_bits(128, (FCH / 8) * 128);   // weight chunk: 32 columns
      uint32_t f = 0;                                   // ring uses so far
      uint32_t ph_acc = 0, ph_x = 0;   // phase parities, bit s for tile slot s (registers, not arrays)
      // descriptor of element 0 of each operand buffer; advancing by 16 bytes adds 1
      const uint64_t dact0 = tc05::smem_desc(sm.act[0], DACT);
      constexpr uint64_t DACT_SLOT = sizeof(sm.act[0]) / 16;      // descriptor step between the slots' buffers
      const uint64_t dw1 = tc05::smem_desc(sm.w1, DCH);
      const uint64_t dring0 = tc05::smem_desc(sm.wring[0], DCH);
      constexpr uint64_t DRING_SLOT = sizeof(sm.wring[0]) / 16;   // descriptor step between ring slots
      bool ok = wait_bar(sm, &sm.w1_full, 0);
      for (int64_t k = 0; ok && k < nsteps; ++k)
        for (int s = 0; ok && s < 2; ++s) {
          int l;
          int64_t t;
          if (!step_work(k, s, per_slot, l, t)) continue;
          const uint32_t dst = tmem + (uint32_t)(s * FW);
          if (l == 0) {
            // layer 1: x -> accumulator (holding b1)
            if (!(ok = wait_bar(sm, &sm.acc_ready[s], (ph_acc >> s) & 1u) && wait_bar(sm, &sm.x_ready[s], (ph_x >> s) & 1u)))
              break;
            ph_acc ^= 1u << s;
            ph_x ^= 1u << s;
            tc05::fence_after_sync();
            for (int kk = 0; kk < FK1 / 16; ++kk)   // 128 elements = 256 bytes per K step of 16
              tc05::mma_bf16(dst, dact0 + DACT_SLOT * s + 16 * kk, dw1 + 16 * kk, IDESC, 1u);
            tc05::mma_commit(&sm.acc_full[s]);
          } else {
            // the slot's epilogue has written every activation chunk, read the
            // accumulator and stored the bias
            if (!(ok = wait_bar(sm, &sm.acc_ready[s], (ph_acc >> s) & 1u))) break;
            ph_acc ^= 1u << s;
            tc05::fence_after_sync();
            for (int i = 0; i < FNCH; ++i, ++f) {
              const int c = chunk_at(i);
              const uint32_t r = f % FNSLOT;
              if (!(ok = wait_bar(sm, &sm.w_full[r], (f / FNSLOT) & 1u))) break;
#pragma unroll
              for (int j = 0; j < FCH / 16; ++j)
                tc05::mma_bf16(dst, dact0 + DACT_SLOT * s + (uint64_t)(16 * (2 * c + j)),
                               dring0 + DRING_SLOT * r + (uint64_t)(16 * j), IDESC, 1u);
              tc05::mma_commit(&sm.w_empty[r]);   // the producer may refill ring slot r
            }
            if (!ok) break;
            tc05::mma_commit(&sm.acc_full[s]);
          }
      }
      if (!ok) sm.abort = 1;
      // drain: every MMA issued by this thread
      tc05::mma_commit(&sm.drain);
      if (!tc05::mbar_wait(&sm.drain, 0, kTimeoutNs)) sm.abort = 1;
    }
    __syncwarp();
  } else {
    // ========================== epilogue warps ==========================
    const int q = warp & 3, g = warp >> 2;
    const int row = q * 32 + lane;   // tile row = TMEM lane
    const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
    uint32_t ph_full = 0, ph_head = 0;   // phase parities, bit s for tile slot s
    bool ok = true;
    // both accumulators start holding b1; both slots' first features
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int cc = 0; cc < FGCH; ++cc) {
        const int c0 = g * FGCOLS + cc * FCH;
        store_bias(trow + (uint32_t)(s * FW + c0), &sm.bias[0][c0]);
      }
    tc05::tmem_wait_st();
    tc05::fence_before_sync();
    __syncwarp();
    if (lane == 0) {
      arrive(&sm.acc_ready[0]);
      arrive(&sm.acc_ready[1]);
    }
    if (per_slot > 0) {
#pragma unroll
      for (int s = 0; s < 2; ++s) store_x(sm.act[s], load_x(a, tile_of(0, s), npairs, tid), tid);
      tc05::fence_proxy_async();
      __syncwarp();
      if (lane == 0) {
        arrive(&sm.x_ready[0]);
        arrive(&sm.x_ready[1]);
      }
    }
    // the next features of a slot live from its layer-3 epilogue to its head, and the
    // two slots' intervals never overlap (slot 1 trails by two layers): one register
    // group holds them (an array indexed by the slot would live in local memory, and
    // its store would wait for the global load)
    uint4 xnext = make_uint4(0u, 0u, 0u, 0u);
    for (int64_t k = 0; ok && k < nsteps; ++k)
      for (int s = 0; s < 2; ++s) {
        int l;
        int64_t t;
        if (!step_work(k, s, per_slot, l, t)) continue;
        const int64_t tile = tile_of(t, s);
        const bool more = t + 1 < per_slot;   // the slot has a next tile
        if (!(ok = wait_bar(sm, &sm.acc_full[s], (ph_full >> s) & 1u))) break;
        ph_full ^= 1u << s;
        tc05::fence_after_sync();
        const uint32_t tacc = trow + (uint32_t)(s * FW);
        const int nl = (l + 1) & 3;      // the layer that accumulates here next
        if (l < 3) {
          // a = 2 gelu(z) -> BF16 activation chunks for the next layer
#pragma unroll
          for (int cc = 0; cc < FGCH; ++cc) {
            const int c0 = (g * FGCH + cc) * FCH;
            uint32_t r[32];
            tc05::tmem_ld32_async(tacc + (uint32_t)c0, r);
            tc05::tmem_wait_ld(r);
            store_bias(tacc + (uint32_t)c0, &sm.bias[nl][c0]);
            uint32_t pk[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const float2 y = gelu2_twice(make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1])));
              pk[i] = pack_bf16(y.x, y.y);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
              *reinterpret_cast<uint4*>(&sm.act[s][kmajor_index(row, c0 + 8 * j, FW)]) =
                  make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
          }
          // activations visible to the MMAs (async proxy), bias in TMEM: hand over
          tc05::fence_proxy_async();
          tc05::tmem_wait_st();
          tc05::fence_before_sync();
          __syncwarp();
          if (lane == 0) arrive(&sm.acc_ready[s]);
          // the slot's next features, loaded early, are written at its head
          if (l == 2 && more) xnext = load_x(a, tile_of(t + 1, s), npairs, tid);
        } else {
          // layer 4 has finished reading this slot's activations: its next features
          if (more) {
            store_x(sm.act[s], xnext, tid);
            tc05::fence_proxy_async();
            __syncwarp();
            if (lane == 0) arrive(&sm.x_ready[s]);
          }
          // the row's output inputs, loaded now and used after the dot products
          const int64_t p = tile * FM + row;
          const bool out = g == 0 && p < npairs;
          int64_t e = 0;
          float cpl = 0.f;
          double win = 0.0;
          if (out) {
            int j;
            pair_of(tile_origin(tile, a.k), row, (uint32_t)a.k, e, j);
            cpl = a.ptab[j].z;
            if (a.w_out) win = a.w_in[e];
          }
          float2 ye = make_float2(0.f, 0.f);   // (y, e) partial sums over this warp's columns
          const float4* w5 = reinterpret_cast<const float4*>(&sm.w5[0][0]);   // two columns' (y, e) weights
#pragma unroll
          for (int cc = 0; cc < FGCH; ++cc) {
            const int c0 = g * FGCOLS + cc * FCH;
            uint32_t r[32];
            tc05::tmem_ld32_async(tacc + (uint32_t)c0, r);
            tc05::tmem_wait_ld(r);
            store_bias(tacc + (uint32_t)c0, &sm.bias[nl][c0]);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const float2 y = gelu2_twice(make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1])));
              const uint32_t h = pack_bf16(y.x, y.y);   // the BF16 activations, as the next layer would take them
              const float a0 = __uint_as_float(h << 16), a1 = __uint_as_float(h & 0xffff0000u);
              const float4 w = w5[(c0 >> 1) + i];
              ye = __ffma2_rn(make_float2(a0, a0), make_float2(w.x, w.y), ye);
              ye = __ffma2_rn(make_float2(a1, a1), make_float2(w.z, w.w), ye);
            }
          }
          tc05::tmem_wait_st();
          tc05::fence_before_sync();
          __syncwarp();
          if (lane == 0) arrive(&sm.acc_ready[s]);
          if (g > 0) {
            sm.red[s][g - 1][row][0] = ye.x;
            sm.red[s][g - 1][row][1] = ye.y;
            __syncwarp();
            if (lane == 0) arrive(&sm.head_ready[s]);
          } else {
            if (!(ok = wait_bar(sm, &sm.head_ready[s], (ph_head >> s) & 1u))) break;
            ph_head ^= 1u << s;
            if (out) {
              float y = ye.x, er = ye.y;
#pragma unroll
              for (int h = 0; h < FGROUPS - 1; ++h) {
                y += sm.red[s][h][row][0];
                er += sm.red[s][h][row][1];
              }
              y += sm.b5[0] + cpl;
              er += sm.b5[1];
              if (a.pred) a.pred[p] = y;
              if (a.err) a.err[p] = er;
              if (a.w_out) a.w_out[p] = win * (double)expf(y);
              if (a.flag && !(er <= a.tau)) a.flag[e] = 1;   // NaN errors fall back too
            }
          }
        }
      }
    if (!ok) sm.abort = 1;
  }

  // ---- release TMEM once no MMA, copy or TMEM access of this CTA is in flight ----
  tc05::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc05::fence_after_sync();
    tc05::tmem_dealloc(tmem, FTMEM_COLS);
  }
  if (tid == 0 && sm.abort) atomicExch(a.status, 1);
}

}  // namespace rex
