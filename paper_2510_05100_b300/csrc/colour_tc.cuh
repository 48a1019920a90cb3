// Colour quadratic form on tensor cores (mixed precision), sm_103a.
//
// For one antitop helicity every lane holds the jamps A[ht][s] (ht = 0, 1 top
// helicities, s = 0..NF-1 colour flows).  The colour sum of a lane is
//   sum_ht sum_{s,s'} (Re A_s Cint_ss' Re A_s' + Im A_s Cint_ss' Im A_s'),
// a quadratic form over the real row vectors x = Re A[ht], Im A[ht].  Per top
// helicity the warp stages its 64 row vectors (row = 2 lane + re/im) in shared
// memory as FP16 hi + lo parts of x * 2^-q (q: an exact power of two per event,
// so that the event's largest jamp is O(1); hi + lo carries ~22 bits), computes
// Y = X Cint with mma.sync m16n8k16 (FP16 operands, FP32 accumulation; Cint is a
// matrix of small integers, exact in FP16), and forms the row dots x . y from
// the A fragments, which hold exactly the columns of each lane's D fragment.
//
// The rows of one m16 tile are lanes 8t..8t+7, which belong to one event when an
// event has 8 or more lanes.  The four tile dots are reduced across the warp by
// a transposing butterfly (6 shuffles), after which lane 8t holds tile t's
// colour sum; the other lanes return 0, so a sum over the event's lanes gives
// the event's colour sum.
//
// The B fragments of Cint (constant per warp) live in shared memory, one 32-bit
// word per lane and fragment register, so that they hold no registers across
// the amplitude evaluation.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "helas.cuh"

namespace rex {

template <int NF>
struct ColourTc {
  static constexpr int KP = ((NF + 15) / 16) * 16;   // flows padded to the MMA k
  static constexpr int KS = KP / 16;                   // k16 steps
  static constexpr int NT = (NF + 7) / 8;              // n8 tiles of the result
  static constexpr int LD = KP + 8;                    // smem row stride (halves): spreads ldmatrix banks
  static constexpr int NB = KS * NT * 2;               // B fragment registers per lane
  // per warp: hi and lo planes of 64 rows, then the B fragments (NB words x 32 lanes)
  static constexpr int WARP_HALVES = 2 * 64 * LD + NB * 32 * 2;
  static_assert((LD * 2) % 16 == 0, "rows must stay 16-byte aligned for vector stores");

  // Write this warp's B fragments of Cint (k = flow s, n = flow s') into smem.
  __device__ __forceinline__ static void load(const int (&C)[NF][NF], __half* smem) {
    uint32_t* bw = reinterpret_cast<uint32_t*>(smem + 2 * 64 * LD);
    const int lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int ks = 0; ks < KS; ++ks)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const int k0 = ks * 16 + tig * 2 + r * 8, n = nt * 8 + gid;
          float c0 = 0.f, c1 = 0.f;
          if (n < NF) {
            if (k0 < NF) c0 = float(C[k0][n]);
            if (k0 + 1 < NF) c1 = float(C[k0 + 1][n]);
          }
          const __half2 h = __floats2half2_rn(c0, c1);
          bw[((ks * NT + nt) * 2 + r) * 32 + lane] = *reinterpret_cast<const uint32_t*>(&h);
        }
    __syncwarp();
  }

  // Quadratic form of this lane's jamps; must be called by all 32 lanes.
  // NH: lanes per event (8, 16 or 32).  smem: WARP_HALVES halves for this warp.
  template <int NH>
  __device__ __forceinline__ static float form(const cx<float> (&A)[2][NF], __half* smem) {
    static_assert(NH == 8 || NH == 16 || NH == 32, "events of 8, 16 or 32 lanes");
    const int lane = threadIdx.x & 31;
    // exact power-of-two scale per event
    float amax = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int s = 0; s < NF; ++s) amax = fmaxf(amax, fmaxf(fabsf(A[h][s].re), fabsf(A[h][s].im)));
#pragma unroll
    for (int off = NH >> 1; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
    int ex = 0;
    frexpf(amax > 0.f ? amax : 1.f, &ex);
    const float sc = ldexpf(1.f, -ex), inv2 = ldexpf(1.f, 2 * ex);
    __half* hi = smem;
    __half* lo = smem + 64 * LD;
    const uint32_t* bw = reinterpret_cast<const uint32_t*>(smem + 2 * 64 * LD);
    float v[4] = {0.f, 0.f, 0.f, 0.f};   // dot of m16 tile t (rows of lanes 8t..8t+7)
#pragma unroll
    for (int ht = 0; ht < 2; ++ht) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int row = lane * 2 + c;
#pragma unroll
        for (int s8 = 0; s8 < KP; s8 += 8) {   // 8 flows -> one 16-byte store per plane
          uint32_t ph[4], pl[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int s = s8 + 2 * j;
            float x0 = 0.f, x1 = 0.f;
            if (s < NF) x0 = (c == 0 ? A[ht][s].re : A[ht][s].im) * sc;
            if (s + 1 < NF) x1 = (c == 0 ? A[ht][s + 1].re : A[ht][s + 1].im) * sc;
            const __half2 h2 = __floats2half2_rn(x0, x1);
            const float2 hb = __half22float2(h2);
            const __half2 l2 = __floats2half2_rn(x0 - hb.x, x1 - hb.y);
            ph[j] = *reinterpret_cast<const uint32_t*>(&h2);
            pl[j] = *reinterpret_cast<const uint32_t*>(&l2);
          }
          *reinterpret_cast<uint4*>(&hi[row * LD + s8]) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
          *reinterpret_cast<uint4*>(&lo[row * LD + s8]) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
        }
      }
      __syncwarp();
#pragma unroll
      for (int t = 0; t < 4; ++t) {   // m16 tiles: rows 16t..16t+15 = lanes 8t..8t+7
        uint32_t ah[KS][4], al[KS][4];
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
          const int r = t * 16 + (lane & 15), col = ks * 16 + (lane >> 4) * 8;
          const uint32_t ph = static_cast<uint32_t>(__cvta_generic_to_shared(&hi[r * LD + col]));
          const uint32_t pl = static_cast<uint32_t>(__cvta_generic_to_shared(&lo[r * LD + col]));
          asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                       : "=r"(ah[ks][0]), "=r"(ah[ks][1]), "=r"(ah[ks][2]), "=r"(ah[ks][3])
                       : "r"(ph));
          asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                       : "=r"(al[ks][0]), "=r"(al[ks][1]), "=r"(al[ks][2]), "=r"(al[ks][3])
                       : "r"(pl));
        }
        float dot = 0.f;
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int ks = 0; ks < KS; ++ks) {
            const uint32_t b0 = bw[((ks * NT + nt) * 2 + 0) * 32 + lane];
            const uint32_t b1 = bw[((ks * NT + nt) * 2 + 1) * 32 + lane];
#pragma unroll
            for (int part = 0; part < 2; ++part) {
              const uint32_t* a = part == 0 ? ah[ks] : al[ks];
              asm volatile(
                  "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                  "{%0,%1,%2,%3};\n"
                  : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                  : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
            }
          }
          // x at the D fragment's columns n = 8 nt + 2 tig (+1): k step nt/2, fragment half nt%2
          const int ks = nt >> 1, hsel = (nt & 1) * 2;
          const __half2 h0 = *reinterpret_cast<const __half2*>(&ah[ks][hsel]);       // row gid
          const __half2 l0 = *reinterpret_cast<const __half2*>(&al[ks][hsel]);
          const __half2 h1 = *reinterpret_cast<const __half2*>(&ah[ks][hsel + 1]);   // row gid + 8
          const __half2 l1 = *reinterpret_cast<const __half2*>(&al[ks][hsel + 1]);
          const float2 x0 = __half22float2(h0), y0 = __half22float2(l0);
          const float2 x1 = __half22float2(h1), y1 = __half22float2(l1);
          dot += d[0] * (x0.x + y0.x) + d[1] * (x0.y + y0.y) + d[2] * (x1.x + y1.x) + d[3] * (x1.y + y1.y);
        }
        v[t] += dot;
      }
      __syncwarp();
    }
    // transposing butterfly: after it lane l holds the warp sum of tile l >> 3
    const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0;
    const float k0 = b4 ? v[2] : v[0], k1 = b4 ? v[3] : v[1];   // the pair this lane keeps
    const float s0 = b4 ? v[0] : v[2], s1 = b4 ? v[1] : v[3];   // the pair its partner keeps
    const float w0 = k0 + __shfl_xor_sync(0xffffffffu, s0, 16);
    const float w1 = k1 + __shfl_xor_sync(0xffffffffu, s1, 16);
    float u = (b3 ? w1 : w0) + __shfl_xor_sync(0xffffffffu, b3 ? w0 : w1, 8);
    u += __shfl_xor_sync(0xffffffffu, u, 4);
    u += __shfl_xor_sync(0xffffffffu, u, 2);
    u += __shfl_xor_sync(0xffffffffu, u, 1);
    // lane l is in tile l >> 3, whose rows belong to lane l's own event: its scale applies
    return (lane & 7) == 0 ? u * inv2 : 0.f;
  }
};

}  // namespace rex
