// BF16 tensor-core GEMM with FP32 accumulation for the surrogate MLP (sm_103a).
//
//   C[M x N] = op(A)[M x K] . op(B)[K x N]   (+ fused epilogue)
//
// A is stored row-major [M][K] (A_T = false) or as its transpose [K][M]
// (A_T = true); B is stored [K][N] (B_T = false) or [N][K] (B_T = true).  Tiles
// of 128 x 128 x 32 are staged global -> shared with cp.async (16-byte chunks,
// rows beyond M or N zero-filled, two buffers), fragments are read with
// ldmatrix (.trans when the stored layout is the transpose of the fragment's),
// and each of 8 warps computes a 64 x 32 block with mma.sync m16n8k16 BF16.
// K must be a multiple of 32 and the leading dimensions multiples of 8.
//
// Epilogues: EPI_F32     store the FP32 accumulator (split-K partials);
//            EPI_FWD     z = acc + bias[n]; store z (FP32, optional) and gelu(z) (BF16);
//            EPI_BWD     dz = acc * gelu'(zprev[m][n]); store dz (BF16).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace rex {

enum GemmEpi : int { EPI_F32 = 0, EPI_FWD = 1, EPI_BWD = 2 };

constexpr int GBM = 128, GBN = 128, GBK = 32, GTHREADS = 256;
constexpr int GPAD = 8;   // bf16 elements of padding per smem row (bank spread for ldmatrix)

// GELU in its tanh form (Hendrycks & Gimpel 2016):
//   gelu(z) = h (1 + t), h = z / 2, t = tanh(u), u = sqrt(2/pi) (z + 0.044715 z^3)
//   gelu'(z) = (1 + t) / 2 + h (1 - t^2) sqrt(2/pi) (1 + 3 * 0.044715 z^2)
// with tanh from the hardware approximation (tanh.approx.f32, relative error
// about 2^-11, one MUFU operation).
__device__ __forceinline__ float tanh_hw(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
constexpr float GELU_C0 = 0.7978845608028654f;               // sqrt(2/pi)
constexpr float GELU_C1 = 0.7978845608028654f * 0.044715f;   // sqrt(2/pi) * 0.044715
__device__ __forceinline__ float gelu_f(float z) {
  const float u = z * fmaf(GELU_C1, z * z, GELU_C0);
  const float h = 0.5f * z;
  return fmaf(h, tanh_hw(u), h);
}
__device__ __forceinline__ float gelu_grad_f(float z) {
  const float z2 = z * z;
  const float t = tanh_hw(z * fmaf(GELU_C1, z2, GELU_C0));
  const float du = fmaf(3.0f * GELU_C1, z2, GELU_C0);
  return fmaf(0.5f * z * (1.0f - t * t), du, 0.5f * (1.0f + t));
}

struct GemmArgs {
  int M, N, K;
  const __nv_bfloat16* A;
  int lda;
  const __nv_bfloat16* B;
  int ldb;
  // epilogue operands
  float* C32;                  // EPI_F32 output, or EPI_FWD pre-activation (may be null)
  int ldc;
  __nv_bfloat16* C16;          // EPI_FWD activation / EPI_BWD gradient output
  int ldc16;
  const float* bias;           // EPI_FWD
  const float* zprev;          // EPI_BWD
  int ldz;
  int k_per_split;             // split-K: blockIdx.z covers K range [z*kps, (z+1)*kps)
  int64_t split_stride;        // EPI_F32: elements between split partials
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const int bytes = valid ? 16 : 0;   // 0: zero-fill the 16 destination bytes
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(smem)), "l"(gmem), "r"(bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldsm_x4(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Shared-memory tile geometry for the two stored layouts.
template <bool TRANS, int ROWS_MN>
struct TileGeom {
  // not transposed: [ROWS_MN][GBK] (k contiguous); transposed: [GBK][ROWS_MN] (m/n contiguous)
  static constexpr int R = TRANS ? GBK : ROWS_MN;
  static constexpr int C = (TRANS ? ROWS_MN : GBK) + GPAD;
  static constexpr int ELEMS = R * C;
};

template <bool A_T, bool B_T, int EPI>
__global__ void __launch_bounds__(GTHREADS) gemm_bf16_kernel(const GemmArgs g) {
  using GA = TileGeom<A_T, GBM>;
  using GB = TileGeom<!B_T, GBN>;   // B fragment wants [n][k]; stored [k][n] is the "transposed" case
  __shared__ __align__(16) __nv_bfloat16 sa[2][GA::ELEMS];
  __shared__ __align__(16) __nv_bfloat16 sb[2][GB::ELEMS];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 2, wn = warp & 3;           // 2 x 4 warps, 64 x 32 each
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  const int kbeg = blockIdx.z * g.k_per_split;
  const int kend = min(g.K, kbeg + g.k_per_split);
  const int nk = (kend - kbeg) / GBK;

  auto load_tile = [&](int buf, int k0) {
    // A: 128 x 32 bf16 = 512 chunks of 16 B; B: 32 x 128 = 512 chunks
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int c = tid + i * GTHREADS;
      if (!A_T) {   // [m][k]: row m, 4 chunks per row
        const int r = c >> 2, kc = (c & 3) * 8;
        const int gm = m0 + r;
        const bool ok = gm < g.M;
        cp_async16(&sa[buf][r * GA::C + kc], g.A + (int64_t)(ok ? gm : 0) * g.lda + k0 + kc, ok);
      } else {      // [k][m]: row k, 16 chunks per row
        const int r = c >> 4, mc = (c & 15) * 8;
        const int gm = m0 + mc;
        const bool ok = gm < g.M;   // M is a multiple of 8 for transposed A
        cp_async16(&sa[buf][r * GA::C + mc], g.A + (int64_t)(k0 + r) * g.lda + (ok ? gm : 0), ok);
      }
      if (B_T) {    // stored [n][k]: row n, 4 chunks per row
        const int r = c >> 2, kc = (c & 3) * 8;
        const int gn = n0 + r;
        const bool ok = gn < g.N;
        cp_async16(&sb[buf][r * GB::C + kc], g.B + (int64_t)(ok ? gn : 0) * g.ldb + k0 + kc, ok);
      } else {      // stored [k][n]: row k, 16 chunks per row
        const int r = c >> 4, nc = (c & 15) * 8;
        const int gn = n0 + nc;
        const bool ok = gn < g.N;   // N is a multiple of 8
        cp_async16(&sb[buf][r * GB::C + nc], g.B + (int64_t)(k0 + r) * g.ldb + (ok ? gn : 0), ok);
      }
    }
    cp_async_commit();
  };

  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

  if (nk > 0) load_tile(0, kbeg);
  for (int kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < nk) {
      load_tile(buf ^ 1, kbeg + (kt + 1) * GBK);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const __nv_bfloat16* A_s = sa[buf];
    const __nv_bfloat16* B_s = sb[buf];
#pragma unroll
    for (int kk = 0; kk < GBK; kk += 16) {
      uint32_t af[4][4], bf[4][2];
#pragma unroll
      for (int mt = 0; mt < 4; ++mt) {
        const int mb = wm * 64 + mt * 16;
        if (!A_T) {
          const int r = mb + (lane & 15), c = kk + (lane >> 4) * 8;
          ldsm_x4(af[mt][0], af[mt][1], af[mt][2], af[mt][3], &A_s[r * GA::C + c]);
        } else {
          const int kr = kk + (lane & 7) + (lane >> 4) * 8, mc = mb + ((lane >> 3) & 1) * 8;
          ldsm_x4_t(af[mt][0], af[mt][1], af[mt][2], af[mt][3], &A_s[kr * GA::C + mc]);
        }
      }
#pragma unroll
      for (int np = 0; np < 2; ++np) {   // two n8 tiles per ldmatrix.x4
        const int nb = wn * 32 + np * 16;
        uint32_t r0, r1, r2, r3;
        if (B_T) {   // smem [n][k]
          const int nr = nb + ((lane >> 4) << 3) + (lane & 7), kc = kk + ((lane >> 3) & 1) * 8;
          ldsm_x4(r0, r1, r2, r3, &B_s[nr * GB::C + kc]);
        } else {     // smem [k][n]
          const int kr = kk + ((lane >> 3) & 1) * 8 + (lane & 7), nc = nb + ((lane >> 4) << 3);
          ldsm_x4_t(r0, r1, r2, r3, &B_s[kr * GB::C + nc]);
        }
        bf[np * 2][0] = r0;
        bf[np * 2][1] = r1;
        bf[np * 2 + 1][0] = r2;
        bf[np * 2 + 1][1] = r3;
      }
#pragma unroll
      for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], af[mt], bf[nt]);
    }
    __syncthreads();
  }

  // epilogue: thread owns rows gid, gid+8 and columns 2 tig, 2 tig + 1 of each 16 x 8 tile
  const int gid = lane >> 2, tig = lane & 3;
#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int m = m0 + wm * 64 + mt * 16 + gid + h * 8;
        const int n = n0 + wn * 32 + nt * 8 + tig * 2;
        if (m >= g.M) continue;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          if (n + e >= g.N) continue;
          const float v = acc[mt][nt][h * 2 + e];
          if (EPI == EPI_F32) {
            g.C32[blockIdx.z * g.split_stride + (int64_t)m * g.ldc + n + e] = v;
          } else if (EPI == EPI_FWD) {
            const float z = v + g.bias[n + e];
            if (g.C32) g.C32[(int64_t)m * g.ldc + n + e] = z;
            g.C16[(int64_t)m * g.ldc16 + n + e] = __float2bfloat16(gelu_f(z));
          } else {
            const float d = v * gelu_grad_f(g.zprev[(int64_t)m * g.ldz + n + e]);
            g.C16[(int64_t)m * g.ldc16 + n + e] = __float2bfloat16(d);
          }
        }
      }
}

}  // namespace rex
