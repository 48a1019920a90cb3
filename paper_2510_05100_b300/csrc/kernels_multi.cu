// Persistent multi-process reweighting kernel (sm_103a).
//
// One launch reweights several subprocess batches of uneven size (e.g. 10k
// e+e- -> mu+mu-, 1M g g -> t t~, 500k g g -> t t~ g, 100k g g -> t t~ g g) to the
// same parameter points (q q~ -> t t~ batches too).  The paper runs subprocesses one after another and
// finds multi-channel GPU runs latency bound (Sec. 4.2); here every (batch,
// event tile) is a work item of a single persistent grid (one block per SM
// slot), and blocks take items from a global atomic counter in
// heaviest-process-first order so that the cheap tiles fill the tail.
// The per-tile code is exactly the single-process kernels' (QcdTile, QqTile, ee_tile).
#include <cuda_runtime.h>

#include "ee_kernel.cuh"
#include "qcd_kernel.cuh"
#include "qq_kernel.cuh"

namespace rex {

static_assert(QQ_BLOCK == QCD_BLOCK, "every tile runs on the multi kernel's block size");

template <typename R, bool WIDTH, int MINB, int S_TTX, int S_TTXG, int S_TTXGG, bool TC_TTXGG>
__global__ void __launch_bounds__(QCD_BLOCK, MINB)
    multi_reweight_kernel(const __grid_constant__ MultiLaunch ml, unsigned long long* __restrict__ counter) {
  using T1 = QcdTile<PROC_GG_TTX, R, WIDTH, S_TTX>;
  using T2 = QcdTile<PROC_GG_TTXG, R, WIDTH, S_TTXG>;
  using T3 = QcdTile<PROC_GG_TTXGG, R, WIDTH, S_TTXGG, TC_TTXGG>;
  using T4 = QqTile<R>;
  union Smem {
    typename T1::Smem a;
    typename T2::Smem b;
    typename T3::Smem c;
    typename T4::Smem d;
  };
  __shared__ Smem sm;
  __shared__ unsigned long long item_s;
  for (;;) {
    if (threadIdx.x == 0) item_s = atomicAdd(counter, 1ull);
    __syncthreads();
    const long long item = (long long)item_s;
    __syncthreads();
    if (item >= ml.total) break;
    int b = 0;
    while (b + 1 < ml.nbatch && item >= ml.b[b].tile_end) ++b;
    const MultiBatch& B = ml.b[b];
    const int64_t tile = item - B.tile_begin;
    switch (B.kind) {
      case PROC_EE_MUMU: ee_tile(B.mom, B.w_in, B.nev, tile, ml.ew, B.out); break;
      case PROC_GG_TTX: T1::run(sm.a, B.mom, B.w_in, B.nev, tile, B.t, B.out); break;
      case PROC_GG_TTXG: T2::run(sm.b, B.mom, B.w_in, B.nev, tile, B.t, B.out); break;
      case PROC_GG_TTXGG: T3::run(sm.c, B.mom, B.w_in, B.nev, tile, B.t, B.out); break;
      case PROC_QQ_TTX: T4::run(sm.d, B.mom, B.w_in, B.nev, tile, B.t, B.out); break;
      default: break;
    }
    __syncthreads();
  }
}

// Lanes-per-event split of each QCD process in the multi kernel (the defaults of
// the single-process kernels: no split, scalar colour form).  One register budget
// serves every process: min blocks per SM follows g g -> t t~ g g, the heaviest.
#ifndef REX_MULTI_MINB
#define REX_MULTI_MINB 1
#endif
template <typename R>
struct MultiSplit;
template <>
struct MultiSplit<double> {
  static constexpr int TTX = 0, TTXG = 0, TTXGG = 0, MINB = 1;
  static constexpr bool TC_TTXGG = false;
};
template <>
struct MultiSplit<float> {
  static constexpr int TTX = 0, TTXG = 0, TTXGG = 0, MINB = REX_MULTI_MINB;
  static constexpr bool TC_TTXGG = false;
};

template <typename R, bool WIDTH>
static auto multi_kernel_ptr() {
  using S = MultiSplit<R>;
  return multi_reweight_kernel<R, WIDTH, S::MINB, S::TTX, S::TTXG, S::TTXGG, S::TC_TTXGG>;
}

int multi_events_per_tile(int kind, int mixed) {
  switch (kind) {
    case PROC_EE_MUMU: return 128;
    case PROC_GG_TTX: return QCD_BLOCK / (4 << (mixed ? MultiSplit<float>::TTX : 0));
    case PROC_GG_TTXG: return QCD_BLOCK / (8 << (mixed ? MultiSplit<float>::TTXG : 0));
    case PROC_GG_TTXGG: return QCD_BLOCK / (16 << (mixed ? MultiSplit<float>::TTXGG : 0));
    case PROC_QQ_TTX: return QqTile<float>::EPB;
    default: return 0;
  }
}

int multi_grid_size(int mixed, int width, int* blocks) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return (int)e;
  if (mixed)
    e = width ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, multi_kernel_ptr<float, true>(), QCD_BLOCK, 0)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, multi_kernel_ptr<float, false>(), QCD_BLOCK, 0);
  else
    e = width ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, multi_kernel_ptr<double, true>(), QCD_BLOCK, 0)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, multi_kernel_ptr<double, false>(), QCD_BLOCK, 0);
  if (e != cudaSuccess) return (int)e;
  *blocks = sms * (per_sm > 0 ? per_sm : 1);
  return 0;
}

template <typename R, bool WIDTH>
static void launch_multi_t(int blocks, const MultiLaunch& ml, unsigned long long* counter, cudaStream_t st) {
  using S = MultiSplit<R>;
  multi_reweight_kernel<R, WIDTH, S::MINB, S::TTX, S::TTXG, S::TTXGG, S::TC_TTXGG><<<blocks, QCD_BLOCK, 0, st>>>(ml, counter);
}

int launch_multi(int mixed, int width, int blocks, const MultiLaunch& ml, unsigned long long* counter,
                 void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return (int)e;
  if (mixed) {
    if (width) launch_multi_t<float, true>(blocks, ml, counter, st);
    else launch_multi_t<float, false>(blocks, ml, counter, st);
  } else {
    if (width) launch_multi_t<double, true>(blocks, ml, counter, st);
    else launch_multi_t<double, false>(blocks, ml, counter, st);
  }
  return (int)cudaGetLastError();
}

}  // namespace rex
