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

#include <type_traits>

#include "ee_kernel.cuh"
#include "qcd_kernel.cuh"
#include "qq_kernel.cuh"
#include "qqg_kernel.cuh"

namespace rex {

static_assert(QQ_BLOCK == QCD_BLOCK && QQG_BLOCK == QCD_BLOCK, "every tile runs on the multi kernel's block size");

// Register classes: the persistent kernel is compiled once per class with only
// the tiles the class admits, and a multi-process call launches one kernel per
// class present, so each process runs at the occupancy its class allows:
//   class 0: e+e- -> mu+mu-, g g -> t t~, q q~ -> t t~
//   class 1: class 0, g g -> t t~ g and q q~ -> t t~ g
//   class 2: every process (g g -> t t~ g g sets the budget)
template <typename R, bool WIDTH, int MINB, int CLASS, int S_TTX, int S_TTXG, int S_TTXGG, bool TC_TTXGG>
__global__ void __launch_bounds__(QCD_BLOCK, MINB)
    multi_reweight_kernel(const __grid_constant__ MultiLaunch ml, unsigned long long* __restrict__ counter) {
  using T1 = QcdTile<PROC_GG_TTX, R, WIDTH, S_TTX>;
  using T2 = QcdTile<PROC_GG_TTXG, R, WIDTH, S_TTXG>;
  using T3 = QcdTile<PROC_GG_TTXGG, R, WIDTH, S_TTXGG, TC_TTXGG>;
  using T4 = QqTile<R>;
  using T5 = QqgTile<R>;
  using T6 = QqgTile<R, true>;   // crossed light line (q g, q~ g): the t-channel tile
  union Smem {
    typename T1::Smem a;
    typename std::conditional<(CLASS >= 1), typename T2::Smem, char>::type b;
    typename std::conditional<(CLASS >= 2), typename T3::Smem, char>::type c;
    typename T4::Smem d;
    typename std::conditional<(CLASS >= 1), typename T5::Smem, char>::type e;
    typename std::conditional<(CLASS >= 1), typename T6::Smem, char>::type f;
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
    // a g g batch's item: (tile, slot group); slots 1 .. nmass-1 split evenly over the
    // groups, slot 0 evaluated by each and its outputs written by group 0
    const int64_t local = item - B.tile_begin;
    const int64_t tile = local / B.ngroup;
    const int grp = (int)(local - tile * B.ngroup);
    const int nm1 = B.t.nmass - 1;
    const int s_lo = 1 + (nm1 * grp) / B.ngroup, s_hi = 1 + (nm1 * (grp + 1)) / B.ngroup;
    switch (B.kind) {
      case PROC_EE_MUMU: ee_tile(B.mom, B.w_in, B.nev, tile, ml.ew, B.out); break;
      case PROC_GG_TTX: T1::run(sm.a, B.mom, B.w_in, B.nev, tile, B.t, B.out, nullptr, s_lo, s_hi, grp == 0); break;
      case PROC_GG_TTXG:
        if constexpr (CLASS >= 1) T2::run(sm.b, B.mom, B.w_in, B.nev, tile, B.t, B.out, nullptr, s_lo, s_hi, grp == 0);
        break;
      case PROC_GG_TTXGG:
        if constexpr (CLASS >= 2) T3::run(sm.c, B.mom, B.w_in, B.nev, tile, B.t, B.out, nullptr, s_lo, s_hi, grp == 0);
        break;
      case PROC_QQ_TTX: T4::run(sm.d, B.mom, B.w_in, B.nev, tile, B.t, B.out); break;
      case PROC_QQ_TTXG:
        if constexpr (CLASS >= 1) {
          if (B.cross.neg[0] || B.cross.neg[1])
            T6::run(sm.f, B.mom, B.w_in, B.nev, tile, B.t, B.out, nullptr, B.cross);
          else
            T5::run(sm.e, B.mom, B.w_in, B.nev, tile, B.t, B.out, nullptr, B.cross);
        }
        break;
      default: break;
    }
    __syncthreads();
  }
}

int multi_class_of(int kind) {
  return kind == PROC_GG_TTXGG ? 2 : ((kind == PROC_GG_TTXG || kind == PROC_QQ_TTXG) ? 1 : 0);
}

// Lanes-per-event split of each QCD process in the multi kernel (the defaults of
// the single-process kernels: no split, scalar colour form) and the resident
// blocks per SM the register allocator must allow, per register class: the
// single-process kernels' best for the heaviest process of the class.
#ifndef REX_MULTI_MINB
#define REX_MULTI_MINB 1
#endif
template <typename R, int CLASS>
struct MultiSplit;
template <int CLASS>
struct MultiSplit<double, CLASS> {
  static constexpr int TTX = 0, TTXG = 0, TTXGG = 0;
  static constexpr int MINB = CLASS == 0 ? 3 : 1;
  static constexpr bool TC_TTXGG = false;
};
template <int CLASS>
struct MultiSplit<float, CLASS> {
  static constexpr int TTX = 0, TTXG = 0, TTXGG = 0;
  static constexpr int MINB = CLASS == 0 ? 4 : (CLASS == 1 ? 4 : REX_MULTI_MINB);
  static constexpr bool TC_TTXGG = false;
};

template <typename R, bool WIDTH, int CLASS>
static auto multi_kernel_ptr() {
  using S = MultiSplit<R, CLASS>;
  return multi_reweight_kernel<R, WIDTH, S::MINB, CLASS, S::TTX, S::TTXG, S::TTXGG, S::TC_TTXGG>;
}

int multi_events_per_tile(int kind, int mixed) {
  (void)mixed;   // every class uses the unsplit mapping
  switch (kind) {
    case PROC_EE_MUMU: return 128;
    case PROC_GG_TTX: return QCD_BLOCK / 4;
    case PROC_GG_TTXG: return QCD_BLOCK / 8;
    case PROC_GG_TTXGG: return QCD_BLOCK / 16;
    case PROC_QQ_TTX: return QqTile<float>::EPB;
    case PROC_QQ_TTXG: return QqgTile<float>::EPB;
    default: return 0;
  }
}

template <typename R, bool WIDTH, int CLASS>
static cudaError_t occupancy(int* per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, multi_kernel_ptr<R, WIDTH, CLASS>(), QCD_BLOCK, 0);
}

template <typename R, bool WIDTH>
static cudaError_t occupancy_c(int cls, int* per_sm) {
  switch (cls) {
    case 0: return occupancy<R, WIDTH, 0>(per_sm);
    case 1: return occupancy<R, WIDTH, 1>(per_sm);
    default: return occupancy<R, WIDTH, 2>(per_sm);
  }
}

int multi_grid_size(int mixed, int width, int cls, int* blocks) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return (int)e;
  if (mixed) e = width ? occupancy_c<float, true>(cls, &per_sm) : occupancy_c<float, false>(cls, &per_sm);
  else e = width ? occupancy_c<double, true>(cls, &per_sm) : occupancy_c<double, false>(cls, &per_sm);
  if (e != cudaSuccess) return (int)e;
  *blocks = sms * (per_sm > 0 ? per_sm : 1);
  return 0;
}

template <typename R, bool WIDTH, int CLASS>
static void launch_multi_t(int blocks, const MultiLaunch& ml, unsigned long long* counter, cudaStream_t st) {
  using S = MultiSplit<R, CLASS>;
  multi_reweight_kernel<R, WIDTH, S::MINB, CLASS, S::TTX, S::TTXG, S::TTXGG, S::TC_TTXGG>
      <<<blocks, QCD_BLOCK, 0, st>>>(ml, counter);
}

template <typename R, bool WIDTH>
static void launch_multi_c(int cls, int blocks, const MultiLaunch& ml, unsigned long long* counter,
                           cudaStream_t st) {
  switch (cls) {
    case 0: launch_multi_t<R, WIDTH, 0>(blocks, ml, counter, st); break;
    case 1: launch_multi_t<R, WIDTH, 1>(blocks, ml, counter, st); break;
    default: launch_multi_t<R, WIDTH, 2>(blocks, ml, counter, st); break;
  }
}

int launch_multi(int mixed, int width, int cls, int blocks, const MultiLaunch& ml, unsigned long long* counter,
                 void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return (int)e;
  if (mixed) {
    if (width) launch_multi_c<float, true>(cls, blocks, ml, counter, st);
    else launch_multi_c<float, false>(cls, blocks, ml, counter, st);
  } else {
    if (width) launch_multi_c<double, true>(cls, blocks, ml, counter, st);
    else launch_multi_c<double, false>(cls, blocks, ml, counter, st);
  }
  return (int)cudaGetLastError();
}

}  // namespace rex
