// C ABI of the reweighting library (declared in include/rex.h).
//
// Host side only: argument validation, the per-launch parameter table
// (distinct mass slots, coupling factors), chunking of large point lists,
// and the kernel launches.  No call here reaches the CPU for any step of the
// computation: every |M|^2 and weight is produced by the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <utility>
#include <string>
#include <vector>

#include "../../include/rex.h"
#include "dev_alloc.h"
#include "generated/qcd_amplitudes.cuh"
#include "rex_internal.cuh"

using namespace rex;

namespace rex {

cudaError_t dev_malloc(void** p, size_t bytes) {
  static std::mutex mu;
  static std::string armed;     // the value the countdown belongs to
  static long made = 0;         // allocations since it took that value
  *p = nullptr;
  {
    std::lock_guard<std::mutex> lock(mu);
    const char* v = std::getenv("REX_FAIL_DEVICE_ALLOC");
    char* end = nullptr;
    const long n = (v && *v) ? std::strtol(v, &end, 10) : 0;
    if (n >= 1 && end && *end == '\0') {
      if (armed != v) {
        armed = v;
        made = 0;
      }
      if (++made >= n) return cudaErrorMemoryAllocation;
    } else {
      armed.clear();
    }
  }
  return cudaMalloc(p, bytes);
}

}  // namespace rex

struct rex_proc {
  int kind;
  int precision;
  unsigned flags;
  int variant;        // QCD thread-mapping variant (qcd_kernel.cuh)
  int has_orig;
  rex_params orig;
  QqgCrossing cross;  // q q~ -> t t~ g channels: how the kernel reads an event
  double avg;         // q q~ -> t t~ g channels: the spin-colour average's denominator
  // rex_reweight_host buffers (device), grown on demand
  double* d_mom;
  double* d_win;
  double* d_wout;
  size_t cap_mom, cap_win, cap_wout;
  // rex_reweight_host pipeline: two streams forked from the caller's, created on first use
  cudaStream_t hs[2];
  cudaEvent_t hfork, hjoin[2];
};

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(int err, const char* what) {
  return fail(REX_ECUDA, "%s: %s", what, cudaGetErrorString(static_cast<cudaError_t>(err)));
}

// A CUDA error left by earlier work on this thread (another library's failed launch,
// an asynchronous fault) would otherwise be picked up by the launch check after this
// call's own kernel and reported as that kernel's.  Report it before enqueueing
// anything, under its own message, without clearing it.
int pending_error() {
  const cudaError_t e = cudaPeekAtLastError();
  if (e == cudaSuccess) return REX_OK;
  return fail(REX_ECUDA, "CUDA error pending from earlier work, before this call enqueued anything: %s",
              cudaGetErrorString(e));
}

struct ProcInfo {
  const char* name;
  int kind;
  int npart;
  int ngluon;
  int colour_den;
};

const ProcInfo kProcs[] = {
    {"ee_mumu", PROC_EE_MUMU, 4, 0, 1},
    {"gg_ttx", PROC_GG_TTX, 4, gg_ttx_info::NGLUON, gg_ttx_info::COLOUR_DEN},
    {"gg_ttxg", PROC_GG_TTXG, 5, gg_ttxg_info::NGLUON, gg_ttxg_info::COLOUR_DEN},
    {"gg_ttxgg", PROC_GG_TTXGG, 6, gg_ttxgg_info::NGLUON, gg_ttxgg_info::COLOUR_DEN},
    {"qq_ttx", PROC_QQ_TTX, 4, 0, 1},
    {"qq_ttxg", PROC_QQ_TTXG, 5, 0, 1},
};
static_assert(sizeof(kProcs) / sizeof(kProcs[0]) == PROC_LAST + 1, "one table row per process kind");

// The crossed channels of q q~ -> t t~ g with one light-quark line (record order: the
// two incoming partons, t, t~, the outgoing parton), run by the q q~ -> t t~ g
// kernels; avg: 4 spins x 9 colours for q q~, x 24 for q g.
struct QqgChannel {
  const char* name;
  QqgCrossing cross;
  double avg;
};
const QqgChannel kQqgChannels[] = {
    {"qq_ttxg", {{0, 1, 2, 3, 4}, {0, 0, 0, 0, 0}}, 36.0},
    {"qxq_ttxg", {{1, 0, 2, 3, 4}, {0, 0, 0, 0, 0}}, 36.0},
    {"qg_ttxq", {{0, 4, 2, 3, 1}, {0, 1, 0, 0, 1}}, 96.0},
    {"gq_ttxq", {{1, 4, 2, 3, 0}, {0, 1, 0, 0, 1}}, 96.0},
    {"qxg_ttxqx", {{4, 0, 2, 3, 1}, {1, 0, 0, 0, 1}}, 96.0},
    {"gqx_ttxqx", {{4, 1, 2, 3, 0}, {1, 0, 0, 0, 1}}, 96.0},
};

bool is_direct(const QqgCrossing& c) {
  for (int i = 0; i < 5; ++i)
    if (c.src[i] != i || c.neg[i] != 0) return false;
  return true;
}

const ProcInfo& info_of(int kind) { return kProcs[kind]; }

// processes with one kernel (no thread-mapping variants to choose from)
bool single_variant(const rex_proc* p) {
  return p->precision == REX_DF64 || p->kind == PROC_EE_MUMU || p->kind == PROC_QQ_TTX || p->kind == PROC_QQ_TTXG;
}

// Default thread-mapping variant per (process, precision), the fastest of every
// variant timed on a B300 at 2^20 (gg_ttx, gg_ttxg) / 2^16 (gg_ttxgg) events;
// rex_autotune picks again on the caller's device and data.
int default_variant(int kind, int precision) {
  static const int table[PROC_LAST + 1][2] = {
      {0, 0},   // ee_mumu (single variant)
      {0, 0},   // gg_ttx:   FP64 v0, mixed v0
      {0, 4},   // gg_ttxg:  FP64 v0, mixed v4 (min 4 blocks/SM: 16 warps, 128 registers)
      {0, 0},   // gg_ttxgg: FP64 v0, mixed v0
      {0, 0},   // qq_ttx (single variant)
      {0, 0},   // qq_ttxg (single variant)
  };
  return table[kind][precision == REX_MIXED ? 1 : 0];
}

int launch_qcd(const rex_proc* p, const double* mom, const double* w_in, int64_t nev, const QcdLaunch& lp,
               double* out, void* stream, const signed char* hel) {
  const int mixed = p->precision == REX_MIXED;
  if (p->precision == REX_DF64) {   // gg_ttx, gg_ttxg, qq_ttxg (rex_init_process); exclusive: gg_ttxg
    if (hel) return launch_gg_ttxg_df64_exclusive(mom, w_in, nev, lp, out, stream, hel);
    if (p->kind == PROC_QQ_TTXG) return launch_qq_ttxg_df64(mom, w_in, nev, lp, out, stream, p->cross);
    return p->kind == PROC_GG_TTX ? launch_gg_ttx_df64(mom, w_in, nev, lp, out, stream)
                                  : launch_gg_ttxg_df64(mom, w_in, nev, lp, out, stream);
  }
  switch (p->kind) {
    case PROC_GG_TTX:
      return hel ? launch_gg_ttx_exclusive(mixed, mom, w_in, nev, lp, out, stream, hel)
                 : launch_gg_ttx(mixed, p->variant, mom, w_in, nev, lp, out, stream);
    case PROC_GG_TTXG:
      return hel ? launch_gg_ttxg_exclusive(mixed, mom, w_in, nev, lp, out, stream, hel)
                 : launch_gg_ttxg(mixed, p->variant, mom, w_in, nev, lp, out, stream);
    case PROC_GG_TTXGG:
      return hel ? launch_gg_ttxgg_exclusive(mixed, mom, w_in, nev, lp, out, stream, hel)
                 : launch_gg_ttxgg(mixed, p->variant, mom, w_in, nev, lp, out, stream);
    case PROC_QQ_TTX: return launch_qq_ttx(mixed, mom, w_in, nev, lp, out, stream, hel);
    case PROC_QQ_TTXG: return launch_qq_ttxg(mixed, mom, w_in, nev, lp, out, stream, hel, p->cross);
    default: return (int)cudaErrorInvalidValue;
  }
}

bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// avg * (4 pi alphas)^n / colour_den for a pure-gluon tree amplitude with n gluons;
// q q~ -> t t~: (4 pi alphas)^2 * colour sum (N^2 - 1)/4 = 2 / (4 spins * 9 colours)
double qcd_factor(const rex_proc* p, double alphas) {
  const ProcInfo& pi = info_of(p->kind);
  const double gs2 = 4.0 * M_PI * alphas;
  if (pi.kind == PROC_QQ_TTX) return gs2 * gs2 * 2.0 / 36.0;
  // q q~ -> t t~ g and its crossings: g^6, the integer colour matrix's 1/3, and the
  // channel's average (1/(4 spins * 9 colours) for q q~, 1/(4 * 24) for q g)
  if (pi.kind == PROC_QQ_TTXG) return gs2 * gs2 * gs2 / (3.0 * p->avg);
  double f = 1.0;
  for (int i = 0; i < pi.ngluon; ++i) f *= gs2;
  int nfinal = pi.ngluon - 2;
  double sym = 1.0;
  for (int i = 2; i <= nfinal; ++i) sym *= i;
  return f / (4.0 * 64.0 * sym * pi.colour_den);
}

int check_qcd_point(const rex_params& p) {
  if (!(p.mt > 0.0) || !std::isfinite(p.mt) || !(p.alphas > 0.0) || !std::isfinite(p.alphas) ||
      !(p.wt >= 0.0) || !std::isfinite(p.wt))
    return fail(REX_EINVAL, "QCD point needs finite mt > 0, alphas > 0, wt >= 0 (got mt=%g alphas=%g wt=%g)",
                p.mt, p.alphas, p.wt);
  return REX_OK;
}

int check_ew_point(const rex_params& p) {
  if (!(p.mz > 0.0) || !(p.wz >= 0.0) || !(p.sw2 > 0.0 && p.sw2 < 1.0) || !(p.alpha > 0.0) ||
      !std::isfinite(p.mz) || !std::isfinite(p.wz) || !std::isfinite(p.alpha))
    return fail(REX_EINVAL, "ee_mumu point needs mz > 0, wz >= 0, 0 < sw2 < 1, alpha > 0");
  return REX_OK;
}

EwPoint ew_point(const rex_params& p) {
  EwPoint c;
  const double e2 = 4.0 * M_PI * p.alpha;
  const double cw2 = 1.0 - p.sw2;
  const double gz2 = e2 / (p.sw2 * cw2);
  const double q = -1.0, t3 = -0.5;
  const double gl = t3 - q * p.sw2, gr = -q * p.sw2;
  c.e2qq = e2 * q * q;
  c.gzz[0] = gz2 * gl * gl;
  c.gzz[1] = gz2 * gl * gr;
  c.gzz[2] = gz2 * gr * gl;
  c.gzz[3] = gz2 * gr * gr;
  c.mz2 = p.mz * p.mz;
  c.mzwz = p.mz * p.wz;
  c.avg = 0.25;
  return c;
}

// Enqueue one QCD launch for points [j0, j1) writing columns j0.. of rows with stride k.
int run_qcd_chunk(rex_proc* p, const double* mom, const double* w_in, int64_t nev,
                  const rex_params* pts, int j0, int j1, int mode, double* out, int64_t stride,
                  void* stream, int* next_j, const signed char* hel = nullptr) {
  QcdLaunch lp;
  std::memset(&lp, 0, sizeof lp);
  lp.mode = mode;
  lp.out_stride = stride;
  lp.nmass = 1;
  lp.mass[0] = p->orig.mt;
  lp.width[0] = p->orig.wt;
  lp.factor0 = qcd_factor(p, p->orig.alphas);
  const bool dedupe = !(p->flags & REX_FLAG_NO_DEDUPE);
  int j = j0;
  for (; j < j1 && j - j0 < MAX_POINTS; ++j) {
    const rex_params& q = pts[j];
    int slot = -1;
    if (dedupe) {
      for (int s = 0; s < lp.nmass; ++s)
        if (lp.mass[s] == q.mt && lp.width[s] == q.wt) {
          slot = s;
          break;
        }
    }
    if (slot < 0) {
      if (lp.nmass == MAX_MASS) break;
      slot = lp.nmass++;
      lp.mass[slot] = q.mt;
      lp.width[slot] = q.wt;
    }
    lp.slot[j - j0] = slot;
    lp.factor[j - j0] = qcd_factor(p, q.alphas);
  }
  lp.k = j - j0;
  for (int s = 0; s < lp.nmass; ++s)
    if (lp.width[s] != 0.0) lp.has_width = 1;
  *next_j = j;
  double* o = (mode == OUT_RATIO) ? out + j0 : out;
  const int err = launch_qcd(p, mom, w_in, nev, lp, o, stream, hel);
  if (err != 0) return cuda_fail(err, "kernel launch");
  return REX_OK;
}

int run_ee_chunk(rex_proc* p, const double* mom, const double* w_in, int64_t nev,
                 const rex_params* pts, int j0, int j1, int mode, double* out, int64_t stride,
                 void* stream, int* next_j, const signed char* hel = nullptr) {
  EwLaunch lp;
  std::memset(&lp, 0, sizeof lp);
  lp.mode = mode;
  lp.out_stride = stride;
  lp.pt[0] = ew_point(p->orig);
  int j = j0;
  for (; j < j1 && j - j0 < MAX_EW_POINTS; ++j) lp.pt[1 + j - j0] = ew_point(pts[j]);
  lp.k = j - j0;
  *next_j = j;
  double* o = (mode == OUT_RATIO) ? out + j0 : out;
  const int err = launch_ee(mom, w_in, nev, lp, o, stream, hel);
  if (err != 0) return cuda_fail(err, "kernel launch");
  return REX_OK;
}

int validate_proc(const rex_proc* p) {
  if (!p) return fail(REX_EINVAL, "null process handle");
  if (p->kind < 0 || p->kind > PROC_LAST) return fail(REX_EINVAL, "corrupt process handle");
  return REX_OK;
}

int reweight_impl(rex_proc* p, const double* momenta, const double* w_in, int64_t nev,
                  const rex_params* param_sets, int k, double* w_out, void* stream,
                  const signed char* hel = nullptr) {
  int rc = validate_proc(p);
  if (rc) return rc;
  if (nev < 0) return fail(REX_EINVAL, "nev < 0");
  if (k < 0) return fail(REX_EINVAL, "k < 0");
  if (!p->has_orig) return fail(REX_ENOTINIT, "rex_set_params has not been called");
  if (nev == 0 || k == 0) return REX_OK;
  if (!momenta || !w_in || !w_out || !param_sets) return fail(REX_EINVAL, "null array pointer");
  if (!aligned16(momenta) || !aligned8(w_in) || !aligned8(w_out))
    return fail(REX_EINVAL, "momenta must be 16-byte and weights 8-byte aligned");
  for (int j = 0; j < k; ++j) {
    rc = p->kind == PROC_EE_MUMU ? check_ew_point(param_sets[j]) : check_qcd_point(param_sets[j]);
    if (rc) return rc;
  }
  if ((rc = pending_error())) return rc;
  int j = 0;
  while (j < k) {
    int next = j;
    rc = p->kind == PROC_EE_MUMU
             ? run_ee_chunk(p, momenta, w_in, nev, param_sets, j, k, OUT_RATIO, w_out, k, stream, &next, hel)
             : run_qcd_chunk(p, momenta, w_in, nev, param_sets, j, k, OUT_RATIO, w_out, k, stream, &next, hel);
    if (rc) return rc;
    j = next;
  }
  return REX_OK;
}

// ---------------------------------------------------------------------------
// persistent multi-process launch
// ---------------------------------------------------------------------------
int fill_multi_table(const rex_proc* p, const rex_params* pts, int j0, int j1, int64_t stride, MultiTable& t) {
  std::memset(&t, 0, sizeof t);
  t.mode = OUT_RATIO;
  t.out_stride = stride;
  t.nmass = 1;
  t.mass[0] = p->orig.mt;
  t.width[0] = p->orig.wt;
  t.factor0 = qcd_factor(p, p->orig.alphas);
  const bool dedupe = !(p->flags & REX_FLAG_NO_DEDUPE);
  for (int j = j0; j < j1; ++j) {
    const rex_params& q = pts[j];
    int slot = -1;
    if (dedupe)
      for (int s = 0; s < t.nmass; ++s)
        if (t.mass[s] == q.mt && t.width[s] == q.wt) {
          slot = s;
          break;
        }
    if (slot < 0) {
      slot = t.nmass++;
      t.mass[slot] = q.mt;
      t.width[slot] = q.wt;
    }
    t.slot[j - j0] = slot;
    t.factor[j - j0] = qcd_factor(p, q.alphas);
  }
  t.k = j1 - j0;
  for (int s = 0; s < t.nmass; ++s)
    if (t.width[s] != 0.0) t.has_width = 1;
  return REX_OK;
}

}  // namespace

struct rex_multi {
  int precision;
  int mode;                      // REX_MULTI_PERSISTENT or REX_MULTI_STREAMS
  cudaStream_t side[MULTI_MAX_BATCH];   // stream mode: one forked stream per batch
  cudaEvent_t fork, join[MULTI_MAX_BATCH];
  int device;
  unsigned long long* counter;   // device work counter (scratch), reset by every launch
  int blocks[MULTI_NCLASS][2];   // persistent grid size per register class, without / with complex propagators
  cudaStream_t cap_stream;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  int slot_groups;               // work items per g g tile (rex_multi_set_slot_groups / rex_multi_autotune)
  double tile_us[PROC_LAST + 2]; // measured time of one tile per tile kind (tile_kind), 0 when not measured
};

namespace {

// The tile a process's batch runs on in the persistent kernel: one per process, and a
// second one for the q q~ -> t t~ g channels whose light line is crossed (q g, q~ g and
// their beam swaps: the t-channel tile).
int tile_kind(const rex_proc* p) {
  return (p->kind == PROC_QQ_TTXG && (p->cross.neg[0] || p->cross.neg[1])) ? PROC_LAST + 1 : p->kind;
}

// Cost of one tile of each batch; items are handed out longest tiles first, so that
// short ones fill the tail.  The measured times (rex_multi_autotune,
// rex_multi_set_tile_cost) when every batch with events has one (returns true);
// otherwise an estimate: events per tile x flops per event / issue rate of the pipe
// the tile runs on (FP64 is 1/64 of FP32 on B300; e+e- tiles always run in FP64).
bool tile_costs(const rex_multi* m, const rex_batch* batches, int nbatch, int k, double* cost) {
  bool measured = true;
  for (int i = 0; i < nbatch; ++i) {
    cost[i] = batches[i].nev > 0 ? m->tile_us[tile_kind(batches[i].proc)] : 0.0;
    if (batches[i].nev > 0 && !(cost[i] > 0.0)) measured = false;
  }
  if (measured) return true;
  const int mixed_p = m->precision == REX_MIXED;
  for (int i = 0; i < nbatch; ++i) {
    static const double flops_per_event_slot[PROC_LAST + 1] = {160.0, 5.0e3, 4.8e4, 5.7e5, 3.0, 2.4e4};   // per mass slot
    static const double flops_per_event_fixed[PROC_LAST + 1] = {6.4e3, 4.0e2, 6.6e3, 1.1e5, 6.0e2, 4.0e3};
    const int kind = batches[i].proc->kind;
    const double rate = (kind == PROC_EE_MUMU || !mixed_p) ? 1.0 : 64.0;
    const double slots = kind == PROC_EE_MUMU ? (k < MULTI_MAX_POINTS ? k : MULTI_MAX_POINTS) + 1.0 : 9.0;
    cost[i] = multi_events_per_tile(kind, mixed_p) *
              (flops_per_event_fixed[kind] + slots * flops_per_event_slot[kind]) / rate;
  }
  return false;
}

int multi_impl(rex_multi* m, const rex_batch* batches, int nbatch, const rex_params* pts, int k, void* stream) {
  if (!m) return fail(REX_EINVAL, "null multi handle");
  if (nbatch < 1 || nbatch > MULTI_MAX_BATCH)
    return fail(REX_EINVAL, "nbatch must be in [1, %d] (got %d)", MULTI_MAX_BATCH, nbatch);
  if (!batches) return fail(REX_EINVAL, "null batch array");
  if (k < 0) return fail(REX_EINVAL, "k < 0");
  if (k > 0 && !pts) return fail(REX_EINVAL, "null parameter array");
  int nee = 0;
  for (int i = 0; i < nbatch; ++i) {
    const rex_batch& b = batches[i];
    int rc = validate_proc(b.proc);
    if (rc) return rc;
    // ee_mumu is FP64 only and its tile always runs in FP64: it may join a mixed launch
    if (b.proc->precision != m->precision && b.proc->kind != PROC_EE_MUMU)
      return fail(REX_EINVAL, "batch %d precision differs from the multi handle", i);
    if (!b.proc->has_orig) return fail(REX_ENOTINIT, "batch %d: rex_set_params has not been called", i);
    if (b.nev < 0) return fail(REX_EINVAL, "batch %d: nev < 0", i);
    if (b.nev > 0 && (!b.momenta || !b.w_in || !b.w_out)) return fail(REX_EINVAL, "batch %d: null array", i);
    if (b.nev > 0 && (!aligned16(b.momenta) || !aligned8(b.w_in) || !aligned8(b.w_out)))
      return fail(REX_EINVAL, "batch %d: misaligned array", i);
    if (b.proc->kind == PROC_EE_MUMU) ++nee;
    for (int j = 0; j < k; ++j) {
      rc = b.proc->kind == PROC_EE_MUMU ? check_ew_point(pts[j]) : check_qcd_point(pts[j]);
      if (rc) return rc;
    }
  }
  if (nee > 1) return fail(REX_EINVAL, "at most one ee_mumu batch per multi launch");
  if (k == 0) return REX_OK;
  if (const int pe = pending_error()) return pe;
  if (m->mode == REX_MULTI_STREAMS) {
    // fork: every batch's own tuned single-process kernel on its side stream; join
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaEventRecord(m->fork, st);
    if (e != cudaSuccess) return cuda_fail((int)e, "fork event");
    for (int i = 0; i < nbatch; ++i) {
      if (batches[i].nev == 0) continue;
      e = cudaStreamWaitEvent(m->side[i], m->fork, 0);
      if (e != cudaSuccess) return cuda_fail((int)e, "fork wait");
      const int rc = reweight_impl(batches[i].proc, batches[i].momenta, batches[i].w_in, batches[i].nev, pts, k,
                                   batches[i].w_out, m->side[i]);
      if (rc) return rc;
      e = cudaEventRecord(m->join[i], m->side[i]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st, m->join[i], 0);
      if (e != cudaSuccess) return cuda_fail((int)e, "join");
    }
    return REX_OK;
  }
  // longest tiles first: items are handed out in this order
  double tile_cost[MULTI_MAX_BATCH];
  tile_costs(m, batches, nbatch, k, tile_cost);
  int order[MULTI_MAX_BATCH];
  for (int i = 0; i < nbatch; ++i) order[i] = i;
  for (int i = 0; i < nbatch; ++i)
    for (int j = i + 1; j < nbatch; ++j)
      if (tile_cost[order[j]] > tile_cost[order[i]]) std::swap(order[i], order[j]);
  const int mixed = m->precision == REX_MIXED;
  static thread_local MultiLaunch ml;   // ~20 KB: kept off the stack
  bool forked = false;
  // one persistent launch per register class present, heaviest class first (one graph
  // when captured): each class runs at the occupancy its own tiles allow instead of
  // the heaviest process's.  With side streams (a multi handle) the classes run on
  // streams forked from the caller's, each with its own work counter, so a lighter
  // class fills the SMs the heavier one's blocks leave at its tail; without them
  // (the allocation-free entry point) they run back to back on one counter.
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool fork = m->side[0] != nullptr;
  for (int j0 = 0; j0 < k; j0 += MULTI_MAX_POINTS) {
    const int j1 = (k - j0) < MULTI_MAX_POINTS ? k : j0 + MULTI_MAX_POINTS;
    for (int cls = MULTI_NCLASS - 1; cls >= 0; --cls) {
      std::memset(&ml, 0, sizeof ml);
      int64_t total = 0;
      int nb = 0, width = 0;
      for (int oi = 0; oi < nbatch; ++oi) {
        const rex_batch& b = batches[order[oi]];
        if (b.nev == 0 || multi_class_of(b.proc->kind) != cls) continue;
        MultiBatch& B = ml.b[nb++];
        B.kind = b.proc->kind;
        B.cross = b.proc->cross;
        B.nev = b.nev;
        B.mom = b.momenta;
        B.w_in = b.w_in;
        B.out = b.w_out + j0;
        const int epb = multi_events_per_tile(B.kind, mixed);
        B.ngroup = 1;
        if (B.kind == PROC_EE_MUMU) {
          ml.ew.k = j1 - j0;
          ml.ew.mode = OUT_RATIO;
          ml.ew.out_stride = k;
          ml.ew.pt[0] = ew_point(b.proc->orig);
          for (int j = j0; j < j1; ++j) ml.ew.pt[1 + j - j0] = ew_point(pts[j]);
        } else {
          fill_multi_table(b.proc, pts, j0, j1, k, B.t);
          if (B.t.has_width) width = 1;
          // g g batches: the handle's slot groups per tile, at most one slot each
          const bool gg = B.kind == PROC_GG_TTX || B.kind == PROC_GG_TTXG || B.kind == PROC_GG_TTXGG;
          if (gg && m->slot_groups > 1 && B.t.nmass > 2)
            B.ngroup = m->slot_groups < B.t.nmass - 1 ? m->slot_groups : B.t.nmass - 1;
        }
        B.tile_begin = total;
        total += (b.nev + epb - 1) / epb * B.ngroup;
        B.tile_end = total;
      }
      if (nb == 0) continue;
      ml.nbatch = nb;
      ml.total = total;
      const int64_t grid = total < m->blocks[cls][width] ? total : m->blocks[cls][width];
      void* ls = stream;
      unsigned long long* counter = m->counter;
      if (fork) {
        cudaError_t e = cudaSuccess;
        if (!forked) {
          e = cudaEventRecord(m->fork, st);
          forked = true;
        }
        if (e == cudaSuccess) e = cudaStreamWaitEvent(m->side[cls], m->fork, 0);
        if (e != cudaSuccess) return cuda_fail((int)e, "fork");
        ls = m->side[cls];
        counter = m->counter + cls;
      }
      const int err = launch_multi(mixed, width, cls, (int)grid, ml, counter, ls);
      if (err != 0) return cuda_fail(err, "multi kernel launch");
      if (fork) {
        cudaError_t e = cudaEventRecord(m->join[cls], m->side[cls]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, m->join[cls], 0);
        if (e != cudaSuccess) return cuda_fail((int)e, "join");
      }
    }
    // the next 64-point chunk re-forks after this one's joins
    forked = false;
  }
  return REX_OK;
}

int ensure_host_pipeline(rex_proc* p) {
  if (p->hs[0]) return REX_OK;
  cudaError_t e = cudaEventCreateWithFlags(&p->hfork, cudaEventDisableTiming);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&p->hs[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->hjoin[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) return REX_OK;
  for (int i = 0; i < 2; ++i) {
    if (p->hs[i]) cudaStreamDestroy(p->hs[i]);
    if (p->hjoin[i]) cudaEventDestroy(p->hjoin[i]);
    p->hs[i] = nullptr;
    p->hjoin[i] = nullptr;
  }
  if (p->hfork) cudaEventDestroy(p->hfork);
  p->hfork = nullptr;
  return cuda_fail((int)e, "host-copy pipeline streams");
}

}  // namespace

extern "C" {

int rex_multi_create(int precision, rex_multi** out) {
  if (!out) return fail(REX_EINVAL, "null output handle pointer");
  *out = nullptr;
  if (precision == REX_DF64)
    return fail(REX_EUNSUPPORTED, "the persistent multi-process kernels are built in FP64 and mixed precision");
  if (precision != REX_FP64 && precision != REX_MIXED) return fail(REX_EINVAL, "unknown precision %d", precision);
  rex_multi* m = new (std::nothrow) rex_multi;
  if (!m) return fail(REX_ENOMEM, "out of host memory");
  std::memset(m, 0, sizeof *m);
  m->precision = precision;
  cudaError_t e = cudaGetDevice(&m->device);
  if (e == cudaSuccess) e = dev_malloc(&m->counter, 256);
  if (e != cudaSuccess) {
    delete m;
    return fail(REX_ENOMEM, "work-counter allocation failed: %s", cudaGetErrorString(e));
  }
  for (int c = 0; c < MULTI_NCLASS; ++c)
    for (int w = 0; w < 2; ++w) {
      const int err = multi_grid_size(precision == REX_MIXED, w, c, &m->blocks[c][w]);
      if (err != 0) {
        cudaFree(m->counter);
        delete m;
        return cuda_fail(err, "occupancy query");
      }
    }
  e = cudaEventCreateWithFlags(&m->fork, cudaEventDisableTiming);
  for (int i = 0; i < MULTI_MAX_BATCH && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&m->side[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->join[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    rex_multi_free(m);
    return cuda_fail((int)e, "stream/event creation");
  }
  *out = m;
  return REX_OK;
}

int rex_multi_set_mode(rex_multi* m, int mode) {
  if (!m) return fail(REX_EINVAL, "null multi handle");
  if (mode != REX_MULTI_PERSISTENT && mode != REX_MULTI_STREAMS) return fail(REX_EINVAL, "unknown mode %d", mode);
  m->mode = mode;
  return REX_OK;
}

int rex_reweight_multi(rex_multi* m, const rex_batch* batches, int nbatch, const rex_params* param_sets, int k,
                       void* stream) {
  return multi_impl(m, batches, nbatch, param_sets, k, stream);
}

int rex_multi_set_slot_groups(rex_multi* m, int groups) {
  if (!m) return fail(REX_EINVAL, "null multi handle");
  if (groups < 1 || groups > REX_MULTI_MAX_SLOT_GROUPS)
    return fail(REX_EINVAL, "slot groups must be in [1, %d] (got %d)", REX_MULTI_MAX_SLOT_GROUPS, groups);
  m->slot_groups = groups;
  return REX_OK;
}

int rex_multi_get_slot_groups(const rex_multi* m) {
  if (!m) return fail(REX_EINVAL, "null multi handle");
  return m->slot_groups > 1 ? m->slot_groups : 1;
}

int rex_multi_get_tile_cost(const rex_multi* m, const rex_proc* proc, double* us) {
  if (!m) return fail(REX_EINVAL, "null multi handle");
  if (!us) return fail(REX_EINVAL, "null output pointer");
  const int rc = validate_proc(proc);
  if (rc) return rc;
  *us = m->tile_us[tile_kind(proc)];
  return REX_OK;
}

int rex_multi_set_tile_cost(rex_multi* m, const rex_proc* proc, double us) {
  if (!m) return fail(REX_EINVAL, "null multi handle");
  const int rc = validate_proc(proc);
  if (rc) return rc;
  if (!(us >= 0.0) || !std::isfinite(us)) return fail(REX_EINVAL, "tile cost must be finite and >= 0 (got %g)", us);
  m->tile_us[tile_kind(proc)] = us;
  return REX_OK;
}

int rex_multi_autotune(rex_multi* m, const rex_batch* batches, int nbatch, const rex_params* param_sets, int k,
                       void* stream, float* ms_out) {
  if (!m) return fail(REX_EINVAL, "null multi handle");
  static const int cand[REX_MULTI_TUNE_CANDIDATES] = {1, 2, 3, 4, 6, 8};
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_fail((int)e, "autotune events");
  }
  const int keep = m->slot_groups;
  double keep_us[PROC_LAST + 2];
  std::memcpy(keep_us, m->tile_us, sizeof keep_us);
  // mean ms per call of `reps` calls on these batches, after a warm-up call
  auto timed = [&](const rex_batch* b, int nb, int reps, float* ms) -> int {
    int r = multi_impl(m, b, nb, param_sets, k, stream);
    if (r) return r;
    cudaError_t ce = cudaEventRecord(e0, st);
    for (int i = 0; i < reps && r == REX_OK && ce == cudaSuccess; ++i) r = multi_impl(m, b, nb, param_sets, k, stream);
    if (r) return r;
    if (ce == cudaSuccess) ce = cudaEventRecord(e1, st);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    float t = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
    if (ce != cudaSuccess) return cuda_fail((int)ce, "autotune timing");
    *ms = t / reps;
    return REX_OK;
  };
  m->slot_groups = 1;
  int rc = multi_impl(m, batches, nbatch, param_sets, k, stream);   // validates the arguments
  // one tile's time per tile kind, from the first batch of that kind run alone in its
  // persistent launch: with fewer tiles than blocks each tile has a block of its own
  // and the launch lasts one tile, otherwise the blocks share out the tiles
  bool seen[PROC_LAST + 2] = {};
  for (int i = 0; i < nbatch && rc == REX_OK && k > 0; ++i) {
    const rex_batch& b = batches[i];
    const int key = tile_kind(b.proc);
    if (b.nev == 0 || seen[key]) continue;
    seen[key] = true;
    float ms = 0.f;
    rc = timed(&b, 1, 2, &ms);
    if (rc) break;
    const int epb = multi_events_per_tile(b.proc->kind, m->precision == REX_MIXED);
    const double tiles = (double)((b.nev + epb - 1) / epb);
    const int launches = (k + MULTI_MAX_POINTS - 1) / MULTI_MAX_POINTS;
    int width = 0;
    if (b.proc->kind != PROC_EE_MUMU) {
      width = b.proc->orig.wt != 0.0;
      for (int j = 0; j < k; ++j)
        if (param_sets[j].wt != 0.0) width = 1;
    }
    const double grid = m->blocks[multi_class_of(b.proc->kind)][width];
    const double us = 1e3 * ms / launches * (tiles < grid ? tiles : grid) / tiles;
    m->tile_us[key] = us > 0.0 ? us : 1e-3;
  }
  int best = 1;
  float best_ms = 0.f;
  for (int c = 0; c < REX_MULTI_TUNE_CANDIDATES && rc == REX_OK; ++c) {
    m->slot_groups = cand[c];
    float ms = 0.f;
    rc = timed(batches, nbatch, 3, &ms);
    if (rc) break;
    if (ms_out) ms_out[c] = ms;
    if (c == 0 || ms < best_ms) {
      best_ms = ms;
      best = cand[c];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  m->slot_groups = rc == REX_OK ? best : keep;
  if (rc != REX_OK) std::memcpy(m->tile_us, keep_us, sizeof keep_us);
  return rc;
}

int rex_multi_capture(rex_multi* m, const rex_batch* batches, int nbatch, const rex_params* param_sets, int k) {
  if (!m) return fail(REX_EINVAL, "null multi handle");
  if (m->exec) {
    cudaGraphExecDestroy(m->exec);
    m->exec = nullptr;
  }
  if (m->graph) {
    cudaGraphDestroy(m->graph);
    m->graph = nullptr;
  }
  if (!m->cap_stream) {
    const cudaError_t e = cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail((int)e, "capture stream");
  }
  cudaError_t e = cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail((int)e, "cudaStreamBeginCapture");
  const int rc = multi_impl(m, batches, nbatch, param_sets, k, m->cap_stream);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(m->cap_stream, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail((int)e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&m->exec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail((int)e, "cudaGraphInstantiate");
  }
  m->graph = g;
  return REX_OK;
}

int rex_multi_replay(rex_multi* m, void* stream) {
  if (!m) return fail(REX_EINVAL, "null multi handle");
  if (!m->exec) return fail(REX_ENOTINIT, "rex_multi_capture has not been called");
  const cudaError_t e = cudaGraphLaunch(m->exec, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail((int)e, "cudaGraphLaunch");
  return REX_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free multi-process entry point
// ---------------------------------------------------------------------------
// Scratch of rex_reweight_multi_noalloc: the persistent kernel's 64-bit work
// counter, held in this fixed device array instead of a handle's cudaMalloc'd
// buffer.  Every GPU that loads the library holds these 256 bytes until exit.
constexpr int NOALLOC_COUNTERS = 1;   // one 64-point chunk per call; its per-class launches reuse it in stream order
static __device__ __align__(256) unsigned long long g_noalloc_counter[NOALLOC_COUNTERS];

namespace {

constexpr int NOALLOC_MAX_DEVICES = 64;

struct NoallocDevice {
  bool ready;
  unsigned long long* counter;   // device address of g_noalloc_counter on this device
  int blocks[2][MULTI_NCLASS][2];   // persistent grid size [mixed][register class][width]
};

std::mutex g_noalloc_mutex;
NoallocDevice g_noalloc[NOALLOC_MAX_DEVICES];

// Once per device, with that device current: look up the array's device
// address and the persistent grid sizes.  Neither call allocates.
int noalloc_setup(NoallocDevice** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail((int)e, "cudaGetDevice");
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(REX_EINVAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  NoallocDevice& d = g_noalloc[dev];
  if (!d.ready) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_counter);
    if (e != cudaSuccess) return cuda_fail((int)e, "cudaGetSymbolAddress of the static work counter");
    for (int mixed = 0; mixed < 2; ++mixed)
      for (int c = 0; c < MULTI_NCLASS; ++c)
        for (int width = 0; width < 2; ++width) {
          const int err = multi_grid_size(mixed, width, c, &d.blocks[mixed][c][width]);
          if (err != 0) return cuda_fail(err, "occupancy query");
        }
    d.counter = static_cast<unsigned long long*>(ptr);
    d.ready = true;
  }
  *out = &d;
  return REX_OK;
}

}  // namespace

extern "C" {

int rex_reweight_multi_noalloc(const rex_batch* batches, int nbatch, const rex_params* param_sets, int k,
                               int precision, void* stream) {
  if (precision == REX_DF64)
    return fail(REX_EUNSUPPORTED, "the persistent multi-process kernels are built in FP64 and mixed precision");
  if (precision != REX_FP64 && precision != REX_MIXED) return fail(REX_EINVAL, "unknown precision %d", precision);
  if (k > MULTI_MAX_POINTS * NOALLOC_COUNTERS)
    return fail(REX_EINVAL,
                "rex_reweight_multi_noalloc takes at most %d points per call (one launch on its static "
                "work counter); got k = %d: split the points over several calls",
                MULTI_MAX_POINTS * NOALLOC_COUNTERS, k);
  NoallocDevice* d = nullptr;
  const int rc = noalloc_setup(&d);
  if (rc) return rc;
  rex_multi tmp;
  std::memset(&tmp, 0, sizeof tmp);
  tmp.precision = precision;
  tmp.counter = d->counter;
  std::memcpy(tmp.blocks, d->blocks[precision == REX_MIXED], sizeof tmp.blocks);
  return multi_impl(&tmp, batches, nbatch, param_sets, k, stream);
}

void rex_multi_free(rex_multi* m) {
  if (!m) return;
  if (m->exec) cudaGraphExecDestroy(m->exec);
  if (m->graph) cudaGraphDestroy(m->graph);
  if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
  for (int i = 0; i < MULTI_MAX_BATCH; ++i) {
    if (m->side[i]) cudaStreamDestroy(m->side[i]);
    if (m->join[i]) cudaEventDestroy(m->join[i]);
  }
  if (m->fork) cudaEventDestroy(m->fork);
  if (m->counter) cudaFree(m->counter);
  delete m;
}


int rex_init_process(const char* name, int precision, rex_proc** out) {
  if (!out) return fail(REX_EINVAL, "null output handle pointer");
  *out = nullptr;
  if (!name) return fail(REX_EINVAL, "null process name");
  if (precision != REX_FP64 && precision != REX_MIXED && precision != REX_DF64)
    return fail(REX_EINVAL, "unknown precision %d", precision);
  int kind = -1;
  for (const ProcInfo& pi : kProcs)
    if (std::strcmp(pi.name, name) == 0) kind = pi.kind;
  const QqgChannel* channel = nullptr;
  for (const QqgChannel& c : kQqgChannels)
    if (std::strcmp(c.name, name) == 0) {
      kind = PROC_QQ_TTXG;
      channel = &c;
    }
  if (kind < 0) return fail(REX_EINVAL, "unknown process '%s'", name);
  if (kind == PROC_EE_MUMU && precision != REX_FP64)
    return fail(REX_EUNSUPPORTED, "ee_mumu is implemented in FP64 only");
  if (precision == REX_DF64 && kind != PROC_GG_TTX && kind != PROC_GG_TTXG && kind != PROC_QQ_TTXG)
    return fail(REX_EUNSUPPORTED, "REX_DF64 is built for gg_ttx, gg_ttxg, qq_ttxg and its crossings");
  rex_proc* p = new (std::nothrow) rex_proc;
  if (!p) return fail(REX_ENOMEM, "out of host memory");
  std::memset(p, 0, sizeof *p);
  p->kind = kind;
  p->precision = precision;
  p->variant = default_variant(kind, precision);
  if (channel) {
    p->cross = channel->cross;
    p->avg = channel->avg;
  }
  *out = p;
  return REX_OK;
}

int rex_process_npart(const rex_proc* proc) {
  const int rc = validate_proc(proc);
  if (rc) return rc;
  return info_of(proc->kind).npart;
}

int rex_set_flags(rex_proc* proc, unsigned flags) {
  const int rc = validate_proc(proc);
  if (rc) return rc;
  if (flags & ~REX_FLAG_NO_DEDUPE) return fail(REX_EINVAL, "unknown flag bits 0x%x", flags);
  proc->flags = flags;
  return REX_OK;
}

int rex_set_params(rex_proc* proc, const rex_params* original) {
  int rc = validate_proc(proc);
  if (rc) return rc;
  if (!original) return fail(REX_EINVAL, "null parameter pointer");
  rc = proc->kind == PROC_EE_MUMU ? check_ew_point(*original) : check_qcd_point(*original);
  if (rc) return rc;
  proc->orig = *original;
  proc->has_orig = 1;
  return REX_OK;
}

int rex_reweight(rex_proc* proc, const double* momenta, const double* w_in, int64_t nev,
                 const rex_params* param_sets, int k, double* w_out, void* stream) {
  return reweight_impl(proc, momenta, w_in, nev, param_sets, k, w_out, stream);
}

int rex_reweight_helicity(rex_proc* proc, const double* momenta, const signed char* helicities,
                          const double* w_in, int64_t nev, const rex_params* param_sets, int k, double* w_out,
                          void* stream) {
  const int rc = validate_proc(proc);
  if (rc) return rc;
  if (proc->precision == REX_DF64 && proc->kind != PROC_GG_TTXG)
    return fail(REX_EUNSUPPORTED, "helicity-exclusive double-float reweighting is built for gg_ttxg");
  if (proc->kind == PROC_QQ_TTXG && !is_direct(proc->cross))
    return fail(REX_EUNSUPPORTED,
                "helicity-exclusive reweighting of q q~ -> t t~ g is built for the direct channel only; its "
                "crossings evaluate the helicity sum");
  if (nev > 0 && k > 0 && !helicities) return fail(REX_EINVAL, "null helicity array");
  return reweight_impl(proc, momenta, w_in, nev, param_sets, k, w_out, stream, helicities);
}

static int grow(double** buf, size_t* cap, size_t need) {
  if (*cap >= need) return REX_OK;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  const cudaError_t e = dev_malloc(buf, need * sizeof(double));
  if (e != cudaSuccess) {
    *buf = nullptr;
    return fail(REX_ENOMEM, "device allocation of %zu doubles failed: %s", need, cudaGetErrorString(e));
  }
  *cap = need;
  return REX_OK;
}

int rex_reweight_host(rex_proc* proc, const double* momenta, const double* w_in, int64_t nev,
                      const rex_params* param_sets, int k, double* w_out, void* stream) {
  int rc = validate_proc(proc);
  if (rc) return rc;
  if (nev < 0 || k < 0) return fail(REX_EINVAL, "nev < 0 or k < 0");
  if (!proc->has_orig) return fail(REX_ENOTINIT, "rex_set_params has not been called");
  if (nev == 0 || k == 0) return REX_OK;
  if (!momenta || !w_in || !w_out || !param_sets) return fail(REX_EINVAL, "null array pointer");
  const size_t npart = (size_t)info_of(proc->kind).npart;
  const size_t nm = (size_t)nev * npart * 4, nw = (size_t)nev, no = (size_t)nev * (size_t)k;
  if ((rc = grow(&proc->d_mom, &proc->cap_mom, nm))) return rc;
  if ((rc = grow(&proc->d_win, &proc->cap_win, nw))) return rc;
  if ((rc = grow(&proc->d_wout, &proc->cap_wout, no))) return rc;
  if ((rc = ensure_host_pipeline(proc))) return rc;
  // Chunks of events alternate between two streams forked from the caller's: while one
  // chunk's kernel runs, the next chunk's inputs come in and the previous chunk's weights
  // go out (the copy engines of each direction work beside the SMs).  At least 2^16
  // events per chunk, so that a launch still fills the GPU; the two streams' kernels
  // overlap at the chunk boundaries.
  const int64_t chunk = std::max<int64_t>(int64_t(1) << 16, (nev + 7) / 8);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaEventRecord(proc->hfork, st);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(proc->hs[i], proc->hfork, 0);
  if (e != cudaSuccess) return cuda_fail((int)e, "host-copy pipeline fork");
  int c = 0;
  for (int64_t e0 = 0; e0 < nev && rc == REX_OK; e0 += chunk, ++c) {
    const int64_t n = std::min(chunk, nev - e0);
    cudaStream_t cs = proc->hs[c & 1];
    const size_t om = (size_t)e0 * npart * 4, oo = (size_t)e0 * (size_t)k;
    e = cudaMemcpyAsync(proc->d_mom + om, momenta + om, (size_t)n * npart * 4 * sizeof(double),
                        cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(proc->d_win + e0, w_in + e0, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) {
      rc = cuda_fail((int)e, "host-to-device copy");
      break;
    }
    rc = reweight_impl(proc, proc->d_mom + om, proc->d_win + e0, n, param_sets, k, proc->d_wout + oo, cs);
    if (rc) break;
    e = cudaMemcpyAsync(w_out + oo, proc->d_wout + oo, (size_t)n * (size_t)k * sizeof(double),
                        cudaMemcpyDeviceToHost, cs);
    if (e != cudaSuccess) rc = cuda_fail((int)e, "device-to-host copy");
  }
  // join back into the caller's stream (also after an error, so that no copy into the
  // caller's arrays is still in flight when the call returns)
  for (int i = 0; i < 2; ++i) {
    cudaError_t ej = cudaEventRecord(proc->hjoin[i], proc->hs[i]);
    if (ej == cudaSuccess) ej = cudaStreamWaitEvent(st, proc->hjoin[i], 0);
    if (ej != cudaSuccess) {
      cudaStreamSynchronize(proc->hs[i]);
      if (rc == REX_OK) rc = cuda_fail((int)ej, "host-copy pipeline join");
    }
  }
  e = cudaStreamSynchronize(st);
  if (rc != REX_OK) return rc;
  if (e != cudaSuccess) return cuda_fail((int)e, "device-to-host copy");
  return REX_OK;
}

int rex_me2(rex_proc* proc, const double* momenta, int64_t nev, const rex_params* point, double* me2_out,
            void* stream) {
  int rc = validate_proc(proc);
  if (rc) return rc;
  if (nev < 0) return fail(REX_EINVAL, "nev < 0");
  if (!point) return fail(REX_EINVAL, "null parameter pointer");
  rc = proc->kind == PROC_EE_MUMU ? check_ew_point(*point) : check_qcd_point(*point);
  if (rc) return rc;
  if (nev == 0) return REX_OK;
  if (!momenta || !me2_out) return fail(REX_EINVAL, "null array pointer");
  if (!aligned16(momenta) || !aligned8(me2_out)) return fail(REX_EINVAL, "misaligned array pointer");
  if ((rc = pending_error())) return rc;
  // evaluate with the point as the original: slot 0 only
  rex_proc tmp = *proc;
  tmp.orig = *point;
  tmp.has_orig = 1;
  int next = 0;
  return proc->kind == PROC_EE_MUMU
             ? run_ee_chunk(&tmp, momenta, nullptr, nev, point, 0, 0, OUT_ME2, me2_out, 1, stream, &next)
             : run_qcd_chunk(&tmp, momenta, nullptr, nev, point, 0, 0, OUT_ME2, me2_out, 1, stream, &next);
}

int rex_num_variants(const rex_proc* proc) {
  const int rc = validate_proc(proc);
  if (rc) return rc;
  return single_variant(proc) ? 1 : QCD_NVARIANT;
}

int rex_get_variant(const rex_proc* proc) {
  const int rc = validate_proc(proc);
  if (rc) return rc;
  return single_variant(proc) ? 0 : proc->variant;
}

int rex_set_variant(rex_proc* proc, int variant) {
  const int rc = validate_proc(proc);
  if (rc) return rc;
  const int n = single_variant(proc) ? 1 : QCD_NVARIANT;
  if (variant < 0 || variant >= n) return fail(REX_EINVAL, "variant %d out of range [0, %d)", variant, n);
  proc->variant = variant;
  return REX_OK;
}

int rex_autotune(rex_proc* proc, const double* momenta, const double* w_in, int64_t nev,
                 const rex_params* param_sets, int k, double* w_out, void* stream, float* ms_out) {
  int rc = validate_proc(proc);
  if (rc) return rc;
  if (single_variant(proc)) return REX_OK;
  if (nev <= 0 || k <= 0) return fail(REX_EINVAL, "autotune needs nev > 0 and k > 0");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(REX_ECUDA, "cudaEventCreate failed");
  const int keep = proc->variant;
  int best = keep;
  float best_ms = 3.0e38f;
  for (int v = 0; v < QCD_NVARIANT; ++v) {
    proc->variant = v;
    rc = reweight_impl(proc, momenta, w_in, nev, param_sets, k, w_out, stream);   // warm-up
    if (!rc) {
      cudaEventRecord(e0, st);
      rc = reweight_impl(proc, momenta, w_in, nev, param_sets, k, w_out, stream);
      cudaEventRecord(e1, st);
    }
    cudaError_t ce = cudaEventSynchronize(e1);
    if (rc || ce != cudaSuccess) {
      proc->variant = keep;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return rc ? rc : cuda_fail((int)ce, "autotune");
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms_out) ms_out[v] = ms;
    if (ms < best_ms) {
      best_ms = ms;
      best = v;
    }
  }
  proc->variant = best;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return REX_OK;
}

void rex_free_process(rex_proc* proc) {
  if (!proc) return;
  if (proc->d_mom) cudaFree(proc->d_mom);
  if (proc->d_win) cudaFree(proc->d_win);
  if (proc->d_wout) cudaFree(proc->d_wout);
  for (int i = 0; i < 2; ++i) {
    if (proc->hs[i]) cudaStreamDestroy(proc->hs[i]);
    if (proc->hjoin[i]) cudaEventDestroy(proc->hjoin[i]);
  }
  if (proc->hfork) cudaEventDestroy(proc->hfork);
  delete proc;
}

const char* rex_last_error(void) { return g_last_error.c_str(); }

const char* rex_version(void) { return "rex-b300 0.1.0 (sm_103a)"; }

}  // extern "C"
