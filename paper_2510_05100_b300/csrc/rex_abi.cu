// C ABI of the reweighting library (declared in include/rex.h).
//
// Host side only: argument validation, the per-launch parameter table
// (distinct mass slots, coupling factors), chunking of large point lists,
// and the kernel launches.  No call here reaches the CPU for any step of the
// computation: every |M|^2 and weight is produced by the kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/rex.h"
#include "generated/qcd_amplitudes.cuh"
#include "rex_internal.cuh"

using namespace rex;

struct rex_proc {
  int kind;
  int precision;
  unsigned flags;
  int has_orig;
  rex_params orig;
  // rex_reweight_host buffers (device), grown on demand
  double* d_mom;
  double* d_win;
  double* d_wout;
  size_t cap_mom, cap_win, cap_wout;
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
};

const ProcInfo& info_of(int kind) { return kProcs[kind]; }

bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// avg * (4 pi alphas)^n / colour_den for a pure-gluon tree amplitude with n gluons
double qcd_factor(const ProcInfo& pi, double alphas) {
  const double gs2 = 4.0 * M_PI * alphas;
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
                  void* stream, int* next_j) {
  const ProcInfo& pi = info_of(p->kind);
  QcdLaunch lp;
  std::memset(&lp, 0, sizeof lp);
  lp.mode = mode;
  lp.out_stride = stride;
  lp.nmass = 1;
  lp.mass[0] = p->orig.mt;
  lp.width[0] = p->orig.wt;
  lp.factor0 = qcd_factor(pi, p->orig.alphas);
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
    lp.factor[j - j0] = qcd_factor(pi, q.alphas);
  }
  lp.k = j - j0;
  for (int s = 0; s < lp.nmass; ++s)
    if (lp.width[s] != 0.0) lp.has_width = 1;
  *next_j = j;
  double* o = (mode == OUT_RATIO) ? out + j0 : out;
  const int err = launch_qcd(p->kind, p->precision == REX_MIXED, mom, w_in, nev, lp, o, stream);
  if (err != 0) return cuda_fail(err, "kernel launch");
  return REX_OK;
}

int run_ee_chunk(rex_proc* p, const double* mom, const double* w_in, int64_t nev,
                 const rex_params* pts, int j0, int j1, int mode, double* out, int64_t stride,
                 void* stream, int* next_j) {
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
  const int err = launch_ee(mom, w_in, nev, lp, o, stream);
  if (err != 0) return cuda_fail(err, "kernel launch");
  return REX_OK;
}

int validate_proc(const rex_proc* p) {
  if (!p) return fail(REX_EINVAL, "null process handle");
  if (p->kind < 0 || p->kind > PROC_GG_TTXGG) return fail(REX_EINVAL, "corrupt process handle");
  return REX_OK;
}

int reweight_impl(rex_proc* p, const double* momenta, const double* w_in, int64_t nev,
                  const rex_params* param_sets, int k, double* w_out, void* stream) {
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
  int j = 0;
  while (j < k) {
    int next = j;
    rc = p->kind == PROC_EE_MUMU
             ? run_ee_chunk(p, momenta, w_in, nev, param_sets, j, k, OUT_RATIO, w_out, k, stream, &next)
             : run_qcd_chunk(p, momenta, w_in, nev, param_sets, j, k, OUT_RATIO, w_out, k, stream, &next);
    if (rc) return rc;
    j = next;
  }
  return REX_OK;
}

}  // namespace

extern "C" {

int rex_init_process(const char* name, int precision, rex_proc** out) {
  if (!out) return fail(REX_EINVAL, "null output handle pointer");
  *out = nullptr;
  if (!name) return fail(REX_EINVAL, "null process name");
  if (precision != REX_FP64 && precision != REX_MIXED) return fail(REX_EINVAL, "unknown precision %d", precision);
  int kind = -1;
  for (const ProcInfo& pi : kProcs)
    if (std::strcmp(pi.name, name) == 0) kind = pi.kind;
  if (kind < 0) return fail(REX_EINVAL, "unknown process '%s'", name);
  if (kind == PROC_EE_MUMU && precision != REX_FP64)
    return fail(REX_EUNSUPPORTED, "ee_mumu is implemented in FP64 only");
  rex_proc* p = new (std::nothrow) rex_proc;
  if (!p) return fail(REX_ENOMEM, "out of host memory");
  std::memset(p, 0, sizeof *p);
  p->kind = kind;
  p->precision = precision;
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

static int grow(double** buf, size_t* cap, size_t need) {
  if (*cap >= need) return REX_OK;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  const cudaError_t e = cudaMalloc(reinterpret_cast<void**>(buf), need * sizeof(double));
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
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(proc->d_mom, momenta, nm * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(proc->d_win, w_in, nw * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail((int)e, "host-to-device copy");
  rc = reweight_impl(proc, proc->d_mom, proc->d_win, nev, param_sets, k, proc->d_wout, stream);
  if (rc) return rc;
  e = cudaMemcpyAsync(w_out, proc->d_wout, no * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
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
  // evaluate with the point as the original: slot 0 only
  rex_proc tmp = *proc;
  tmp.orig = *point;
  tmp.has_orig = 1;
  int next = 0;
  return proc->kind == PROC_EE_MUMU
             ? run_ee_chunk(&tmp, momenta, nullptr, nev, point, 0, 0, OUT_ME2, me2_out, 1, stream, &next)
             : run_qcd_chunk(&tmp, momenta, nullptr, nev, point, 0, 0, OUT_ME2, me2_out, 1, stream, &next);
}

void rex_free_process(rex_proc* proc) {
  if (!proc) return;
  if (proc->d_mom) cudaFree(proc->d_mom);
  if (proc->d_win) cudaFree(proc->d_win);
  if (proc->d_wout) cudaFree(proc->d_wout);
  delete proc;
}

const char* rex_last_error(void) { return g_last_error.c_str(); }

const char* rex_version(void) { return "rex-b300 0.1.0 (sm_103a)"; }

}  // extern "C"
