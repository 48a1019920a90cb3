// Internal launch descriptors shared by the kernels and the C ABI.
#pragma once
#include <cstdint>

namespace rex {

// Distinct (mass, width) evaluations per launch and parameter points per launch.
// The whole table travels as a __grid_constant__ kernel parameter (< 8 KB), so
// a launch needs no device allocation and no host-to-device copy.
constexpr int MAX_MASS = 64;
constexpr int MAX_POINTS = 256;

enum ProcKind : int {
  PROC_EE_MUMU = 0, PROC_GG_TTX = 1, PROC_GG_TTXG = 2, PROC_GG_TTXGG = 3, PROC_QQ_TTX = 4, PROC_QQ_TTXG = 5
};
constexpr int PROC_LAST = PROC_QQ_TTXG;
enum OutMode : int { OUT_RATIO = 0, OUT_ME2 = 1 };

// QCD processes: the amplitude is evaluated once per mass slot (slot 0 is the
// original point) with unit coupling; point j then takes
//   |M|^2_j = acc[slot[j]] * factor[j],  factor = avg * (4 pi alphas)^n / colour_den
// (q q~ -> t t~: avg * (4 pi alphas)^2 * colour sum 2; q q~ -> t t~ g: (4 pi alphas)^3 / 108).
struct QcdLaunch {
  int nmass;
  int k;
  int mode;           // OutMode
  int has_width;      // any non-zero width among the slots
  int64_t out_stride; // row stride of the output (elements)
  double factor0;     // factor of the original point
  double mass[MAX_MASS];
  double width[MAX_MASS];
  int slot[MAX_POINTS];
  double factor[MAX_POINTS];
};

// e+e- -> mu+mu-: per point, couplings of the photon and Z terms (index 0 is
// the original point, 1..k the new ones).
//   amp = e2qq/s (Je.Jm) + sum_{X,Y in L,R} gzz[XY] / (s - mz2 + i mzwz) (JeX.JmY)
struct EwPoint {
  double e2qq;
  double gzz[4];  // LL, LR, RL, RR
  double mz2, mzwz;
  double avg;     // 1/4 spin average times nothing else
};

constexpr int MAX_EW_POINTS = 128;

struct EwLaunch {
  int k;          // new points (table holds k+1 entries)
  int mode;
  int64_t out_stride;
  EwPoint pt[MAX_EW_POINTS + 1];
};

// A channel of q q~ -> t t~ g as its kernel reads an event: slot s of the
// q q~ -> t t~ g record (q in, q~ in, t, t~, g out) takes the event's particle
// src[s], with its momentum negated where neg[s] (a crossed parton: an outgoing
// quark in the q~ slot, an outgoing antiquark in the q slot, an incoming gluon in
// the g slot).  The direct channel is {{0, 1, 2, 3, 4}, {0, 0, 0, 0, 0}}.
struct QqgCrossing {
  signed char src[5];
  signed char neg[5];
};

// Persistent multi-process launch (kernels_multi.cu): up to MULTI_MAX_BATCH
// subprocess batches, up to MULTI_MAX_POINTS points per launch.
constexpr int MULTI_MAX_BATCH = 8;
constexpr int MULTI_MAX_POINTS = 64;

struct MultiTable {     // QCD batch: the QcdLaunch fields a tile reads
  int nmass, k, mode, has_width;
  int64_t out_stride;
  double factor0;
  double mass[MULTI_MAX_POINTS + 1];
  double width[MULTI_MAX_POINTS + 1];
  int slot[MULTI_MAX_POINTS];
  double factor[MULTI_MAX_POINTS];
};

struct MultiBatch {
  int kind;
  QqgCrossing cross;    // q q~ -> t t~ g channels only
  int ngroup;           // g g batches: slot groups per tile (work items per tile); 1 otherwise
  int64_t nev, tile_begin, tile_end;   // work items [tile_begin, tile_end) of the launch
  const double* mom;
  const double* w_in;
  double* out;
  MultiTable t;
};

struct EwTable {        // the e+e- batch (at most one per launch)
  int k, mode;
  int64_t out_stride;
  EwPoint pt[MULTI_MAX_POINTS + 1];
};

struct MultiLaunch {
  int nbatch;
  int64_t total;        // work items
  MultiBatch b[MULTI_MAX_BATCH];
  EwTable ew;
};

// Register classes of the persistent kernel (kernels_multi.cu): the heaviest
// process of a launch selects the instantiation and hence the register budget.
constexpr int MULTI_NCLASS = 3;
int multi_class_of(int kind);
int multi_events_per_tile(int kind, int mixed);
int multi_grid_size(int mixed, int width, int cls, int* blocks);
int launch_multi(int mixed, int width, int cls, int blocks, const MultiLaunch& ml, unsigned long long* counter,
                 void* stream);

// Thread-mapping variants of the QCD kernels (see qcd_kernel.cuh).
constexpr int QCD_NVARIANT = 9;

// Launchers (defined in the kernel translation units).  Return cudaError_t as int.
int launch_gg_ttx(int mixed, int variant, const double* mom, const double* w_in, int64_t nev,
                  const QcdLaunch& lp, double* out, void* stream);
int launch_gg_ttxg(int mixed, int variant, const double* mom, const double* w_in, int64_t nev,
                   const QcdLaunch& lp, double* out, void* stream);
int launch_gg_ttxgg(int mixed, int variant, const double* mom, const double* w_in, int64_t nev,
                    const QcdLaunch& lp, double* out, void* stream);
// Helicity-exclusive reweighting of the g g processes (the events' helicity
// configurations hel [nev][npart], int8, positive: +1, otherwise -1).
// double-float amplitudes (REX_DF64)
int launch_gg_ttx_df64(const double* mom, const double* w_in, int64_t nev, const QcdLaunch& lp, double* out,
                       void* stream);
int launch_gg_ttxg_df64(const double* mom, const double* w_in, int64_t nev, const QcdLaunch& lp, double* out,
                        void* stream);
int launch_gg_ttxg_df64_exclusive(const double* mom, const double* w_in, int64_t nev, const QcdLaunch& lp,
                                  double* out, void* stream, const signed char* hel);
int launch_qq_ttxg_df64(const double* mom, const double* w_in, int64_t nev, const QcdLaunch& lp, double* out,
                        void* stream, const QqgCrossing& cross);
int launch_gg_ttx_exclusive(int mixed, const double* mom, const double* w_in, int64_t nev, const QcdLaunch& lp,
                            double* out, void* stream, const signed char* hel);
int launch_gg_ttxg_exclusive(int mixed, const double* mom, const double* w_in, int64_t nev, const QcdLaunch& lp,
                             double* out, void* stream, const signed char* hel);
int launch_gg_ttxgg_exclusive(int mixed, const double* mom, const double* w_in, int64_t nev, const QcdLaunch& lp,
                              double* out, void* stream, const signed char* hel);
// hel: null for the helicity sum, else the events' helicity configurations
// [nev][npart] (int8, positive: +1, otherwise -1) for helicity-exclusive reweighting.
int launch_qq_ttx(int mixed, const double* mom, const double* w_in, int64_t nev, const QcdLaunch& lp,
                  double* out, void* stream, const signed char* hel);
int launch_qq_ttxg(int mixed, const double* mom, const double* w_in, int64_t nev, const QcdLaunch& lp,
                   double* out, void* stream, const signed char* hel, const QqgCrossing& cross);
int launch_ee(const double* mom, const double* w_in, int64_t nev, const EwLaunch& lp,
              double* out, void* stream, const signed char* hel);

}  // namespace rex
