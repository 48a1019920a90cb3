/*
 * rex.h -- C ABI of the B300 (sm_103a) LO matrix-element reweighting library.
 *
 * What the library computes (paper Sec. 3, the weight factorisation
 * w' = w |M'|^2 / |M|^2, and the teaRex normaliser of Sec. 3.1.1 that maps 1/0 to 0):
 * for every event e of one subprocess and every parameter point j,
 *
 *     w_out[e][j] = w_in[e] * |M(p_e; theta_j)|^2 / |M(p_e; theta_0)|^2
 *                 = 0                       if |M(p_e; theta_0)|^2 == 0,
 *
 * where |M|^2 is the tree-level, helicity-summed (the paper's tool reweights
 * helicity-summed only, Sec. 4.1.2; rex_reweight_helicity gives the
 * helicity-exclusive alternative) and colour-summed squared matrix element,
 * averaged over initial spins and colours, theta_0 the parameter point set
 * with rex_set_params and theta_j the j-th entry of param_sets.
 *
 * Momenta enter exactly as the paper's amplitude bridge receives them
 * (Sec. 4.1.3: only the particle momenta, the flat per-process momentum
 * vector): one flat FP64 array [nev][npart][4] with components
 * (E, px, py, pz) per particle, particles in the order the process name
 * states.  Events must already be sorted into the subprocess and their
 * partons reordered to that order (Rex's eventBelongs, Sec. 2.1.2).
 *
 * Conventions for all calls:
 *  - return value 0 = success, negative = error (REX_E*); rex_last_error()
 *    returns a message for the calling thread's last failure;
 *  - device pointers must be device (or managed) memory of the current
 *    device, 8-byte aligned (momenta 16-byte aligned); the caller owns every
 *    array passed in;
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default
 *    stream); calls taking a stream only enqueue work on it and return
 *    without synchronising; asynchronous kernel faults surface at the
 *    caller's next synchronisation of that stream;
 *  - nev == 0 or k == 0 is a no-op that returns 0;
 *  - non-finite momenta give NaN in that event's outputs (no trap).
 */
#ifndef REX_B300_H
#define REX_B300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define REX_OK 0
#define REX_EINVAL (-1)      /* bad handle, name, size, null or misaligned pointer */
#define REX_ENOTINIT (-2)    /* rex_reweight before rex_set_params */
#define REX_ECUDA (-3)       /* a CUDA call failed; see rex_last_error().  The
                              * reweighting entry points also return it, before
                              * enqueueing anything, when a CUDA error from earlier
                              * work is already pending on the calling thread
                              * (cudaPeekAtLastError); the message says so and the
                              * error is left pending for its owner. */
#define REX_ENOMEM (-4)      /* a library-owned allocation failed; what was
                              * allocated before the failure is released.  For
                              * tests: while the environment variable
                              * REX_FAIL_DEVICE_ALLOC holds n >= 1, the n-th
                              * library-owned device allocation counted from when
                              * it took that value, and every later one while it
                              * keeps it, fails as out of memory without touching
                              * the device. */
#define REX_EUNSUPPORTED (-5) /* precision mode or helicity-exclusive reweighting not
                                 available for this process */

/* Precision modes (the paper's fptype option, Sec. 4.1.2, re-cut for B300,
 * where FP64 issues at 1/64 of the FP32 rate):
 * REX_FP64: every step in FP64.
 * REX_MIXED: wavefunctions, amplitudes, colour sum and helicity sum (whose
 *            terms are non-negative) in FP32; Lorentz invariants and the
 *            weight ratio in FP64 (q q~ -> t t~: FP32 after the momenta,
 *            except the exact FP64 product for points at the original top
 *            mass).  Kernel variants 5-8 of the g g processes put the colour
 *            sum on tensor cores (FP16 hi/lo operands, FP32 accumulation).
 *            The error against FP64 is bounded per process (gg_ttx 1e-5,
 *            gg_ttxg and gg_ttxgg 1e-3, qq_ttx 1e-5, qq_ttxg and every crossing
 *            of it 1e-4, relative per weight).  For the q g and q~ g crossings
 *            this holds for forward light quarks too: when the light line's
 *            gluon has |t| < s' / 256 the kernel splits the light-quark current
 *            along the gluon momentum (J = J' + a q, J' formed in FP64) and
 *            evaluates the part along q through the Ward identity, so the
 *            diagrams on the t-channel gluon no longer cancel in FP32.
 * REX_DF64:  every step of REX_FP64 whose arithmetic is per gluon configuration
 *            (wavefunctions, currents, amplitudes, colour and helicity sums) in
 *            double-float: each quantity the unevaluated sum of two FP32
 *            numbers, 48-bit significands, 7 to 15 FP32 operations per FP64
 *            one (Dekker's sum and the FMA-based exact product); the Lorentz
 *            invariants and the weight ratio stay FP64.  Same 1e-12 bound as
 *            REX_FP64 against the FP64 oracle (a unit roundoff near 2^-48; the
 *            largest error measured over 10^4 (event, mass) values of
 *            g g -> t t~ g is 1.3e-13).  Built for gg_ttx, gg_ttxg, qq_ttxg and
 *            its crossings, one kernel variant, helicity-summed (and
 *            helicity-exclusive for gg_ttxg); REX_EUNSUPPORTED elsewhere and in
 *            the persistent entry points. */
#define REX_FP64 0
#define REX_MIXED 1
#define REX_DF64 2

/* Options (rex_set_flags). */
#define REX_FLAG_NO_DEDUPE 1u  /* evaluate the amplitude once per parameter
                                  point instead of once per distinct (mt, Gamma_t) */

typedef struct rex_proc rex_proc; /* opaque, library-owned */

/* One parameter point.  Fields a process does not use are ignored.
 *   QCD processes (gg_ttx, gg_ttxg, gg_ttxgg, qq_ttx, qq_ttxg and its crossings): mt, wt (top mass and
 *     width, GeV), alphas (strong coupling, fixed; g_s = sqrt(4 pi alphas)).
 *     mt enters the top propagators and the external top spinors; momenta
 *     are kept as given.  qq_ttx has no top propagator: wt is checked and
 *     ignored.
 *   ee_mumu: mz, wz (Z mass and width, GeV), sw2 (sin^2 theta_W),
 *     alpha (electromagnetic coupling); independent inputs, cW^2 = 1 - sW^2. */
typedef struct {
  double mt, wt, alphas;
  double mz, wz, sw2, alpha;
} rex_params;

/* Create a handle for one subprocess.
 * name: "ee_mumu"  e+(1) e-(2) -> mu+(3) mu-(4), photon + Z, massless leptons;
 *       "gg_ttx"   g(1) g(2) -> t(3) t~(4);
 *       "gg_ttxg"  g(1) g(2) -> t(3) t~(4) g(5);
 *       "gg_ttxgg" g(1) g(2) -> t(3) t~(4) g(5) g(6);
 *       "qq_ttxg"  q(1) q~(2) -> t(3) t~(4) g(5), massless light quark,
 *                  five diagrams;
 *       "qxq_ttxg" q~(1) q(2) -> t(3) t~(4) g(5);
 *       "qg_ttxq"  q(1) g(2) -> t(3) t~(4) q(5);   "gq_ttxq"   g(1) q(2) -> t(3) t~(4) q(5);
 *       "qxg_ttxqx" q~(1) g(2) -> t(3) t~(4) q~(5); "gqx_ttxqx" g(1) q~(2) -> t(3) t~(4) q~(5):
 *                  the crossings of qq_ttxg that complete p p -> t t~ + jet with a
 *                  light-quark line, evaluated by its kernels with the event's
 *                  partons read into its slots (spin-colour average 1/96 for the
 *                  q g channels, 1/36 for q q~); helicity-summed only;
 *       "qq_ttx"   q(1) q~(2) -> t(3) t~(4), massless light quark, one
 *                  s-channel gluon (the quark-initiated leading-order
 *                  channel of p p -> t t~; multi-channel samples with p any
 *                  massless QCD parton are the paper's Sec. 4.2 workload).
 * precision: REX_FP64, REX_MIXED or REX_DF64 (gg_ttx, gg_ttxg, qq_ttxg and its
 *            crossings).
 * On success *out receives a handle the caller releases with rex_free_process.
 * Errors: REX_EINVAL (null out, unknown name or precision). */
int rex_init_process(const char *name, int precision, rex_proc **out);

/* Number of particles (npart) of the handle's process, or REX_EINVAL. */
int rex_process_npart(const rex_proc *proc);

/* Set option flags (REX_FLAG_*).  Errors: REX_EINVAL. */
int rex_set_flags(rex_proc *proc, unsigned flags);

/* Set the original parameter point theta_0 (host pointer, copied).
 * This is the point the input weights were generated at (paper Sec. 3.1.1:
 * the normaliser is |M|^2 at the original card).
 * Errors: REX_EINVAL (null pointer, non-positive mass or coupling). */
int rex_set_params(rex_proc *proc, const rex_params *original);

/* Reweight nev events to k parameter points (paper Sec. 3, the factorised
 * weight w' = w |M'|^2/|M|^2; Sec. 3.1.1 normaliser 1/0 -> 0).
 *   momenta    device, [nev][npart][4] FP64, (E, px, py, pz)
 *   w_in       device, [nev] FP64 original weights
 *   param_sets host, [k] points (copied before return)
 *   w_out      device, [nev][k] FP64, row-major (event-major), written
 * One launch evaluates |M|^2 at theta_0 and at every point.  The call only
 * enqueues on stream; it allocates nothing and may be captured in a CUDA graph.
 * Errors: REX_EINVAL, REX_ENOTINIT, REX_ECUDA. */
int rex_reweight(rex_proc *proc, const double *momenta, const double *w_in,
                 int64_t nev, const rex_params *param_sets, int k,
                 double *w_out, void *stream);

/* Helicity-exclusive reweighting: the alternative to the helicity-summed default
 * that MG5aMC reweighting offers (Sec. 4.1.2).  Each event keeps the helicity
 * configuration it was generated with, and
 *     w'_e = w_e |M_h(theta')|^2 / |M_h(theta_0)|^2,   h = the event's configuration,
 * with |M_h|^2 colour-summed (and averaged) as in the helicity sum, so that summing
 * it over configurations gives |M|^2.  A configuration whose |M_h(theta_0)|^2 is 0
 * (in particular one that the chirality of a massless fermion pair forbids) gives 0
 * (Sec. 3.1.1's 1/0 -> 0 rule).
 *   helicities  device, [nev][npart] int8 in the process's particle order:
 *               helicities in the frame of the momenta, +1 / -1 (a positive value
 *               reads as +1, any other as -1); no alignment requirement
 *   other arguments as rex_reweight.
 * Processes: ee_mumu, qq_ttx and qq_ttxg evaluate helicity amplitudes directly
 * (the q q~ -> t t~ g gluon in the helicity basis).  gg_ttx, gg_ttxg and gg_ttxgg
 * evaluate the jamps of every real linear polarisation configuration of the
 * gluons (one lane each) and combine them into the event's helicity amplitude,
 * e_lambda = (e1 - i lambda e2)/sqrt(2) up to a phase, before the colour sum; only
 * the event's own top and antitop helicities are evaluated.  The crossings of
 * qq_ttxg use the helicity sum's freedom in their wavefunctions and return
 * REX_EUNSUPPORTED.  In REX_DF64 only gg_ttxg is built (REX_EUNSUPPORTED for the
 * others).
 * Error against FP64 per weight: the helicity sum's bound of the mode (1e-12 in
 * REX_FP64, the process's REX_MIXED bound), or, for a term far below its event's
 * helicity sum, up to 64 eps (sqrt(kappa_0) + sqrt(kappa_j)) with eps the mode's
 * unit roundoff (2^-48 in REX_DF64) and kappa = |M|^2 / |M_h|^2 at the original point and at point j:
 * the amplitudes that cancel into a small |M_h| are of the size of the whole sum's
 * and leave their rounding on it.
 * Enqueue only.  Errors: REX_EUNSUPPORTED, REX_EINVAL (as rex_reweight, null
 * helicities), REX_ENOTINIT, REX_ECUDA. */
int rex_reweight_helicity(rex_proc *proc, const double *momenta, const signed char *helicities,
                          const double *w_in, int64_t nev, const rex_params *param_sets, int k,
                          double *w_out, void *stream);

/* Same computation with HOST arrays: copies momenta and w_in to the device,
 * reweights, copies w_out back and synchronises stream before returning.
 * The events go in chunks (at least 2^16 events, at most 8 chunks) on two
 * streams of the handle, forked from stream after the work already on it and
 * joined back into it: a chunk's kernel runs while the next chunk's inputs are
 * copied in and the previous chunk's weights copied out.  Page-locked host
 * memory makes the copies asynchronous DMA, which this overlap needs.  Device
 * buffers and the two streams are library-owned, made on first use and kept
 * until rex_free_process.  On an error the call still waits for every copy it
 * had enqueued.  Errors: as rex_reweight, plus REX_ENOMEM. */
int rex_reweight_host(rex_proc *proc, const double *momenta, const double *w_in,
                      int64_t nev, const rex_params *param_sets, int k,
                      double *w_out, void *stream);

/* |M|^2 per event at one parameter point (spin/colour summed and averaged).
 *   momenta device [nev][npart][4]; me2_out device [nev].  Enqueue only.
 * Errors: REX_EINVAL, REX_ECUDA. */
int rex_me2(rex_proc *proc, const double *momenta, int64_t nev,
            const rex_params *point, double *me2_out, void *stream);

/* Kernel thread-mapping variants (QCD processes: lanes per event and
 * register budget, colour form; ee_mumu, qq_ttx and qq_ttxg have one).  Every variant
 * computes the same quantity within its mode's tolerance (the summation order
 * and, for the tensor-core variants 5-8 in REX_MIXED, the colour arithmetic
 * differ); they differ in speed.  rex_num_variants returns the count,
 * rex_get_variant / rex_set_variant read and select the handle's variant.
 * Errors: REX_EINVAL (bad handle or index). */
int rex_num_variants(const rex_proc *proc);
int rex_get_variant(const rex_proc *proc);
int rex_set_variant(rex_proc *proc, int variant);

/* Time every variant on the caller's data (one warm-up and one timed launch
 * each, enqueued on stream, which this call synchronises) and keep the
 * fastest in the handle.  Arguments as rex_reweight; w_out is overwritten.
 * ms_out (host, rex_num_variants floats, may be NULL) receives the timings.
 * Errors: as rex_reweight. */
int rex_autotune(rex_proc *proc, const double *momenta, const double *w_in,
                 int64_t nev, const rex_params *param_sets, int k,
                 double *w_out, void *stream, float *ms_out);

/* ---- Several subprocesses in one persistent launch -------------------------
 * The paper reweights subprocesses one after another and finds multi-channel
 * GPU runs latency bound (Sec. 4.2).  rex_reweight_multi instead puts every
 * (batch, event tile) of up to 8 subprocess batches into one persistent grid
 * that takes work items from a device counter, heaviest process first. */
typedef struct rex_multi rex_multi; /* opaque, library-owned */

typedef struct {
  rex_proc *proc;          /* handle: process, original point, flags */
  const double *momenta;   /* device [nev][npart][4] */
  const double *w_in;      /* device [nev] */
  int64_t nev;
  double *w_out;           /* device [nev][k], written */
} rex_batch;

/* Create a multi-launch handle for one precision (all its batches' handles
 * must have it, except ee_mumu batches, which are always FP64).  Allocates a small device work counter (scratch) on the
 * current device, so call it outside stream capture.
 * Errors: REX_EINVAL, REX_ENOMEM, REX_ECUDA. */
int rex_multi_create(int precision, rex_multi **out);

/* Execution mode of a multi handle (rex_multi_set_mode; errors: REX_EINVAL):
 * REX_MULTI_PERSISTENT (default): persistent kernels over the batches' event
 *   tiles, fed by the device work counter, one per register class present
 *   (e+e-, g g -> t t~ and q q~ -> t t~; g g -> t t~ g and q q~ -> t t~ g;
 *   g g -> t t~ g g), heaviest first, back to back on the stream, so light
 *   batches keep the occupancy of their own kernels;
 * REX_MULTI_STREAMS: each batch's own tuned single-process kernel on a
 *   stream forked from (and joined back into) the caller's stream. */
#define REX_MULTI_PERSISTENT 0
#define REX_MULTI_STREAMS 1
int rex_multi_set_mode(rex_multi *m, int mode);

/* Reweight every batch to the same k points (host array, copied).  Each
 * batch's original point is its handle's.  Enqueues a counter reset and one
 * kernel per 64 points and register class present on stream; allocates
 * nothing, so it can be captured.
 * At most one ee_mumu batch.  Errors: REX_EINVAL, REX_ENOTINIT, REX_ECUDA. */
int rex_reweight_multi(rex_multi *m, const rex_batch *batches, int nbatch,
                       const rex_params *param_sets, int k, void *stream);

/* Slot groups of the persistent mode (the paper's observation that small
 * subprocess batches leave a GPU latency bound, Sec. 4.2): each g g tile's
 * distinct top-mass slots (beyond the original one) are split over `groups` work
 * items, each of which evaluates the original slot and its share and writes the
 * weights at those slots.  A batch of few tiles then spreads over more SMs, at
 * the cost of re-evaluating the original slot once per group; large batches lose
 * by it.  groups in [1, REX_MULTI_MAX_SLOT_GROUPS] (default 1; at most one slot
 * per group is used).  Errors: REX_EINVAL.  rex_multi_get_slot_groups returns the
 * setting (or REX_EINVAL). */
#define REX_MULTI_MAX_SLOT_GROUPS 16
int rex_multi_set_slot_groups(rex_multi *m, int groups);
int rex_multi_get_slot_groups(const rex_multi *m);

/* Tile costs of the persistent mode.  Its work items are handed out longest
 * tiles first, so that short ones fill the tail.  The cost is one value per tile
 * kind: one per process, plus one for the q q~ -> t t~ g channels whose light
 * line is crossed (q g, q~ g and their beam swaps run on a tile of their own).
 * A launch orders its batches by the measured costs when every batch with events
 * has one; otherwise by an estimate from counted flops per event and the issue
 * rate of the pipe each tile runs on.
 * rex_multi_get_tile_cost writes the cost of proc's tile kind to *us (host; 0 if
 * not measured).  rex_multi_set_tile_cost sets it (us finite and >= 0; 0 clears
 * it), e.g. from a stored tuning.  Costs are in microseconds of one block and
 * depend on the point list they were measured with.  Errors: REX_EINVAL. */
int rex_multi_get_tile_cost(const rex_multi *m, const rex_proc *proc, double *us);
int rex_multi_set_tile_cost(rex_multi *m, const rex_proc *proc, double us);

/* Tune the persistent mode by measurement, in two steps.
 * 1. Tile costs: the first batch of each tile kind runs alone in its persistent
 *    launch (a warm-up and two timed launches).  Its time, times the blocks its
 *    tiles occupied, divided by its tiles, is stored as that kind's cost.
 * 2. Slot groups: rex_reweight_multi runs with these arguments for each of 1, 2,
 *    3, 4, 6 and 8 groups (a warm-up and three timed launches each).  The fastest
 *    is kept in the handle, and the mean times (ms, REX_MULTI_TUNE_CANDIDATES
 *    floats) go to ms_out (host, may be NULL).
 * Timing uses CUDA events on stream.  Overwrites the batches' w_out and
 * synchronises stream.  On an error the handle keeps its earlier settings.
 * Errors: as rex_reweight_multi. */
#define REX_MULTI_TUNE_CANDIDATES 6
int rex_multi_autotune(rex_multi *m, const rex_batch *batches, int nbatch,
                       const rex_params *param_sets, int k, void *stream, float *ms_out);

/* Capture one rex_reweight_multi call (same arguments) into a CUDA graph kept
 * in the handle, replacing any earlier capture; rex_multi_replay launches it
 * on stream.  The graph reads the batch pointers given at capture time.
 * Errors: as rex_reweight_multi; rex_multi_replay: REX_ENOTINIT, REX_ECUDA. */
int rex_multi_capture(rex_multi *m, const rex_batch *batches, int nbatch,
                      const rex_params *param_sets, int k);
int rex_multi_replay(rex_multi *m, void *stream);

/* Release a multi handle (NULL is ignored). */
void rex_multi_free(rex_multi *m);

/* Allocation-free form of rex_reweight_multi.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc, and so
 * cannot create the rex_multi handle (whose creation allocates its device
 * work counter).  Such callers are applications whose device memory belongs
 * to a framework's caching allocator or to a fixed budget (a serving process
 * that sizes its memory once at start-up, a plug-in inside a host program that
 * owns the device), which forbid allocations made outside it.
 *
 * Same computation and arguments as rex_reweight_multi, with the precision
 * given here instead of by a handle.  The caller still owns and passes every
 * input and output.  The only scratch, the persistent kernel's 64-bit work
 * counter, lives in a static device array that every GPU which loads the
 * library holds until the process exits; the call allocates nothing and
 * calls no allocating routine.
 *
 * Limits: at most 64 points per call (one launch on the one static counter)
 * and 8 batches; a larger k is rejected with REX_EINVAL and a message.
 * Set-up: the first call on each device (with that device current) looks up
 * the counter's device address with cudaGetSymbolAddress and the persistent
 * grid size; make that first call before any stream capture.  Each call
 * clears the counter on stream before its kernel.  Every call shares the same
 * counter, so calls whose kernels overlap on the GPU race with each other:
 * enqueue them on one stream, or otherwise serialise them.
 * Errors: REX_EINVAL, REX_ENOTINIT, REX_ECUDA. */
int rex_reweight_multi_noalloc(const rex_batch *batches, int nbatch,
                               const rex_params *param_sets, int k,
                               int precision, void *stream);

/* ---- Reweighted cross sections (Sec. 3.1.2) --------------------------------
 * For a sample with cross section sigma, error dsigma, original weights w_i and
 * reweighted weights w'_ij (i = events, j = points):
 *   sigma'_j  = C sum_i w'_ij,  C = sigma / sum_i w_i (the sample's normalisation);
 *   dsigma'_j = dsigma * mean_i(w'_ij / w_i) + sigma * std_i(w'_ij),
 * with std the population standard deviation and the mean of w'/w taken over
 * the events with w_i != 0.  When dsigma'_j is infinite, NaN or non-positive it
 * is replaced by dsigma * max(sigma'_j / sigma, sigma / sigma'_j) and the
 * point's fallback flag is set.
 * The statistics accumulate in FP64 over any number of calls (a sample spread
 * over several processes or batches) in a fixed order: results are bitwise
 * reproducible.  Calls on one handle must be issued on one stream (or
 * otherwise serialised).  Errors: REX_EINVAL, REX_ENOMEM, REX_ECUDA; the message
 * is in rex_xsec_last_error(). */
typedef struct rex_xsec rex_xsec; /* opaque, library-owned */

const char *rex_xsec_last_error(void);

/* Accumulator for k points (1 <= k <= 2^20), zeroed; device memory owned by the handle. */
int rex_xsec_create(int k, rex_xsec **out);

/* Zero the accumulator (enqueued on stream). */
int rex_xsec_reset(rex_xsec *x, void *stream);

/* Add nev events: w_in (device [nev]) and w_out (device [nev][k], e.g. the
 * rex_reweight output).  Enqueued on stream; nev = 0 is a no-op.  Growing the
 * internal partials buffer (a call with more events than any before)
 * synchronises stream. */
int rex_xsec_accumulate(rex_xsec *x, const double *w_in, const double *w_out, int64_t nev, void *stream);

/* sigma'_j, dsigma'_j (host [k]) and fallback flags (host [k], may be NULL) of
 * everything accumulated so far; synchronises stream. */
int rex_xsec_result(rex_xsec *x, double sigma, double dsigma, double *sigma_out, double *dsigma_out,
                    int *fallback, void *stream);

/* The accumulator's statistics as 5k + 3 doubles: per point j, (n, mean of w',
 * sum of squared deviations of w', sum of w', sum of w'/w), then (events, events
 * with w != 0, sum of w).  get_state copies them to host and synchronises stream;
 * set_state replaces them from host and synchronises stream.  Used to combine the
 * accumulations of several GPUs (one process per GPU): every rank gathers all
 * states and merges them in rank order with rex_xsec_merge_states. */
int rex_xsec_get_state(rex_xsec *x, double *state, void *stream);
int rex_xsec_set_state(rex_xsec *x, const double *state, void *stream);

/* out = state a merged with state b (host arrays of 5k + 3 doubles; out may be a
 * or b), with the pairwise update of Chan, Golub & LeVeque for the moments.  Host
 * only: needs no GPU. */
int rex_xsec_merge_states(const double *a, const double *b, int k, double *out);

void rex_xsec_free(rex_xsec *x);

/* ---- LHE front-end (host; Sec. 2 and Sec. 3.1) ------------------------------
 * Reads an LHE v3 file, selects the events of one process by their external
 * legs and hands their momenta to the reweighting calls in the process's parton
 * order (the paper's eventBelongs sorting, parton reindexing and transposition
 * to a structure of arrays), and writes the file back with new weights appended
 * to every event (<rwgt><wgt id='ID'> %+.10e </wgt>) and declared in the header
 * (<initrwgt><weightgroup name='rex_b300'><weight id='ID'>ID</weight>).  Nothing
 * else of the file changes.  Host memory only; no GPU needed.  Errors:
 * REX_EINVAL (unreadable or malformed file, bad argument), REX_ENOMEM; the
 * message is in rex_lhe_last_error(). */
typedef struct rex_lhe rex_lhe; /* opaque, library-owned */

const char *rex_lhe_last_error(void);

/* Parse path with nthreads threads (<= 0: all hardware threads). */
int rex_lhe_read(const char *path, int nthreads, rex_lhe **out);

int64_t rex_lhe_num_events(const rex_lhe *lhe);

/* The events whose status -1 particles carry the PDG codes pdg_in[n_in] and whose
 * status +1 particles carry pdg_out[n_out] (as multisets; other statuses are
 * ignored), in file order.  Writes *nev; if momenta is not NULL, the momenta
 * (E, px, py, pz) in the order pdg_in then pdg_out, identical codes in file order
 * (host [nev][n_in + n_out][4]); if weights is not NULL, each event's xWgtUP
 * (host [nev]); if index is not NULL, each event's position in the file (host
 * [nev]).  Call with NULL arrays to size them. */
int rex_lhe_extract(const rex_lhe *lhe, const int *pdg_in, int n_in, const int *pdg_out, int n_out,
                    int64_t *nev, double *momenta, double *weights, int64_t *index);

/* The same events in the same order, with each particle's SPINUP (the LHE helicity
 * column) rounded to an integer: host int8 [nev][n_in + n_out] in the order of
 * rex_lhe_extract, the layout rex_reweight_helicity takes once copied to the
 * device.  +1 / -1 are helicities; 9 means unknown (the LHE convention; also
 * written for a particle line without the column).  Call with NULL to size. */
int rex_lhe_extract_helicities(const rex_lhe *lhe, const int *pdg_in, int n_in, const int *pdg_out,
                               int n_out, int64_t *nev, signed char *helicities);

/* Set weight id (plain text, no quotes or markup) of the events at positions
 * index[n] (host) to values[n] (host).  Ids are written in the order of their
 * first call; an event without a value for an id gets no line for it. */
int rex_lhe_set_weights(rex_lhe *lhe, const char *id, const int64_t *index, const double *values, int64_t n);

/* Write the file with the weights inserted. */
int rex_lhe_write(const rex_lhe *lhe, const char *path);

void rex_lhe_free(rex_lhe *lhe);

/* ---- Learned surrogate of the weight ratio ---------------------------------
 * The paper has no learned component.  An MLP (22 inputs -> 4 hidden layers of
 * 256 with GELU in its tanh form, z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))) / 2
 * -> 2 outputs) predicts r = log(|M(p;theta)|^2/|M(p;theta_0)|^2)
 * for g g -> t t~ g events (inputs: the 20 momentum components in TeV,
 * (mt - 173)/3, (alphas - 0.118)/0.008) and an estimate of its own absolute
 * error.  Weights are FP32 masters with BF16 copies; GEMMs run on tensor cores
 * in BF16 with FP32 accumulation.  Parameter layout (rex_surrogate_num_params
 * floats, every matrix [in][out] row-major): W1 [32][256] (rows 22..31 zero),
 * b1 [256], W2 [256][256], b2, W3, b3, W4, b4, W5 [256][2], b5 [2].
 * Loss: mean of (y - t)^2 + (e - |y - t|)^2, the error head's target held
 * constant; Adam (beta1 0.9, beta2 0.999, eps 1e-8).
 * All calls return REX_OK or a negative REX_E* code; the message of a
 * surrogate call's failure is in rex_surrogate_last_error(). */
typedef struct rex_surrogate rex_surrogate; /* opaque, library-owned */

int64_t rex_surrogate_num_params(void);
const char *rex_surrogate_last_error(void);

/* Create a network with He-normal weights drawn from seed; allocates its
 * parameters, optimiser state and (on demand) work buffers on the current device. */
int rex_surrogate_create(unsigned long long seed, rex_surrogate **out);

/* Copy all parameters from / to a host FP32 array of num_params floats
 * (setting resets the optimiser state).  Synchronises the device. */
int rex_surrogate_set_weights(rex_surrogate *s, const float *host, int64_t n);
int rex_surrogate_get_weights(rex_surrogate *s, float *host, int64_t n);

/* Loss and gradient (no update) of n samples, n a multiple of 32: sample i is
 * momenta[i] (device [n][5][4]) at point (mt[i], alphas[i]) (device) with
 * target log(ratio[i]) (device).  Writes the mean loss (host float) and the
 * gradient (host, num_params floats); synchronises stream. */
int rex_surrogate_loss_grad(rex_surrogate *s, const double *momenta, const double *ratio,
                            const double *mt, const double *alphas, int64_t n,
                            float *loss, float *grad, void *stream);

/* Train for steps Adam steps of batch samples (a multiple of 128) drawn with
 * SplitMix64 from the nev x k pairs (event e, point j) of momenta (device
 * [nev][5][4]) and exact weight ratios ratio (device [nev][k], e.g. rex_reweight
 * output with w_in = 1).  losses (host, steps floats) may be NULL; if given the
 * call synchronises stream. */
int rex_surrogate_train(rex_surrogate *s, const double *momenta, const double *ratio, int64_t nev,
                        const rex_params *param_sets, int k, int steps, int batch, float lr,
                        unsigned long long seed, float *losses, void *stream);

/* Surrogate reweighting of nev events to k points (k <= 4096):
 * pred, err (device [nev][k] floats, may be NULL) receive the predicted log
 * ratio and error estimate; w_out (device [nev][k], may be NULL) receives
 * w_in * exp(pred) (exp in FP32), and then every event with some err > tau (or NaN) is
 * recomputed exactly with the handle exact (rex_reweight on those events), as is
 * every event outside the guard (rex_surrogate_set_guard).
 * n_fallback (host, may be NULL) receives the number of such events.  With
 * w_out set the call synchronises stream (to size the fallback). */
int rex_surrogate_reweight(rex_surrogate *s, rex_proc *exact, const double *momenta,
                           const double *w_in, int64_t nev, const rex_params *param_sets, int k,
                           float tau, double *w_out, float *pred, float *err,
                           int64_t *n_fallback, void *stream);

/* Input-domain guard of the fallback: with y_min > 0, rex_surrogate_reweight also
 * recomputes exactly every event whose final-gluon invariant
 *     y = min over i in {1, 2, t, t~} of 2 k.p_i / s_hat   (k the final gluon,
 *     s_hat = (p_1 + p_2)^2)
 * is below y_min (or NaN).  Small y is the soft and collinear region, where |M|^2
 * is singular and the weight ratio varies fastest with the top mass: the network's
 * largest errors sit there and its error head does not see them.  y_min = 0 (the
 * default) turns the guard off.  Not saved by rex_surrogate_save.
 * Errors: REX_EINVAL (y_min outside [0, 1)). */
int rex_surrogate_set_guard(rex_surrogate *s, double y_min);

/* Choose the fallback threshold tau and the guard for a stated error bound, on a
 * held-out set of nev events (device momenta [nev][5][4]) at k points: with the
 * exact handle's ratios r (rex_reweight, unit weights) as truth, a kept pair
 * "escapes" when |pred - log r| > bound.  Among the candidate guards (off, and the
 * y quantiles 0.25 % .. 50 %) and every threshold, the call picks the pair that
 * keeps the most events while the kept pairs' escape share stays <= max_escape,
 * sets that guard on the handle and returns tau (pass it to rex_surrogate_reweight),
 * the guard, and the fallback share and escape share on this set (host outputs;
 * fallback_out, escape_out may be NULL).  If no event can be kept, tau is -inf
 * (every event falls back).  Allocates work buffers of about 16 nev k bytes and
 * synchronises stream.  Errors: REX_EINVAL, REX_ENOMEM, REX_ECUDA. */
int rex_surrogate_calibrate(rex_surrogate *s, rex_proc *exact, const double *momenta, int64_t nev,
                            const rex_params *param_sets, int k, double bound, double max_escape,
                            float *tau_out, double *guard_out, double *fallback_out, double *escape_out,
                            void *stream);

/* Exact coupling part of the target.  At tree level |M|^2 is proportional to
 * alphas^power (power = 3 for g g -> t t~ g: one factor g_s^2 per QCD vertex
 * pair, Sec. 3), so log r = power * log(alphas / alphas0) + f(p, mt) with
 * f independent of alphas.  After this call the network learns f only:
 * training targets become log(ratio) - power * log(alphas / alphas0), and
 * inference adds the term back to pred (err is unchanged).  power = 0 (the
 * default) learns the whole log ratio.  alphas0 is the original point's
 * alphas.  Errors: REX_EINVAL for power outside 0..8 or alphas0 <= 0. */
int rex_surrogate_set_exact_alphas(rex_surrogate *s, double alphas0, int power);

/* Save the network (parameters, Adam state and step, the exact coupling setting)
 * to a host file, or load one saved by this library (same parameter count).  Both
 * synchronise the device.  Errors: REX_EINVAL (unreadable, unwritable or foreign
 * file), REX_ECUDA. */
int rex_surrogate_save(rex_surrogate *s, const char *path);
int rex_surrogate_load(rex_surrogate *s, const char *path);

/* Inference kernel of rex_surrogate_reweight.
 *   REX_SURROGATE_FUSED (default): one persistent kernel per call; each tile of
 *     128 (event, point) pairs runs all layers on the tcgen05 tensor cores with
 *     the accumulator in tensor memory and the activations in shared memory.
 *   REX_SURROGATE_LAYERED: layer-by-layer mma.sync GEMMs over event chunks, the
 *     activations stored in global memory between layers.
 * Both compute the same network in the same precision (BF16 operands and
 * activations, FP32 accumulation); their results agree to FP32 summation order.
 * With the fused kernel a bounded internal wait that gives up makes the call
 * return REX_ECUDA when it synchronises (w_out set).  Errors: REX_EINVAL. */
#define REX_SURROGATE_FUSED 0
#define REX_SURROGATE_LAYERED 1
int rex_surrogate_set_kernel(rex_surrogate *s, int kind);

void rex_surrogate_free(rex_surrogate *s);

/* Release a handle (NULL is ignored).  Synchronises nothing; the caller must
 * make sure no work enqueued with the handle is still running. */
void rex_free_process(rex_proc *proc);

/* Message of the calling thread's most recent error ("" if none). */
const char *rex_last_error(void);

/* Library version string. */
const char *rex_version(void);

#ifdef __cplusplus
}
#endif

#endif /* REX_B300_H */
