/*
 * opmm.h -- C ABI of the GB300 OPMM estimation library.
 *
 * The library fits oculomotor plant characteristic (OPC) vectors to recorded
 * saccades: "recorded eye movement data as input ... an OPC vector as output"
 * (paper Sec. 2, "Oculomotor plant mathematical model").  The model is the
 * 18-parameter oculomotor plant (Sec. 2.2.1, Table 1), the estimator the
 * parallel Nelder-Mead search of Sec. 3.3 / Algorithm 1.  All numerical work
 * runs in the library's CUDA kernels on one GPU (sm_103a); there is no CPU
 * fallback: a call on a machine without a usable device fails with
 * OPMM_ECUDA.
 *
 * Conventions
 *  - Every function returns an int status: OPMM_OK (0), OPMM_NOT_READY (1), or
 *    a negative error.  No exception or abort crosses the ABI.  The text of
 *    the calling thread's last error is returned by opmm_last_error.
 *  - Inputs are owned by the caller and only read during the call; outputs
 *    are caller-owned buffers.  Pointers documented as "host or device" may
 *    point to either (the library asks the CUDA runtime which); all pointers
 *    of one kind in one call must be of the same kind.
 *  - OPC vectors are 18 floats in the column order of the paper's example
 *    output (Fig. 4): SE_ag SE_ant LT_ag LT_ant PE_ag PE_ant Vis FV_ag FV_ant
 *    Inert Act_ag Act_ant Deact_ag Deact_ant Step H_ag H_ant W.  Units:
 *    elasticities g/deg, viscosities g*s/deg, inertia g*s^2/deg, the four
 *    activation/deactivation times and the pulse width W in ms, tensions in g
 *    (Table 1's values; the paper states no units, these follow Bahill).
 *  - Positions are in degrees.  A saccade with theta_end < theta_start is
 *    simulated in the mirrored frame and its output mirrored back (Fig. 1
 *    shows the plant for positive saccades).
 *  - A context is not thread-safe except for the serving calls, which may be
 *    made from any thread.
 */
#ifndef OPMM_H
#define OPMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define OPMM_OK 0
#define OPMM_NOT_READY 1     /* serving: result not available yet */
#define OPMM_EINVAL (-1)     /* malformed argument or descriptor */
#define OPMM_ENOMEM (-2)     /* device or pinned host allocation failed */
#define OPMM_ECUDA (-3)      /* CUDA runtime error, or no usable device */
#define OPMM_ETIMEDOUT (-4)  /* a host deadline or a kernel's bounded wait expired */
#define OPMM_EBUSY (-5)      /* serving: admission refused (queue or memory full) */

#define OPMM_NPARAM 18
#define OPMM_MODEL_18 18     /* the 18-parameter OPMM (Sec. 2.2.1) */
/* The 9-parameter OPMM (Sec. 2.2.2, Table 2) on the same plant: nine search
 * coordinates in Table 2's order (K_SE, K_LT, B_AG, B_ANT, B_P, N_C_AG,
 * N_C_ANT, J, N_C_FIX).  The shared K_SE scales K_SE_AG and K_SE_ANT, the
 * shared K_LT scales K_LT_AG and K_LT_ANT; the neural control signal
 * (activation and deactivation times, pulse heights, pulse width) is not
 * estimated and stays at the box centre.  A simplex has 10 vertices and an
 * iteration evaluates 13 trial points, so candidates / 13 simplices run per
 * saccade.  init_opc, when given, must have K_SE_AG == K_SE_ANT and
 * K_LT_AG == K_LT_ANT.  Results are full 18-entry OPC vectors.  Not available
 * with use_surrogate, the request loop or opmm_fit_saccade_static. */
#define OPMM_MODEL_9 9

/* How the box centre (initial OPC vector) is chosen when the caller gives none
 * (Sec. 3.2: the estimator starts from model defaults culled from literature). */
#define OPMM_PULSE_TABLE1 0      /* Table 1 verbatim; W = duration - 6 ms */
#define OPMM_PULSE_CALIBRATED 1  /* Table 1, W = duration - 6 ms, agonist pulse
                                    height set so that the default plant's
                                    saccade from 0 to the amplitude peaks at the
                                    amplitude (Table 1's single 55 g pulse cannot
                                    reach every amplitude) */

typedef struct opmm_ctx opmm_ctx;     /* opaque, library-owned */
typedef struct opmm_plan opmm_plan;   /* opaque, library-owned */

/* One recorded saccade, the OPMM's input in Sec. 3.1 (a saccade extracted
 * from the recording, 1-D horizontal or vertical position).  The window holds fixation, saccade and
 * fixation; the pulse of the neural control signal starts at
 * onset_index / sample_rate_hz. */
typedef struct {
  const float* trace_deg;    /* [n_samples] positions, host or device memory */
  int32_t n_samples;         /* >= 1 */
  float sample_rate_hz;      /* > 0; RK4 uses round(1e4 / rate) substeps per sample */
  int32_t onset_index;       /* 0 <= onset_index < n_samples */
  float theta_start_deg;     /* fixation before the saccade */
  float theta_end_deg;       /* fixation after the saccade */
  float duration_ms;         /* detected duration; nominal W = duration - 6 ms */
} opmm_saccade;

/* Estimator settings (Sec. 3.3, Algorithm 1). */
typedef struct {
  int32_t model;             /* OPMM_MODEL_18 or OPMM_MODEL_9 */
  int32_t candidates;        /* trial points per iteration per saccade; the
                                estimator runs candidates / 22 independent
                                simplices (each iteration of one simplex
                                evaluates its 18 + 4 trial points at once;
                                candidates / 13 with OPMM_MODEL_9) */
  int32_t iterations;        /* iteration cap per simplex (>= 0) */
  float box_lo, box_hi;      /* search box: centre * [box_lo, box_hi], 0 < lo <= 1 <= hi */
  float init_step;           /* initial simplex edge in ln-parameter units (e.g. 0.05) */
  float tol_x, tol_f;        /* exit tolerances: max-norm vertex spread (ln units)
                                and objective spread (deg^2) */
  uint64_t seed;             /* Philox key for the simplex starting points */
  int32_t pulse_init;        /* OPMM_PULSE_* when init_opc is NULL */
  int32_t use_surrogate;     /* 1: centre the box on the surrogate's estimate
                                (requires opmm_surrogate_init or _load) */
  const float* init_opc;     /* nullable, host [n][18] box centres (all > 0) */
} opmm_fit_opts;

/* Result per saccade (Fig. 4: OPC vector and optimisation error). */
typedef struct {
  float opc[18];             /* best OPC vector found */
  float f;                   /* its objective as the search computed it:
                                mean squared error, deg^2, FP32 */
  int32_t iterations_run;    /* iterations of the winning simplex */
  double rms_deg;            /* FP64 recomputation: sqrt(mean squared error) */
  double l1_deg;             /* FP64 recomputation: mean absolute error */
  int32_t status;            /* 0 ok; 1 no finite candidate */
  int32_t winner;            /* index of the winning simplex */
  int32_t evaluations;       /* candidate OPC vectors simulated for this saccade */
  int32_t source;            /* OPMM_SOURCE_*: which search produced opc */
  int32_t pulse_end_evals;   /* of the evaluations, those whose pulse ended
                                inside the recorded window (the sample holding
                                the pulse end is integrated substep by
                                substep); counted like evaluations */
  int32_t reserved;          /* 0 */
} opmm_fit_result;

enum {
  OPMM_SOURCE_PLAIN = 0,     /* box around the given or nominal centres */
  OPMM_SOURCE_SEEDED = 1,    /* narrowed box around the surrogate's estimate */
  OPMM_SOURCE_FALLBACK = 2,  /* plain search run after a seeded fit missed */
  OPMM_SOURCE_REFINED = 3    /* opmm_refine_batch (Levenberg-Marquardt) */
};

/* ------------------------------------------------------------- context */

/* Create a context on CUDA device `device_ordinal`.  Owns a stream, scratch
 * buffers and the autotuner cache. */
int opmm_create(int device_ordinal, opmm_ctx** out);
void opmm_destroy(opmm_ctx* ctx);
/* Message of the last failed call made by the calling thread (never NULL;
 * valid until that thread's next failing call). */
const char* opmm_last_error(const opmm_ctx* ctx);
/* Use the caller's CUDA stream (cudaStream_t) for subsequent calls; NULL
 * restores the context's own stream. */
int opmm_set_stream(opmm_ctx* ctx, void* cuda_stream);

/* Launch-shape override for the search kernel (tuning and testing): variant
 * in [0, count) from opmm_search_variants, or -1 (default) to let plans pick
 * by timing.  All variants of a model compute the same estimator; they differ
 * in simplices per block, register budget and register-lean scheduling. */
int opmm_set_search_variant(opmm_ctx* ctx, int32_t variant);
int opmm_search_variants(int32_t* count);
/* Shape of search variant `variant`: simplices per block and the model whose
 * search coordinates it runs (OPMM_MODEL_18 or OPMM_MODEL_9; a forced variant
 * applies to fits of that model only).  Either output may be NULL.
 * OPMM_EINVAL for a variant out of range. */
int opmm_search_variant_info(int32_t variant, int32_t* simplices_per_block, int32_t* model);
/* How search variant `variant` integrates a candidate (the autotuner's
 * integrator axis): OPMM_WALK_SCALAR (one FMA per matrix element of the
 * one-sample update), OPMM_WALK_PACKED (the same update with two rows per
 * packed FP32 FMA instruction: identical arithmetic, fewer instructions) or
 * OPMM_WALK_LEAN (one phase's propagator live at a time, parameters
 * re-derived when needed).  OPMM_EINVAL for a variant out of range or a NULL
 * output. */
enum { OPMM_WALK_SCALAR = 0, OPMM_WALK_PACKED = 1, OPMM_WALK_LEAN = 2 };
int opmm_search_variant_walk(int32_t variant, int32_t* walk);

/* ------------------------------------------------------------ plant */

/* Simulate n trajectories (the plant of Sec. 2.2.1 integrated by RK4,
 * h ~ 0.1 ms, pulse end split).  Trajectory i uses OPC vector opc[i] and the
 * descriptor sacs[sac_index ? sac_index[i] : i] (its trace pointer is not
 * read).  Output: out_deg[out_offset[i] + k], k < n_samples, positions at
 * t_k = k / rate.
 *   opc:        [n][18] host or device
 *   sacs:       host array of descriptors
 *   sac_index:  nullable host [n]
 *   out_offset: host [n] element offsets into out_deg
 *   out_deg:    host or device, caller-owned
 * n = 0 does nothing and returns OPMM_OK.  Synchronous with respect to the
 * host. */
int opmm_simulate(opmm_ctx* ctx, const float* opc, int32_t n, const opmm_saccade* sacs,
                  int32_t n_sacs, const int32_t* sac_index, const int64_t* out_offset,
                  float* out_deg);

/* Objective of m candidate OPC vectors against one recorded saccade: mean
 * squared error (deg^2) accumulated in FP32 with compensated summation,
 * +inf for candidates outside RK4's stable step range.  opc: [m][18] host or
 * device; out_f: [m] host or device.  m = 0 does nothing (the descriptor is
 * still checked). */
int opmm_score(opmm_ctx* ctx, const float* opc, int32_t m, const opmm_saccade* sac,
               float* out_f);

/* Box centres the estimator would use: the caller's init_opc if given, else
 * Table 1 with W = duration - 6 ms and the agonist pulse chosen by
 * pulse_init.  out_opc: host [n][18].  n = 0 does nothing. */
int opmm_nominal_opc(opmm_ctx* ctx, const opmm_saccade* sacs, int32_t n, int32_t pulse_init,
                     float* out_opc);

/* ---------------------------------------------------------- estimation */

/* Fit every saccade of the batch (Algorithm 1: one optimisation task per
 * saccade, all on the device at once).  sacs: host array; traces host or
 * device.  out: host [n], caller-owned.  Synchronous.  n >= 1: an empty
 * batch is OPMM_EINVAL. */
int opmm_fit_batch(opmm_ctx* ctx, const opmm_saccade* sacs, int32_t n, const opmm_fit_opts* opts,
                   opmm_fit_result* out);

/* Reusable plan for repeated fits of batches of one shape: validates and
 * stages the descriptors, sizes the device buffers, picks the launch shape
 * (autotuned on first use per device and shape class) and captures the whole
 * fit (trace gather, box centres, persistent search, FP64 check) in one CUDA
 * graph.  The descriptors' trace pointers are recorded: each execute re-reads
 * the traces they point to.  opts->init_opc, if given, is copied. */
int opmm_plan_create(opmm_ctx* ctx, const opmm_saccade* sacs, int32_t n, const opmm_fit_opts* opts,
                     opmm_plan** out);
/* Replay the plan's graph and copy the n results to `out` (host). */
int opmm_plan_execute(opmm_plan* plan, opmm_fit_result* out);
/* Launch-shape choice of the plan: simplices per block, threads per block,
 * blocks per SM; and the number of kernels one execute launches. */
int opmm_plan_info(const opmm_plan* plan, int32_t* simplices_per_block, int32_t* threads,
                   int32_t* blocks_per_sm, int32_t* kernels_per_execute);
/* The search variant the plan runs (see opmm_search_variant_info and
 * opmm_search_variant_walk). */
int opmm_plan_variant(const opmm_plan* plan, int32_t* variant);
/* The autotuner's probes for this plan: for each launch-shape variant tried,
 * its id, simplices per block, register bound (minimum resident blocks), the
 * blocks per SM launched, and the probe's device time in ms (iteration cap 2).
 * Writes at most `cap` entries; *count = number of probes (0 when the shape
 * came from the context's cache without a log, or was not tuned). */
int opmm_plan_tuning(const opmm_plan* plan, int32_t* variant, int32_t* simplices_per_block,
                     int32_t* min_blocks, int32_t* blocks_per_sm, float* probe_ms, int32_t cap,
                     int32_t* count);
/* Device time of the persistent search kernel in the last execute, from CUDA
 * events recorded around it on the plan's stream (inside the graph). */
int opmm_plan_last_search_ms(const opmm_plan* plan, float* ms);
void opmm_plan_destroy(opmm_plan* plan);

/* ------------------------------------------------------------ serving */
/* Real-time request loop with continuous batching (the paper's motivation:
 * estimation as fast as the recording, Sec. 5).  Single saccades arrive
 * with opmm_serve_submit; a scheduler thread admits them into device slots
 * while earlier requests are still being searched, advances all resident
 * requests together a few Nelder-Mead iterations per round (search state
 * stays in HBM between rounds), and completes each one after
 * opmm_fit_opts.iterations iterations.  A request's result does not depend
 * on what else is running. */
typedef struct {
  int32_t max_slots;            /* upper bound on requests resident on the device */
  uint64_t max_device_bytes;    /* admission budget for slot state; 0 = half the free HBM */
  int32_t max_queue;            /* queued requests beyond which submit returns OPMM_EBUSY */
  int32_t max_samples;          /* longest accepted trace (<= 16384) */
  int32_t round_iters;          /* iterations per scheduling round (>= 1) */
  int32_t max_admit_per_round;  /* admissions per round (>= 1) */
} opmm_serve_opts;

typedef struct {
  uint64_t submitted, admitted, completed, rejected, rounds;
  int32_t queued, active, slots, reserved;
} opmm_serve_stats;

/* Start the loop with fixed fit options (fit->init_opc, if given, is one
 * host [18] centre used for every request).  The number of slots is
 * min(max_slots, budget / bytes per slot); OPMM_EBUSY if not even one fits. */
int opmm_serve_start(opmm_ctx* ctx, const opmm_serve_opts* cfg, const opmm_fit_opts* fit);
/* Queue one saccade (the trace, host or device, is copied before returning);
 * OPMM_EBUSY when the queue is full (back-pressure), OPMM_EINVAL for a
 * malformed descriptor.  Thread-safe. */
int opmm_serve_submit(opmm_ctx* ctx, const opmm_saccade* sac, uint64_t* ticket);
/* Result of a ticket: OPMM_OK (and the ticket is released), OPMM_NOT_READY
 * (timeout_us == 0), OPMM_ETIMEDOUT (waited timeout_us), OPMM_EINVAL for an
 * unknown ticket.  latency_us (nullable): submit-to-completion time.
 * Thread-safe. */
int opmm_serve_poll(opmm_ctx* ctx, uint64_t ticket, opmm_fit_result* out, int32_t timeout_us,
                    double* latency_us);
int opmm_serve_stats_get(opmm_ctx* ctx, opmm_serve_stats* out);
/* Stop the loop; queued and running requests are dropped. */
int opmm_serve_stop(opmm_ctx* ctx);

/* ------------------------------------------------------------ surrogate */
/* A learned amortised inverse (not in the paper): a multilayer perceptron
 * 512 -> 4 x 512 (GELU) -> 18, BF16 weights with FP32 accumulation on the
 * tensor cores, maps a saccade resampled to 256 points of position and
 * velocity (1 ms apart from onset, position normalised so that the start
 * fixation is 0 and the end fixation 1, velocity = 10 x the per-ms
 * difference) to y with OPC centre = nominal centre * exp(0.2 y).  It only
 * seeds a fit (opmm_fit_opts.use_surrogate) whose box is then narrowed; the
 * plain search is the fallback. */

/* Surrogate-seeded fit with the plain search as fallback and judge: fit all n
 * saccades with `seeded` (use_surrogate must be 1: a narrow box around the
 * network's estimate), then fit every saccade whose seeded result has status
 * != 0 or rms_deg > fallback_rms_deg again with `plain` (use_surrogate must be
 * 0; its init_opc, if given, is indexed by the original saccade index).  A
 * re-fitted saccade keeps whichever result has the lower FP64 rms_deg; its
 * evaluations and pulse_end_evals count both searches and source says which result was kept
 * (OPMM_SOURCE_SEEDED or OPMM_SOURCE_FALLBACK).  n_fallback (nullable)
 * receives the number of saccades re-fitted.  Host descriptors; traces host or
 * device as for opmm_fit_batch.  Errors as for opmm_fit_batch; on error out is
 * unspecified. */
int opmm_fit_batch_seeded(opmm_ctx* ctx, const opmm_saccade* sacs, int32_t n, const opmm_fit_opts* seeded,
                          const opmm_fit_opts* plain, float fallback_rms_deg, opmm_fit_result* out,
                          int32_t* n_fallback);

/* Gradient-based refinement (Sec. 5 proposes testing gradient methods
 * against Nelder-Mead): Levenberg-Marquardt steps on the residual vector
 * theta_k - y_k of each saccade, from start_opc (e.g. a search's or the
 * surrogate's result), in the search's ln coordinates around the box centre,
 * clamped to the box.  The Jacobian is taken by central differences of step
 * fd_step (ln units) through the same RK4 plant, A = J^T J and g = J^T r
 * (FP32 products, compensated sums), (A + lambda D) du = -g with
 * D = diag(max(A_jj, 1e-9 max A_ii)) solved in FP64; a step
 * is kept when it lowers the mean squared error (lambda / 10), else lambda * 10.
 * With OPMM_MODEL_9 the nine Table 2 coordinates are refined (start_opc gives
 * each through its first OPC entry) and the neural signal stays at the centre. */
typedef struct {
  int32_t model;             /* OPMM_MODEL_18 or OPMM_MODEL_9 */
  int32_t iterations;        /* Levenberg-Marquardt iterations, [0, 1e4] */
  float box_lo, box_hi;      /* search box around the centre, as opmm_fit_opts */
  float fd_step;             /* central-difference step, ln units (e.g. 0.01) */
  float lambda0;             /* initial damping (e.g. 1e-3) */
  int32_t pulse_init;        /* OPMM_PULSE_*: centre when centre_opc is NULL */
  const float* centre_opc;   /* nullable, host [n][18] box centres (all > 0) */
} opmm_refine_opts;

/* Refine n saccades from start_opc (host [n][18], all entries > 0) and write
 * one result each: opc, f (MSE of the refined vector, FP64 sum of the FP32
 * trajectory), rms_deg and l1_deg recomputed in FP64 as for the search,
 * iterations_run = accepted steps, evaluations = trajectories simulated
 * (pulse_end_evals of them with the pulse end inside the window), winner 0,
 * source OPMM_SOURCE_REFINED, status 1 when the start cannot be simulated.
 * Descriptors and traces as for opmm_fit_batch.  Errors: OPMM_EINVAL for bad
 * arguments (as opmm_fit_batch for descriptors, box and centres; non-positive
 * or non-finite fd_step or lambda0); OPMM_ECUDA / OPMM_ETIMEDOUT as for
 * opmm_fit_batch; on error out is unspecified. */
int opmm_refine_batch(opmm_ctx* ctx, const opmm_saccade* sacs, int32_t n, const float* start_opc,
                      const opmm_refine_opts* opts, opmm_fit_result* out);

/* ------------------------------------------------------------- front end */

/* Velocity-threshold (I-VT) saccade detection and cleaning of a raw position
 * stream (the paper segments its recordings with I-VT and discards saccades
 * shorter than 6 ms or smaller than 4 deg, Sec. 4; it gives no velocity
 * threshold and no cleaning rule, so both are the caller's).  Step k, between
 * samples k - 1 and k, is fast when both samples are valid (finite and in
 * [valid_min_deg, valid_max_deg]: track loss and blinks appear as NaN or
 * out-of-range positions) and |x_k - x_(k-1)| * fs > threshold_dps, in FP32.
 * A saccade is a maximal run of fast steps [a, b): onset sample s = a - 1,
 * end sample e = b - 1.  It is kept when (e - s) * 1000 / fs >=
 * min_duration_ms, |x_e - x_s| >= min_amplitude_deg, and the window
 * [s - pre_samples, e + post_samples] lies in the stream with every sample
 * valid; that window, with onset index pre_samples, start fixation x_s, end
 * fixation x_e and duration (e - s) / fs, is the descriptor the estimator
 * takes (opmm_saccade). */
typedef struct {
  float threshold_dps;       /* velocity threshold, deg/s (e.g. 30) */
  float min_duration_ms;     /* 6 in the paper */
  float min_amplitude_deg;   /* 4 in the paper */
  float valid_min_deg, valid_max_deg;   /* valid position range, e.g. -90, 90 */
  int32_t pre_samples;       /* window samples before the onset sample */
  int32_t post_samples;      /* window samples after the end sample */
} opmm_ivt_opts;

typedef struct {
  int64_t onset;             /* s: last sample before the movement */
  int64_t end;               /* e: first sample after it */
  int64_t window_start;      /* s - pre_samples */
  int32_t n_samples;         /* window length, e - s + pre + post + 1 */
  int32_t onset_index;       /* s - window_start (= pre_samples) */
  float theta_start_deg;     /* x_s */
  float theta_end_deg;       /* x_e */
  float amplitude_deg;       /* |x_e - x_s| */
  float duration_ms;         /* (e - s) * 1000 / fs */
  float peak_velocity_dps;   /* largest |step| * fs of the run */
  int32_t reserved;          /* 0 */
} opmm_ivt_event;

/* Detect the saccades of stream_deg (n_samples positions at sample_rate_hz,
 * host or device memory, read only).  Writes the first min(max_events, found)
 * kept events to out (host, caller-owned) in onset order and the number found
 * to *n_events.  Errors: OPMM_EINVAL for bad arguments (n_samples < 2,
 * non-positive rate or threshold, negative filters, windows or max_events,
 * valid_min_deg > valid_max_deg); OPMM_ENOMEM when the stream has more than
 * 2^26 runs of fast steps (a threshold below the noise) or scratch allocation
 * fails; OPMM_ECUDA for CUDA errors. */
int opmm_detect_saccades(opmm_ctx* ctx, const float* stream_deg, int64_t n_samples, float sample_rate_hz,
                         const opmm_ivt_opts* opts, opmm_ivt_event* out, int32_t max_events, int32_t* n_events);

/* Fresh weights (uniform +-1/sqrt(512), seeded) and zeroed AdamW state; builds
 * the amplitude -> agonist-pulse table the training data uses. */
int opmm_surrogate_init(opmm_ctx* ctx, uint64_t seed);
/* Number of parameters of the flat FP32 parameter vector: for each hidden
 * layer W [512 out][512 in] then b [512]; then W_out [18][512] and b_out [18]. */
int opmm_surrogate_num_params(int64_t* n);
int opmm_surrogate_get_params(opmm_ctx* ctx, float* out /* host [n] */);
int opmm_surrogate_set_params(opmm_ctx* ctx, const float* in /* host [n] */);
/* Loss (mean over rows and the 18 outputs of (y - t)^2) and its gradient with
 * respect to the flat parameter vector, for m rows of features x [m][512]
 * (rounded to BF16) and targets t [m][18]; m a multiple of 128.  y_out
 * (nullable) receives the network outputs [m][18].  All host memory. */
int opmm_surrogate_grad(opmm_ctx* ctx, const float* x, const float* t, int32_t m, float* loss, float* grad,
                        float* y_out);
/* One AdamW step with a caller-given gradient grad (host [n_params], the flat
 * layout above), as opmm_surrogate_train takes after each batch: step count
 * t += 1; m = 0.9 m + 0.1 g, v = 0.999 v + 0.001 g^2; weight matrices (not
 * biases) w -= lr * weight_decay * w; then every entry
 * w -= lr * (m / (1 - 0.9^t)) / (sqrt(v / (1 - 0.999^t)) + 1e-8), in FP32,
 * and the BF16 working copies are refreshed.  For gradients accumulated
 * outside the library (several batches, another loss).  Errors: OPMM_EINVAL
 * without a surrogate, with a null gradient, lr <= 0 or weight_decay < 0. */
int opmm_surrogate_apply_grad(opmm_ctx* ctx, const float* grad, float lr, float weight_decay);
/* `steps` AdamW steps (betas 0.9, 0.999, eps 1e-8, decoupled weight decay on
 * weight matrices) on fresh batches of `batch` saccades (multiple of 128)
 * generated on the device by the plant itself: rates 250/500/1000 Hz, windows
 * of 40-400 samples, amplitudes log-uniform in 1-40 deg, both directions,
 * hidden OPC = calibrated nominal x U(0.8, 1.2) per entry, N(0, 0.05^2) deg
 * noise; sample i of step s is drawn from Philox4x32-10 (key data_seed,
 * counter sample_base + s * batch + i).  losses (nullable, host [steps]).
 * Deterministic: the same initialisation, data_seed and samples give the
 * same parameters and losses bit for bit, in one call or split over several
 * calls with sample_base continued.  The call returns when every step is
 * done (it uses a stream of its own for the data besides the context's). */
int opmm_surrogate_train(opmm_ctx* ctx, int32_t steps, int32_t batch, float lr, float weight_decay,
                         uint64_t data_seed, int64_t sample_base, float* losses);
/* Box centres the surrogate proposes for n saccades (host descriptors, traces
 * host or device): out_opc host [n][18]. */
int opmm_surrogate_predict(opmm_ctx* ctx, const opmm_saccade* sacs, int32_t n, int32_t pulse_init,
                           float* out_opc);
/* The surrogate's input features of n saccades (host descriptors, traces host
 * or device), as BF16 values widened to float: out host [n][512] (positions
 * 0..255, velocities 256..511). */
int opmm_featurize(opmm_ctx* ctx, const opmm_saccade* sacs, int32_t n, float* out);
/* D[M][N] = A[M][K] . B[N][K]^T on the tensor cores (tcgen05): A, B BF16
 * row-major, D FP32 row-major, all DEVICE pointers (16-byte aligned); M and N
 * multiples of 128, K a multiple of 64.  The surrogate's layer primitive. */
int opmm_gemm_bf16(opmm_ctx* ctx, const void* A, const void* B, int32_t M, int32_t N, int32_t K, float* D);
/* Weights file: 8-byte magic "OPMMSG1", int64 count, float32 parameters. */
int opmm_surrogate_save(opmm_ctx* ctx, const char* path);
int opmm_surrogate_load(opmm_ctx* ctx, const char* path);

/* ------------------------------------------------- allocation-free fit */

/* Fit one saccade without allocating any memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- a real-time loop that must not stall on an allocation
 * (cudaMalloc/cudaFree may synchronise the device), or a program whose device
 * memory belongs to another allocator or a fixed budget.  It needs no
 * context.
 *   sac:        host descriptor; sac->trace_deg must be DEVICE memory
 *   opts:       as for opmm_fit_batch (init_opc, if given, is one host [18]
 *               vector); use_surrogate must be 0
 *   out_device: DEVICE memory for one opmm_fit_result, written by the GPU
 *   cuda_stream: cudaStream_t to run on (NULL = legacy default stream)
 * Limits: n_samples <= 4096 and candidates <= 65536; larger sizes, a host
 * trace or result pointer, or any malformed argument return OPMM_EINVAL
 * before anything runs.  The working memory is one fixed 27,648-byte
 * __device__ array inside the library, held by every GPU that loads the
 * library until the process exits.  Every call (with the device current) looks
 * up that array's address and the search kernel's occupancy for this trace;
 * the first call on a device also loads the library's kernels there, so make
 * it before any stream capture.  Calls share the array: calls that overlap on the GPU race,
 * so run them one at a time (the call returns only after the fit finished).
 * Returns OPMM_ETIMEDOUT if a kernel's bounded wait expired, OPMM_ECUDA on a
 * CUDA error. */
int opmm_fit_saccade_static(const opmm_saccade* sac, const opmm_fit_opts* opts,
                            opmm_fit_result* out_device, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* OPMM_H */
