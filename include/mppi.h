/*
 * mppi.h - C ABI of the GB300 (sm_103a) Hermite-spline MPPI hot path.
 *
 * The library implements one receding-horizon update of "Reference-Free Sampling-Based
 * Model Predictive Control" (arXiv 2511.19204): Alg. 1 (Sec. III-C) with the cubic
 * Hermite knot parameterisation of Sec. III-A, the per-knot noise schedule of Sec. III-B,
 * the min-max softmin weights and knot average of Sec. III-C, and best-trajectory
 * tracking (Sec. III-D). Rollouts use floating-base rigid-body dynamics with soft
 * ground contact in place of the paper's simulator.
 *
 * Conventions used by every entry point:
 *   - Robot state x [nx], FP64 at the boundary, rounded to FP32 on the device:
 *       [p_base(3, world), quat(4: w,x,y,z, Hamilton, body->world), q(nj),
 *        v_base_lin(3, body frame), omega_base(3, body frame), qdot(nj)],
 *     nq = 7 + nj, nv = 6 + nj, nx = nq + nv.
 *   - Knots [nk][2][nj] row-major FP32: [knot][position | velocity][joint]. Knot j sits
 *     at t_j = j * H * dt / (nk - 1) (uniform, both horizon ends included).
 *   - Pointers named h_* are host memory, d_* device memory of the current CUDA device.
 *     Unless stated otherwise the caller owns every buffer it passes; the library
 *     copies inputs before returning and never keeps caller pointers.
 *   - Every call returns an mppi_status: 0 = MPPI_OK, > 0 = MPPI_PENDING, < 0 = error.
 *     No exception crosses the ABI and nothing aborts the process. After
 *     MPPI_ERR_CUDA, mppi_last_error() describes the failing CUDA call.
 *   - A context (mppi_ctx) is not thread-safe; a server (mppi_server) is.
 */
#ifndef MPPI_H_
#define MPPI_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t mppi_status;
#define MPPI_OK 0
#define MPPI_PENDING 1
#define MPPI_ERR_INVALID_ARG (-1)
#define MPPI_ERR_NONFINITE_STATE (-2)
#define MPPI_ERR_ALL_COSTS_NONFINITE (-3)
#define MPPI_ERR_OUT_OF_MEMORY (-4)
#define MPPI_ERR_ADMISSION (-5)
#define MPPI_ERR_TIMEOUT (-6)
#define MPPI_ERR_CUDA (-7)
#define MPPI_ERR_UNSUPPORTED (-8)
#define MPPI_ERR_NOT_FOUND (-9)
#define MPPI_ERR_DEADLINE (-10)   /* a served request waited past the server's deadline and was shed */

/* Rollout mappings (chosen per context, MPPI_MAP_AUTO asks the autotuner). */
#define MPPI_MAP_AUTO (-1)
#define MPPI_MAP_WARP 0       /* one sample per warp, one lane per body             */
#define MPPI_MAP_HALFWARP 1   /* one sample per 16 lanes, one lane per body (nb<=16) */
#define MPPI_MAP_CHAIN 2      /* one sample per 4 lanes, one lane per leg chain (a
                                 floating base with 4 equal 3-body chains)           */
#define MPPI_MAP_THREAD 3     /* reserved: no kernel; contexts reject it (INVALID_ARG) */

/* Weight normalisation. */
#define MPPI_NORM_MINMAX 0    /* Eq. (softmax_minmax): costs min-max normalised first */
#define MPPI_NORM_RAW 1       /* Eq. (omega-weights): exp(-S/lambda)                   */

/* What stays resident as the next solve's warm start. */
#define MPPI_WARM_BEST 0      /* Alg. 1: tau_0 <- tau_best at every control step      */
#define MPPI_WARM_MEAN 1      /* the last weighted mean                               */

/* Spline parameterisation of the joint references (Sec. III-A; the variants of the
 * ablation of Sec. IV-D). Under the position-only variants the velocity knots are not
 * sampled: every sample's (and the nominal's) velocity knots are set to the variant
 * spline's node derivatives, so knots stay [knots][2][nj] and the rollout is the same. */
#define MPPI_SPLINE_HERMITE 0    /* cubic Hermite, positions and velocities sampled     */
#define MPPI_SPLINE_CUBIC 1      /* natural cubic spline through the position nodes     */
#define MPPI_SPLINE_QUADRATIC 2  /* C1 quadratic spline through the nodes, from rest    */

#define MPPI_MAX_BODIES 32
#define MPPI_MAX_CONTACTS 32
#define MPPI_MAX_CHILDREN 8
#define MPPI_MAX_KNOTS 16

/*
 * Robot description. Body 0 is the base (6-DoF floating unless fixed_base != 0); body
 * i >= 1 hangs from parent[i] < i on a revolute joint whose frame sits at jpos[i] in
 * the parent frame, parallel to it at q = 0, rotating by q_i about the unit axis[i]
 * (child coordinates). Joint j (state index) belongs to body j + 1.
 * Inertia of body b: mass[b], centre of mass com[b] (body frame), rotational inertia
 * about it inertia[b] = (Ixx, Iyy, Izz, Ixy, Ixz, Iyz). armature[b] is the joint's
 * reflected rotor inertia. PD gains, torque limits and joint limits are per joint
 * (Eq. pd-controller; Eq. vel-clamp uses q_min/q_max, +-INFINITY disables it).
 * Contacts are points contact_pos[c] on body contact_body[c] against the ground plane
 * z = 0: f_n = max(0, k*depth - c*v_z), f_t = -mu f_n v_t / sqrt(|v_t|^2 + eps_f^2).
 * Cost S = sum_{h<H} c(x_h, u_h) + c_T(x_H) (Sec. IV-A) on the pre-step state of each
 * step. c sums two groups of terms; a zero weight disables its term.
 *  - Quadratic terms of the synthetic workloads: w_z (z - z_des)^2 + w_vx (vx - vx_des)^2
 *    + w_tilt tilt^2 + w_tau |u|^2, with z and tilt of body cost_body and vx the world-x
 *    velocity of the base origin.
 *  - The modular running cost of Sec. IV-A (Eq. running cost): w_h |p_base,z - z_des|
 *    + w_orient ||log3(R_base^T R_des)||^2 + w_q ||q - q_init||^2
 *    + w_cvel sum_c ||v_c||_1 + w_cforce sum_c ||f_c - f0||_1, with R_des the rotation of
 *    the unit quaternion quat_des (w, x, y, z), v_c the world velocity of contact point c
 *    summed over the points in contact (depth > 0), f_c its world contact force (zero
 *    off contact) summed over all points, f0 the same for every point.
 *  - Terminal cost c_T = w_term ||p_base(x_H) - p_target||_1 with
 *    p_target = p_base(x_0) + pdot_des H dt (Sec. IV-A Eq. terminal cost).
 * q_init (nullable, [nj]) seeds the initial nominal theta^q = q_init, theta^v = 0
 * (Alg. 1 initialisation) and is q0 of the w_q term; NULL means zeros. All arrays are
 * read during the call only. Weights must be finite and >= 0.
 */
typedef struct mppi_model_desc {
    int32_t nb;                   /* bodies, 1..MPPI_MAX_BODIES */
    int32_t nc;                   /* contacts, 0..MPPI_MAX_CONTACTS */
    int32_t fixed_base;
    int32_t cost_body;
    const int32_t* parent;        /* [nb], parent[0] = -1 */
    const double* axis;           /* [nb][3] */
    const double* jpos;           /* [nb][3] */
    const double* mass;           /* [nb] */
    const double* com;            /* [nb][3] */
    const double* inertia;        /* [nb][6] */
    const double* armature;       /* [nb] */
    const double* q_min;          /* [nb-1] */
    const double* q_max;          /* [nb-1] */
    const double* kp;             /* [nb-1] */
    const double* kd;             /* [nb-1] */
    const double* tau_max;        /* [nb-1] */
    const int32_t* contact_body;  /* [nc] */
    const double* contact_pos;    /* [nc][3] */
    const double* q_init;         /* [nb-1] or NULL */
    double contact_k, contact_c, mu, eps_f, gravity;
    double z_des, vx_des, w_z, w_vx, w_tilt, w_tau;
    /* modular cost of Sec. IV-A (Tab. II weight sets) */
    double w_h, w_orient, w_q, w_cvel, w_cforce, w_term;
    double quat_des[4];           /* R_des as a quaternion (w, x, y, z), normalised here; all zeros = identity */
    double f0[3];                 /* f0, world frame */
    double pdot_des[3];           /* desired base velocity of p_target, world frame */
} mppi_model_desc;

typedef struct mppi_params {
    double dt;            /* simulation step (s) */
    double scale_q;       /* position-knot noise scale (Alg. 1 scale_q), default 1 */
    double scale_v;       /* velocity-knot noise scale; <= 0 selects 1 / knot spacing */
    int32_t normalize;    /* MPPI_NORM_MINMAX (default) or MPPI_NORM_RAW */
    int32_t warm_from;    /* MPPI_WARM_BEST (default) or MPPI_WARM_MEAN */
    uint64_t seed;        /* Philox key */
    uint32_t instance_id; /* Philox counter word 3: results depend on it, not on scheduling */
    int32_t mapping;      /* MPPI_MAP_* */
    int32_t block_size;   /* threads per block of the rollout kernel, 0 = default */
    int32_t spline;       /* MPPI_SPLINE_* (default MPPI_SPLINE_HERMITE) */
    void* stream;         /* cudaStream_t for all work of this context, NULL = own stream */
} mppi_params;

/* Per-solve information. Costs are the last iteration's unless stated. */
typedef struct mppi_result {
    double cost_min;      /* S_min over finite costs */
    double cost_max;      /* S_max over finite costs */
    double best_cost;     /* lowest cost seen in any iteration of this solve (Sec. III-D) */
    double ess;           /* 1 / sum w^2 */
    double lse;           /* log sum_j exp(-S_hat_j / lambda) */
    int32_t best_index;   /* sample of best_cost (ties -> lowest index) */
    int32_t best_iter;    /* iteration of best_cost */
    int32_t n_finite;     /* finite costs in the last iteration */
    int32_t status;       /* MPPI_OK or MPPI_ERR_ALL_COSTS_NONFINITE */
} mppi_result;

typedef struct mppi_model mppi_model;
typedef struct mppi_ctx mppi_ctx;
typedef struct mppi_server mppi_server;

/* ---------------------------------------------------------------------------------- */
/* Models and contexts                                                                 */
/* ---------------------------------------------------------------------------------- */

/* Validate desc and upload the model's constants to the current device.
 * Errors: INVALID_ARG (sizes, parents, non-unit axes, negative masses, cost_body),
 * OUT_OF_MEMORY, CUDA. *out is owned by the caller (mppi_model_destroy). */
mppi_status mppi_model_create(const mppi_model_desc* desc, mppi_model** out);
void mppi_model_destroy(mppi_model* model);

/* One MPC instance (Alg. 1 parameters): K samples (sample 0 is the unperturbed nominal,
 * Alg. 1 samples n = 1..K-1), H simulation steps, `knots` Hermite knots
 * (2..MPPI_MAX_KNOTS), temperature lambda > 0, `iters` MPPI iterations per solve and
 * the noise schedule sigma_schedule[iters][knots] (standard deviations, rad; the
 * cached table of Eq. overall-noise-kernel). All device buffers are allocated here and
 * owned by the context; the model must outlive it.
 * Errors: INVALID_ARG (K < 1, H < 1, knots out of range, lambda <= 0, sigma < 0 or not
 * finite, dt <= 0, unsupported mapping), OUT_OF_MEMORY, CUDA. */
mppi_status mppi_create(const mppi_model* model, int32_t K, int32_t H, int32_t knots,
                        double lambda, const float* h_sigma_schedule, int32_t iters,
                        const mppi_params* params, mppi_ctx** out);
void mppi_destroy(mppi_ctx* ctx);

/* The annealed noise schedule of Sec. III-B Eq. (overall-noise-kernel), computed once on
 * the host as the paper caches it: h_sigma[it][k] = scale * exp(-(I - i)/(beta1 I) -
 * (K - k)/(beta2 K)) for iterations i = I..1 (row it = I - i: the first iteration uses
 * factor 1 on the trajectory term) and knots k = 0..K-1 (K = knots). The isotropic factor
 * of the covariance is used as the per-knot standard-deviation factor, the table
 * mppi_create takes. Errors: INVALID_ARG (iters, knots < 1, beta <= 0, scale < 0). */
mppi_status mppi_noise_schedule(int32_t iters, int32_t knots, double beta1, double beta2, double scale,
                                float* h_sigma);

/* One MPPI update (Alg. 1 inner loop over `iters` iterations) from state h_state.
 * h_warm_start [knots][2][nj] replaces the resident nominal if non-NULL; NULL keeps the
 * resident one (initially theta^q = q_init, theta^v = 0; after each solve the best
 * knots, or the mean under MPPI_WARM_MEAN). Writes the weighted-mean knots of the last
 * iteration to h_out_mean and, if non-NULL, the best knots (tau_best) to h_out_best and
 * the information to h_info. Blocks until the results are on the host.
 * Errors: INVALID_ARG, NONFINITE_STATE (state not finite, nothing launched),
 * ALL_COSTS_NONFINITE (some iteration had no finite cost; that iteration left the
 * nominal unchanged, outputs are still written), CUDA. */
mppi_status mppi_solve(mppi_ctx* ctx, const double* h_state, const float* h_warm_start,
                       float* h_out_mean, float* h_out_best, mppi_result* h_info);

/* Same update on device-resident data, enqueued on the context's stream without a host
 * synchronisation: d_state [nx] FP64, d_warm_start nullable, d_out_mean [knots*2*nj],
 * d_out_best nullable, d_info nullable (device mppi_result). The CUDA-graph-captured
 * iteration sequence runs as one graph launch. Finiteness of the state is not checked.
 * Errors: INVALID_ARG, CUDA. */
mppi_status mppi_solve_device(mppi_ctx* ctx, const double* d_state, const float* d_warm_start,
                              float* d_out_mean, float* d_out_best, mppi_result* d_info);

/* Wait for all work of the context. */
mppi_status mppi_sync(mppi_ctx* ctx);

/* Rollout step only (Alg. 1 "simulate") on caller-given knots, bypassing the noise:
 * h_knots [K][knots][2][nj] -> h_costs [K] (FP32 sums with Kahan compensation, widened to
 * FP64) and, if non-NULL, h_final_states [K][nx]. Uses the context's rollout mapping. */
mppi_status mppi_rollout_explicit(mppi_ctx* ctx, const double* h_state, const float* h_knots,
                                  double* h_costs, double* h_final_states);

/* Noise step only (Alg. 1 sampling, clamp of Eq. vel-clamp): the knots of iteration
 * `iter` (selects the sigma row) drawn around h_nominal with Philox counter word 2 =
 * iter_counter. h_out [K][knots][2][nj]. */
mppi_status mppi_sample_knots(mppi_ctx* ctx, int32_t iter, uint32_t iter_counter,
                              const float* h_nominal, float* h_out);

/* Counter of the next solve's first iteration (Philox counter word 2); it advances by
 * `iters` per solve. Set it to replay a solve. */
mppi_status mppi_get_iter_counter(const mppi_ctx* ctx, uint32_t* out);
mppi_status mppi_set_iter_counter(mppi_ctx* ctx, uint32_t value);

/* Deterministic resume: the resident warm start and the noise counter, as bytes.
 * Call with buf = NULL to query *len. */
mppi_status mppi_export_state(const mppi_ctx* ctx, void* buf, size_t* len);
mppi_status mppi_import_state(mppi_ctx* ctx, const void* buf, size_t len);

/* ---------------------------------------------------------------------------------- */
/* Receding horizon (Sec. III-E)                                                        */
/* ---------------------------------------------------------------------------------- */

/* State prediction over the compute delay, Eq. of Sec. III-E: the state the robot reaches
 * after `steps` control steps (steps * dt seconds; steps = floor(delay / dt)) from
 * h_state while it executes the resident warm start (tau_best after a solve under
 * MPPI_WARM_BEST), simulated with the rollout's dynamics and PD tracking of the first
 * `steps` of the H steps (FP32; FP64 under mppi_ctx_set_fp64_check). 0 <= steps <= H;
 * steps = 0 returns h_state. h_state, h_out [nx] FP64 host, may alias. Blocks.
 * Errors: INVALID_ARG, NONFINITE_STATE, CUDA, TIMEOUT (a bounded device wait gave up). */
mppi_status mppi_predict_state(mppi_ctx* ctx, const double* h_state, int32_t steps, double* h_out);

/* Same on device buffers, enqueued on the context's stream after any solve enqueued
 * there (so it reads that solve's warm start): d_state, d_out [nx] FP64 device. The
 * result can be passed straight to mppi_solve_device. A bounded-wait failure is
 * reported by the next mppi_sync. Errors: INVALID_ARG, CUDA. */
mppi_status mppi_predict_state_device(mppi_ctx* ctx, const double* d_state, int32_t steps, double* d_out);

/* Shift of the resident warm start by `steps` executed actions, Sec. III-E, with the tail
 * padded. The knots parameterise a spline over T = H dt with knot j at t_j = j T /
 * (knots - 1); the shifted knot j is the old spline's value and time derivative at
 * t_j + steps dt, and past T the final knot is repeated. steps = 0 leaves the knots
 * unchanged; steps >= H repeats the final knot everywhere. Evaluated in FP64 from the
 * FP32 knots, rounded once; enqueued on the context's stream. Errors: INVALID_ARG
 * (steps < 0), CUDA. */
mppi_status mppi_shift_warm_start(mppi_ctx* ctx, int32_t steps);

/* Copy of the resident warm start [knots][2][nj] to h_out (synchronises the stream). */
mppi_status mppi_get_warm_start(const mppi_ctx* ctx, float* h_out);

/* ---------------------------------------------------------------------------------- */
/* Kernel-level entry points (each runs one kernel of the path on host buffers)         */
/* ---------------------------------------------------------------------------------- */

/* The rollout's own FP32 elementary functions (no counterpart in the paper, which leaves
 * the arithmetic to its simulator): sine and cosine (a reduction by pi/2 and Taylor
 * polynomials) and the arctangent of the tilt cost (atan2 for y >= 0) on n argument
 * pairs: h_out [n][3] = (sin x, cos x, atan2(y, x)). For accuracy checks. */
mppi_status mppi_selftest_math(int32_t n, const float* h_x, const float* h_y, float* h_out);

/* The knot average's exact FP32 -> FP64 widening by integer operations (no counterpart in
 * the paper: the FP64 pipe of this part is narrow, so the average converts knots without
 * it): h_out[i] = (double)h_x[i] for every float, NaNs quieted. For exactness checks. */
mppi_status mppi_selftest_widen(int32_t n, const float* h_x, double* h_out);

/* Philox4x32-10 (Salmon et al., SC'11) words for n counters: h_ctr [n][4], key [2],
 * h_out [n][4]. */
mppi_status mppi_philox_words(int32_t n, const uint32_t* h_ctr, const uint32_t* h_key,
                              uint32_t* h_out);

/* Weights of Eq. (softmax_minmax) (normalize = MPPI_NORM_MINMAX) or Eq. (omega-weights)
 * (MPPI_NORM_RAW) for K costs, FP64 log-sum-exp. Non-finite costs get weight 0.
 * h_w [K] FP64. Returns ALL_COSTS_NONFINITE when no cost is finite (w = 0). */
mppi_status mppi_weights(int32_t K, const float* h_costs, double lambda, int32_t normalize,
                         double* h_w, mppi_result* h_info);

/* Eq. (update-nominal) on the knots: h_out[e] = sum_n h_w[n] h_knots[n][e] with FP64
 * accumulation in a fixed order (chunks of 64 samples). h_knots [K][E], h_out [E]. */
mppi_status mppi_average(int32_t K, int32_t E, const float* h_knots, const double* h_w,
                         double* h_out);

/* Allocation-free variant of mppi_average, for callers that cannot call cudaMalloc where
 * they need the average: real-time loops that must not block on the allocator
 * (cudaMalloc / cudaFree can synchronise the device), code with a fixed pre-reserved
 * footprint, hosts whose allocator belongs to another framework. The paper has no
 * counterpart; this is a deployment convenience.
 * d_knots [K][E] FP32, d_w [K] FP64 and d_out [E] FP64 are the caller's device buffers;
 * the work is enqueued on `stream` (cudaStream_t, NULL = legacy default stream) and
 * nothing is allocated or freed. The FP64 partial sums live in one file-scope device
 * array of 2^20 doubles (8 MiB held on every device that loads the library), so
 * ceil(K / 64) * E must not exceed 1048576 (else MPPI_ERR_INVALID_ARG). The first call in
 * each CUDA context looks up that array's device address (cudaGetSymbolAddress, with the
 * device current) and caches it under the context's unique id; a device reset gives the
 * device a new context, whose first call looks the address up again. Make the first call
 * on a device (and the first after a reset) before any stream capture. Every call shares
 * the array and leaves its contents behind; each call writes every element it reads
 * before reading it, so nothing needs clearing, but calls that overlap on the GPU (on
 * different streams) race. Results equal mppi_average's. */
mppi_status mppi_average_noalloc(int32_t K, int32_t E, const float* d_knots, const double* d_w, double* d_out,
                                 void* stream);

/* Bounds-check word of a check build of the library (compiled with -DMPPI_CHECK; no
 * counterpart in the paper): every index check on the path (noise, segment, split
 * records, persistent queue items, chunk sums, best sample) that failed since the last
 * reset set its bit here (1 noise, 2 segment, 4 queue, 8 chunk, 16 split record, 32 best
 * sample); the kernel skipped or clamped that access instead of trapping. reset != 0
 * clears the word after reading it. Returns MPPI_ERR_UNSUPPORTED (word 0) in the product
 * build, which has no checks. */
mppi_status mppi_check_word(uint32_t* h_word, int32_t reset);

/* ---------------------------------------------------------------------------------- */
/* Sample shards: one iteration's weights and knot average over samples split into     */
/* shards (on several devices, or several launches of one)                              */
/* ---------------------------------------------------------------------------------- */
/* The weights of Sec. III-C (Eq. (softmax_minmax)) need the global S_min and S_max of
 * the iteration's costs before any exponential, so a sharded iteration exchanges twice:
 * (1) each shard scans its costs (mppi_shard_range_local) and the ranges are merged
 * (mppi_shard_range_merge); (2) each shard forms, with the merged range, its
 * unnormalised weight sum and weighted knot sums (mppi_shard_moments), the sums are
 * merged (mppi_shard_moments_merge) and divided (mppi_shard_mean) into the updated
 * nominal of Eq. (update-nominal). The sample with the global best_index (Sec. III-D)
 * belongs to exactly one shard, which supplies its knots. Both merges are associative
 * and commutative (the second up to FP64 rounding: merge in a fixed shard order for
 * run-to-run identical results). Costs are FP32, sums FP64. The library itself moves no
 * data between devices; the exchange is the caller's (an all-gather of 4 doubles, then
 * of E + 1 doubles). */
typedef struct {
    double s_min;       /* smallest finite cost (+inf if the shard has none) */
    double s_max;       /* largest finite cost (-inf if none) */
    int64_t best_index; /* global sample index of the first smallest cost (-1 if none) */
    int64_t n_finite;   /* number of finite costs */
} mppi_shard_range;

/* Range of a shard's K costs d_costs [K] (device); the shard's sample n is global
 * sample index_base + n. Ties go to the lowest index, non-finite costs are left out
 * (as in the single-instance weights). Synchronous on `stream` (NULL = legacy default
 * stream); allocates and frees a few bytes of device memory. Errors: INVALID_ARG
 * (K < 1, index_base < 0, null pointers), CUDA. */
mppi_status mppi_shard_range_local(int32_t K, const float* d_costs, int64_t index_base,
                                   mppi_shard_range* h_out, void* stream);

/* out = the range of the union of a's and b's samples (host only; out may alias a or
 * b). Associative and commutative. */
void mppi_shard_range_merge(const mppi_shard_range* a, const mppi_shard_range* b, mppi_shard_range* out);

/* A shard's moments under the merged range `global`: h_out[0] = sum_n w_n and
 * h_out[1 + e] = sum_n w_n theta_n[e] for e < E, with w_n = exp(-(S_n - S_min) k),
 * k = 1 / ((S_max - S_min) lambda) for MPPI_NORM_MINMAX (0 when S_max = S_min, i.e.
 * uniform weights) or 1 / lambda for MPPI_NORM_RAW, and w_n = 0 for a non-finite cost:
 * the single-instance weights before their division by the total. d_knots [K][E] and
 * d_costs [K] are the shard's samples (device), h_out [E + 1] host FP64. Synchronous on
 * `stream`; allocates its scratch on the device for the call (like mppi_average).
 * Errors: INVALID_ARG (also when global's s_min is not an FP32 value, as a merge of
 * mppi_shard_range_local results always gives, or s_max < s_min), ALL_COSTS_NONFINITE
 * (global->n_finite == 0: the iteration leaves the nominal unchanged), CUDA. */
mppi_status mppi_shard_moments(int32_t K, int32_t E, const float* d_knots, const float* d_costs,
                               const mppi_shard_range* global, double lambda, int32_t normalize,
                               double* h_out, void* stream);

/* out[i] = a[i] + b[i] for i <= E (host only; out may alias a or b). */
void mppi_shard_moments_merge(int32_t E, const double* a, const double* b, double* out);

/* The updated nominal from merged moments: h_mean[e] = sums[1 + e] / sums[0] (FP32).
 * Errors: INVALID_ARG (E < 1, null pointers, sums[0] not positive and finite). */
mppi_status mppi_shard_mean(int32_t E, const double* sums, float* h_mean);

/* Single-step state derivative: generalised accelerations h_acc [n][nv] (base spatial
 * acceleration (w_dot, v_dot) in body coordinates, then qdd) of n states under
 * torques h_tau [n][nj], contact forces included, by the warp-per-sample articulated-
 * body recursion. */
mppi_status mppi_forward_dynamics(const mppi_model* model, int32_t n, const double* h_states,
                                  const double* h_tau, double* h_acc);
/* Same with fp64 != 0 selecting the FP64 check build of the kernel. */
mppi_status mppi_forward_dynamics_ex(const mppi_model* model, int32_t n, const double* h_states,
                                     const double* h_tau, double* h_acc, int32_t fp64);

/* ---------------------------------------------------------------------------------- */
/* Batched solves: many contexts in one persistent launch                               */
/* ---------------------------------------------------------------------------------- */

/* Solve `count` independent contexts (uneven models, K, H, knots, lambda) in one
 * persistent kernel that walks a device work queue of (instance, sample tile) items;
 * the last tile of an instance computes its weights and average and enqueues its next
 * iteration. h_states[i] [nx_i], h_warm[i] nullable, h_out_mean[i] [E_i],
 * h_out_best[i] nullable, h_info [count] nullable. Every instance's result equals its
 * mppi_solve result for the same inputs (noise depends only on seed, instance_id and
 * the iteration counter). Blocks until done. Device waits inside the kernel are bounded
 * (MPPI_ERR_TIMEOUT). Errors: INVALID_ARG, UNSUPPORTED (contexts on other devices or
 * with foreign streams), OUT_OF_MEMORY, TIMEOUT, CUDA. */
mppi_status mppi_solve_batch(mppi_ctx* const* ctxs, int32_t count, const double* const* h_states,
                             const float* const* h_warm, float* const* h_out_mean,
                             float* const* h_out_best, mppi_result* h_info);

/* Self-test of failure detection: launches the persistent kernel on a queue whose only
 * item is never published. Its bounded wait must give up after budget_us (1 us .. 10 s)
 * and set the error word; the call then returns MPPI_ERR_TIMEOUT and writes the device
 * error bits (2 = queue wait timed out) to h_error_bits (nullable). Nothing traps or
 * faults and the device stays usable. Returns MPPI_OK only if the wait did not give up
 * (which would be a defect). */
mppi_status mppi_selftest_queue_timeout(int64_t budget_us, int32_t* h_error_bits);

/* ---------------------------------------------------------------------------------- */
/* Serving: continuous batching of controller requests on one GPU                       */
/* ---------------------------------------------------------------------------------- */

/* A request loop on `device` that admits solves while their device memory fits in
 * mem_budget_bytes and at most max_inflight launch groups are on the GPU; requests that
 * arrive while others run are admitted as slots and memory free up, and their work
 * overlaps on the device (separate streams). Each of the max_inflight launch slots gets a
 * device launch block (queue, descriptors, packed inputs and outputs) and two pinned host
 * images of slot_bytes = min(4 MiB, floor(mem_budget_bytes / (4 max_inflight)) rounded
 * down to 256 B) when the server is created; that reservation (max_inflight * slot_bytes,
 * at most a quarter of the budget) counts against the budget for the server's lifetime, so
 * the contexts of admitted requests may use the rest, and nothing is allocated while
 * requests run. A batch is closed when the next request's launch block would overflow its
 * slot. Errors: INVALID_ARG (slot_bytes below 16 KiB, max_inflight outside 1..64),
 * OUT_OF_MEMORY, CUDA. *out owned by the caller. */
mppi_status mppi_server_create(int32_t device, size_t mem_budget_bytes, int32_t max_inflight,
                               mppi_server** out);
void mppi_server_destroy(mppi_server* server);

/* Queue one solve of ctx from h_state (copied now) with the resident warm start (or
 * h_warm_start, copied now). The context must not be used elsewhere until its ticket
 * is polled complete. Errors: INVALID_ARG, NONFINITE_STATE, ADMISSION (the request
 * alone exceeds the memory budget). */
mppi_status mppi_submit(mppi_server* server, mppi_ctx* ctx, const double* h_state,
                        const float* h_warm_start, uint64_t* ticket);

/* Result of a ticket: MPPI_PENDING while running (after waiting up to timeout_us,
 * < 0 = wait forever), else the solve's status with h_out_mean [E], h_out_best
 * (nullable) and h_info (nullable) written. A completed ticket is released; polling it
 * again returns NOT_FOUND. */
mppi_status mppi_poll(mppi_server* server, uint64_t ticket, float* h_out_mean,
                      float* h_out_best, mppi_result* h_info, int64_t timeout_us);

/* Next completed ticket, in completion order: MPPI_PENDING if none completes within
 * timeout_us (< 0 = wait forever, 0 = do not wait). times_ns (nullable, [2]) receives the
 * ticket's submit and completion times on CLOCK_MONOTONIC. The ticket still has to be
 * polled to fetch its results and release it. */
mppi_status mppi_next_completed(mppi_server* server, int64_t timeout_us, uint64_t* ticket, int64_t* times_ns);

/* Load shedding: a request still waiting for admission deadline_us after it was submitted
 * completes with MPPI_ERR_DEADLINE without running (its context's warm start and noise
 * counter are unchanged), so the queue and the latency of the requests that run stay
 * bounded when the offered load exceeds the server's capacity. 0 (the default) never
 * sheds. A control loop sets it to the control period: a solve that starts later is of no
 * use to it. Errors: INVALID_ARG (deadline_us < 0). */
mppi_status mppi_server_set_deadline(mppi_server* server, int64_t deadline_us);

/* Server counters: [0] submitted, [1] completed (shed requests included), [2] launches,
 * [3] peak device bytes charged to the budget (the slots' reservation plus the admitted
 * contexts' buffers), [4] admissions deferred by the memory budget. */
mppi_status mppi_server_stats(mppi_server* server, int64_t* h_out5);
/* The same counters and more: h_out[k] for k < n (n <= 11): [0..4] as above, [5] requests
 * shed by the deadline, [6] bytes reserved for the launch slots, [7] bytes per slot, and
 * the worker thread's longest pass of its loop [8], longest launch call [9] and longest
 * result unpacking [10] since creation or mppi_server_reset_timing, in ns (host time, where
 * a request waited when the device was not busy). */
mppi_status mppi_server_stats_ex(mppi_server* server, int64_t* h_out, int32_t n);
/* Restart the maxima [8..10] of mppi_server_stats_ex. Errors: INVALID_ARG. */
mppi_status mppi_server_reset_timing(mppi_server* server);

/* ---------------------------------------------------------------------------------- */
/* Autotuning and introspection                                                         */
/* ---------------------------------------------------------------------------------- */

/* Time every supported rollout mapping and block size for this context's model and
 * sizes (a few timed launches each) and switch the context to the fastest. h_ms (nullable,
 * [4*4]) receives the timings in ms per rollout launch (mapping-major: warp, half-warp,
 * lanes-per-chain and the reserved mapping 3, whose row is always negative; block sizes 32,
 * 64, 128, 256; negative = not supported). Writes the choice to *mapping / *block_size. */
mppi_status mppi_autotune(mppi_ctx* ctx, int32_t* mapping, int32_t* block_size, float* h_ms);

/* Persist the autotuner's choices in a JSON file (an array with one object per tuned
 * shape: device type as name|SMs|compute capability, model hash, K, H, knots, mapping,
 * block, the 16 timings). The file's entries are loaded now (a missing file is created
 * by the next tuning) and every new tuning rewrites it; later processes on the same kind
 * of GPU reuse the entries without timing. NULL or "" keeps the choices in the process
 * only. Errors: INVALID_ARG (the file exists but is not in this format). */
mppi_status mppi_autotune_cache_file(const char* path);

/* Switch a context's rollout mapping and block size (MPPI_MAP_WARP/HALFWARP/CHAIN). */
mppi_status mppi_ctx_set_mapping(mppi_ctx* ctx, int32_t mapping, int32_t block_size);

/* FP64 check build: when on, mppi_rollout_explicit runs the same rollout source in double
 * precision (the warp mappings) so that comparisons with an FP64 reference separate
 * algorithmic differences from FP32 rounding. The product path is unaffected. */
mppi_status mppi_ctx_set_fp64_check(mppi_ctx* ctx, int32_t on);

/* Profiling: with on != 0 the captured solve graph records CUDA events around each
 * iteration's rollout launch; mppi_ctx_rollout_ms then returns the rollout kernel
 * durations of the last completed solve (h_ms [iters], milliseconds; synchronises). */
mppi_status mppi_ctx_profile(mppi_ctx* ctx, int32_t on);
mppi_status mppi_ctx_rollout_ms(mppi_ctx* ctx, float* h_ms);

/* Dimensions of a context: [0] K, [1] H, [2] knots, [3] iters, [4] nj, [5] nx,
 * [6] mapping, [7] block_size. */
mppi_status mppi_ctx_info(const mppi_ctx* ctx, int32_t* h_out8);

/* Bytes that one mppi_solve moves between host and device: h_out2[0] host -> device (the
 * state; a warm start adds knots x 2 x nj x 4), h_out2[1] device -> host (the mean, the
 * best knots and the result). */
mppi_status mppi_ctx_io_bytes(const mppi_ctx* ctx, int64_t* h_out2);

/* What the library derived from a model: h_out4 = (topology: 0 generic tree, 1 base + 4
 * chains of <= 3, 2 base + 2 chains + a branch body with 2 chains; axis plan of the
 * lanes-per-chain kernels: 0 any axes, 1 the quadruped layout (every chain turns about +x,
 * +y, +y, hip offsets in the base's xy-plane, thigh and knee offsets on one axis, contact
 * points only on the calves), 2 the humanoid layout run by the two-warp split kernel
 * (legs z, x, y, y, y, x; waist z; arms y, x, z, y; offsets on one axis, in the yz-plane
 * or zero; contact points only on the feet; the cost body not on a leg); 1 when the
 * modular cost of Sec. IV-A is on,
 * else 0; the number of bodies). With plan 2 the lanes-per-chain mapping needs blocks of
 * 64, 128 or 256 threads. */
mppi_status mppi_model_info(const mppi_model* model, int32_t* h_out4);

/* Device bytes one solve of a context occupies (its buffers). */
size_t mppi_ctx_device_bytes(const mppi_ctx* ctx);

/* Number of kernels one solve launches (for launch accounting). */
int32_t mppi_ctx_kernels_per_solve(const mppi_ctx* ctx);

const char* mppi_status_str(mppi_status status);
/* Text of the last CUDA error seen by this context (or by the library when ctx is NULL). */
const char* mppi_last_error(const mppi_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* MPPI_H_ */
