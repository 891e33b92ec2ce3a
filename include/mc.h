/*
 * mc.h -- C ABI of the GB300 Monte Carlo closed-loop library.
 *
 * The library runs many independent stochastic closed-loop simulations of a
 * continuous stirred tank reactor (CSTR) on one NVIDIA GB300 GPU, following
 * Kaysfeld, Zanon, Joergensen, "Performance Quantification of a Nonlinear
 * Model Predictive Controller by Parallel Monte Carlo Simulations of a
 * Closed-loop System" (arXiv 2212.02197):
 *
 *   plant     three-state CSTR SDE, Eq. (CSTR) of Sec. VI, integrated by
 *             Euler-Maruyama with N_s substeps per sample (Sec. VII-A),
 *   sensor    y_i = c_T(t_i) + v_i, v_i ~ N(0, R) (Sec. II, Eq. CDS),
 *   NMPC      CD-EKF prediction/filtering (Sec. III-A, Eqs. predictionEquations
 *             and Josph) on the one-state model, and the regulator OCP
 *             (Eq. OPC_general) in multiple-shooting form (Eq. OCP_NLP),
 *             solved by SQP (Sec. IV): structured QP subproblem
 *             (Eq. QP-subproblem), Powell l1-merit backtracking line search
 *             (Eq. Armijo), damped block BFGS, scaled convergence test
 *             (Eq. convergence),
 *   PI        the reference controller with anti-windup, Eq. (PI) of Sec. V,
 *   result    the performance index Phi of Eq. (Phi), Sec. VII-C, per
 *             trajectory, plus the OCP statistics of Table II.
 *
 * Conventions for every function below:
 *   - Pointers named *_host are host memory; *_dev are device memory; a
 *     `dst_is_device` flag says which one a destination is.
 *   - Nothing aborts.  Every function returns an mc_status; on failure the
 *     handle (if any) keeps a message available from mc_last_error().
 *   - The handle owns all device memory it allocates (cudaMalloc in
 *     mc_create, freed by mc_destroy).  Input arrays are copied at the call,
 *     so the caller may free them when the call returns.
 *   - Work is enqueued on the CUDA stream given as `cuda_stream`
 *     (a cudaStream_t; NULL means the legacy default stream) and is
 *     asynchronous until mc_stats / mc_copy_* / mc_sync.
 *   - Units: time s, volume L, amount mol, temperature K; flows at this
 *     interface in mL/min.
 */
#ifndef MC_GB300_H
#define MC_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MC_MAX_SETPOINTS 16
#define MC_MAX_HORIZON 64
#define MC_MAX_BINS 256
#define MC_N_COUNTERS 8

typedef enum {
  MC_OK = 0,
  MC_EINVAL = 1,          /* invalid argument or configuration               */
  MC_ENOMEM = 2,          /* device allocation failed                        */
  MC_ECUDA = 3,           /* a CUDA call failed (message in mc_last_error)   */
  MC_ETIMEOUT = 4,        /* the GPU did not finish within the wait limit    */
  MC_ENOTRUN = 5,         /* results requested before any mc_run             */
  MC_WARN_NONFINITE = 100 /* finished; some trajectories became non-finite   */
} mc_status;

typedef enum { MC_CTRL_NMPC = 0, MC_CTRL_PI = 1 } mc_ctrl_kind;
typedef enum { MC_FP64 = 0, MC_MIXED = 1 } mc_precision;
typedef enum {
  MC_QP_ACTIVE_SET = 0,   /* Riccati-based primal active-set method          */
  MC_QP_IPM = 1,          /* Riccati-based primal-dual interior point (Mehrotra) */
  MC_QP_ACTIVE_SET_WARP = 2  /* the active-set method with a parallel-in-horizon
                                Riccati recursion, one warp per QP (the lanes
                                over the stages); mc_qp_solve_batch only --
                                the closed loop runs one trajectory per lane */
} mc_qp_solver;

/* Plant, NMPC model and closed-loop set-up (Sec. VI, VII-A). */
typedef struct {
  double V, k0, EaR, beta, cA_in, cB_in, T_in; /* CSTR parameters, Eq. (CSTR)   */
  double sigma[3];        /* diagonal of sigma-bar (mol/L, mol/L, K)           */
  double meas_sd;         /* sqrt(R), measurement noise sd (K); > 0           */
  double Ts, t0;          /* sample time and start time (s)                    */
  int32_t n_steps;        /* control steps K (Phi has K+1 terms)               */
  int32_t n_em;           /* Euler-Maruyama substeps per sample, N_s           */
  int32_t n_setpoints;    /* 1..MC_MAX_SETPOINTS                               */
  int32_t Ea_plant_only;  /* 0: the E_a/R perturbation is known to the
                             controller (its EKF and OCP model use the
                             trajectory's E_a/R); 1: model mismatch, the
                             perturbation acts on the plant only and the
                             controller keeps the nominal E_a/R              */
  const double* sp_time;  /* host, n_setpoints: segment start times, ascending */
  const double* sp_value; /* host, n_setpoints: set-point temperatures (K)     */
  double Ea_logsd;        /* lognormal sd of E_a/R per trajectory, 0 = off     */
  double dT_in_step;      /* +- step of T_in at a uniform random time, 0 = off */
} mc_model_t;

/* Controller (Sec. III-V, VII-A). */
typedef struct {
  int32_t kind;           /* mc_ctrl_kind                                      */
  int32_t precision;      /* mc_precision                                      */
  double u_min, u_max;    /* input bounds (mL/min)                             */
  double kP, kI, kaw;     /* PI gains; act on F in L/s and e in K             */
  int32_t N;              /* prediction horizon, 1..MC_MAX_HORIZON             */
  int32_t n_rk4;          /* classical RK4 steps per interval, N_c             */
  double Qz;              /* output weight of the NMPC objective               */
  double P0;              /* initial EKF covariance P_{-1|-1} ((K L)^2)        */
  int32_t sqp_max_it;     /* SQP iteration limit (a hit counts as failed OCP)  */
  int32_t ls_max;         /* maximum step halvings of the line search          */
  double sqp_tol;         /* epsilon of the scaled KKT test                    */
  int32_t qp_solver;      /* mc_qp_solver                                      */
  int32_t ip_max_it;      /* interior-point iteration limit                   */
  double ip_tol;          /* interior-point residual/complementarity tolerance */
  double u_scale;         /* OCP input unit (mL/min)                           */
  double x_scale;         /* OCP state unit (K L); V makes it kelvin           */
  /* uneven batches: > 0 draws each trajectory's horizon uniformly from
   * N_min..N and its SQP iteration limit from sqp_max_it_min..sqp_max_it
   * (Philox counter (2, j, 3, 0)); 0 keeps N and sqp_max_it for all         */
  int32_t N_min;
  int32_t sqp_max_it_min;
  int32_t schedule;       /* mc_schedule                                       */
  int32_t threads_per_sm; /* persistent schedule: resident threads per SM,
                             0 = one per trajectory up to the GPU's capacity   */
  int32_t nx_model;       /* NMPC model: 0 or 1 = the one-state model of Sec. VI
                             (the paper's); 3 = the three-state model of
                             Eq. (CSTR) with a 3x3 CD-EKF (FP64, active-set
                             QP, either schedule)                             */
  /* extended NMPC objective (the paper's has both 0):
   *   + sum_{k=1..N} Ru (v_{k-1} - vbar_k)^2 T_s + Qn (z_N - zbar_N)^2,
   * v the OCP input (flow / u_scale), vbar_k the steady-state input of the
   * set-point zbar_k; one-state model only                                  */
  double Ru;
  double Qn;
  /* persistent schedule: a backtracking line search shoots its next halvings
   * together (speculative backtracking; the same iterates and counters as
   * one trial at a time) while at most this many lanes of its warp hold a
   * trajectory; 0 = always, negative = never, 1..32 = that many lanes    */
  int32_t ls_spec_lanes;
} mc_controller_t;

typedef enum {
  MC_SCHED_STATIC = 0,    /* one thread per trajectory, OCPs in lock-step      */
  MC_SCHED_PERSISTENT = 1 /* per-lane state machine; each round the warp
                             shoots all pending intervals (trial points and
                             OCP starts) as one pool and draws the plant noise
                             of the OCPs it starts; trajectories taken from a
                             queue (longest horizons first when horizons
                             differ).  Same results as the static schedule,
                             bit for bit                                       */
} mc_schedule;

/* Reduced results of the last run (Table II and Fig. 3 of Sec. VII). */
typedef struct {
  int64_t n_traj;         /* trajectories in the last run                      */
  int64_t n_ocp;          /* OCPs solved (NMPC: n_traj * n_steps)              */
  int64_t n_ocp_failed;   /* OCPs stopped by the SQP iteration limit           */
  int64_t n_ls_fail;      /* OCPs stopped by a failed line search              */
  int64_t n_hess_reset;   /* block-BFGS resets to the identity                 */
  int64_t n_nonfinite;    /* trajectories whose state became non-finite        */
  int64_t sqp_iters;      /* QP subproblems solved                             */
  int64_t ls_trials;      /* merit evaluations in the line searches            */
  int64_t qp_iters;       /* QP solver iterations (active-set or IPM)          */
  int64_t qp_fail;        /* QP subproblems that hit their iteration limit     */
  double phi_mean, phi_var, phi_min, phi_max; /* over finite trajectories      */
  int32_t n_bins;         /* histogram of Phi                                  */
  int32_t reserved0;
  double bin_lo, bin_hi;
  int64_t hist[MC_MAX_BINS];
  double gpu_ms;          /* device time of the last mc_run (CUDA events)      */
} mc_stats_t;

typedef struct mc_handle mc_handle;

/* Validate the configuration and allocate device buffers for n_sims
 * trajectories (indices 0 .. n_sims-1).  Trajectory j draws its noise from
 * Philox4x32-10 with key `seed` and counters carrying j, so handles with the
 * same seed (an NMPC and a PI handle, say) see common random numbers, and any
 * trajectory's result is independent of how runs are split.
 * Returns MC_EINVAL (with the reason in mc_last_error(NULL)) or MC_ENOMEM. */
mc_status mc_create(const mc_model_t* model, const mc_controller_t* ctrl,
                    int64_t n_sims, uint64_t seed, mc_handle** out);

/* Histogram of Phi with n_bins (1..MC_MAX_BINS) equal bins on [lo, hi);
 * lo >= hi selects the [min, max] of the run itself.  Values outside are
 * counted in the first/last bin. */
mc_status mc_set_histogram(mc_handle* h, int32_t n_bins, double lo, double hi);

/* Simulate all trajectories (Sec. VII-C: Monte Carlo over process and
 * measurement noise) and reduce the statistics, asynchronously on the stream. */
mc_status mc_run(mc_handle* h, void* cuda_stream);

/* Simulate trajectories j0 .. j1-1 only (0 <= j0 <= j1 <= n_sims) and reduce
 * the statistics over that range.  Per-trajectory results of other indices
 * are kept. */
mc_status mc_run_range(mc_handle* h, int64_t j0, int64_t j1, void* cuda_stream);

/* CUDA graphs: with on = 1 each trajectory range's launch sequence is
 * captured into a graph on its first mc_run/mc_run_range and replayed from
 * then on; on = 0 (default) launches directly.  Needs a stream other than the
 * legacy default stream (with NULL the launches stay direct).  Changing the
 * histogram or autotuning drops the captured graphs. */
mc_status mc_set_graph(mc_handle* h, int on);

/* Persistent NMPC schedule only: time short probe runs (the first probe_steps
 * samples of every trajectory) for a range of resident threads per SM, keep
 * the fastest in the handle and return it in *threads_per_sm (may be NULL).
 * Blocks until done; overwrites the per-trajectory results of earlier runs. */
mc_status mc_autotune(mc_handle* h, int32_t probe_steps, void* cuda_stream,
                      int32_t* threads_per_sm);

/* Wait for the last run (polling, at most timeout_ms; <= 0 waits without limit)
 * and copy its statistics.  Returns MC_ETIMEOUT if the GPU has not finished,
 * MC_WARN_NONFINITE if some trajectory became non-finite. */
mc_status mc_stats(mc_handle* h, mc_stats_t* out, int64_t timeout_ms);

/* Copy Phi of trajectories j0 .. j0+n-1 (after a run) to dst. */
mc_status mc_copy_phi(mc_handle* h, int64_t j0, int64_t n, double* dst, int dst_is_device);

/* Copy the per-trajectory counters of trajectories j0 .. j0+n-1, row-major
 * n x MC_N_COUNTERS int32: [n_ocp_failed, sqp_iters, ls_trials, n_hess_reset,
 * n_ls_fail, qp_iters, nonfinite, qp_fail]. */
mc_status mc_copy_counters(mc_handle* h, int64_t j0, int64_t n, int32_t* dst,
                           int dst_is_device);

/* Per-warp record of the last one-state NMPC launch on the persistent
 * schedule (mc_run, mc_run_range, mc_nmpc_grad's closed loop; the paper has no
 * counterpart: it describes where a launch's time goes).  Waits for that
 * launch, then copies min(max_warps, W) records of MC_WARP_TRACE_WORDS uint64
 * each into out_host (host memory) and writes the launch's warp count W to
 * *n_warps_out.  Record w (warp = block w): [0] the pool rounds the warp ran,
 * [1] its lane-rounds (the sum over those rounds of its lanes still holding a
 * trajectory; over all warps, the launch's OCP starts plus line-search
 * rounds, where a backtracking line search tests several trials per round),
 * [2] and [3] the GPU's global timer in ns when the warp started and
 * finished, [4] the SM it ran on.  MC_ENOTRUN if no such launch has run on h;
 * MC_EINVAL for a null h or n_warps_out, a negative max_warps, or a null
 * out_host with max_warps > 0. */
#define MC_WARP_TRACE_WORDS 5
mc_status mc_copy_warp_trace(mc_handle* h, uint64_t* out_host, int64_t max_warps,
                             int64_t* n_warps_out);

/* Block until all work of the handle's last run has finished (timeout as in
 * mc_stats). */
mc_status mc_sync(mc_handle* h, int64_t timeout_ms);

/* Restrict the handle's kernels to a partition of at least n_sms SMs (a green
 * context; the driver rounds up to its partition granularity, 8 SMs on
 * sm_90 and later); n_sms = 0 or >= the device's SM count restores the whole
 * GPU.  *n_sms_out (may be NULL) receives the SMs the handle now uses.  The
 * paper measures how its study scales with CPU cores (Sec. VII-B, Fig. 2);
 * this is the GPU's counterpart.  Runs are launched on the partition's own
 * stream, ordered after the caller's stream and joined back into it, so the
 * stream semantics of mc_run_range are unchanged; CUDA-graph replay is not
 * used while a partition is set.  Waits for the device to be idle.
 * MC_ECUDA if the driver has no green contexts. */
mc_status mc_set_sm_partition(mc_handle* h, int32_t n_sms, int32_t* n_sms_out);

void mc_destroy(mc_handle* h);
const char* mc_status_str(mc_status s);
/* last error message of a handle; NULL gives the last mc_create failure */
const char* mc_last_error(const mc_handle* h);

/* ---------------------------------------------------------------------------
 * Gradients of the PI study.  The paper proposes the Monte Carlo study as a
 * tool for tuning the controller (Sec. VIII); these calls give the derivative
 * of the performance index Phi_j, Eq. (Phi), with respect to the gains of the
 * PI law, Eq. (PI), by a discrete adjoint (reverse mode) of the simulated
 * closed loop, so that mean Phi can be minimised by gradient methods.  The
 * derivative is that of the discrete simulation the library runs (Euler-
 * Maruyama substeps, Philox noise fixed by seed and trajectory index); where
 * the input clip of Eq. (PI) saturates, the derivative through it is zero.
 * ------------------------------------------------------------------------- */

/* Replace the gains (k_P, k_I, k_aw; units as in mc_controller_t) of a PI
 * handle.  MC_EINVAL for an NMPC handle or non-finite gains. */
mc_status mc_set_pi_gains(mc_handle* h, double kP, double kI, double kaw);

/* Run trajectories j0 .. j1-1 of a PI handle (FP64 only) forward and
 * backward on cuda_stream, asynchronously.  Writes what mc_run_range writes
 * (Phi_j, the counters, the statistics for mc_stats) and, per trajectory,
 * dPhi_j/d(k_P, k_I, k_aw).  The forward sweep stores the plant state and
 * the integral state every checkpoint_every samples (1..32); the backward
 * sweep recomputes each segment from its checkpoint.  The first call
 * allocates the gradient buffers (24 B per trajectory) and the checkpoints
 * (32 B per trajectory and checkpoint), kept until mc_destroy.
 * MC_EINVAL for an NMPC or mixed-precision handle, a bad range or
 * checkpoint interval, or n_em > 32; MC_ENOMEM if the buffers cannot be had. */
mc_status mc_pi_grad(mc_handle* h, int64_t j0, int64_t j1, int32_t checkpoint_every,
                     void* cuda_stream);

/* Replace the objective weights (Q_z, R_u, Q_n) of an NMPC handle.  MC_EINVAL
 * for a PI handle, negative or non-finite weights, or R_u, Q_n != 0 on the
 * three-state model. */
mc_status mc_set_nmpc_weights(mc_handle* h, double Qz, double Ru, double Qn);

/* Device memory the persistent schedule's mc_nmpc_grad may take for its
 * sample records (the paper has no counterpart): bytes >= the records of one
 * trajectory, (n_steps + 1) (5 (N + 1) + 8) doubles; 0 restores the default
 * of 8 GB.  Smaller budgets split the trajectories into more chunks, each a
 * recording launch and a tangent launch; the results do not change.  Takes
 * effect at the next mc_nmpc_grad, which reallocates the records only when
 * they must grow.  MC_EINVAL for a null or non-NMPC handle, a negative
 * budget, or one below a trajectory's records. */
mc_status mc_set_grad_record_budget(mc_handle* h, int64_t bytes);

/* Run trajectories j0 .. j1-1 of an NMPC handle (one-state model, FP64) and
 * the tangents of Phi_j with respect to the weights (Q_z, R_u, Q_n) of the
 * extended objective (mc_controller_t.Ru, .Qn; the paper's has both 0), on
 * cuda_stream, asynchronously.  Every OCP enters through its solution map
 * u_0(x-hat, theta) at the KKT point the SQP returns, differentiated
 * implicitly (Lagrangian Hessian from second-order shooting sensitivities,
 * active bounds held); the plant, the measurement and the CD-EKF are
 * differentiated exactly (forward mode).  The warm start does not enter.
 * Writes Phi_j, the counters (counter 7 also counts OCPs whose reduced
 * Hessian was not positive definite; their input tangent is 0) and
 * dPhi_j/d(Q_z, R_u, Q_n) per trajectory (read with mc_grad_mean,
 * mc_copy_grad).  Runs on the handle's schedule, with the same results bit
 * for bit: the static one carries the tangents along the closed loop; the
 * persistent one records each sample's starting state and KKT point while it
 * runs the closed loop, then propagates the tangents through the records with
 * every lane of a warp on the same sample (records of at most 8 GB, chunks of
 * trajectories beyond that).  Allocates on its first call 3 doubles per
 * trajectory, 27 per scratch column and, on the persistent schedule, the
 * records ((n_steps + 1) (5 (N + 1) + 8) doubles per trajectory of a chunk).
 * MC_EINVAL for a PI, mixed-precision or
 * three-state handle or a bad range; MC_ENOMEM if the gradient buffers
 * cannot be had. */
mc_status mc_nmpc_grad(mc_handle* h, int64_t j0, int64_t j1, void* cuda_stream);

/* Wait for the last mc_pi_grad or mc_nmpc_grad (as mc_stats does) and write
 * the mean of the three derivatives over its trajectories with a finite
 * Phi_j to out (3 doubles, host).  MC_ENOTRUN before any gradient run;
 * MC_WARN_NONFINITE (out still written) when some trajectory was non-finite. */
mc_status mc_grad_mean(mc_handle* h, double out[3], int64_t timeout_ms);

/* Copy the per-trajectory derivatives of the last gradient run of
 * trajectories j0 .. j0+n-1, row-major n x 3 doubles (NaN rows for
 * non-finite trajectories). */
mc_status mc_copy_grad(mc_handle* h, int64_t j0, int64_t n, double* dst, int dst_is_device);

/* ---------------------------------------------------------------------------
 * Building blocks of the hot path, exposed for batched use and for testing
 * each step against an independent implementation.  All pointers are host
 * memory; the call copies in, runs one kernel and copies out (blocking).
 * ------------------------------------------------------------------------- */

/* Philox4x32-10 (Salmon et al., SC'11) on n counters: ctr_host (n x 4),
 * key (2 words), out_host (n x 4). */
mc_status mc_philox(const uint32_t* ctr_host, const uint32_t key[2], int64_t n,
                    uint32_t* out_host);

/* The closed loop's noise for trajectory j, as the simulation draws it:
 * process noise of substeps k0 .. k0+nk-1 (out_host, nk x 3 standard
 * normals, Sec. II d-omega) and measurement noise of samples k0 .. k0+nk-1
 * (meas_host, nk standard normals).  precision selects the FP64 or FP32
 * transform of the same Philox words. */
mc_status mc_noise(uint64_t seed, int64_t j, int64_t k0, int64_t nk, int32_t precision,
                   double* out_host, double* meas_host);

/* The FP64 exponential every rate-law evaluation of the simulation uses
 * (k = k0 exp(-(E_a/R)/T) = exp(log k0 - (E_a/R)/T), Eq. (CSTR)): y = e^x for
 * n values, host arrays.  Tang's table-driven method; within about 1 ulp of
 * the exact value. */
mc_status mc_exp_batch(const double* x_host, int64_t n, double* out_host);

/* The FP64 reciprocal the one-state rate law takes of the temperature
 * (1/T in (E_a/R)/T and in dr/dT, Sec. VI): y = 1/x for n values, host
 * arrays.  Two Newton-Raphson steps on the hardware's approximate
 * reciprocal; within about 1 ulp of the exact value for normal x, the
 * approximation's own value (exact) for zeros, infinities and NaN. */
mc_status mc_rcp_batch(const double* x_host, int64_t n, double* out_host);

/* Throughput probe of one arithmetic pipe on the current device, for the
 * roofline of the simulation kernels (the paper has no counterpart: its
 * timings are wall-clock on CPU cores).  kind: 0 FP64 fma chain, 1 fma + add,
 * 2 the rate law's table-driven exp, 3 the library exp, 4 FP64 division,
 * 5 log, 6 sqrt, 7 sincospi, 8 FP32 fma chain, 9 fma + expf, 10 FP32 fma +
 * add, 11 the rate law's Newton-refined reciprocal.  One launch of 16 four-warp blocks per SM, every thread with 8
 * independent chains of `iters` steps (1 .. 2^30).  *ms_out receives the
 * launch's device time (CUDA events, after a short warm-up launch) and
 * *steps_out the number of chain steps it ran, so steps / time is the
 * probed operation's throughput.  Synchronises the device; allocates and
 * frees one small device buffer.  MC_EINVAL for a bad kind or count. */
mc_status mc_pipe_probe(int32_t kind, int64_t iters, double* ms_out, double* steps_out);

/* Solve n structured QP subproblems, Eq. (QP-subproblem)/(nlpsqp_qp), with the
 * selected solver.  Inputs are n x N (A, B, b, r, lb, ub) and n x (N+1)
 * (Wxx, Wxu, Wuu, q) row-major host arrays (A[.,0], Wxx[.,0], Wxu[.,0],
 * Wxu[.,N], Wuu[.,N], q[.,0] unused); outputs du, mu, nul, nuu (n x N),
 * dx (n x (N+1)), iters and status (n; 0 = solved, 1 = iteration limit,
 * 2 = not positive definite). */
mc_status mc_qp_solve_batch(int32_t N, int64_t n, int32_t solver, int32_t max_it,
                            double tol, const double* A, const double* B, const double* b,
                            const double* Wxx, const double* Wxu, const double* Wuu,
                            const double* q, const double* r, const double* lb,
                            const double* ub, double* du, double* dx, double* mu,
                            double* nul, double* nuu, int32_t* iters, int32_t* status);

/* Solve n NMPC OCPs (Sec. III-B) by the SQP of Sec. IV from the given warm
 * starts.  x0 (n): initial OCP states; EaR (n): activation energies;
 * zbar (n x (N+1), column 0 unused): set-points z-bar(t_{i+k}); u (n x N),
 * x (n x (N+1)), lam, pil, piu (n x N) are read as the warm start and
 * overwritten with the solution; info (n x 4 int32): [iters, status
 * (0 converged, 1 iteration limit, 2 line search), ls_trials, qp_iters];
 * kkt (n x 3 double): [||grad L / s_d||_inf, ||g||_inf, f]. */
mc_status mc_ocp_solve_batch(const mc_model_t* model, const mc_controller_t* ctrl,
                             int64_t n, const double* x0, const double* EaR,
                             const double* zbar, double* u, double* x, double* lam,
                             double* pil, double* piu, int32_t* info, double* kkt);

/* Sensitivity of n OCP solutions (as mc_ocp_solve_batch returns them): the
 * derivatives of the first input u_0 with respect to the initial state x_0
 * (OCP units) and the weights (Q_z, R_u, Q_n), by implicit differentiation of
 * the KKT conditions (one-state model).  x0, EaR (n); zbar, x (n x (N+1));
 * u, lam, pil, piu (n x N); sens (n x 4) out; status (n) out: 0, or 1 when
 * the reduced Hessian is not positive definite (sens 0). */
mc_status mc_ocp_sens_batch(const mc_model_t* model, const mc_controller_t* ctrl, int64_t n,
                            const double* x0, const double* EaR, const double* zbar,
                            const double* u, const double* x, const double* lam,
                            const double* pil, const double* piu, double* sens,
                            int32_t* status);

/* ---------------------------------------------------------------------------
 * Statistics without allocation.  The paper has no counterpart to this call;
 * it exists for callers that cannot call cudaMalloc: code that runs under a
 * device-memory budget fixed up front, or in a loop that must never enter the
 * allocator (cudaMalloc may synchronise the device and its latency is
 * unbounded), or a host framework that owns all device memory itself.
 * ------------------------------------------------------------------------- */

/* Largest n one mc_reduce_noalloc call accepts: 1024 blocks of 256 threads. */
#define MC_NOALLOC_MAX_TRAJ 262144

/* Reduce per-trajectory results that already live on the device -- phi_dev
 * (n doubles) and counters_dev (n x MC_N_COUNTERS int32, the layout of
 * mc_copy_counters; must not be NULL) -- into *out_host, exactly as mc_stats
 * reduces a run: mean/variance/min/max of the finite Phi, the histogram
 * (n_bins bins on [lo, hi), lo >= hi meaning [min, max]) and the counter sums.
 * n_ocp and gpu_ms are left 0 (this call does not know the run).
 *
 * Nothing is allocated.  The scratch (1024 block partials and one result
 * record, about 120 KB) is a file-scope __device__ array in the library: every
 * GPU that loads the library holds it until the process exits.  The first
 * call on a device looks up the array's device address with that device
 * current; make that first call before any stream capture.  The address is
 * kept for the life of the process, so it assumes the device is not reset
 * (cudaDeviceReset) while the library is loaded.  All calls share
 * the one array and each call overwrites what it reads, so calls that overlap
 * on the GPU (other streams, other host threads) race: serialise them.
 * The call enqueues two kernels on cuda_stream, waits for that stream and
 * copies the result to out_host.  Returns MC_EINVAL for n < 0,
 * n > MC_NOALLOC_MAX_TRAJ, n_bins outside 1..MC_MAX_BINS or NULL pointers;
 * MC_WARN_NONFINITE if some Phi is not finite. */
mc_status mc_reduce_noalloc(const double* phi_dev, const int32_t* counters_dev, int64_t n,
                            int32_t n_bins, double lo, double hi, void* cuda_stream,
                            mc_stats_t* out_host);

#ifdef __cplusplus
}
#endif
#endif
