/*
 * oracle.h -- plain FP64 CPU oracle for the parallel Monte Carlo closed-loop
 * study of Kaysfeld, Zanon and Joergensen (arXiv 2212.02197).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path; only
 * the test-suite, the smoke check and the CPU-baseline leg of the benchmark
 * load it.  It shares no source, header, table or helper with the CUDA path:
 * configuration reaches it as plain data through the structs below.
 *
 * Everything is straightforward double-precision C, one trajectory at a time,
 * in the order and notation of the paper:
 *   Sec. II   stochastic continuous-discrete system, Eq. (CDS)
 *   Sec. III  CD-EKF prediction (predictionEquations) and filtering (Josph),
 *             regulator OCP (OPC_general) and its multiple-shooting NLP (OCP_NLP)
 *   Sec. IV   SQP: QP subproblem (QP-subproblem), Powell l1-merit backtracking
 *             line search (Armijo), damped block BFGS, scaled convergence test
 *   Sec. V    PI controller with anti-windup, Eq. (PI)
 *   Sec. VI   CSTR model, Eq. (CSTR), three-state plant and one-state model
 *   Sec. VII  closed-loop set-up and the performance index, Eq. (Phi)
 *
 * The QP subproblem is solved here by condensing the state increments away
 * and running a dense primal active-set method to the exact KKT point; the
 * paper's solver (a Riccati interior-point method) is deliberately not used,
 * so that the GPU path and this oracle reach the unique QP minimiser by
 * independent routes.
 *
 * Pins for every function are in tests/test_oracle_*.py.
 */
#ifndef MC_ORACLE_H
#define MC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAX_SP 16   /* set-point schedule segments            */
#define OR_MAX_N 64    /* longest prediction horizon supported   */

/* Plant and NMPC model (Sec. VI) plus the closed-loop set-up (Sec. VII).
 * Units: s, L, mol, K.  The state of the plant is n = c V (mol, mol, K L). */
typedef struct {
  double V, k0, EaR, beta, cA_in, cB_in, T_in;
  double sigma[3];      /* diagonal of sigma-bar, (mol/L, mol/L, K)          */
  double meas_sd;       /* square root of the measurement covariance R (K)   */
  double Ts, t0;        /* sample time and start time (s)                    */
  int32_t n_steps;      /* control steps K; Phi has K+1 terms                */
  int32_t n_em;         /* Euler-Maruyama substeps per sample, N_s           */
  int32_t n_sp;         /* number of set-point segments                      */
  int32_t Ea_plant_only; /* 1: the E_a/R perturbation acts on the plant only;
                            the controller's model keeps the nominal E_a/R  */
  double sp_time[OR_MAX_SP];   /* segment s starts at sp_time[s]             */
  double sp_value[OR_MAX_SP];  /* set-point temperature of segment s (K)     */
  double Ea_logsd;      /* per-trajectory lognormal sd of E_a/R, 0 = off    */
  double dTin_step;     /* magnitude of the inlet-temperature step, 0 = off */
} or_model;

/* Controller: NMPC (Sec. III, IV) or PI (Sec. V). */
typedef struct {
  int32_t kind;         /* 0 = NMPC, 1 = PI                                  */
  int32_t N;            /* prediction horizon (control intervals)            */
  int32_t n_rk4;        /* classical RK4 steps per interval, N_c             */
  int32_t sqp_max_it;   /* SQP iteration limit                               */
  int32_t ls_max;       /* maximum number of step halvings                   */
  int32_t nx_model;     /* NMPC model: 0 or 1 = one-state (Sec. VI),
                           3 = the three-state model of Eq. (CSTR)           */
  double u_min, u_max;  /* input bounds (mL/min)                             */
  double kP, kI, kaw;   /* PI gains, acting on F in L/s and e in K           */
  double Qz;            /* output weight of the NMPC objective               */
  double P0;            /* initial EKF covariance P_{-1|-1} ((K L)^2)        */
  double sqp_tol;       /* epsilon of the scaled convergence test            */
  double u_scale;       /* unit of the OCP input variable, in mL/min         */
  double x_scale;       /* unit of the OCP state variable, in K L            */
  int32_t N_min;        /* > 0: per-trajectory horizon uniform on N_min..N   */
  int32_t it_min;       /* > 0: per-trajectory SQP limit on it_min..max_it   */
  double Ru;            /* input-deviation weight of the NMPC objective      */
  double Qn;            /* terminal output weight of the NMPC objective      */
} or_ctrl;

/* Per-trajectory result of one closed-loop simulation. */
typedef struct {
  double phi;            /* performance index, Eq. (Phi)                     */
  int32_t n_ocp;         /* OCPs solved (= K for NMPC)                       */
  int32_t n_ocp_failed;  /* OCPs that hit the SQP iteration limit            */
  int32_t sqp_iters;     /* QP subproblems solved, summed over the OCPs      */
  int32_t ls_trials;     /* merit evaluations in the line searches           */
  int32_t n_hess_reset;  /* block-BFGS resets to the identity                */
  int32_t n_ls_fail;     /* line searches that ran out of halvings           */
  int32_t qp_iters;      /* active-set iterations, summed                    */
  int32_t nonfinite;     /* 1 if the state became non-finite                 */
} or_traj_out;

/* Per-OCP diagnostics of one SQP solve. */
typedef struct {
  int32_t iters;         /* QP subproblems solved                            */
  int32_t status;        /* 0 converged, 1 iteration limit, 2 line search    */
  int32_t ls_trials;
  int32_t n_hess_reset;
  int32_t qp_iters;
  int32_t pad0;
  double kkt_grad;       /* ||grad L / s_d||_inf at the returned point       */
  double kkt_eq;         /* ||g||_inf at the returned point                  */
  double f;              /* objective at the returned point                  */
} or_sqp_info;

/* ---- counter-based random numbers (Philox4x32-10, Salmon et al. SC'11) ---- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_uniform52(uint32_t hi, uint32_t lo);
void or_normal_pair(const uint32_t w[4], double z[2]);
/* normals used by the closed loop: tag 0/1 process noise, 2 measurement, 3 params */
void or_process_noise(uint64_t seed, int64_t j, int64_t substep, double xi[3]);
double or_meas_noise(uint64_t seed, int64_t j, int64_t step);
void or_traj_params(const or_model* m, uint64_t seed, int64_t j,
                    double* EaR_j, double* t_d, double* dTin);
void or_traj_horizon(const or_ctrl* c, uint64_t seed, int64_t j, int* N, int* max_it);

/* ---- CSTR model, Eq. (CSTR) ---- */
void or_plant_drift(const or_model* m, double EaR, double T_in, const double n[3],
                    double F, double f[3]);
void or_model1(const or_model* m, double EaR, double x, double F,
               double* f, double* fx, double* fF);
double or_zbar(const or_model* m, double t);
double or_Fss(const or_model* m, double EaR, double Tbar);
void or_em_step(const or_model* m, double EaR, double T_in, double n[3], double F,
                double h, const double xi[3]);

/* ---- one shooting interval with classical RK4 and forward sensitivities ---- */
void or_rk4_interval(const or_model* m, double EaR, int n_rk4, double Ts, double x0,
                     double F, double Fconv, double* xF, double* A, double* B);

/* ---- CD-EKF ---- */
void or_ekf_predict(const or_model* m, double EaR, int n_rk4, double F, double* x,
                    double* P);
void or_ekf_filter(const or_model* m, double y, double* x, double* P,
                   double* P_short);

/* ---- structured QP subproblem, solved by condensing + primal active set ---- */
int or_qp_solve(int N, const double* A, const double* B, const double* b,
                const double* Wxx, const double* Wxu, const double* Wuu,
                const double* q, const double* r, const double* lb, const double* ub,
                double* du, double* dx, double* mu, double* nul, double* nuu,
                int* iters);

/* ---- damped BFGS update of one packed 1x1 or 2x2 Hessian block ---- */
void or_bfgs_block(int n, double* w, const double* s, const double* y);

/* ---- SQP for one OCP; warm start in u, x, lam, pil, piu (updated in place) ---- */
int or_sqp(const or_model* m, const or_ctrl* c, double EaR, double x0,
           const double* zbar /* zbar[k], k = 1..N */, double* u, double* x,
           double* lam, double* pil, double* piu, or_sqp_info* info);

/* One row per SQP iteration l (Sec. IV): what the
 * penalty update (Sec. IV-B), the Armijo backtracking (Eq. Armijo), the scaled
 * convergence test (Eq. convergence) and the Hessian reset (Sec. IV-C) saw and
 * decided, so that tests can check each decision against the paper's rules. */
#define OR_TRACE_MAX_TRIALS 64
typedef struct {
  int32_t l;            /* iteration index                                    */
  int32_t reset;        /* 1: the block update that opened this iteration
                           found a block not positive definite and reset all */
  int32_t n_trials;     /* merit evaluations of this line search              */
  int32_t accepted;     /* 1: a trial point was accepted                      */
  int32_t stop;         /* -1: the iteration went on to the QP; else the SQP
                           stopped here with this status (0 converged,
                           1 iteration limit)                                */
  int32_t pad0;
  double s_d;           /* scaling of the convergence test                    */
  double kkt_grad_raw;  /* ||grad_xi L||_inf before the scaling               */
  double kkt_grad;      /* the scaled value the test compared                 */
  double kkt_eq;        /* ||g||_inf                                          */
  double f;             /* objective at the iterate                           */
  double T0, DT0;       /* merit T(0) and its directional derivative          */
  double lam[OR_MAX_N], pil[OR_MAX_N], piu[OR_MAX_N];  /* multipliers at the
                           iterate (the ones the convergence test used)      */
  double g[OR_MAX_N];   /* constraint residuals g_k at the iterate            */
  double q[OR_MAX_N + 1], r[OR_MAX_N];   /* objective gradient at the iterate */
  double A[OR_MAX_N], B[OR_MAX_N];       /* shooting sensitivities there      */
  double du[OR_MAX_N], dx[OR_MAX_N + 1]; /* QP step                           */
  double mu[OR_MAX_N];  /* QP multipliers of the dynamics                     */
  double sigma[OR_MAX_N];                /* penalty weights after the update  */
  double alpha[OR_TRACE_MAX_TRIALS];     /* step length of each trial         */
  double f_trial[OR_TRACE_MAX_TRIALS];   /* objective at each trial point     */
  double pen_trial[OR_TRACE_MAX_TRIALS]; /* sigma^T |g| at each trial point   */
} or_sqp_trace_row;

/* or_sqp with the trace: rows[0 .. *n_rows-1] (at most max_rows). */
int or_sqp_traced(const or_model* m, const or_ctrl* c, double EaR, double x0,
                  const double* zbar, double* u, double* x, double* lam, double* pil,
                  double* piu, or_sqp_info* info, or_sqp_trace_row* rows, int max_rows,
                  int* n_rows);

/* The block-BFGS step of Sec. IV-C on all N + 1 packed blocks
 * (W[3k .. 3k+2] = W11, W12, W22 of block k; block 0 = [u_0], blocks
 * 1..N-1 = [x_k u_k], block N = [x_N]): each block is updated by the damped
 * BFGS formula with s = (s_x[k], s_u[k]) and y = (y_x[k], y_u[k]), then, if any
 * block is not positive definite, every block is reset to the identity.
 * Returns 1 after a reset, else 0. */
int or_bfgs_update_blocks(int N, double* W, const double* s_u, const double* s_x,
                          const double* y_u, const double* y_x);

/* ---- PI controller, Eq. (PI) ---- */
double or_pi_step(const or_ctrl* c, double Ts, double ybar, double y, double ubar,
                  double* Ihat);

/* du_0/d(x_0, Q_z, R_u, Q_n) at an OCP solution of or_sqp (implicit
 * differentiation of its KKT conditions); 0 or -1 (singular KKT matrix). */
int or_ocp_sens(const or_model* m, const or_ctrl* c, double EaR, double x0, const double* zbar,
                const double* u, const double* x, const double* lam, const double* pil,
                const double* piu, double* out);

/* ---- closed loop and Monte Carlo driver ---- */
/* trace (optional, may be NULL): per step i = 0..K-1 the row
 * (T_plant, y, xhat, u_applied_mLmin, sqp_iters)                        */
void or_traj(const or_model* m, const or_ctrl* c, uint64_t seed, int64_t j,
             or_traj_out* out, double* trace);
void or_run(const or_model* m, const or_ctrl* c, uint64_t seed, int64_t j0,
            int64_t j1, int n_threads, or_traj_out* out);

/* ---- three-state NMPC model (or_nmpc3.c) ---- */
void or_drift3(const or_model* m, double EaR, double T_in, const double n[3], double F,
               double f[3], double J[9], double fF[3]);
void or_rk4_interval3(const or_model* m, double EaR, int n_rk4, double Ts, const double x0[3],
                      double v, double Fconv, double xF[3], double A[9], double B[3]);
void or_ekf3_predict(const or_model* m, double EaR, int n_rk4, double F, double x[3],
                     double P[9]);
void or_ekf3_filter(const or_model* m, double y, double x[3], double P[9], double* P_short);
int or_qp3_solve(int N, const double* A, const double* B, const double* b, const double* Wxx,
                 const double* Wxu, const double* Wuu, const double* q, const double* r,
                 const double* lb, const double* ub, double* du, double* dx, double* mu,
                 double* nul, double* nuu, int* iters);
void or_bfgs_blockn(int n, double* W, const double* s, const double* y);
int or_sqp3(const or_model* m, const or_ctrl* c, double EaR, const double x0[3],
            const double* zbar, double* u, double* x, double* lam, double* pil, double* piu,
            or_sqp_info* info);

/* ---- derivatives of Phi_j with respect to the PI gains (or_grad.c) ---- */
/* Complex-step derivative of Phi_j with respect to gain `which` (0 = k_P,
 * 1 = k_I, 2 = k_aw), step h_cs (imaginary); returns Phi_j, *dphi = dPhi_j/dk. */
double or_pi_phi_cs(const or_model* m, const or_ctrl* c, uint64_t seed, int64_t j,
                    int which, double h_cs, double* dphi);
/* phi[j - j0] and dphi[3 (j - j0) + q] for q = k_P, k_I, k_aw, on n_threads
 * host threads (h_cs = 1e-20 |k|). */
void or_pi_grad_run(const or_model* m, const or_ctrl* c, uint64_t seed, int64_t j0,
                    int64_t j1, int n_threads, double* phi, double* dphi);
/* dPhi_j/d(Q_z, R_u, Q_n) of the one-state NMPC closed loop: complex step
 * through plant, measurement and CD-EKF, each OCP by its solution map with
 * the implicit derivative of or_ocp_sens (which = 0 Q_z, 1 R_u, 2 Q_n);
 * *n_sens_fail counts OCPs whose KKT matrix was singular. */
double or_nmpc_phi_cs(const or_model* m, const or_ctrl* c, uint64_t seed, int64_t j, int which,
                      double h_cs, double* dphi, int* n_sens_fail);
void or_nmpc_grad_run(const or_model* m, const or_ctrl* c, uint64_t seed, int64_t j0,
                      int64_t j1, int n_threads, double* phi, double* dphi, int* fails);

#ifdef __cplusplus
}
#endif
#endif
