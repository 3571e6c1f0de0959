/*
 * parareal.h - C ABI of the GB300 (sm_103a) hot path of the MOR-based adaptive parareal
 * method of arXiv 2601.10981 for  u_t + b.grad(u) = eps Lap(u) + f  on a periodic cube.
 *
 * Plain C: every argument is a pointer, a size or a scalar.  "host" pointers are CPU
 * memory owned by the caller and only read (or written) during the call; "device"
 * pointers are CUDA global memory on the current device, owned by the caller unless
 * stated otherwise.  Grid functions are n^3 doubles laid out [z][y][x] (x fastest).
 * Every call returns a pr_status; on failure pr_last_error() describes it.  Phase calls
 * are asynchronous on the stream set by pr_set_stream (default: the legacy stream);
 * calls documented as "synchronises" wait for that stream.  A context is used by one
 * host thread at a time.
 */
#ifndef PARAREAL_H
#define PARAREAL_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pr_ctx pr_ctx;

typedef enum pr_status {
    PR_OK = 0,
    PR_ERR_INVALID_ARG = 1,    /* bad size, pointer or option                          */
    PR_ERR_OOM = 2,            /* device memory could not be allocated / bound buffer too small */
    PR_ERR_CUDA = 3,           /* a CUDA runtime call failed                           */
    PR_ERR_NOT_CONVERGED = 4,  /* BiCGStab hit lin_maxit in some fine step             */
    PR_ERR_BREAKDOWN = 5,      /* BiCGStab breakdown, or a non-positive Cholesky pivot */
    PR_ERR_TIMEOUT = 6,        /* an in-kernel barrier exceeded its spin limit          */
    PR_ERR_NONFINITE = 7,      /* NaN/Inf in the initial data or in an iterate          */
    PR_ERR_STATE = 8,          /* phase called out of order                            */
    PR_ERR_UNSUPPORTED = 9     /* valid request this build does not implement          */
} pr_status;

/* Velocity fields b(x).  Each component is a sum of 1-D functions of the two other
 * coordinates (b_x(y,z), b_y(x,z), b_z(x,y)), which is what makes central advection
 * exactly skew-symmetric on the periodic grid. */
enum pr_flow_kind {
    PR_FLOW_ABC = 0,        /* (A sin z + C cos y, B sin x + A cos z, C sin y + B cos x) */
    PR_FLOW_KOLMOGOROV = 1, /* (sin(k y), 0, 0)                                          */
    PR_FLOW_CONST = 2,      /* (b[0], b[1], b[2])                                        */
    /* the time-dependent flows of Sec. 4, with their forcing added to the given f:       */
    PR_FLOW_PAPER_KOLMOGOROV = 3, /* eq. (koleq): (cos y, cos z, cos x) +
                                     (sin z, sin x, sin y) cos t, f += -cos y - sin z cos t */
    PR_FLOW_PAPER_ABC = 4   /* Sec. 4.2: ABC (A = B = C = 1) with every argument shifted
                               by sin(w t), f += -sin(z + sin wt) - cos(y + sin wt)      */
};

/* Arithmetic of the fine Krylov solves.  Interface states U^k_n, fine states and end
 * states, snapshots, POD bases, Grams, eigenproblems and reduced systems are FP64 in both
 * modes: the augmentation of eq. (eqaug) resolves U^k_n against the POD space to
 * ||d~||/||U|| ~ 1e-9, which a basis rounded to FP32 cannot. */
enum pr_precision {
    PR_FP64 = 0,            /* everything FP64                                           */
    PR_FP32 = 1             /* fine sweep: FP64 state, FP32 BiCGStab for the increment
                               ("delta form"), FP64 residual of the state               */
};

typedef struct pr_grid {
    int n;                  /* points per direction, 4 <= n <= 1024                      */
    double L;               /* cube edge; <= 0 means 2*pi                               */
} pr_grid;

typedef struct pr_flow {
    int kind;               /* enum pr_flow_kind                                        */
    double A, B, C;         /* ABC coefficients                                         */
    int k;                  /* Kolmogorov wave number                                   */
    double b[3];            /* constant velocity                                        */
    double w;               /* time frequency of PR_FLOW_PAPER_ABC                       */
    const double* pert;     /* optional stored velocity perturbation added to a steady
                               kind: host array [3][n^3] (b'_x, b'_y, b'_z, each [z][y][x],
                               x fastest), copied by pr_create, caller keeps ownership;
                               NULL: none.  Time-dependent kinds and PR_FINE_RK4 with a
                               perturbation return PR_ERR_UNSUPPORTED.  The advection
                               stencil reads it per point (no skew-symmetry is assumed).  */
} pr_flow;

/* Options; pr_opts_init fills the defaults.  Values marked "0: derive" are computed from
 * the problem in pr_create following the paper's parameter ratios (Sec. 4). */
typedef struct pr_opts {
    double T0;              /* Case-I window [0,T0] (Sec. 2.3); 0: derive = DeltaT        */
    double dT;              /* coarse step; 0: derive = DeltaT/10 (ratio of Sec. 4.1)     */
    int n_snap;             /* snapshots per window; 0: one every delta_M = 5 fine steps,
                               n_s = floor(S/delta_M)+1 (Case I); else delta_M =
                               floor(S/(n_snap-1))                                       */
    int m_cap;              /* cap on every POD dimension; 0: none                       */
    int m_l, p;             /* left neighbours / previous iterations in W^k_n, eq. (W^k_n);
                               each 0 or 1; default 1, 1                                  */
    double pod_tol3;        /* gamma3 = 1 - pod_tol3; 0: derive = pod_tol * 4e-3          */
    double rank_tau;        /* eigenvalues <= rank_tau*lambda_1 count as zero (Alg. 1);
                               0: derive = 1e-13                                         */
    int precision;          /* enum pr_precision; default PR_FP64                        */
    double lin_tol;         /* BiCGStab stops at ||r|| <= lin_tol ||rhs||;
                               0: derive = 1e-14 (FP64) or 1e-9 (FP32)                   */
    int lin_maxit;          /* BiCGStab iteration cap per fine step; default 200         */
    double aug_tol;         /* no augmentation if ||d~|| <= aug_tol ||U||; default 1e-12  */
    int group_ctas;         /* CTAs cooperating on one subinterval in the fine sweep (its
                               tile-planes split evenly over them; capped at their count);
                               0: every co-resident CTA slot over the subintervals        */
    int ctas_per_sm;        /* resident CTAs per SM for the fine sweep; 0: occupancy max  */
    long long spin_limit;   /* polls of an in-kernel barrier or mbarrier before
                               PR_ERR_TIMEOUT (default 1<<22, a few seconds; 0: one
                               non-blocking check, so a wait not already complete fails) */
    int method;             /* enum pr_method; default PR_METHOD_ADAPTIVE                 */
    int fine;               /* enum pr_fine; default PR_FINE_IMPLICIT_EULER               */
    int wave;               /* adaptive method only.  0 (default): pr_fine_sweep covers all
                               active subintervals in one launch, the snapshot store holds
                               all their windows and the level-2 bases of all of them.
                               w > 0 (w < n_sub): pr_fine_sweep streams iteration k in waves
                               of w subintervals (n = k-1, k, ... in order): per wave the
                               fine sweep, the level-1 POD, the level-2 POD and Galerkin
                               matrices of its subintervals and their share of the
                               sequential coarse sweep; pr_pod_update and pr_coarse_sweep
                               then only advance the phase.  The workspace holds one wave's
                               snapshots, level-2 bases and scratch and one generation of
                               level-1 bases (replaced wave by wave), which is what lets the
                               128^3 x 256 and 256^3 x 128 problems fit one GPU.  Every step
                               sees the inputs it has with w = 0, in the same order, so the
                               iterates are bit-identical for a fixed group_ctas.
                               pr_rewind can only undo iteration 1; pr_get_snapshots and
                               pr_get_basis(level 2) reach the last wave's subintervals only. */
    int gram_mode;          /* enum pr_gram_mode: which kernel forms the FP32 mode's symmetric
                               POD Grams (level 1, Cholesky QR); default PR_GRAM_AUTO        */
} pr_opts;

/* Fine integrator.  PR_FINE_IMPLICIT_EULER: the paper's, eq. (semi-dis-eq), BiCGStab per
 * step.  PR_FINE_RK4: the classical explicit fourth-order Runge-Kutta method on
 * u' = f(t) - L_h(t) u with the same step (no counterpart in the paper; the caller keeps
 * dt within its stability bound, about 2.78 / (12 eps / h^2) for diffusion and
 * 2.8 h / (|b_x| + |b_y| + |b_z|) for advection). */
enum pr_fine { PR_FINE_IMPLICIT_EULER = 0, PR_FINE_RK4 = 1 };

/* PR_METHOD_ADAPTIVE: Algorithm 2.  PR_METHOD_PARAREAL_I: the comparator "Parareal-I" of
 * Sec. 4, plain parareal whose coarse space is the iteration-0 POD space V0 for every
 * subinterval and iteration (no level-1/2 POD, no augmentation; pr_pod_update does
 * nothing, snapshots are not taken); the paper gives it a longer window T0 = 10.
 * PR_METHOD_PARAREAL_II: the comparator "Parareal-II", plain parareal whose coarse
 * propagator is implicit Euler with step dT on the grid coarsened by 2 (n even, n/2 >= 4):
 * G(x) = P G_c(R x), restriction by injection, trilinear prolongation; iteration 0 keeps
 * the Case-I window [0, T0] and then U^0_{n+1} = G(U^0_n). */
enum pr_method { PR_METHOD_ADAPTIVE = 0, PR_METHOD_PARAREAL_I = 1, PR_METHOD_PARAREAL_II = 2 };

/* Symmetric Gram kernels of the FP32 mode.  PR_GRAM_DF: double-float arithmetic on the
 * FP32 pipe (up to 126 columns, windows wider than 54 columns in several passes over the
 * data; FP64 beyond).  PR_GRAM_TENSOR: the tensor cores, with the values cut into
 * error-free BF16 digits (FP64-accurate, see pr_op_gram; up to 64 columns, double-float
 * beyond).  PR_GRAM_AUTO: the tensor cores for snapshot windows of 20..32 columns (where
 * the narrow tensor-core form is faster) and 55..64 columns (where the double-float
 * kernel would need two passes), double-float otherwise (and for the Cholesky-QR Grams,
 * whose column counts are POD dimensions known only on the device).  The FP64 mode always
 * forms its Grams in FP64. */
enum pr_gram_mode { PR_GRAM_AUTO = 0, PR_GRAM_DF = 1, PR_GRAM_TENSOR = 2 };

/* Per-solve report (pr_solve).  Times are seconds measured with CUDA events. */
typedef struct pr_report {
    int k;                  /* parareal iterations performed (k >= 1)                    */
    int converged;          /* criterion met                                             */
    double max_inc;         /* max_n ||U^k_n - U^{k-1}_n|| / ||U^k_n|| at the last k      */
    double max_err;         /* max_n error of eq. (error) against the reference; -1 if none */
    double t_iter0, t_fine, t_pod, t_coarse, t_check, t_total;
    double fine_dof_steps;  /* grid points x fine steps propagated by F (all iterations) */
    double lin_iters_mean;  /* BiCGStab iterations per fine step, mean                   */
    int lin_iters_max;
    int m0;                 /* dimension of V0 (iteration 0)                              */
    int m1_max, m2_max;     /* largest level-1 / level-2 POD dimension at the last k     */
} pr_report;

/* Fill *opts with defaults. */
void pr_opts_init(pr_opts* opts);

/* Create a solver for Algorithm 2 on [0, T0 + T]: the fine propagator on [0, T0] (Case I)
 * and parareal with n_sub subintervals of length DeltaT = T / n_sub on [T0, T0 + T].
 *   grid, flow: problem (host structs, copied).   eps > 0: diffusion.   T > 0.
 *   dt_fine: requested fine step; the step used is DeltaT / S, S = ceil(DeltaT/dt_fine)
 *            (ratios within 1e-9 of an integer are rounded).
 *   pod_tol: gamma1 = gamma2 = 1 - pod_tol (Algorithm 1); the paper uses 5e-6.
 *   opts: NULL for defaults.   *out receives the context (free with pr_destroy).
 * Selects the current CUDA device; allocates nothing on it yet. */
pr_status pr_create(const pr_grid* grid, const pr_flow* flow, double eps, double T,
                    int n_sub, double dt_fine, double pod_tol, const pr_opts* opts,
                    pr_ctx** out);
void pr_destroy(pr_ctx* ctx);

/* Derived sizes: fine steps per subinterval S, steps on [0,T0] S0, snapshot stride and
 * counts, coarse steps per subinterval; any pointer may be NULL. */
pr_status pr_get_sizes(const pr_ctx* ctx, int* S, int* S0, int* dM, int* n_s, int* n_s0,
                       int* Lc, double* dt_eff, double* DeltaT);

/* Device bytes the context needs.  pr_bind_workspace hands it a caller-owned device
 * buffer of at least that size (e.g. a torch tensor); otherwise the first phase call
 * allocates it with cudaMalloc and pr_destroy frees it. */
size_t pr_workspace_bytes(const pr_ctx* ctx);
pr_status pr_bind_workspace(pr_ctx* ctx, void* device_ptr, size_t bytes);

/* Stream (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream) for all work. */
pr_status pr_set_stream(pr_ctx* ctx, void* cuda_stream);

/* Initial state u0 and forcing f (n^3 host doubles each, copied; f may be NULL for 0).
 * Resets the iteration state.  PR_ERR_NONFINITE if u0 or f holds NaN/Inf. */
pr_status pr_set_initial(pr_ctx* ctx, const double* u0, const double* f);

/* Iteration 0 (Case I, Algorithm 2): fine propagator on [0,T0] with snapshots,
 * V0 = POD_Mode(W, gamma1), U^0_0 = u_hat0, U^0_{n+1} = G_0(P_{V0} U^0_n). */
pr_status pr_iteration0(pr_ctx* ctx);

/* Parareal iteration k >= 1, three phases that must run in this order:
 *  pr_fine_sweep:   F_n = F(t_n, t_{n+1}, U^{k-1}_n) and snapshots W^k_{n,0} for
 *                   n = k-1..N-1, all subintervals in one persistent launch.
 *  pr_pod_update:   R^k_{n,0} = POD_Mode(W^k_{n,0}, gamma2) for n = k-1..N-1, the level-2
 *                   basis R^k_n = POD_Mode(W^k_n, gamma3) of eq. (W^k_n) and its Galerkin
 *                   matrices for n = k..N-1.
 *  pr_coarse_sweep: sequential over n = k..N-1: augmentation (eqs. (eqaug), (eq12)), the
 *                   bordered reduced system (eq13) and the update of eq. (formula4),
 *                   U^k_{n+1} = G(U^k_n) + F_n - G(P U^{k-1}_n); U^k_n = U^{k-1}_n (n<k),
 *                   U^k_k = F_{k-1}. */
pr_status pr_fine_sweep(pr_ctx* ctx, int k);
pr_status pr_pod_update(pr_ctx* ctx, int k);
pr_status pr_coarse_sweep(pr_ctx* ctx, int k);

/* pr_fine_sweep for several contexts at once (no counterpart in the paper: it serves
 * several problems on one GPU).  ks[i] is the iteration of ctxs[i]; all contexts need
 * the same n, box and precision, count <= 16, each context at most once.  Their
 * subintervals share one persistent launch of the fine kernel, one job per context,
 * issued on the stream of the context with the most CTA groups and ordered after each
 * context's earlier work and before its later work; each context then continues with
 * pr_pod_update.  With a fixed pr_opts.group_ctas the results are bit-identical to
 * pr_fine_sweep on each context alone.  A launch-wide device error (barrier time-out) is
 * recorded in that owning context only.  Asynchronous. */
pr_status pr_fine_sweep_batch(pr_ctx* const* ctxs, const int* ks, int count);

/* Autotuner of the fine launch shape (no counterpart in the paper): times `steps` fine
 * steps of all n_sub subintervals from the current iterate for CTA-group sizes G = the
 * co-resident CTA count / n_sub and G = (n / tile rows) * 2^j up to the co-resident CTA
 * count, keeps the fastest in the
 * context (pr_opts.group_ctas) and returns it (best_ms: its time, may be NULL).  Needs
 * iteration 0 done and no phase of the next iteration started; leaves the iterate
 * unchanged.  Synchronises. */
pr_status pr_tune_fine(pr_ctx* ctx, int steps, int* best_group_ctas, double* best_ms);

/* Convergence after pr_coarse_sweep(k): max increment max_n ||U^k_n-U^{k-1}_n||/||U^k_n||
 * and, if a reference is set, the max error of eq. (error).  Synchronises; also returns
 * any error a kernel recorded since the last check. */
pr_status pr_check(pr_ctx* ctx, int k, double* max_inc, double* max_err);

/* Whole Algorithm 2: iteration 0 (if not yet done), then k = 1, 2, ... until the
 * criterion holds (error against the reference <= tol if ref or a set reference exists,
 * else increment <= tol), k = n_sub or k = k_max (<= 0: n_sub).  ref: NULL or host
 * (n_sub+1) x n^3 doubles U_0..U_N of the sequential fine solution.  Synchronises. */
pr_status pr_solve(pr_ctx* ctx, double tol, int k_max, const double* ref, pr_report* out);

/* Sequential fine solution U_n = F(0, t_n, u0), n = 0..N, one subinterval after another
 * on the GPU (the cost_seq form of Sec. 3.3); kept as the context's reference.
 * fp64: 1 computes it with FP64 Krylov solves whatever the context precision. */
pr_status pr_compute_reference(pr_ctx* ctx, int fp64);
/* Reference from the caller: (N+1) x n^3 doubles, host (on_device = 0) or device (1). */
pr_status pr_set_reference(pr_ctx* ctx, const double* U, int on_device);

/* Interface states of the latest iteration (U^k after pr_coarse_sweep(k), U^0 after
 * pr_iteration0).  pr_get_interface copies U_n, pr_get_interfaces all N+1 of them, to
 * host memory.  Synchronise. */
pr_status pr_get_interface(pr_ctx* ctx, int n, double* host_out);
pr_status pr_get_interfaces(pr_ctx* ctx, double* host_out);
/* Replace the latest iterate by host (N+1) x n^3 doubles and declare it iteration k_done
 * (0 <= k_done < N): the next phase is pr_fine_sweep(k_done+1).  Needs iteration 0 done
 * (V0 is part of the state). */
pr_status pr_set_interfaces(pr_ctx* ctx, const double* host_U, int k_done);

/* Undo the latest completed iteration k >= 1 (its predecessor U^{k-1} and the level-1
 * bases of iteration k-1 are still resident): the next phase is pr_fine_sweep(k) again.
 * One level deep; used to repeat an iteration on identical inputs. */
pr_status pr_rewind(pr_ctx* ctx);

/* Read back, to host memory, what the latest phases produced for subinterval n:
 * F_n of the last fine sweep (n^3 doubles); its snapshots W^k_{n,0} (n_s x n^3 doubles;
 * slot 0 holds the Case-I window after pr_iteration0); and a basis:
 * level 0 = V0 (n ignored), 1 = R^k_{n,0}, 2 = R^k_n, m_out receives its dimension and
 * host_out (may be NULL) m x n^3 doubles.  Synchronise. */
pr_status pr_get_fine_end(pr_ctx* ctx, int n, double* host_out);
pr_status pr_get_snapshots(pr_ctx* ctx, int n, void* host_out);
pr_status pr_get_basis(pr_ctx* ctx, int level, int n, void* host_out, int* m_out);

/* Per-subinterval diagnostics of the last pr_check: increments and errors (N+1 each,
 * host, may be NULL), and POD dimensions m0 / m^k_{n,0} / m^k_n (N each, may be NULL).
 * Synchronise. */
pr_status pr_get_diagnostics(pr_ctx* ctx, double* inc, double* err, int* m0, int* m1,
                             int* m2);
/* BiCGStab iteration counts of the last fine sweep: total and max over steps, per
 * subinterval n (N each, host; entries of inactive subintervals are 0).  Synchronises. */
pr_status pr_get_lin_stats(pr_ctx* ctx, int* total, int* max_per_step);

/* Device time of the fine-kernel launches of the last pr_fine_sweep (one launch, or one a
 * wave in wave mode, measured with CUDA events around each launch on the context stream):
 * *ms their summed milliseconds, *launches (may be NULL) their count.  PR_ERR_STATE before
 * the first fine sweep.  Synchronises on the last launch. */
pr_status pr_get_fine_ms(pr_ctx* ctx, double* ms, int* launches);

/* Wait for the stream; return the first error any kernel recorded. */
pr_status pr_sync(pr_ctx* ctx);
const char* pr_last_error(const pr_ctx* ctx);
const char* pr_status_string(pr_status s);
/* Number of kernels this library has launched in this process. */
long long pr_launch_count(void);

/* ---- single steps on caller data (device pointers), same kernels as the phases ---- */

/* out = L_h u (transpose = 0) or L_h^T u (1) for `count` grid functions, the FD operator
 * of eq. (eq1) (central advection, 7-point Laplacian).  d_in, d_out: count x n^3. */
pr_status pr_op_apply_L(pr_ctx* ctx, const double* d_in, double* d_out, int count,
                        int transpose);

/* out = L_h u as the FP32 mode's Galerkin projection forms it (Algorithm 2, the reduced
 * operator R^T L R): the stencil weights and values split into float pairs and summed with
 * error-free products and TwoSums on the FP32 pipe, within ~1e-14 of the sum of the seven
 * terms' magnitudes at each point (pr_op_apply_L computes the same operator in FP64).
 * d_in, d_out: count x n^3 device doubles.  Steady flows only (PR_ERR_UNSUPPORTED for a
 * time-dependent one).  Synchronises the context stream. */
pr_status pr_op_apply_L_df(pr_ctx* ctx, const double* d_in, double* d_out, int count);

/* Fine propagator on B independent states: d_out[b] = F(t0, t0 + steps*dt, d_in[b]) with
 * snapshots of the states at steps 0, dM, ... (n_snap of them; d_snap may be NULL when
 * n_snap = 0).  d_in, d_out: B x n^3 doubles.  d_snap: B x n_snap x n^3 doubles (snapshots
 * are FP64 in both precision modes).  1 <= B <= n_sub.  The forcing is
 * the one given to pr_set_initial (zero before the first call). */
pr_status pr_op_fine(pr_ctx* ctx, const double* d_in, double* d_out, void* d_snap, int B,
                     double t0, int steps, int dM, int n_snap);

/* POD_Mode (Algorithm 1) with one Cholesky-QR re-orthonormalisation pass on B snapshot matrices:
 * d_W: B x n_cols x n^3 doubles (w_f32 = 0; the level-1 path, numerical zero 1e-13) or
 * floats (w_f32 = 1; Gram accumulated over 32-point blocks in FP32, numerical zero 1e-6);
 * d_R: B x m_max x n^3 doubles, m_max = min(cap, n_cols) or
 * n_cols when cap = 0; gamma in (0,1]; m_out: host, B ints.  n_cols <= the largest window
 * the context was built for (max(n_s, n_s0, (m_l+1+p) * level-1 cap)); B <= n_sub. */
pr_status pr_op_pod(pr_ctx* ctx, const void* d_W, int w_f32, int n_cols, int B, double gamma,
                    int cap, void* d_R, int* m_out);

/* Gram matrices G_b = W_b^T W_b of B snapshot matrices, step 1 of POD_Mode (Algorithm 1)
 * (M = I).  d_W: B x n_cols x n^3 device doubles (column-major blocks as for pr_op_pod);
 * d_G: B x n_cols x n_cols device doubles (row-major, symmetric).  tensor selects the
 * arithmetic:
 *   1: the tensor cores (tcgen05.mma, BF16 operands, FP32 accumulation; n_cols <= 64).
 *      Each column is aligned to its largest magnitude and each value truncated to 56
 *      bits and cut into eight balanced base-128 integer digits, which BF16 holds
 *      exactly; digit products are summed exactly in FP32 over windows of points.  Up to
 *      32 columns the windows are folded into 128-bit integers, so the result is the
 *      digit sum rounded once to FP64 (bit-reproducible); 33..64 columns fold them into
 *      FP64 every 1024 points.  Either way FP64-accurate.
 *   2: double-float arithmetic on the FP32 pipe (the FP32 mode's default kernel).
 *   0: FP64 arithmetic.
 * B <= n_sub + 1, n_cols <= the context's largest POD window.  Synchronises. */
pr_status pr_op_gram(pr_ctx* ctx, const double* d_W, int n_cols, int B, double* d_G, int tensor);

/* One coarse update of eq. (formula4) on subinterval [t, t+DeltaT] with the augmented
 * space [R, d(U)]:  d_out = G(U) + F - G(P U_prev).  d_R: m x n^3 doubles (orthonormal
 * columns), d_U, d_Uprev, d_F, d_out: n^3 doubles. */
pr_status pr_op_coarse_update(pr_ctx* ctx, const void* d_R, int m, const double* d_U,
                              const double* d_Uprev, const double* d_F, double* d_out);

/* The operator of pr_op_apply_L without any device allocation, for callers that cannot
 * call cudaMalloc (another framework's allocator owns the device memory budget, or the
 * caller must not trigger the allocator's synchronisation).  It does not need a bound
 * workspace: its scratch (velocity tables, pointer lists) is one static device array of
 * 13 568 bytes that every GPU loading this library holds until the process exits.
 * Limits: n <= 256 and count <= 64 grid functions per call (PR_ERR_INVALID_ARG beyond).
 * d_in, d_out: count x n^3 device doubles.  Runs on the context stream and synchronises
 * it before returning.  A stored velocity perturbation (pr_flow.pert) lives in the
 * workspace: with one, bind the workspace and call pr_set_initial first
 * (PR_ERR_UNSUPPORTED otherwise).  The first call on a device looks up the array's device
 * address and keeps it for the life of the process; do not use the library across a
 * cudaDeviceReset (the kept address would be stale).  All calls share the array and leave
 * the last call's contents; each call rewrites what it reads, but calls that overlap on
 * the GPU (different streams, no ordering) race on it.  The paper has no counterpart: this is library plumbing. */
pr_status pr_op_apply_L_noalloc(pr_ctx* ctx, const double* d_in, double* d_out, int count,
                                int transpose);

/* ---------------------------------------------------------------------------------------
 * Serving (no counterpart in the paper, which solves one problem at a time on a CPU
 * cluster): parareal solves of different n, flows and eps arrive over time and share the
 * GPU by continuous batching.
 *
 * A submitted request waits in arrival order until its workspace (pr_workspace_bytes)
 * fits the memory budget next to the resident requests and the resident cap allows it;
 * it is then admitted (device workspace and stream of its own, initial state copied,
 * iteration 0 issued) and stays resident until it finishes.  Requests advance on their
 * own iteration clocks, not in lock-step: each has at most one iteration in flight on its
 * stream.  Each pr_server_step admits waiting requests; finds the requests whose work in
 * flight has completed (polling for up to about a millisecond if none has), checks their
 * convergence and retires the finished ones (max increment
 * max_n ||U^k_n - U^{k-1}_n|| / ||U^k_n|| <= tol or k = k_max: U^k_N is copied to host
 * memory, the workspace released and waiting requests admitted at once); and issues the
 * next iteration of every ready request: fine sweeps of ready requests with the same n,
 * box and precision share persistent launches (pr_fine_sweep_batch, up to 16 requests
 * each), then each request's POD update and coarse sweep on its own stream, so that the
 * requests' work overlaps on the device.  A small request thus finishes while a large
 * one is mid-solve.  The fine CTA-group size is tuned once per (n, box, precision) by
 * pr_tune_fine on the first request admitted with opts.group_ctas = 0 and used for every
 * later request of that shape; a request with group_ctas > 0 keeps its own, and then
 * gives the same result alone and in a mix.
 * Single-threaded: one thread calls the pr_server_* functions of a server.
 * ------------------------------------------------------------------------------------ */
typedef struct pr_server pr_server;
typedef struct pr_server_opts {
    size_t hbm_budget;   /* bytes of request workspaces resident at once; 0: 90% of the
                            device memory free at pr_server_create */
    int max_active;      /* resident requests at once; 0: memory is the only limit */
    int batch_fine;      /* 1 (default): shared fine launches; 0: one launch per request */
} pr_server_opts;
typedef struct pr_request {
    pr_grid grid;
    pr_flow flow;
    double eps, T;
    int n_sub;
    double dt_fine;
    double pod_tol;
    pr_opts opts;        /* as for pr_create */
    const double* u0;    /* host n^3 doubles, copied by pr_server_submit */
    const double* f;     /* host n^3 doubles or NULL, copied */
    double tol;          /* increment tolerance, > 0 */
    int k_max;           /* <= 0 or > n_sub: n_sub */
} pr_request;
enum { PR_REQ_PENDING = 0, PR_REQ_ACTIVE = 1, PR_REQ_DONE = 2, PR_REQ_FAILED = 3 };

void pr_server_opts_init(pr_server_opts* opts);
/* opts may be NULL (defaults).  Allocates nothing on the device. */
pr_status pr_server_create(const pr_server_opts* opts, pr_server** out);
/* Releases every request's device memory and stream. */
void pr_server_destroy(pr_server* srv);
/* Queue a request; *id numbers requests 0, 1, 2, ... in submission order. */
pr_status pr_server_submit(pr_server* srv, const pr_request* req, int* id);
/* Admit; check the requests whose iteration in flight completed (polling up to about a
 * millisecond for one), retire finished ones and admit again; issue the next iteration of
 * every ready request.  n_active / n_pending (may be NULL): resident and waiting requests
 * after the step.  Call it repeatedly; it does not wait for all resident requests. */
pr_status pr_server_step(pr_server* srv, int* n_active, int* n_pending);
/* state: PR_REQ_*, k: iterations done, max_inc: increment of the last check. */
pr_status pr_server_query(pr_server* srv, int id, int* state, int* k, double* max_inc);
/* U^k_N of a finished request (n^3 doubles, host).  PR_ERR_STATE if not finished. */
pr_status pr_server_result(pr_server* srv, int id, double* host_out);
/* Why a request failed ("" otherwise), and the last error of a server call. */
const char* pr_server_request_error(const pr_server* srv, int id);
const char* pr_server_last_error(const pr_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* PARAREAL_H */
