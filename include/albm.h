/*
 * albm.h - C ABI of the GB300 adjoint Lattice Boltzmann library (libalbm.so).
 *
 * The operations follow the paper's statement of the problem
 * (Laniewski-Wollk & Rokicki, "Adjoint Lattice Boltzmann for Topology
 * Optimization on multi-GPU architecture"):
 *
 *   lattice L = {0..Lx-1} x {0..Ly-1} x {0..Lz-1}, densities f: L -> R^M,
 *   one step  f^{n+1}_j(x + e_j) = W^x_j(f^n(x), theta)      (Sec. 2.1,
 *             Eq. "normal:iteration", shifts periodic),
 *   objective J = sum_n c_n sum_x F^x(f^n(x))                (Eq.
 *             "objective:function", with time weights c_n),
 *   adjoint   lambda^n_k(x) = sum_j lambda^{n+1}_j(x + e_j) dW^x_j/df_k
 *                             + c_n dF^x/df_k                (Eqs.
 *             "adjoint:iteration" and "adjoint:operator", unsteady form),
 *   gradient  dJ/dtheta(x) = sum_n sum_j lambda^{n+1}_j(x + e_j) dW^x_j/dtheta
 *                            + sum_n c_n dF^x/dtheta         (Eq.
 *             "adjoint:derivative", accumulated over the time steps).
 *
 * Conventions shared by every call:
 *  - Node index idx = x + Lx*(y + Ly*z) (x fastest).  Per-node arrays hold N =
 *    Lx*Ly*Lz entries.  Population arrays are structure-of-arrays: density m
 *    of node idx at [m*N + idx], m = 0..M-1 with the Q fluid populations
 *    first (paper order e1..e19, or its z = 0 members in 2D) followed by
 *    each scalar lattice's Qs populations.
 *  - theta is the solid fraction per node (0 = fluid, 1 = solid), i.e.
 *    1 - w for the paper's w of Sec. 3.2.
 *  - Pointer arguments marked "host or device" may point to host memory
 *    (pageable or pinned) or to device memory of the handle's device; the
 *    library copies through unified addressing.  The caller keeps ownership
 *    of every pointer it passes; the library keeps none of them.
 *  - Every call returns an lbm_status and never throws; lbm_last_error()
 *    gives a message for the last failure on a handle.
 *  - Calls are asynchronous on the handle's CUDA stream unless stated.
 *  - A handle is not thread-safe: one host thread drives it at a time.
 */
#ifndef ALBM_H
#define ALBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx* lbm_handle;

typedef enum {
  LBM_OK = 0,
  LBM_ERR_ARG = 1,        /* invalid argument or unsupported combination   */
  LBM_ERR_OOM = 2,        /* device allocation failed                      */
  LBM_ERR_CUDA = 3,       /* a CUDA runtime call or kernel launch failed   */
  LBM_ERR_NONFINITE = 4,  /* a non-finite value was found in the state     */
  LBM_ERR_TIMEOUT = 5,    /* a bounded device wait expired                 */
  LBM_ERR_STATE = 6       /* call out of order (e.g. adjoint before primal)*/
} lbm_status;

typedef enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1 } lbm_lattice;
typedef enum { LBM_BGK = 0, LBM_MRT = 1 } lbm_collision;
typedef enum { LBM_FP32 = 0, LBM_BF16 = 1, LBM_FP16 = 2 } lbm_precision;
typedef enum { LBM_POR_LINEAR = 0, LBM_POR_POWER = 1, LBM_POR_RAMP = 2 } lbm_porosity;
typedef enum {
  LBM_OBJ_NONE = 0,
  LBM_OBJ_DISSIPATION = 1, /* sum over FLUID nodes of 2 rho nu S:S            */
  LBM_OBJ_VARIANCE = 2,    /* outlet variance of scalar 0                     */
  LBM_OBJ_HEATFLUX_DP = 3, /* outlet sum u_x T (Eq. exchanger:obj) - 0.1 dp   */
  LBM_OBJ_MIXFLUX = 4,     /* outlet sum u_x (1 - T^2) (Eq. mixing:obj)        */
  LBM_OBJ_HEATFLUX = 5     /* outlet sum u_x T alone (Eq. exchanger:obj)       */
} lbm_objective_kind;

/* Node types of the uint8 flag array (Sec. 3: interior, inlet/outlet, wall). */
enum {
  LBM_NODE_FLUID = 0,  /* FMRT/BGK with Exact-Difference forcing and porosity */
  LBM_NODE_WALL = 1,   /* full-way bounce-back of every lattice               */
  LBM_NODE_INLET = 2,  /* Zou-He inlet on the x = 0 face (velocity/pressure) */
  LBM_NODE_OUTLET = 3, /* Zou-He pressure outlet on the x = Lx-1 face         */
  LBM_NODE_HOT = 4     /* fluid bounce-back, scalars at equilibrium T_hot     */
};

/* Problem description (plain values; copied by lbm_create). */
typedef struct {
  int lattice;          /* lbm_lattice                                       */
  int nx, ny, nz;       /* lattice size; nz = 1 for D2Q9                      */
  int collision;        /* lbm_collision (Sec. 3.1: Eq. SRT or FMRT)          */
  double tau;           /* 1/omega = tau = 0.5 + 3 nu (0.5 < tau)             */
  double s_other;       /* MRT rate of the non-stress, non-conserved moments  */
  double force[3];      /* body acceleration g (Exact-Difference forcing)     */
  int walls;            /* bit 0: wall planes y = 0, Ly-1; bit 1: z = 0, Lz-1 */
  int inlet_outlet;     /* 0: periodic x; 1: Zou-He inlet x=0, outlet x=Lx-1 */
  double u_in;          /* inlet velocity (x component)                      */
  double rho_out;       /* outlet density                                    */
  int nscalars;         /* passive scalar lattices: 0, 1 or 2                 */
  double alpha_fluid;   /* scalar diffusivity at theta = 0                    */
  double alpha_solid;   /* scalar diffusivity at theta = 1 (Sec. 3.2 interp.) */
  int scalar_inlet;     /* 0: zero; 1: halves (0 for y < Ly/2, else 1; odd
                           scalars carry the complement 1 - c); 2: signed
                           (-1 for y < Ly/2, else +1, the paper's mixer
                           inlet, Sec. 4.1; odd scalars carry -c)            */
  int hot[4];           /* x0, x1, z0, z1 of the T_hot patch on y = 0; x1<=x0
                           means none                                        */
  double T_hot;
  int porosity;         /* lbm_porosity: G(theta) of the Darcy damping        */
  double porosity_q;
  int objective;        /* lbm_objective_kind                                */
  int obj_window;       /* 0: J = F(f^N); K > 0: J = (1/K) sum_{N-K<n<=N} F(f^n) */
  int nsteps;           /* horizon N of the unsteady problem                 */
  int precision;        /* lbm_precision of the stored populations           */
  int ckpt_every;       /* level-1 checkpoint stride (0 = automatic)         */
  double mem_budget;    /* bytes for stored states (0 = 0.90 of the free
                           device memory at lbm_create)                      */
  int kernel;           /* 0: automatic (one thread per node); 1: one thread
                           per node, gathers from global memory; 2 or 3:
                           tile-staged, x-row segments of 128-node tiles
                           copied to shared memory by TMA bulk copies (2)
                           or by per-thread cp.async (3); nx a multiple of
                           128                                              */
  int adjoint_mode;     /* 0: unsteady adjoint over the trajectory (exact
                           gradient of J over the horizon); 1: the paper's
                           fixed-point ALBS at the held state f-hat = f^N
                           (Sec. 2.2, Eqs. adjoint:iteration/adjoint:operator
                           at the stationary state), needs obj_window 0      */
  int inlet_kind;       /* inlet_outlet channels: 0 velocity inlet u_x = u_in;
                           1 pressure inlet (Sec. 4): rho = rho_out + 3 dp
                           (the pressure drop dp over the outlet, p = rho/3),
                           with the inlet velocity capped at u_in (a node
                           whose pressure condition would exceed the cap is
                           a velocity inlet at the cap)                      */
  double dp;            /* pressure drop of a pressure inlet                 */
} lbm_params;

/* Create a solver.  Defines the lattice, node types, collision (Sec. 3,
 * Sec. 3.1), porosity parametrisation (Sec. 3.2) and objective.
 *   out     : receives the handle (owned by the library until lbm_destroy).
 *   p       : problem description (copied).
 *   theta   : N floats, host or device; copied.
 *   flags   : N uint8 node types (LBM_NODE_*), host or device, copied; NULL
 *             builds the channel geometry described by p.
 *   stream  : cudaStream_t the handle launches on (NULL = legacy default).
 * The state starts at f^0 = rest equilibrium (rho = 1, u = 0), scalars 0.
 * Errors: LBM_ERR_ARG (bad sizes or parameters), LBM_ERR_OOM, LBM_ERR_CUDA. */
lbm_status lbm_create(lbm_handle* out, const lbm_params* p, const float* theta,
                      const uint8_t* flags, void* stream);

/* Release every device allocation of the handle.  NULL is ignored. */
void lbm_destroy(lbm_handle h);

/* Message describing the last failure on h (static string if h is NULL). */
const char* lbm_last_error(lbm_handle h);

/* Replace theta (N floats, host or device) and reset the handle to f^0. */
lbm_status lbm_set_theta(lbm_handle h, const float* theta);

/* Return to f^0, drop stored states, objective record, adjoint and gradient. */
lbm_status lbm_reset(lbm_handle h);

/* Advance k primal steps (Eq. normal:iteration, pull form: the fused
 * kernel gathers f_j(x - e_j) and writes W(f(x)) at x).  Objective terms
 * c_n F(f^n) are recorded on the way, and states are kept for the adjoint
 * as the checkpoint schedule requires.  Errors: LBM_ERR_STATE if the
 * adjoint of this trajectory has started. */
lbm_status lbm_primal_step(lbm_handle h, int k);

/* Current primal time n (number of steps taken since f^0). */
int lbm_time(lbm_handle h);

/* J = sum over recorded n of c_n F(f^n) (Eq. objective:function), FP64.
 * Synchronises the stream.  J_host: host pointer to one double. */
lbm_status lbm_objective(lbm_handle h, double* J_host);

/* Run k adjoint steps.
 * adjoint_mode 0 (unsteady; Eq. adjoint:iteration applied backward in
 * time): the first call starts at the current primal time n = T with
 * lambda^T = c_T dF/df(f^T) and zeroes the gradient; each step computes
 * lambda^{n} from lambda^{n+1} and f^n (restored from checkpoints by
 * recomputation when it was not kept) and adds its theta terms to the FP64
 * gradient.  Errors: LBM_ERR_STATE when k exceeds the remaining steps.
 * adjoint_mode 1 (the paper's ALBS, Sec. 2.2): k iterations of
 *   v^k = (d(SW)/df(f-hat))^T v^{k-1} + dF/df(f-hat)
 * at the held state f-hat = the current primal state (f^N after a full
 * primal run), starting from v^0 = 0 (or the lbm_adjoint_seed vector) on
 * the first call.  Each iteration overwrites the gradient with Eq.
 * adjoint:derivative evaluated with the iterate it consumes,
 *   dJ/dtheta = (d(SW)/dtheta(f-hat))^T v^{k-1} + dF/dtheta(f-hat),
 * which converges to the gradient of the stationary objective F(f-hat)
 * when f-hat is a fixed point of the primal.  Any k >= 0 is allowed;
 * lbm_get_adjoint returns v^k.  The batched adjoint does not take this
 * mode (LBM_ERR_ARG). */
lbm_status lbm_adjoint_step(lbm_handle h, int k);

/* Start the adjoint at the current primal time T with lambda^T = lam (M*N
 * floats, host or device) instead of the objective source, and zero the
 * gradient; later lbm_adjoint_step calls continue from there.  Used to
 * apply the transposed step to an arbitrary vector. */
lbm_status lbm_adjoint_seed(lbm_handle h, const float* lam);

/* Current adjoint time n (lambda^n is held); -1 before the adjoint starts. */
int lbm_adjoint_time(lbm_handle h);

/* Full sensitivity solve: reset, nsteps primal steps, nsteps adjoint steps
 * (unsteady), or nsteps primal steps followed by the same number of ALBS
 * iterations at f^N (adjoint_mode 1, the schedule of Sec. 3.3).
 * Equivalent to lbm_reset + lbm_primal_step(N) + lbm_adjoint_step(N). */
lbm_status lbm_run(lbm_handle h);

/* Copy dJ/dtheta (N doubles, Eq. adjoint:derivative) into dst, host or
 * device.  Synchronises the stream when dst is host memory. */
lbm_status lbm_gradient(lbm_handle h, double* dst);

/* Copy populations of the current primal time into dst (M*N floats, host or
 * device), as full values f (not deviations).
 *   which = 0: pre-collision f^n(x) (the paper's state);
 *   which = 1: post-collision W(f^{n-1}(x)) at x, before streaming. */
lbm_status lbm_get_populations(lbm_handle h, float* dst, int which);

/* As lbm_get_populations for the state of an earlier time that the handle
 * still holds (a checkpoint, or the state the adjoint last used);
 * LBM_ERR_STATE when that state is not held. */
lbm_status lbm_get_populations_at(lbm_handle h, int time, float* dst, int which);

/* Overwrite the current state with pre-collision populations src (M*N
 * floats, host or device, full values); drops stored states. */
lbm_status lbm_set_populations(lbm_handle h, const float* src);

/* Copy lambda^n of the current adjoint time into dst (M*N floats, host or
 * device).  Errors: LBM_ERR_STATE before the adjoint starts. */
lbm_status lbm_get_adjoint(lbm_handle h, float* dst);

/* Copy the node-type array (N bytes, host or device). */
lbm_status lbm_get_flags(lbm_handle h, uint8_t* dst);

/* Count non-finite values in the current state (0 = healthy); synchronises.
 * Returns LBM_ERR_NONFINITE when the count is positive. */
lbm_status lbm_check_finite(lbm_handle h, long long* count_host);

/* Bound of the tile-staged kernels' (lbm_params.kernel 2) waits for the
 * shared-memory copies of a stage: polls >= 0 polls (0: give up at the first
 * wait), polls < 0: the default of 2^22 polls.  A block that gives up records
 * the failure, waits (with the default bound) for every copy it still has
 * in flight and returns; the next synchronising call (lbm_objective,
 * lbm_gradient to host memory, lbm_check_finite, ...) returns
 * LBM_ERR_TIMEOUT, the state of that step is not valid and lbm_reset starts
 * over.  Lets a test drive the timeout path without a fault.  Errors:
 * LBM_ERR_ARG. */
lbm_status lbm_set_wait_polls(lbm_handle h, long long polls);

/* Move the handle to another CUDA stream (NULL = legacy default).  Work
 * already queued for the handle on its old stream is ordered before any
 * later work on the new one (an event recorded on the old stream, waited
 * for on the new one); nothing is synchronised on the host.  Lets a
 * scheduler give each group of batched handles its own stream.  Errors:
 * LBM_ERR_ARG, LBM_ERR_CUDA. */
lbm_status lbm_set_stream(lbm_handle h, void* stream);

/* Sizes: M densities per node and N nodes. */
lbm_status lbm_sizes(lbm_handle h, int* M, long long* N);

/* Device time of the kernels of the last lbm_primal_step / lbm_adjoint_step
 * call, measured with CUDA events on the handle's stream (ms; synchronises). */
lbm_status lbm_last_timing(lbm_handle h, float* primal_ms, float* adjoint_ms);

/* Kernel timing: with enable != 0 every primal, recompute and adjoint
 * kernel launch is bracketed by CUDA events on the handle's stream. */
lbm_status lbm_profile(lbm_handle h, int enable);

/* Read and clear the kernel timing record (synchronises): out[8] =
 * {primal launches, primal ms, recompute launches, recompute ms,
 *  adjoint launches, adjoint ms, other launches (objective and record
 *  folding), total launches}. */
lbm_status lbm_profile_read(lbm_handle h, double* out);

/* Primal steps recomputed by the checkpoint schedule since the last reset. */
long long lbm_recompute_steps(lbm_handle h);

/* Batched primal steps (continuous batching): advance each of
 * the n handles by up to k steps, one kernel launch per step covering every
 * handle below 2^20 nodes that has not reached its horizon (at most 64
 * handles per launch; larger batches are split); a handle of 2^20 nodes or
 * more fills the GPU alone and gets its own single-instance launch within
 * the step.  The per-node arithmetic, and the grouping of the per-step
 * objective sums, are those of lbm_primal_step, so results are
 * bit-identical to driving each handle alone (16-bit storage with even nx,
 * whose single-instance primal updates node pairs, groups its per-step
 * objective sums differently: equal up to rounding).  All handles must
 * share lattice, collision, scalar count, storage precision and stream.
 * Errors: LBM_ERR_ARG, LBM_ERR_STATE (an adjoint has started on a handle),
 * LBM_ERR_OOM. */
lbm_status lbm_batch_primal_step(const lbm_handle* hs, int n, int k);

/* Batched adjoint steps: each handle that has adjoint steps left goes back
 * up to k steps (Eq. adjoint:iteration), one launch per step for all of
 * them (handles of 2^20 nodes or more: their own launch, as for the
 * primal); states are restored per handle by its own checkpoint schedule.  A
 * handle whose adjoint has not started starts at its current primal time.
 * Same requirements and errors as lbm_batch_primal_step. */
lbm_status lbm_batch_adjoint_step(const lbm_handle* hs, int n, int k);

/* As lbm_batch_primal_step / lbm_batch_adjoint_step with a step count per
 * handle: handle i advances by up to ks[i] >= 0 steps (host array of n
 * ints); every step's launch covers the handles that still have steps left
 * in this call.  A scheduler that gives requests of different sizes
 * different step counts (equal work per request) makes one call per group
 * instead of one per step.  Same requirements and errors. */
lbm_status lbm_batch_primal_steps(const lbm_handle* hs, int n, const int* ks);
lbm_status lbm_batch_adjoint_steps(const lbm_handle* hs, int n, const int* ks);

/* ---- one-shot optimisation (Sec. 3.3) -------------------------------------
 * The design theta is optimised together with the flow.  One iteration:
 *   1. one primal step f^{k+1} = S W(f^k, theta^k)        (Eq. normal:iteration)
 *   2. one ALBS step at the current primal state, with the objective source
 *      every iteration: v^{k+1} = (d(SW)/df(f^k))^T v^k + dF/df(f^k)
 *                                                        (Eq. adjoint:iteration)
 *   3. the gradient estimate g^k = (d(SW)/dtheta(f^k))^T v^k from the adjoint
 *      iterate step 2 consumes                           (Eq. adjoint:derivative)
 *   4. on design nodes, the update of Eq. gradient:update on the penalised
 *      objective s J - penalty P, with P = sum theta (1 - theta) of Eq. P:
 *        theta <- min(max(theta + zeta (s g - penalty (1 - 2 theta)), 0), 1)
 *      s = +1 when J is maximised, -1 when it is minimised; evaluated and
 *      stored in FP32 (zeta and penalty are rounded to FP32).
 * The objective is F of the current state: the horizon and time weights of
 * lbm_params do not apply.  theta is the handle's own array (lbm_set_theta
 * sets the starting design; a one-shot run changes it in place).  While a
 * one-shot run is active the current state is the state of time 0 for
 * lbm_get_populations, lbm_set_populations (which replaces f^k),
 * lbm_adjoint_seed (which replaces v^k), lbm_get_adjoint (v^k) and
 * lbm_gradient (the last estimate g); lbm_primal_step, lbm_adjoint_step and
 * the batched steps return LBM_ERR_STATE until lbm_reset or lbm_set_theta. */

/* Design mask: N bytes (host or device, copied); nonzero marks a node whose
 * theta the one-shot update may change.  NULL restores the default: every
 * FLUID node.  Errors: LBM_ERR_ARG, LBM_ERR_CUDA. */
lbm_status lbm_set_design(lbm_handle h, const uint8_t* mask);

/* Start a one-shot run: f^0 = rest state, v^0 = 0, g = 0 (asynchronous). */
lbm_status lbm_oneshot_reset(lbm_handle h);

/* iters one-shot iterations, asynchronous on the handle's stream: per
 * iteration one primal launch and one adjoint launch that also writes g and
 * updates theta (and, for the outlet-variance objective, the fold of the
 * outlet mean the adjoint source needs).  The iteration always runs the
 * one-thread-per-node kernels, whatever lbm_params.kernel selects.  zeta >= 0 and penalty >= 0 are finite; maximize:
 * nonzero ascends J, zero descends.  Errors: LBM_ERR_ARG, LBM_ERR_STATE (no
 * one-shot run started), LBM_ERR_OOM (the pool cannot hold two states). */
lbm_status lbm_oneshot_step(lbm_handle h, int iters, double zeta, double penalty, int maximize);

/* F(f^k) of the current one-shot state and the penalty P over the design
 * nodes, into host doubles (either may be NULL); synchronises.  The sums
 * are taken per block and folded in a fixed order (reproducible). */
lbm_status lbm_oneshot_eval(lbm_handle h, double* J, double* P);

/* Threshold scan of Sec. 3.2.  For each level eta[i] the design nodes are
 * set solid (theta = 1) where w = 1 - theta < eta[i], both in FP32, and
 * fluid (theta = 0) otherwise; the primal runs nsteps >= 1 steps from rest
 * on that design and J_out[i] = F(f^nsteps).  The continuous theta is
 * restored afterwards and the handle is reset (any one-shot or unsteady run
 * ends).  eta and J_out: host arrays of n >= 1 doubles; synchronises.
 * Errors: LBM_ERR_ARG, LBM_ERR_OOM, LBM_ERR_CUDA. */
lbm_status lbm_threshold_scan(lbm_handle h, const double* eta, int n, int nsteps, double* J_out);

/* ---- MMA design iterations (Sec. 3.3) -------------------------------------
 * The paper's second optimiser, Svanberg's Method of Moving Asymptotes,
 * for 0 <= theta <= 1 without further constraints.  A design iteration is a
 * full solve (lbm_run: primal, unsteady adjoint, dJ/dtheta) followed by
 * lbm_mma_update, which changes theta on the design nodes (lbm_set_design):
 *   asymptotes L < theta < U: iterations 0 and 1: theta -/+ 0.5; later the
 *     previous distances scaled by 0.7 where theta oscillated (its last two
 *     changes of opposite sign), by 1.2 where it moved monotonically, by 1
 *     otherwise, and held within [0.01, 10];
 *   move limits alpha = max(0, L + 0.1 (theta - L), theta - move),
 *               beta  = min(1, U - 0.1 (U - theta), theta + move);
 *   with g the gradient of f = -J when maximising, f = J otherwise,
 *     p = (U - theta)^2 (1.001 g+ + 0.001 g- + 1e-5),
 *     q = (theta - L)^2 (0.001 g+ + 1.001 g- + 1e-5),
 *     theta <- min(max((sqrt p L + sqrt q U) / (sqrt p + sqrt q), alpha), beta),
 *   the minimiser of the convex separable approximation
 *   sum p / (U - theta) + q / (theta - L) on [alpha, beta].
 * FP32 arithmetic; the history (two previous designs, last asymptotes:
 * 4 N floats) is owned by the handle. */

/* Start MMA at iteration 0 (allocates the history on first use). */
lbm_status lbm_mma_reset(lbm_handle h);

/* One MMA update with the handle's dJ/dtheta, after the adjoint has reached
 * time 0 (lbm_run); then lbm_reset, so that the next solve starts from rest
 * with the new theta.  maximize: nonzero maximises J.  move in (0, 1].
 * Errors: LBM_ERR_STATE (no completed adjoint, no lbm_mma_reset, or a
 * one-shot run active), LBM_ERR_ARG. */
lbm_status lbm_mma_update(lbm_handle h, int maximize, double move);

/* The same update with a caller's gradient dF/dtheta instead (N doubles,
 * host or device; F is maximised when maximize is nonzero), e.g. of an
 * objective composed outside the library; no completed adjoint is needed
 * and the handle is not reset. */
lbm_status lbm_mma_update_with(lbm_handle h, const double* grad, int maximize, double move);

/* Binarise the handle's theta in place with one level eta (the rule of
 * lbm_threshold_scan) and reset the handle.  Errors: LBM_ERR_ARG, LBM_ERR_CUDA. */
lbm_status lbm_threshold_apply(lbm_handle h, double eta);

/* Copy the handle's current theta (N floats) into dst (host or device);
 * synchronises when dst is host memory. */
lbm_status lbm_get_theta(lbm_handle h, float* dst);

/* Objective F(f) of one pre-collision state, evaluated without allocating
 * any device memory.  The paper has no counterpart: this entry point exists
 * for callers that cannot allocate at the point of the call - a serving
 * process whose device memory is fully reserved in advance for resident
 * states, plugins inside a host framework that owns the device allocator
 * and forbids allocations behind its back, and code that must not pay the
 * device-wide synchronisation cudaFree implies while other streams run.
 *   p      : problem description (lattice, collision, objective, ...); the
 *            time weights are ignored, F is the objective of this one state.
 *   f      : device, M*N floats, full pre-collision populations (the layout
 *            of lbm_get_populations with which = 0).
 *   theta  : device, N floats.   flags: device, N node types.
 *   stream : cudaStream_t the two kernels run on.
 *   F_host : host pointer receiving F; the call synchronises the stream.
 * The C ABI takes no buffer sizes: f, theta and flags must hold the M*N,
 * N and N elements that p implies.  Scratch lives in a fixed static device
 * array of about 1.5 MiB that every GPU loading the library keeps until
 * exit; lattices above 8,388,608 nodes are rejected with LBM_ERR_ARG.  The
 * first call on a device, with that device current, resolves the array's
 * device address and loads the entry point's kernels; later calls on that
 * device only launch.  All calls share the array, so calls that overlap on
 * the GPU race and must be serialised by the caller.  Errors: LBM_ERR_ARG,
 * LBM_ERR_CUDA; the message is returned by lbm_noalloc_last_error(). */
lbm_status lbm_state_objective_noalloc(const lbm_params* p, const float* f,
                                       const float* theta, const uint8_t* flags,
                                       void* stream, double* F_host);

/* Message of the last failed lbm_state_objective_noalloc call on this thread. */
const char* lbm_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ALBM_H */
