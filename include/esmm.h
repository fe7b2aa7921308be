/*
 * esmm.h -- C ABI of libesmm, the GB300 (sm_103a) implementation of the
 * high-order entropy-stable adaptive moving-mesh finite difference scheme of
 * Duan & Tang, "High-order accurate entropy stable adaptive moving mesh finite
 * difference schemes for special relativistic (magneto)hydrodynamics"
 * (arXiv 2107.12027): 2D special relativistic hydrodynamics (RHD), 2D
 * special relativistic magnetohydrodynamics (RMHD, with the Godunov-Powell
 * source of eq. RMHDSymm) and 3D RMHD (the nested metrics of eq. SCLCoeff).
 *
 * Conventions shared by every entry point
 *   - Every function returns an int status: ESMM_OK (0) or one ESMM_ERR_*.
 *     On error nothing the caller owns has been written, except where stated;
 *     esmm_last_error() returns a message.
 *   - Arrays are structure of arrays, FP64, node-ordered with i (the xi
 *     index, along x) fastest: element (c, j, i) of an array with C
 *     components is at c*N + j*nx + i, N = nx*ny.  No ghost nodes.
 *     3D grids (dim = 3, RMHD): element (c, k, j, i) at c*N + (k*ny + j)*nx + i,
 *     N = nx*ny*nz, and x, xdot have 3 components.
 *       prim  [m][N]  RHD (m = 4): rho, v_x, v_y, p
 *                     RMHD (m = 8): rho, v_1, v_2, v_3, p, B_1, B_2, B_3
 *       cons  [m][N]  the curvilinear unknown J*U, U = (D, m_x, m_y, E)
 *                     (RMHD: U = (D, m_1, m_2, m_3, E, B_1, B_2, B_3))
 *       J     [N]     the evolved Jacobian (volume) of each node
 *       x     [d][N]  physical node coordinates (x, y[, z]), d = 2 or 3
 *       xdot  [d][N]  mesh velocity
 *   - The computational coordinates are node indices (Delta xi_k = 1), so
 *     metrics, J and fluxes are per unit index.
 *   - mem = ESMM_MEM_HOST: pointers are host memory; the call copies in,
 *     computes on the grid's stream and copies out before returning.
 *     mem = ESMM_MEM_DEVICE: pointers are device memory on the grid's device;
 *     the call only enqueues work on the grid's stream and returns (the
 *     caller synchronises).  Caller pointers are borrowed for the call only.
 *   - A grid owns all device memory it allocates; esmm_grid_destroy frees it.
 *   - Calls on one grid must not overlap; different grids are independent.
 */
#ifndef ESMM_H
#define ESMM_H

#ifdef __cplusplus
extern "C" {
#endif

#define ESMM_OK 0
#define ESMM_ERR_ARG 1      /* invalid argument                               */
#define ESMM_ERR_CUDA 2     /* a CUDA call failed (message in esmm_last_error) */
#define ESMM_ERR_C2P 3      /* conservative-to-primitive recovery failed at
                               some node (non-admissible state)               */
#define ESMM_ERR_TIMEOUT 4  /* an iteration limit was reached                 */
#define ESMM_ERR_STATE 5    /* the grid has no state yet                      */

#define ESMM_RHD 0          /* physics: special relativistic hydrodynamics    */
#define ESMM_RMHD 1         /* physics: special relativistic MHD, 3-component
                               v and B; 2D grids (FP64 or ESMM_MIXED, single
                               problems) and every 3D grid (FP64)            */

#define ESMM_PERIODIC 0     /* boundary: periodic (mesh shifted by the period) */
#define ESMM_OUTFLOW 1      /* boundary: zero-gradient data, fixed boundary
                               nodes, linearly extrapolated mesh ghosts        */
#define ESMM_INFLOW 2       /* boundary: the ghosts beyond the LOW end of the
                               direction hold the state of esmm_set_inflow (the
                               inflow boundary of the shock-cloud examples of
                               Sec. 6); the high end is ESMM_OUTFLOW; the mesh
                               treats both ends as outflow ends              */

#define ESMM_MEM_HOST 0
#define ESMM_MEM_DEVICE 1

#define ESMM_FP64 0         /* every step in FP64                              */
#define ESMM_MIXED 1        /* fluxes, WENO and metrics in FP32; FP64 for the
                               primitive recovery, near-equal log means, the
                               state, and all totals                            */

#define ESMM_MONITOR_RHO 0  /* monitor variable sigma = rho                    */
#define ESMM_MONITOR_LNRHO 1/* monitor variable sigma = ln rho                 */

#define ESMM_GET_PRIM 0     /* [m][N] primitive variables                      */
#define ESMM_GET_CONS 1     /* [m][N] J*U                                       */
#define ESMM_GET_J 2        /* [N]                                              */
#define ESMM_GET_X 3        /* [2][N]                                           */
#define ESMM_GET_XDOT 4     /* [2][N] mesh velocity of the last step            */

typedef struct esmm_grid esmm_grid;

/* Scheme parameters (Sec. 5 and 6 of the paper; defaults in brackets). */
typedef struct {
    double cfl;        /* CFL number of eq. cfl                       [0.4]  */
    double weno_eps;   /* WENO smoothness epsilon                     [1e-6] */
    int monitor;       /* ESMM_MONITOR_RHO or ESMM_MONITOR_LNRHO   [LNRHO]   */
    double alpha;      /* monitor strength alpha of eq. monitor       [20]   */
    int n_filter;      /* passes of the monitor's low-pass filter     [4]    */
    int mu;            /* Jacobi iterations of the mesh equations     [10]   */
    int move_mesh;     /* 0: static mesh (uniform-mesh scheme)        [1]    */
    int precision;     /* ESMM_FP64 or ESMM_MIXED                     [FP64] */
    double alpha_lap;  /* strength of a Laplacian term added to the
                          monitor: omega = sqrt(1 + alpha |grad sigma|/max
                          + alpha_lap |lap sigma|/max), the monitor of the
                          vortex examples of Sec. 6 (there sigma = rho,
                          alpha = 20, alpha_lap = 10); 0: eq. monitor   [0]   */
    int sweep;         /* 2D RHD flux kernels of a sweep direction:
                          ESMM_SWEEP_AUTO, ESMM_SWEEP_FUSED or
                          ESMM_SWEEP_SPLIT (below)                     [AUTO] */
} esmm_params;

/* The flux kernels of one 2D RHD sweep direction (esmm_params.sweep).  Both
 * compute the same interface fluxes bit for bit:
 *   ESMM_SWEEP_FUSED: one launch; the pair fluxes of a tile and its node
 *                     data stay in shared memory;
 *   ESMM_SWEEP_SPLIT: a pair-flux launch writing every two-point flux to
 *                     global memory, then an interface launch reading them;
 *   ESMM_SWEEP_AUTO:  the fused kernel until esmm_tune has timed both and
 *                     kept the faster per direction.
 * RMHD and 3D grids sum their pair fluxes inside the interface kernel and
 * ignore the field. */
#define ESMM_SWEEP_AUTO 0
#define ESMM_SWEEP_FUSED 1
#define ESMM_SWEEP_SPLIT 2

/* Create a grid of n[0] x n[1] nodes on [lo, hi] (dim 2, phys ESMM_RHD or
 * ESMM_RMHD), or of n[0] x n[1] x n[2] nodes (dim 3, phys ESMM_RMHD: the
 * nested metrics of eq. SCLCoeff, FP64; defaults Gamma = 4/3, CFL 0.3,
 * alpha = 800), bc[k] ESMM_PERIODIC, ESMM_OUTFLOW or ESMM_INFLOW, n[k] >= 4.  3D grids
 * accept the single-problem calls, the adjoint and profiling; batches, the
 * tuner and ESMM_MIXED return ESMM_ERR_ARG for them (RMHD 2D grids take
 * ESMM_MIXED and, in FP64, the adjoint; batches are RHD).  A periodic
 * direction has n[k] distinct nodes with spacing (hi-lo)/n[k]; an outflow
 * direction has nodes on both ends.  stream is a cudaStream_t (NULL: the
 * legacy default stream) on the current device; the grid stays on that device.
 * Defaults: Gamma = 5/3, p = 2, w = 5, the parameter defaults above. */
int esmm_grid_create(esmm_grid **g, int dim, const int n[3], const double lo[3],
                     const double hi[3], int phys, const int bc[3], void *stream);
int esmm_grid_destroy(esmm_grid *g);
int esmm_set_stream(esmm_grid *g, void *stream);

/* Ideal-gas EOS p = (Gamma - 1) rho e (eq. EOS); 1 < Gamma <= 2. */
int esmm_set_eos(esmm_grid *g, double gamma);
/* 2p-th order EC flux (eq. ECFlux_O2p), p in {1, 2, 3}; WENO order w of
 * the ES dissipation (eq. ESFlux_HO), w in {0 (EC scheme), 3, 5}. */
int esmm_set_order(esmm_grid *g, int p, int w);
/* Scheme parameters of Sec. 5 (monitor, filter passes, Jacobi sweeps) and
 * Sec. 6 (the CFL number of eq. cfl), and the precision form.  ESMM_ERR_ARG
 * for an out-of-range value, and for ESMM_MIXED on a 3D grid (2D RHD and 2D
 * RMHD grids take both forms). */
int esmm_set_params(esmm_grid *g, const esmm_params *prm);
int esmm_get_params(const esmm_grid *g, esmm_params *prm);

/* Set the state from primitive variables and a mesh (x NULL: the uniform
 * mesh of the grid's box).  cons = J * U(prim) with U(prim) of eq.
 * RMHDdiv2's conservative variables (Sec. 1; RHD: B = 0) and J^0 the
 * Jacobian of Sec. 3.3 from the mesh by the same central differences as the
 * metrics (2D: delta_xi[x] delta_eta[y] - delta_eta[x] delta_xi[y]; 3D: the
 * determinant of delta_k[x_j]); after that J evolves by eq. VCL.  t = 0.
 * ESMM_ERR_ARG for a non-admissible state (rho <= 0, p <= 0 or |v| >= 1).
 * prim and cons have m = 4 (RHD) or 8 (RMHD) components. */
int esmm_state_set(esmm_grid *g, const double *prim, const double *x, int mem);
/* Set the curvilinear state directly (e.g. to resume from esmm_state_get). */
int esmm_state_set_cons(esmm_grid *g, const double *cons, const double *J,
                        const double *x, double t, int mem);
/* Copy one field of the state (ESMM_GET_*) to out. */
int esmm_state_get(esmm_grid *g, int what, double *out, int mem);
int esmm_get_time(esmm_grid *g, double *t);

/* One evaluation of the semi-discrete ES scheme, eqs. RMHDSemiU_O2p_ES and
 * RMHDSemiJ_O2p_ES of Sec. 4 (RHD: B = 0; RMHD: with the Godunov-Powell
 * source -Phi'(V_i)^T sum_k (B~_{i+1/2} - B~_{i-1/2})): d(cons)/dt and dJ/dt
 * for the given
 * (cons, J, x, xdot) (xdot NULL: static mesh).  Independent of the grid's
 * state; uses its EOS, order, boundary conditions and precision.
 * ESMM_ERR_C2P if the primitive recovery failed at some node (outputs are then
 * undefined at those nodes). */
int esmm_rhs(esmm_grid *g, const double *cons, const double *J, const double *x,
             const double *xdot, double *dcons, double *dJ, int mem);

/* CFL time step of eq. cfl for the grid's state (static-mesh spectral
 * radius).  Synchronises. */
int esmm_cfl_dt(esmm_grid *g, double *dt);

/* Domain decomposition into slabs (multi-GPU, the paper's parallel design:
 * a structured grid split into subdomains that exchange halos; Sec. 6 runs
 * on a PLUTO-based MPI code).  A 2D grid of n[0] x n[1] nodes is split along
 * the second index into nslab slabs of consecutive rows (sizes differing by
 * at most one, each at least ESMM_SLAB_HALO rows).  Slab s holds its own rows
 * plus ESMM_SLAB_HALO rows beyond each cut (a periodic second direction has
 * cuts at both ends of every slab).  A rank's slab is an ordinary grid of
 * those rows with outflow treatment at its cuts; only its own rows take part
 * in reductions.  The halo is wide enough that one step's monitor, filter
 * passes and Jacobi sweeps (1 + n_filter + 1 + mu rows of reach) stay exact
 * on the own rows, so the step communicates:
 *   - allreduce max of the spectral radius, max |grad sigma| (and the
 *     Laplacian's max) and the displacement terms; allreduce min of the
 *     limiter Delta tau; per Newton evaluation of the eq. cfl solve an
 *     allreduce max of each direction's value and an allreduce min of the
 *     slope among the slabs that attain it;
 *   - a halo exchange of the mesh velocity after the mesh step, and of
 *     (cons, J, x) after each of the three stages;
 *   - an allreduce sum for esmm_totals.
 * The transport is the caller's: comm->allreduce(ctx, buf, n, op) combines
 * n host doubles in place over all slabs (op ESMM_OP_MAX, _MIN or _SUM);
 * comm->exchange(ctx, send_lo, send_hi, recv_lo, recv_hi, count) sends count
 * host doubles to the slab below (send_lo) and above (send_hi) and receives
 * theirs (recv_lo from below, recv_hi from above; a side without a
 * neighbour is NULL).  Both return 0 on success; every slab must make the
 * same calls in the same order.  With max, min and the Newton rule the
 * result on the own rows equals the undecomposed grid's bit for bit; the
 * totals differ only by the order of the sum.
 * Slab handles accept esmm_set_eos, esmm_set_order, esmm_set_params (not
 * ESMM_INFLOW ends), esmm_state_set (the GLOBAL arrays [m][n1][n0]; every
 * slab copies its rows), esmm_state_get (the slab's OWN rows), esmm_rhs
 * (arrays of the slab's rows, halo included), esmm_rk_step, esmm_advance,
 * esmm_totals, esmm_last_error, esmm_profile* and esmm_grid_destroy; other
 * calls return ESMM_ERR_ARG.  esmm_slab_rows gives the global row ranges:
 * own rows [own0, own1), held rows [ext0, ext1) (ext0 < 0 or ext1 > n[1]
 * wrap periodically).  2D grids only. */
#define ESMM_SLAB_HALO 16
#define ESMM_OP_MAX 0
#define ESMM_OP_MIN 1
#define ESMM_OP_SUM 2
typedef struct {
    void *ctx;
    int (*allreduce)(void *ctx, double *buf, int n, int op);
    int (*exchange)(void *ctx, const double *send_lo, const double *send_hi, double *recv_lo, double *recv_hi,
                    long long count);
} esmm_comm;
int esmm_slab_create(esmm_grid **g, const int n[2], const double lo[2], const double hi[2], int phys,
                     const int bc[2], int nslab, int slab, const esmm_comm *comm, void *stream);
int esmm_slab_rows(const esmm_grid *g, int *own0, int *own1, int *ext0, int *ext1);

/* Adaptive mesh redistribution of Sec. 5 for the grid's state and time step
 * dt: monitor, low-pass filter, mu Jacobi sweeps, movement limiter, and the
 * mesh velocity xdot = Delta tau (x^[mu] - x^n)/dt.
 * dt <= 0 selects the step of eq. cfl with that mesh velocity in the spectral
 * radius: dt solves dt sum_k max_i rho_{k,i} = CFL with rho the spectral
 * radius of d(F_k)/d(JU) including the temporal metric (solved by Newton's
 * method on the convex piecewise-linear left side, at most 6 evaluations,
 * else the safe bound (CFL - C_m)/S).  The limiter Delta tau is kept, unless
 * the displacement's own Courant number C_m = Delta tau sum_k max_i
 * |(x^[mu] - x^n).(J xi_k,x)|/J reaches CFL (no step exists then): there it is
 * scaled to C_m = CFL/2.  A given dt > 0 is used as is (the same rule for
 * Delta tau).  Stores the mesh velocity in the grid and, when given, writes it
 * to xdot [d][N], the limiter value to *dtau and the step to *dt_used (host
 * scalars). */
int esmm_mesh_redistribute(esmm_grid *g, double dt, double *xdot, double *dtau, double *dt_used, int mem);

/* One time step of the fully discrete scheme of Sec. 3.3 (Prop. 3.2) and
 * Sec. 6: CFL step of eq. cfl (dt <= 0, with the mesh motion as in
 * esmm_mesh_redistribute) or the given dt, mesh redistribution of Sec. 5
 * (unless move_mesh = 0), and the three stages of the third-order SSP
 * Runge-Kutta method (Shu-Osher form) applied to (cons, J) and to the mesh
 * with the step's mesh velocity.
 * Asynchronous on the grid's stream; when dt_used is not NULL the call
 * synchronises and writes the step used.  A recovery failure is reported by
 * esmm_last_error / the next synchronising call. */
int esmm_rk_step(esmm_grid *g, double dt, double *dt_used);
/* The inflow boundary of the shock-cloud examples of Sec. 6: the primitive
 * state prim[m] (host array; m = 4 for 2D RHD, 8 for RMHD: rho, v, p (, B))
 * held by the ghost nodes beyond every ESMM_INFLOW end.  A
 * grid with an inflow end returns ESMM_ERR_STATE from every call that
 * evaluates the scheme until this is set; ESMM_ERR_ARG for rho <= 0, p <= 0
 * or |v| >= 1.  The adjoint calls return ESMM_ERR_ARG for grids with an
 * inflow end (the adjoint covers periodic and outflow ends). */
int esmm_set_inflow(esmm_grid *g, const double *prim);
/* One time step with a prescribed mesh motion (the given-mesh runs of the
 * vortex examples of Sec. 6): the caller's mesh velocity xdot [d][N] (host or
 * device per mem, d = 2 or 3) is held over the step, the mesh of stage s is
 * x^n + c_s dt xdot with the SSP-RK3 weights, and J follows eq. VCL, so the
 * GCL holds for any xdot.  dt > 0 is the caller's (no CFL check); the params'
 * move_mesh is ignored.  Synchronises; ESMM_ERR_ARG for dt <= 0, a NULL xdot
 * or a batch, ESMM_ERR_STATE without a state, ESMM_ERR_C2P if a recovery
 * failed. */
int esmm_rk_step_given(esmm_grid *g, const double *xdot, double dt, int mem);
/* nsteps asynchronous esmm_rk_step calls (dt as there).  On a grid or batch
 * with its own stream (not the legacy or per-thread default stream) the step
 * is captured once as a CUDA graph, for nsteps >= 2, and replayed for every
 * later step with the same dt argument, including single-step calls, until
 * the parameters, order, EOS, launch shapes, stream or profiling mask
 * change.  With profiling on, the graph holds event nodes around the
 * profiled kinds; each replay's times are read (the call then waits for the
 * previous replay) before the next replay records them again. */
int esmm_advance(esmm_grid *g, int nsteps, double dt);

/* Batches: nprob independent problems of (possibly) different sizes in one
 * handle (the batched form).  n, lo, hi and bc are [nprob][2]; each problem
 * obeys the rules of esmm_grid_create.  All problems share the EOS, order and
 * parameters; every kernel of a step covers the whole batch in one launch
 * (a block -> (problem, tile) map, blocks never span two problems), and
 * esmm_advance replays one CUDA graph per step.  Each problem has its own CFL
 * time step, time, monitor maximum and mesh limiter.  stream NULL: the batch
 * creates its own non-blocking stream.  Batch handles accept esmm_set_*,
 * esmm_rk_step (dt_used: problem 0's step), esmm_advance, esmm_tune,
 * esmm_profile*, esmm_last_error, esmm_grid_destroy and the esmm_batch_*
 * calls; the single-problem state, rhs, CFL, mesh and totals calls return
 * ESMM_ERR_ARG for them.  Batches are RHD (phys must be ESMM_RHD). */
int esmm_batch_create(esmm_grid **g, int nprob, const int *n, const double *lo, const double *hi, const int *bc,
                      int phys, void *stream);
int esmm_batch_size(const esmm_grid *g, int *nprob);
/* state of problem b (arrays of that problem's size, as esmm_state_set) */
int esmm_batch_state_set(esmm_grid *g, int b, const double *prim, const double *x, int mem);
int esmm_batch_state_get(esmm_grid *g, int b, int what, double *out, int mem);
/* t[nprob]: the time of every problem (synchronises) */
int esmm_batch_times(esmm_grid *g, double *t);
/* out[nprob][3]: the FP64 totals of esmm_totals for every problem */
int esmm_batch_totals(esmm_grid *g, double *out);

/* Adjoint: gradients of a final-time functional with respect to the initial
 * data, single problems (2D RHD, 2D RMHD in the FP64 form, 3D RMHD;
 * ESMM_ERR_ARG for batches and mixed-form RMHD grids), FP64.  m = 4 (RHD) or
 * 8 (RMHD) components and d = 2 or 3 mesh components below.
 * esmm_adjoint_record advances nsteps steps (dt as esmm_rk_step) from the
 * current state, keeping per-step checkpoints (state, mesh velocity, step) on
 * the device ((m + 1 + 2 d) N doubles per step).  The adjoint differentiates the
 * recorded map: each step with its recorded mesh velocity and dt held fixed
 * (the monitor's maximum and the limiter's minimum are not differentiable),
 * the sign switch Y and the lambda^ maximum frozen at their forward
 * selection; esmm_adjoint_replay re-runs that map from the current state (for
 * finite-difference checks).  esmm_adjoint_vjp takes lam_final [m][N] =
 * dF/d(cons) at the last recorded step and returns lam_cons0 = dF/d(cons) at
 * the first (may be NULL) and lam_prim0 = dF/d(prim) of the first state (may
 * be NULL), recomputing the RK stages of each step backwards from its
 * checkpoint.  esmm_rhs_vjp returns lam = (d rhs/d cons)^T mu at (cons, J, x,
 * xdot) (J, x and xdot held fixed), through the implicit-function adjoint of
 * the Newton recovery, the log means, the scaled eigenvectors (RMHD: the
 * first-order perturbation of the 8-wave construction, a cluster of
 * near-equal speeds through its span), the WENO weights and, for RMHD, the
 * Godunov-Powell source; in 3D also through the angle by which the Sec. 4
 * rotation is turned to the tangential B (or v) of the interface state. */
int esmm_adjoint_record(esmm_grid *g, int nsteps, double dt);
int esmm_adjoint_steps(esmm_grid *g, int *nsteps, double *dt);
int esmm_adjoint_checkpoint(esmm_grid *g, int step, int what, double *out, int mem);
int esmm_adjoint_replay(esmm_grid *g, int nsteps);
int esmm_adjoint_vjp(esmm_grid *g, const double *lam_final, double *lam_cons0, double *lam_prim0, int mem);
int esmm_rhs_vjp(esmm_grid *g, const double *cons, const double *J, const double *x, const double *xdot,
                 const double *mu, double *lam, int mem);

/* Launch autotuner: for each kernel kind (node pass, pair fluxes, interface
 * fluxes, per-node kernels) time the candidates on the current state and keep
 * the fastest: block sizes, for batches the tile order (natural / largest
 * problem first), and for the 2D RHD fluxes, per sweep direction, the
 * variant (the fused sweep kernel against the pair and interface kernels,
 * unless esmm_params.sweep fixes one), with, for the pair and interface
 * kernels, the tile shape (flat runs of sites along the sweep, or tiles of
 * tx sites along x_1 by bs/tx along x_2), and for every variant whether a
 * persistent grid (the blocks the SMs hold at once) strides over the
 * (problem, tile) queue or each tile gets its own block.  Requires a state.
 * When block_sizes is given it receives ESMM_TUNE_SLOTS ints: [0, 13) the
 * block size of each launch domain (negative: largest problem first; the
 * interface slots hold the fused kernel's when it was kept), [13, 17) the
 * tile shape of the pair (x_1, x_2) and interface (x_1, x_2) launches: tx
 * (0: flat runs; -1 in the interface slots: the fused sweep kernel, whose
 * tiles are one line segment per warp) plus 1000 for a persistent grid. */
#define ESMM_TUNE_SLOTS 17
int esmm_tune(esmm_grid *g, int *block_sizes);

/* FP64 totals of the grid's state: out[0] = sum J eta, the total entropy of
 * the Sec. 6 entropy plots (without their 1/N normalisation; eta the entropy
 * of the entropy pair of Sec. 2), out[1] = sum J D (mass), out[2] = sum J
 * (volume, conserved by eq. VCL).  Synchronises. */
int esmm_totals(esmm_grid *g, double out[3]);

/* Synchronise and return the accumulated error state: the number of nodes
 * whose primitive recovery failed since the last call (then reset), and the
 * last error message (copied into msg, at most len bytes, NUL-terminated). */
int esmm_last_error(esmm_grid *g, int *n_c2p_fail, char *msg, int len);

/* Profiling, an addition for measurement (the paper has no counterpart).
 * Every kernel launch is counted under one kind; the kinds set in mask also
 * get a CUDA event pair recorded on the grid's stream around each launch, so
 * their device time can be read back.  esmm_profile() clears the counters
 * and times and sets the mask (0: counting only).  esmm_profile_read()
 * synchronises and returns, per kind, the summed device milliseconds of the
 * timed launches, the number of launches, and how many of them were timed. */
#define ESMM_KIND_NODE 0    /* per-node pass: recovery, logs, metrics          */
#define ESMM_KIND_PAIRS 1   /* two-point EC pair fluxes                         */
#define ESMM_KIND_IFACE 2   /* ES interface fluxes: EC sum + WENO dissipation   */
#define ESMM_KIND_UPDATE 3  /* flux differences fused with the SSP-RK3 stage    */
#define ESMM_KIND_MESH 4    /* mesh redistribution                              */
#define ESMM_KIND_OTHER 5   /* CFL reduction, time step, totals                 */
#define ESMM_NKINDS 6
int esmm_profile(esmm_grid *g, int mask);
int esmm_profile_read(esmm_grid *g, double ms[ESMM_NKINDS], long long launches[ESMM_NKINDS],
                      long long timed[ESMM_NKINDS]);

/* FMA throughput of one pipe, a measurement addition (the paper has no
 * counterpart): precision ESMM_FP64 or ESMM_MIXED (FP32) selects the pipe.
 * A kernel of independent FMA chains (8 blocks of 256 threads per SM) runs
 * for about `seconds` (0 < seconds <= 60) on a private stream of the current
 * device, timed with CUDA events; *flops_per_s receives 2 x FMAs / second,
 * *ms_per_launch (may be NULL) the time of one launch.  Synchronises. */
int esmm_fma_peak(int precision, double seconds, double *flops_per_s, double *ms_per_launch);

/* Algorithmic operation counts of the 2D RHD flux arithmetic, a
 * measurement addition (the paper has no counterpart): the library's own
 * flux templates evaluated on a counting number type for one node pair and
 * one interface of a generic state (no near-equal log means), every add,
 * subtract, multiply, divide, reciprocal, square root and reciprocal square
 * root counted once.  ops[0]: one two-point EC flux (k_pairs computes p per
 * anchor node); ops[1]: the ES dissipation of one interface with WENO order w
 * (3 or 5); ops[2]: the interface kernel's combination of the stored pair
 * fluxes and the metric flux (eq. ECFlux_O2p, MetricsFlux_O2p) for order p.
 * Runs one thread on the current device; synchronises. */
int esmm_flux_ops(double gamma, int p, int w, double ops[3]);

/* Allocation-free right-hand side.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory -- code
 * running under an allocator or memory budget it does not own (a plug-in, a
 * solver embedded in another framework, a library driven from inside a
 * captured or pooled context) cannot call cudaMalloc or create a grid.
 *
 * Same arithmetic as esmm_rhs in the FP64 form (WENO epsilon 1e-6): d(cons)/dt
 * and dJ/dt of the ES scheme for an nx x ny grid with boundaries bc[2] on the
 * box [lo, hi].  All array pointers are DEVICE pointers on the current device
 * with the layouts above (xdot may be NULL); the caller owns inputs and
 * outputs.  The call only enqueues work on stream (a cudaStream_t, NULL for
 * the legacy default stream) and returns; it allocates nothing (no cudaMalloc,
 * no cudaFree, no allocating library routine).
 *
 * Scratch: one file-scope device array sized for (nx+6)*(ny+6) <=
 * ESMM_STATIC_MAX_PADDED_NODES (e.g. grids up to 256 x 256), 48 doubles per
 * padded node (~26 MB), held by every GPU that loads the library until the
 * process exits.  Larger grids return ESMM_ERR_ARG, as do invalid arguments.
 * With CUDA's default lazy module loading the driver reserves that array
 * when the first call on a device looks up its address, so that first call
 * can fail with ESMM_ERR_CUDA on a device that has no 26 MB left: callers
 * with a fixed budget make one call up front (any small grid), or load the
 * library with CUDA_MODULE_LOADING=EAGER.  The first call on a device sets
 * up the address (with that device current) and must come before any stream
 * capture; a first call inside a capture returns ESMM_ERR_CUDA.  Calls
 * outside a capture look the address up again, so a cudaDeviceReset between
 * calls is harmless; calls inside a capture use the address of the last call
 * outside one (do not reset the device between that call and the capture).
 * Every call shares the one array and overwrites it, so calls that overlap
 * on the GPU (other streams, other threads) race; serialise them.
 * A CUDA error already pending on the calling thread (cudaPeekAtLastError)
 * makes the call return ESMM_ERR_CUDA at once, enqueuing nothing and leaving
 * that error for its owner; a launch error of the call itself is consumed
 * and returned as ESMM_ERR_CUDA.  Primitive-recovery failures are counted
 * in the scratch only and not reported (those nodes' outputs are
 * undefined). */
#define ESMM_STATIC_MAX_PADDED_NODES 68644
int esmm_rhs_static(int nx, int ny, const int bc[2], const double lo[2], const double hi[2], double gamma,
                    int p, int w, const double *cons, const double *J, const double *x, const double *xdot,
                    double *dcons, double *dJ, void *stream);

/* The scaled eigen-system of the symmetrized RMHD x_1 system (Sec. 4) that
 * the ES dissipation uses, for n rotated primitive states w [n][8] (rho,
 * v_1..3, p, B_1..3): lam [n][8] (the entropy and divergence waves first,
 * then the other six ascending) and R [n][8][8] (row = component, column =
 * wave; R R^T = dU/dV; for a cluster of speeds closer than 1e-5 the canonical
 * basis of its span).  With dw non-NULL also the tangents dlam, dR along the
 * directions dw [n][8]: the first-order perturbation of that construction (a
 * cluster through its span) as the adjoint uses it.  Host arrays, computed on
 * the current device; dlam and dR may be NULL when dw is.  ESMM_ERR_ARG for
 * n < 1 or missing arrays, ESMM_ERR_CUDA on a CUDA failure. */
int esmm_mhd_eigen(double gamma, int n, const double *w, const double *dw, double *lam, double *R, double *dlam,
                   double *dR);

/* Library version string. */
const char *esmm_version(void);

#ifdef __cplusplus
}
#endif
#endif
