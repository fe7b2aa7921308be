/*
 * esmm_oracle.h -- plain FP64 CPU oracle for the entropy-stable adaptive
 * moving-mesh finite difference scheme of Duan & Tang, "High-order accurate
 * entropy stable adaptive moving mesh finite difference schemes for special
 * relativistic (magneto)hydrodynamics" (arXiv 2107.12027), 2D RHD case.
 *
 * TEST INFRASTRUCTURE.  This is the checker, not the product: only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg load it.  It
 * shares no code with the CUDA library.
 *
 * Conventions (all arrays are caller-owned, FP64, structure of arrays):
 *   nodes (i, j), i along xi (fastest), j along eta; N = nx * ny;
 *   index(i, j) = j * nx + i;
 *   RHD:  prim[4][N] = (rho, v_x, v_y, p),  cons[4][N] = J * (D, m_x, m_y, E);
 *   RMHD: prim[8][N] = (rho, v_1, v_2, v_3, p, B_1, B_2, B_3),
 *         cons[8][N] = J * (D, m_1, m_2, m_3, E, B_1, B_2, B_3)
 *   (cons is the curvilinear unknown "J U");
 *   J[N], x[2][N] (physical coordinates), xdot[2][N] (mesh velocity).
 * The computational coordinates are node indices (Delta xi_k = 1).
 */
#ifndef ESMM_ORACLE_H
#define ESMM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* OREF_INFLOW: the ghost data beyond the low end of that direction take the
 * fixed primitive state cfg.inflow (the inflow boundary of the shock-cloud
 * examples of Sec. 6); the high end is outflow, and the mesh treats both ends
 * as outflow ends (extrapolated ghosts, fixed boundary nodes). */
enum { OREF_PERIODIC = 0, OREF_OUTFLOW = 1, OREF_INFLOW = 2 };
enum { OREF_MONITOR_RHO = 0, OREF_MONITOR_LNRHO = 1 };
enum { OREF_RHD = 0, OREF_RMHD = 1 };

typedef struct {
    int nx, ny;
    int bc[2];            /* per direction: OREF_PERIODIC, OREF_OUTFLOW or
                             OREF_INFLOW                                      */
    double period[2];     /* physical period added to x (or y) across a
                             periodic boundary                              */
    double gamma;         /* ideal-gas adiabatic index, 1 < gamma <= 2        */
    int p;                /* EC flux order 2p, p in {1, 2, 3}                 */
    int w;                /* WENO order: 0 (EC only), 3 or 5                  */
    double weno_eps;      /* WENO smoothness epsilon                          */
    double cfl;           /* CFL number                                       */
    int monitor;          /* OREF_MONITOR_RHO or OREF_MONITOR_LNRHO           */
    double alpha;         /* monitor strength                                 */
    int n_filter;         /* low-pass filter passes                           */
    int mu;               /* Jacobi iterations per redistribution             */
    int move_mesh;        /* 0: static mesh (xdot = 0)                        */
    int phys;             /* OREF_RHD (4 unknowns) or OREF_RMHD (8 unknowns)  */
    double alpha_lap;     /* strength of the monitor's Laplacian term (the
                             vortex examples of Sec. 6; 0: eq. monitor)     */
    double inflow[8];     /* primitive inflow state (OREF_INFLOW ends)        */
} oref_cfg;

/* Sec. 3.2, constraint eq. HOCoeff: alpha_{p,1..p}. */
void oref_alpha(int p, double *alpha);
/* Sec. 3.1 logarithmic mean [[a]]/[[ln a]]. */
double oref_logmean(double a, double b);

/* Sec. 1, eq. RMHDdiv2 with B = 0: primitive -> conservative, and back. */
void oref_prim2cons(double gamma, const double *w, double *U);
int oref_cons2prim(double gamma, const double *U, double *w, int *iters);
void oref_flux(double gamma, const double *w, int dir, double *F);

/* Sec. 2: entropy eta, entropy variables V, potentials phi and psi_k. */
double oref_entropy(double gamma, const double *w);
void oref_entropy_vars(double gamma, const double *w, double *V);
void oref_potentials(const double *w, double *phi, double *psi);

/* Sec. 3.1: the two-point parts U~ and F~_1, F~_2 of the EC flux. */
void oref_ec_flux(double gamma, const double *wl, const double *wr,
                  double *Ut, double *F1t, double *F2t);

/* Sec. 4: eigenvalues lam[4] and scaled eigenvectors R[4][4] (row = component,
 * column = wave) of dF_1/dU at a primitive state whose velocity is already
 * rotated to the interface normal (w = rho, v_n, v_t, p). */
void oref_eigen(double gamma, const double *w_rot, double *lam, double *R);

/* Jiang-Shu WENO value at the right edge of the middle node of s[0..w-1]
 * (w = 3 or 5), the stencil ordered from far upwind to far downwind. */
double oref_weno(int w, double eps, const double *s);

/* Sec. 3.3, eq. SCLCoeff / App. B: node metrics m[4][N] =
 * (J xi_x, J xi_y, J eta_x, J eta_y), and J0[N] from the same differences. */
void oref_metrics(const oref_cfg *c, const double *x, double *m, double *J0);

/* Semi-discrete scheme, eqs. RMHDSemiU_O2p_ES / RMHDSemiJ_O2p_ES (RHD: the
 * same with B = 0, no Powell source). */
int oref_rhs(const oref_cfg *c, const double *cons, const double *J,
             const double *x, const double *xdot, double *dcons, double *dJ);

/* CFL time step, eq. cfl, with the static-mesh spectral radius. */
int oref_cfl_dt(const oref_cfg *c, const double *cons, const double *J,
                const double *x, double *dt);

/* Sec. 5 monitor, before the low-pass filter: om[N] = sqrt(1 + alpha
 * |grad_xi sigma| / max |grad_xi sigma| + alpha_lap |lap_xi sigma| /
 * max |lap_xi sigma|) with central differences in the node indices; a term
 * whose maximum is 0 is left out (alpha_lap = 0 gives eq. monitor). */
int oref_monitor(const oref_cfg *c, const double *cons, const double *J, double *om);

/* Threads of the oracle's parallel loops (n <= 0: all host threads);
 * returns the number in effect.  Results do not depend on it. */
int oref_set_threads(int n);

/* Newton steps of oref_cfl_solve before it falls back to the safe bound. */
#define OREF_CFL_NEWTON 6

/* eq. cfl with the mesh velocity in the spectral radius, solved for dt (the
 * reading and the method are stated at the definition).  a, bmin, bmax are
 * [ndir][N]: the displacement term d.(J xi_k,x)/J and the speed bounds
 * L_k lambda_min/J, L_k lambda_max/J of every node. */
double oref_cfl_solve(int ndir, long N, double cfl, const double *a, const double *bmin, const double *bmax,
                      double dt_given, double *tau, int *iters);

/* Sec. 5 low-pass filter of the monitor, n passes in place (weights
 * (1/2)^{|j1|+|j2|+2} over the 3x3 neighbourhood). */
void oref_filter(const oref_cfg *c, double *om, int n);

/* Sec. 5 Jacobi iteration of the mesh equations: mu sweeps with om frozen
 * from X^[0] = x, result X[2][N]. */
void oref_jacobi(const oref_cfg *c, const double *om, const double *x, int mu, double *X);

/* Sec. 5 mesh redistribution and the step: xdot from the state at t^n; dt > 0
 * is used as given, dt <= 0 selects the CFL step with the mesh motion
 * included (written to *dt_out). */
int oref_mesh(const oref_cfg *c, const double *cons, const double *J,
              const double *x, double dt, double *xdot, double *dtau, double *dt_out);

/* One SSP-RK3 step of (cons, J, x) in place; dt <= 0 selects the CFL step. */
int oref_rk_step(const oref_cfg *c, double *cons, double *J, double *x,
                 double dt, double *dt_used);

/* One SSP-RK3 step with a given mesh velocity and step (the map the adjoint
 * differentiates). */
int oref_rk_step_given(const oref_cfg *c, double *cons, double *J, double *x,
                       const double *xdot, double dt);

/* RMHD pointwise parts (esmm_oracle_mhd.c), 8-component states. */
void oref_mhd_prim2cons(double gamma, const double *w, double *U);
void oref_mhd_flux(double gamma, const double *w, int dir, double *F);
int oref_mhd_cons2prim(double gamma, const double *U, double *w, int *iters);
double oref_mhd_entropy(double gamma, const double *w);
void oref_mhd_entropy_vars(double gamma, const double *w, double *V);
/* phi, psi[3] (eq. EntropyPotential) and Phi (eq. Phi) */
void oref_mhd_potentials(const double *w, double *phi, double *psi, double *Phi);
/* Phi'(V)[8] of eq. Phi */
void oref_mhd_phiprime(const double *w, double *P);
/* U~[8] and F~_j[3][8] (Sec. 3.1) */
void oref_mhd_ec_flux(double gamma, const double *wl, const double *wr,
                      double *Ut, double *Ft);
/* speeds lam[8] and scaled eigenvectors R[8][8] (row = component, column =
 * wave) of the symmetrized x_1 system at a rotated primitive state */
void oref_mhd_eigen(double gamma, const double *w_rot, double *lam, double *R);

/* Initial curvilinear state: J from the mesh and cons = J * U(prim). */
int oref_init_state(const oref_cfg *c, const double *prim, const double *x,
                    double *cons, double *J);
/* Primitive variables of a state. */
int oref_state_prim(const oref_cfg *c, const double *cons, const double *J,
                    double *prim);

/* out = (sum J eta, sum J D, sum J, sum (V . dcons - phi dJ)) -- the last
 * only when dcons and dJ are given (else 0). */
int oref_totals(const oref_cfg *c, const double *cons, const double *J,
                const double *dcons, const double *dJ, double *out);


/* ---- 3D RMHD (esmm_oracle3d.c) --------------------------------------------
 * nodes (i, j, k), i fastest, N = nx ny nz, index (k ny + j) nx + i;
 * prim/cons [8][N], J[N], x[3][N], xdot[3][N]; metrics m[9][N] with
 * m[3 k + j] = J d xi_k/d x_j. */
typedef struct {
    int nx, ny, nz;
    int bc[3];
    double period[3];
    double gamma;
    int p, w;
    double weno_eps;
    double cfl;
    int monitor;
    double alpha;
    int n_filter;
    int mu;
    int move_mesh;
    double alpha_lap;
    double inflow[8];
} oref3_cfg;

/* eq. SCLCoeff (nested CMM) and J0 = det(delta_k[x_j]) */
void oref3_metrics(const oref3_cfg *c, const double *x, double *m, double *J0);
int oref3_init_state(const oref3_cfg *c, const double *prim, const double *x, double *cons, double *J);
int oref3_state_prim(const oref3_cfg *c, const double *cons, const double *J, double *prim);
int oref3_rhs(const oref3_cfg *c, const double *cons, const double *J, const double *x,
              const double *xdot, double *dcons, double *dJ);
int oref3_cfl_dt(const oref3_cfg *c, const double *cons, const double *J, const double *x, double *dt);
int oref3_monitor(const oref3_cfg *c, const double *cons, const double *J, double *om);
void oref3_filter(const oref3_cfg *c, double *om, int n);
void oref3_jacobi(const oref3_cfg *c, const double *om, const double *x, int mu, double *X);
int oref3_mesh(const oref3_cfg *c, const double *cons, const double *J, const double *x, double dt,
               double *xdot, double *dtau, double *dt_out);
int oref3_rk_step(const oref3_cfg *c, double *cons, double *J, double *x, double dt, double *dt_used);
int oref3_rk_step_given(const oref3_cfg *c, double *cons, double *J, double *x, const double *xdot, double dt);
int oref3_totals(const oref3_cfg *c, const double *cons, const double *J, const double *dcons,
                 const double *dJ, double *out);

#ifdef __cplusplus
}
#endif
#endif
