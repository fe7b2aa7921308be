/*
 * esmm_oracle.c -- plain FP64 CPU oracle for the high-order entropy-stable (ES)
 * adaptive moving-mesh finite difference scheme of Duan & Tang
 * (arXiv 2107.12027), two-dimensional special relativistic hydrodynamics.
 *
 * TEST INFRASTRUCTURE.  This is the independent checker of the CUDA library:
 * only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it, and it shares no code with the CUDA path.
 *
 * Style: every step follows the paper's formulas in the paper's order, one
 * node, one node pair and one interface at a time, in double precision.
 * There is no pair sharing, fusion or reordering: the 2p-th order interface
 * flux is the literal double sum of two-point fluxes.  Where the paper is
 * silent the comment says "reading" and states the choice.
 *
 * Parity status of each part (see the tests for the pins):
 *   alpha_{p,n}, delta_k            pinned (constraints, textbook stencil)
 *   log mean                        pinned (high-precision reference)
 *   prim <-> cons, cons2prim        pinned (round trip, flux definition)
 *   V, eta, phi, psi                pinned (V = d eta/dU by finite differences,
 *                                   phi = V.U - eta, psi_k = V.F_k - q_k)
 *   two-point EC flux               pinned (EC condition, consistency, symmetry)
 *   eigen-system                    pinned (dF/dU R = R Lambda, R R^T = dU/dV)
 *   WENO                            pinned (exact on linear data, order)
 *   metrics, J0                     pinned (discrete SCL, affine meshes)
 *   rhs                             pinned (free stream on moving meshes,
 *                                   entropy identity / inequality, telescoping,
 *                                   order of accuracy)
 *   mesh redistribution             pinned (uniform-monitor fixed point,
 *                                   movement limiter bound, no tangling; the
 *                                   filter's Fourier symbol, the Jacobi
 *                                   sweep's damping of a mode, its fixed point
 *                                   = the Euler-Lagrange solution of the
 *                                   adaption functional)
 *   step of eq. cfl                 pinned (dt sum_k max rho = CFL with the
 *                                   mesh velocity, rho from eigenvalues;
 *                                   brute-force root on random data)
 *   SSP-RK3 step                    pinned (free stream, exact advection error)
 *
 * The loops over nodes and interfaces run under OpenMP; they write disjoint
 * outputs and combine across threads only by max or min, so results do not
 * depend on the thread count.
 */
#ifdef _OPENMP
#include <omp.h>
#endif
#include "esmm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NV 4   /* 2D RHD: (D, m_x, m_y, E); RMHD states (8) in esmm_oracle_mhd.c */
#define G 3    /* ghost layers of the node data: WENO5 and p <= 3 pairs */
#define OREF_SIGN_TOL 1.0e-10

/* ------------------------------------------------------------------------ */
/* Coefficients alpha_{p,n} (Sec. 3.2, constraint eq. HOCoeff):
 *   sum_n n alpha_{p,n} = 1,  sum_n n^{2s-1} alpha_{p,n} = 0 (s = 2..p).
 * Solved by hand: p=1: 1;  p=2: 4/3, -1/6;  p=3: 3/2, -3/10, 1/30.          */
/* Threads of the parallel loops (OpenMP; n <= 0: all host threads).  The
 * loops write disjoint outputs and reduce across threads only by max or
 * min, so every result is independent of the thread count. */
int oref_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

void oref_alpha(int p, double *alpha)
{
    if (p == 1) {
        alpha[0] = 1.0;
    } else if (p == 2) {
        alpha[0] = 4.0 / 3.0;
        alpha[1] = -1.0 / 6.0;
    } else {
        alpha[0] = 3.0 / 2.0;
        alpha[1] = -3.0 / 10.0;
        alpha[2] = 1.0 / 30.0;
    }
}

/* Logarithmic mean {{a}}^ln = [[a]] / [[ln a]] (Sec. 3.1).  For nearly equal
 * arguments the quotient cancels; there the series of Ismail & Roe (2009) is
 * used: with f = (a_r - a_l)/(a_r + a_l) and u = f^2,
 *   ln(a_r/a_l) = 2 f (1 + u/3 + u^2/5 + u^3/7 + ...),
 * so the mean is (a_l + a_r) / (2 (1 + u/3 + u^2/5 + u^3/7)).
 * Reading: the switch is at u < 1e-4 (the published 1e-2 leaves a truncation
 * error near 1e-9; at 1e-4 the dropped u^4/9 term is below 1e-17).        */
double oref_logmean(double a, double b)
{
    double f = (b - a) / (b + a);
    double u = f * f;
    if (u < 1.0e-4) {
        double F = 1.0 + u / 3.0 + u * u / 5.0 + u * u * u / 7.0;
        return (a + b) / (2.0 * F);
    }
    return (b - a) / (log(b) - log(a));
}

/* ------------------------------------------------------------------------ */
/* Sec. 1, eq. RMHDdiv2 with B = 0: U = (D, m, E), D = rho W,
 * m = rho h W^2 v, E = rho h W^2 - p, h = 1 + e + p/rho with the ideal-gas
 * EOS p = (Gamma - 1) rho e (eq. EOS).                                      */
void oref_prim2cons(double gamma, const double *w, double *U)
{
    double rho = w[0], vx = w[1], vy = w[2], p = w[3];
    double W = 1.0 / sqrt(1.0 - (vx * vx + vy * vy));
    double e = p / ((gamma - 1.0) * rho);
    double h = 1.0 + e + p / rho;
    U[0] = rho * W;
    U[1] = rho * h * W * W * vx;
    U[2] = rho * h * W * W * vy;
    U[3] = rho * h * W * W - p;
}

/* Flux F_dir(U) of eq. RMHDdiv2 with B = 0. */
void oref_flux(double gamma, const double *w, int dir, double *F)
{
    double U[NV];
    double v[2] = {w[1], w[2]};
    oref_prim2cons(gamma, w, U);
    F[0] = U[0] * v[dir];
    F[1] = U[1] * v[dir] + (dir == 0 ? w[3] : 0.0);
    F[2] = U[2] * v[dir] + (dir == 1 ? w[3] : 0.0);
    F[3] = U[1 + dir];
}

/* Conservative -> primitive recovery (Sec. 1: a nonlinear algebraic equation
 * has to be solved; the paper gives no algorithm).  Reading: Newton's method
 * on the pressure,
 *   f(p) = (Gamma-1)/Gamma * ((E + p)/W^2 - D/W) - p,  v = m/(E + p),
 * safeguarded by bisection on the bracket [0, (Gamma-1) E] (f(0) > 0 and
 * f((Gamma-1)E) < 0 for every admissible state, f strictly decreasing).
 * Stops when a step changes p by at most 1e-15 (E + p): f is evaluated from
 * E + p, so p is resolved only to that level (p << E in cold gas); an
 * iterate at which |f| <= 2e-15 (E + p), f's own rounding level, is taken
 * as the root (where df/dp is small, steps at that level exceed the first
 * bound, and the open bracket would reject them and bisect).
 * Returns 0 on success, -1 for a non-admissible state, -2 without
 * convergence.                                                             */
int oref_cons2prim(double gamma, const double *U, double *w, int *iters)
{
    double D = U[0], mx = U[1], my = U[2], E = U[3];
    double S = sqrt(mx * mx + my * my);
    double gg = (gamma - 1.0) / gamma;
    if (!(D > 0.0) || !(E > sqrt(D * D + S * S))) return -1;
    double lo = 0.0, hi = (gamma - 1.0) * E;
    double p = 0.5 * (lo + hi);
    int it, ok = 0;
    for (it = 1; it <= 200; ++it) {
        double Ep = E + p;
        double iW2 = (Ep - S) * (Ep + S) / (Ep * Ep);  /* 1/W^2 = 1 - v^2 */
        double iW = sqrt(iW2);
        double v2 = S * S / (Ep * Ep);
        double f = gg * (Ep * iW2 - D * iW) - p;
        double df = gg * (1.0 + v2 - D * v2 / (iW * Ep)) - 1.0;
        if (fabs(f) <= 2.0e-15 * (E + p)) { /* residual at rounding level */
            ok = 1;
            break;
        }
        double pn = p;                      /* f = 0: p is a root */
        if (f != 0.0) {
            if (f > 0.0) lo = p; else hi = p;
            pn = p - f / df;
            if (!(pn > lo && pn < hi)) pn = 0.5 * (lo + hi);
        }
        if (fabs(pn - p) <= 1.0e-15 * (E + pn)) {
            p = pn;
            ok = 1;
            break;
        }
        p = pn;
    }
    if (iters) *iters = it;
    double Ep = E + p;
    double iW2 = (Ep - S) * (Ep + S) / (Ep * Ep);
    double W = 1.0 / sqrt(iW2);
    w[0] = D / W;
    w[1] = mx / Ep;
    w[2] = my / Ep;
    w[3] = p;
    return ok ? 0 : -2;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2, eq. EntropyPair: eta = -rho W s/(Gamma - 1), s = ln(p/rho^Gamma). */
double oref_entropy(double gamma, const double *w)
{
    double rho = w[0], p = w[3];
    double W = 1.0 / sqrt(1.0 - (w[1] * w[1] + w[2] * w[2]));
    double s = log(p) - gamma * log(rho);
    return -rho * W * s / (gamma - 1.0);
}

/* Sec. 2 (explicit V, B = 0):
 *   V = ((Gamma - s)/(Gamma - 1) + rho/p, rho W v/p, -rho W/p).            */
void oref_entropy_vars(double gamma, const double *w, double *V)
{
    double rho = w[0], vx = w[1], vy = w[2], p = w[3];
    double W = 1.0 / sqrt(1.0 - (vx * vx + vy * vy));
    double s = log(p) - gamma * log(rho);
    V[0] = (gamma - s) / (gamma - 1.0) + rho / p;
    V[1] = rho * W * vx / p;
    V[2] = rho * W * vy / p;
    V[3] = -rho * W / p;
}

/* Sec. 2, eq. EntropyPotential with B = 0: phi = rho W, psi_k = rho v_k W. */
void oref_potentials(const double *w, double *phi, double *psi)
{
    double rho = w[0], vx = w[1], vy = w[2];
    double W = 1.0 / sqrt(1.0 - (vx * vx + vy * vy));
    *phi = rho * W;
    psi[0] = rho * vx * W;
    psi[1] = rho * vy * W;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1: two-point EC flux parts with ([[V]]^T U~ = [[phi]] and
 * [[V]]^T F~_j = [[psi_j]] when B = 0).
 * U~ is the paper's U~^RMHD with b = 0: in the paper's notation
 *   U~_1 = rho^ln {{W}},  D_ = {{beta}}({{W}}^2 - sum {{u^k}}^2)/{{W}},
 *   R_1 = -alpha_0 U~_1,  R_{k+1} = alpha_1 {{u^k}}/{{W}},  alpha_1 = {{rho}},
 *   alpha_0 = 1 + 1/((Gamma-1) beta^ln),
 *   U~_E = D_^{-1} (sum_k {{u^k}} R_{k+1} - {{beta}} R_1),
 *   U~_{m_k} = {{u^k}} U~_E/{{W}} + R_{k+1}/{{beta}},
 * with beta = rho/p, u = W v.  The spatial parts F~_j (the RHD flux of the
 * paper's cited work is not reproduced in it) are the solution of the same
 * coefficient matching for [[psi_j]] = [[rho u_j]]; reading:
 *   F~_D = rho^ln {{u_j}},
 *   F~_E = {{W}} (alpha_0 rho^ln {{u_j}} + {{rho}} {{u_j}}/{{beta}}) / Lambda,
 *   F~_{m_k} = F~_E {{u_k}}/{{W}} + delta_{jk} {{rho}}/{{beta}},
 *   Lambda = {{W}}^2 - sum_k {{u_k}}^2.                                     */
void oref_ec_flux(double gamma, const double *wl, const double *wr,
                  double *Ut, double *F1t, double *F2t)
{
    double rl = wl[0], rr = wr[0];
    double Wl = 1.0 / sqrt(1.0 - (wl[1] * wl[1] + wl[2] * wl[2]));
    double Wr = 1.0 / sqrt(1.0 - (wr[1] * wr[1] + wr[2] * wr[2]));
    double bl = rl / wl[3], br = rr / wr[3];
    double ul[2] = {Wl * wl[1], Wl * wl[2]};
    double ur[2] = {Wr * wr[1], Wr * wr[2]};

    double rho_ln = oref_logmean(rl, rr);
    double beta_ln = oref_logmean(bl, br);
    double rho_m = 0.5 * (rl + rr);
    double beta_m = 0.5 * (bl + br);
    double W_m = 0.5 * (Wl + Wr);
    double u_m[2] = {0.5 * (ul[0] + ur[0]), 0.5 * (ul[1] + ur[1])};
    double usq = u_m[0] * u_m[0] + u_m[1] * u_m[1];

    double alpha0 = 1.0 + 1.0 / (gamma - 1.0) / beta_ln;
    double alpha1 = rho_m;
    double Dcal = beta_m * (W_m * W_m - usq) / W_m;
    double Lam = W_m * W_m - usq;

    /* temporal part U~ */
    double U1 = rho_ln * W_m;
    double R1 = -alpha0 * U1;
    double R2 = alpha1 * u_m[0] / W_m;
    double R3 = alpha1 * u_m[1] / W_m;
    double UE = (u_m[0] * R2 + u_m[1] * R3 - beta_m * R1) / Dcal;
    Ut[0] = U1;
    Ut[1] = u_m[0] * UE / W_m + R2 / beta_m;
    Ut[2] = u_m[1] * UE / W_m + R3 / beta_m;
    Ut[3] = UE;

    /* spatial parts F~_1, F~_2 */
    for (int j = 0; j < 2; ++j) {
        double *F = (j == 0) ? F1t : F2t;
        double FD = rho_ln * u_m[j];
        double FE = W_m * (alpha0 * rho_ln * u_m[j] + rho_m * u_m[j] / beta_m) / Lam;
        F[0] = FD;
        F[1] = FE * u_m[0] / W_m + (j == 0 ? rho_m / beta_m : 0.0);
        F[2] = FE * u_m[1] / W_m + (j == 1 ? rho_m / beta_m : 0.0);
        F[3] = FE;
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 4: eigenvalues and scaled eigenvectors of dF_1/dU with dU/dV = R R^T.
 * (The paper defers the formulas to its cited works.)  Construction used
 * here, at w = (rho, v_n, v_t, p):
 *   lambda_+- = (v_n (1 - c^2) +- c sqrt((1 - v^2)(1 - v^2 c^2 - v_n^2 (1 - c^2))))
 *               / (1 - v^2 c^2),   c^2 = Gamma p/(rho h);
 *   lambda_2 = lambda_3 = v_n.
 * Each wave is written as a primitive perturbation dw: the contact waves are
 * d rho = 1 (entropy) and d v_t = 1 (shear); an acoustic wave of speed lam
 * has dp = 1 and, from dF = lam dU across the wave,
 *   dv_n = (1 - v_n lam)/((lam - v_n) Q),  dv_t = -lam v_t/((lam - v_n) Q),
 *   d rho = rho dv_n/(lam - v_n) - rho W^2 (v_n dv_n + v_t dv_t),  Q = rho h W^2.
 * Column m of R is dU_m / sqrt(dU_m . dV_m) with dU = (dU/dw) dw and
 * dV = (dV/dw) dw: the four columns are orthogonal in the dV/dU inner
 * product (the two contact columns are orthogonal by direct computation), so
 * R^T (dV/dU) R = I, i.e. R R^T = dU/dV.  Reading: this fixed basis of the
 * double eigenvalue's eigenspace.                                           */
static void dU_dw(double gamma, const double *w, const double *dw, double *dU)
{
    double rho = w[0], vn = w[1], vt = w[2], p = w[3];
    double W = 1.0 / sqrt(1.0 - (vn * vn + vt * vt));
    double W2 = W * W;
    double rh = rho + gamma * p / (gamma - 1.0);     /* rho h */
    double g1 = gamma / (gamma - 1.0);
    double drho = dw[0], dvn = dw[1], dvt = dw[2], dp = dw[3];
    double vdv = vn * dvn + vt * dvt;
    /* D = rho W */
    dU[0] = W * drho + rho * W2 * W * vdv;
    /* m_a = rho h W^2 v_a */
    dU[1] = W2 * vn * (drho + g1 * dp) + rh * (2.0 * W2 * W2 * vn * vdv + W2 * dvn);
    dU[2] = W2 * vt * (drho + g1 * dp) + rh * (2.0 * W2 * W2 * vt * vdv + W2 * dvt);
    /* E = rho h W^2 - p */
    dU[3] = W2 * (drho + g1 * dp) - dp + rh * 2.0 * W2 * W2 * vdv;
}

static void dV_dw(double gamma, const double *w, const double *dw, double *dV)
{
    double rho = w[0], vn = w[1], vt = w[2], p = w[3];
    double W = 1.0 / sqrt(1.0 - (vn * vn + vt * vt));
    double W3 = W * W * W;
    double beta = rho / p;
    double drho = dw[0], dvn = dw[1], dvt = dw[2], dp = dw[3];
    double dbeta = drho / p - beta * dp / p;
    double vdv = vn * dvn + vt * dvt;
    double dW = W3 * vdv;
    double un = W * vn, ut = W * vt;
    /* V_1 = Gamma/(Gamma-1) + ln rho + ln beta/(Gamma-1) + beta */
    dV[0] = drho / rho + (drho / rho - dp / p) / (gamma - 1.0) + dbeta;
    /* V_m = beta u,  u = W v */
    dV[1] = dbeta * un + beta * (W * dvn + vn * dW);
    dV[2] = dbeta * ut + beta * (W * dvt + vt * dW);
    /* V_E = -beta W */
    dV[3] = -(dbeta * W + beta * dW);
}

void oref_eigen(double gamma, const double *w, double *lam, double *R)
{
    double rho = w[0], vn = w[1], vt = w[2], p = w[3];
    double v2 = vn * vn + vt * vt;
    double W = 1.0 / sqrt(1.0 - v2);
    double h = 1.0 + gamma * p / ((gamma - 1.0) * rho);
    double c2 = gamma * p / (rho * h);
    double c = sqrt(c2);
    double disc = sqrt((1.0 - v2) * (1.0 - v2 * c2 - vn * vn * (1.0 - c2)));
    double lm = (vn * (1.0 - c2) - c * disc) / (1.0 - v2 * c2);
    double lp = (vn * (1.0 - c2) + c * disc) / (1.0 - v2 * c2);
    double Q = rho * h * W * W;
    double dw[4][4];
    double speeds[4] = {lm, vn, vn, lp};
    for (int m = 0; m < 4; ++m)
        for (int a = 0; a < 4; ++a) dw[m][a] = 0.0;
    for (int s = 0; s < 2; ++s) {
        int m = (s == 0) ? 0 : 3;
        double l = speeds[m];
        double dvn = (1.0 - vn * l) / ((l - vn) * Q);
        double dvt = -l * vt / ((l - vn) * Q);
        dw[m][0] = rho * dvn / (l - vn) - rho * W * W * (vn * dvn + vt * dvt);
        dw[m][1] = dvn;
        dw[m][2] = dvt;
        dw[m][3] = 1.0;
    }
    dw[1][0] = 1.0;   /* entropy wave */
    dw[2][2] = 1.0;   /* shear wave   */
    for (int m = 0; m < 4; ++m) {
        double dU[4], dV[4];
        dU_dw(gamma, w, dw[m], dU);
        dV_dw(gamma, w, dw[m], dV);
        double nrm = dU[0] * dV[0] + dU[1] * dV[1] + dU[2] * dV[2] + dU[3] * dV[3];
        double s = 1.0 / sqrt(nrm);
        for (int a = 0; a < 4; ++a) R[a * 4 + m] = dU[a] * s;
        lam[m] = speeds[m];
    }
}

/* ------------------------------------------------------------------------ */
/* WENO reconstruction of Jiang & Shu (1996), cited in Sec. 4.  s[0..w-1] is
 * the stencil from far upwind to far downwind; the value returned sits at the
 * downwind edge of the middle node s[(w-1)/2].  Linear weights, smoothness
 * indicators and the power 2 are the published ones.                       */
double oref_weno(int w, double eps, const double *s)
{
    if (w == 3) {
        double q0 = (-s[0] + 3.0 * s[1]) / 2.0;
        double q1 = (s[1] + s[2]) / 2.0;
        double b0 = (s[1] - s[0]) * (s[1] - s[0]);
        double b1 = (s[2] - s[1]) * (s[2] - s[1]);
        double a0 = (1.0 / 3.0) / ((eps + b0) * (eps + b0));
        double a1 = (2.0 / 3.0) / ((eps + b1) * (eps + b1));
        return (a0 * q0 + a1 * q1) / (a0 + a1);
    }
    double q0 = (2.0 * s[0] - 7.0 * s[1] + 11.0 * s[2]) / 6.0;
    double q1 = (-s[1] + 5.0 * s[2] + 2.0 * s[3]) / 6.0;
    double q2 = (2.0 * s[2] + 5.0 * s[3] - s[4]) / 6.0;
    double t0 = s[0] - 2.0 * s[1] + s[2], r0 = s[0] - 4.0 * s[1] + 3.0 * s[2];
    double t1 = s[1] - 2.0 * s[2] + s[3], r1 = s[1] - s[3];
    double t2 = s[2] - 2.0 * s[3] + s[4], r2 = 3.0 * s[2] - 4.0 * s[3] + s[4];
    double b0 = 13.0 / 12.0 * t0 * t0 + 0.25 * r0 * r0;
    double b1 = 13.0 / 12.0 * t1 * t1 + 0.25 * r1 * r1;
    double b2 = 13.0 / 12.0 * t2 * t2 + 0.25 * r2 * r2;
    double a0 = 0.1 / ((eps + b0) * (eps + b0));
    double a1 = 0.6 / ((eps + b1) * (eps + b1));
    double a2 = 0.3 / ((eps + b2) * (eps + b2));
    return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

/* ------------------------------------------------------------------------ */
/* Grid helpers: boundary conditions (step "ghost fill").
 * Reading: data ghosts are a periodic wrap or a zero-gradient copy (outflow);
 * mesh ghosts are a periodic wrap plus the period, or a linear extrapolation
 * of the two nodes next to the boundary (outflow).                         */
static int wrapi(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }
static int floordiv(int a, int n) { return (a >= 0) ? a / n : -((-a + n - 1) / n); }
static int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }

static int data_index(const oref_cfg *c, int i, int j)
{
    int ii = c->bc[0] == OREF_PERIODIC ? wrapi(i, c->nx) : clampi(i, 0, c->nx - 1);
    int jj = c->bc[1] == OREF_PERIODIC ? wrapi(j, c->ny) : clampi(j, 0, c->ny - 1);
    return jj * c->nx + ii;
}

/* coordinate comp of array a ([2][N]) at (i, j) with j in range */
static double mesh_row(const oref_cfg *c, const double *a, int comp, int i, int j, int shift)
{
    int nx = c->nx, N = c->nx * c->ny;
    const double *A = a + (size_t)comp * N + (size_t)j * nx;
    if (c->bc[0] == OREF_PERIODIC) {
        double s = (shift && comp == 0) ? floordiv(i, nx) * c->period[0] : 0.0;
        return A[wrapi(i, nx)] + s;
    }
    if (i < 0) return A[0] + i * (A[1] - A[0]);
    if (i > nx - 1) return A[nx - 1] + (i - (nx - 1)) * (A[nx - 1] - A[nx - 2]);
    return A[i];
}

static double mesh_value(const oref_cfg *c, const double *a, int comp, int i, int j, int shift)
{
    int ny = c->ny;
    if (c->bc[1] == OREF_PERIODIC) {
        double s = (shift && comp == 1) ? floordiv(j, ny) * c->period[1] : 0.0;
        return mesh_row(c, a, comp, i, wrapi(j, ny), shift) + s;
    }
    if (j < 0) {
        double a0 = mesh_row(c, a, comp, i, 0, shift), a1 = mesh_row(c, a, comp, i, 1, shift);
        return a0 + j * (a1 - a0);
    }
    if (j > ny - 1) {
        double a0 = mesh_row(c, a, comp, i, ny - 1, shift), a1 = mesh_row(c, a, comp, i, ny - 2, shift);
        return a0 + (j - (ny - 1)) * (a0 - a1);
    }
    return mesh_row(c, a, comp, i, j, shift);
}

/* delta_k[a]_i = 1/2 sum_n alpha_{p,n} (a_{i,k,+n} - a_{i,k,-n}) (Sec. 3.3). */
static double delta(const oref_cfg *c, const double *x, int comp, int i, int j, int k)
{
    double alpha[3];
    oref_alpha(c->p, alpha);
    double d = 0.0;
    for (int n = 1; n <= c->p; ++n) {
        double ap = k == 0 ? mesh_value(c, x, comp, i + n, j, 1) : mesh_value(c, x, comp, i, j + n, 1);
        double am = k == 0 ? mesh_value(c, x, comp, i - n, j, 1) : mesh_value(c, x, comp, i, j - n, 1);
        d += 0.5 * alpha[n - 1] * (ap - am);
    }
    return d;
}

/* App. B with Delta xi = Delta eta = 1 (reading: index-space computational
 * coordinates, which makes App. B's metric formulas and scheme consistent):
 *   J xi_x = delta_eta[y], J xi_y = -delta_eta[x],
 *   J eta_x = -delta_xi[y], J eta_y = delta_xi[x].   M[k][j] = J d xi_k/d x_j. */
static void node_metrics(const oref_cfg *c, const double *x, int i, int j, double M[2][2])
{
    M[0][0] = delta(c, x, 1, i, j, 1);
    M[0][1] = -delta(c, x, 0, i, j, 1);
    M[1][0] = -delta(c, x, 1, i, j, 0);
    M[1][1] = delta(c, x, 0, i, j, 0);
}

void oref_metrics(const oref_cfg *c, const double *x, double *m, double *J0)
{
    int N = c->nx * c->ny;
    for (int j = 0; j < c->ny; ++j)
        for (int i = 0; i < c->nx; ++i) {
            double M[2][2];
            node_metrics(c, x, i, j, M);
            int id = j * c->nx + i;
            m[0 * N + id] = M[0][0];
            m[1 * N + id] = M[0][1];
            m[2 * N + id] = M[1][0];
            m[3 * N + id] = M[1][1];
            /* Reading: J0 = delta_xi[x] delta_eta[y] - delta_eta[x] delta_xi[y]. */
            if (J0) J0[id] = delta(c, x, 0, i, j, 0) * delta(c, x, 1, i, j, 1)
                           - delta(c, x, 0, i, j, 1) * delta(c, x, 1, i, j, 0);
        }
}

/* ------------------------------------------------------------------------ */
/* Physics switch: the RHD and RMHD pointwise parts behind one interface.
 * RHD states have 4 components (pressure at index 3), RMHD states 8
 * (pressure at index 4, B at 5..7).                                        */
#define NVMAX 8
static int nvar(const oref_cfg *c) { return c->phys == OREF_RMHD ? 8 : 4; }

static int c2p(const oref_cfg *c, const double *U, double *w)
{
    return c->phys == OREF_RMHD ? oref_mhd_cons2prim(c->gamma, U, w, NULL)
                                : oref_cons2prim(c->gamma, U, w, NULL);
}

static void p2c(const oref_cfg *c, const double *w, double *U)
{
    if (c->phys == OREF_RMHD) oref_mhd_prim2cons(c->gamma, w, U);
    else oref_prim2cons(c->gamma, w, U);
}

static void entropy_vars(const oref_cfg *c, const double *w, double *V)
{
    if (c->phys == OREF_RMHD) oref_mhd_entropy_vars(c->gamma, w, V);
    else oref_entropy_vars(c->gamma, w, V);
}

/* Primitive state of node (conservative cons[nv][N] / J). */
static int node_prim(const oref_cfg *c, const double *cons, const double *J, int id, double *w)
{
    int N = c->nx * c->ny, nv = nvar(c);
    double U[NVMAX];
    for (int a = 0; a < nv; ++a) U[a] = cons[(size_t)a * N + id] / J[id];
    return c2p(c, U, w);
}

/* ------------------------------------------------------------------------ */
/* Padded node data used by one right-hand-side evaluation. */
typedef struct {
    const oref_cfg *c;
    int px, py;              /* padded extents nx + 2G, ny + 2G */
    double *prim;            /* [nv][P] */
    double *M;               /* [4][P]: M00 M01 M10 M11 */
    double *Mt;              /* [2][P]: J xi_t, J eta_t */
} oref_pad;

static int pad_index(const oref_pad *P, int i, int j) { return (j + G) * P->px + (i + G); }

static void pad_prim(const oref_pad *P, int i, int j, double *w)
{
    int id = pad_index(P, i, j), S = P->px * P->py, nv = nvar(P->c);
    for (int a = 0; a < nv; ++a) w[a] = P->prim[a * S + id];
}

static void pad_M(const oref_pad *P, int i, int j, double M[2][2], double Mt[2])
{
    int id = pad_index(P, i, j), S = P->px * P->py;
    M[0][0] = P->M[0 * S + id];
    M[0][1] = P->M[1 * S + id];
    M[1][0] = P->M[2 * S + id];
    M[1][1] = P->M[3 * S + id];
    Mt[0] = P->Mt[0 * S + id];
    Mt[1] = P->Mt[1 * S + id];
}

static int build_pad(const oref_cfg *c, const double *cons, const double *J,
                     const double *x, const double *xdot, oref_pad *P)
{
    int nx = c->nx, ny = c->ny, N = nx * ny, nv = nvar(c);
    P->c = c;
    P->px = nx + 2 * G;
    P->py = ny + 2 * G;
    int S = P->px * P->py;
    P->prim = (double *)malloc(sizeof(double) * nv * S);
    P->M = (double *)malloc(sizeof(double) * 4 * S);
    P->Mt = (double *)malloc(sizeof(double) * 2 * S);
    double *w = (double *)malloc(sizeof(double) * nv * N);
    int status = 0;
    /* cons2prim at every node: U = (J U)/J */
    #pragma omp parallel for reduction(min : status)
    for (int id = 0; id < N; ++id) {
        double wi[NVMAX];
        if (node_prim(c, cons, J, id, wi) != 0) status = -1;
        for (int a = 0; a < nv; ++a) w[a * N + id] = wi[a];
    }
    #pragma omp parallel for
    for (int j = -G; j < ny + G; ++j)
        for (int i = -G; i < nx + G; ++i) {
            int id = pad_index(P, i, j), src = data_index(c, i, j);
            int in = (c->bc[0] == OREF_INFLOW && i < 0) || (c->bc[1] == OREF_INFLOW && j < 0);
            for (int a = 0; a < nv; ++a) P->prim[a * S + id] = in ? c->inflow[a] : w[a * N + src];
            double M[2][2];
            node_metrics(c, x, i, j, M);
            P->M[0 * S + id] = M[0][0];
            P->M[1 * S + id] = M[0][1];
            P->M[2 * S + id] = M[1][0];
            P->M[3 * S + id] = M[1][1];
            /* eq. VCLCoeff: J xi_k,t = -sum_j xdot_j (J xi_k,x_j) */
            double xd = mesh_value(c, xdot, 0, i, j, 0);
            double yd = mesh_value(c, xdot, 1, i, j, 0);
            P->Mt[0 * S + id] = -(xd * M[0][0] + yd * M[0][1]);
            P->Mt[1 * S + id] = -(xd * M[1][0] + yd * M[1][1]);
        }
    free(w);
    return status;
}

static void free_pad(oref_pad *P)
{
    free(P->prim);
    free(P->M);
    free(P->Mt);
}

static int sgn(double a) { return (a > 0.0) - (a < 0.0); }

/* Rotation T (Sec. 4): T = diag(1, T_0, 1) for RHD and diag(1, T_0, 1, T_0)
 * for RMHD, T_0 with rows n, t (and e_3 for the 3-vectors of RMHD).  In 2D
 * the metric vector has no x_3 part, so varphi = 0 and t = (-n_y, n_x).   */
static void rotate(const oref_cfg *c, double nx_, double ny_, const double *a, double *r)
{
    if (c->phys == OREF_RMHD) {
        r[0] = a[0];
        r[1] = nx_ * a[1] + ny_ * a[2];
        r[2] = -ny_ * a[1] + nx_ * a[2];
        r[3] = a[3];
        r[4] = a[4];
        r[5] = nx_ * a[5] + ny_ * a[6];
        r[6] = -ny_ * a[5] + nx_ * a[6];
        r[7] = a[7];
    } else {
        r[0] = a[0];
        r[1] = nx_ * a[1] + ny_ * a[2];
        r[2] = -ny_ * a[1] + nx_ * a[2];
        r[3] = a[3];
    }
}

static void unrotate(const oref_cfg *c, double nx_, double ny_, const double *r, double *a)
{
    if (c->phys == OREF_RMHD) {
        a[0] = r[0];
        a[1] = nx_ * r[1] - ny_ * r[2];
        a[2] = ny_ * r[1] + nx_ * r[2];
        a[3] = r[3];
        a[4] = r[4];
        a[5] = nx_ * r[5] - ny_ * r[6];
        a[6] = ny_ * r[5] + nx_ * r[6];
        a[7] = r[7];
    } else {
        a[0] = r[0];
        a[1] = nx_ * r[1] - ny_ * r[2];
        a[2] = ny_ * r[1] + nx_ * r[2];
        a[3] = r[3];
    }
}

/* Eigen-system in the rotated frame (Sec. 4). */
static void eigen(const oref_cfg *c, const double *wrot, double *lam, double *R)
{
    if (c->phys == OREF_RMHD) oref_mhd_eigen(c->gamma, wrot, lam, R);
    else oref_eigen(c->gamma, wrot, lam, R);
}

/* The w-th order ES flux at the interface between node (i, j) and its
 * neighbour in direction k (eq. ESFlux_HO), written to F; the 2p-th order
 * temporal-metric flux (eq. MetricsFlux_O2p) to Ft and, for RMHD, the 2p-th
 * order magnetic flux B~ (eqs. BFlux_O2p, BFlux_O2) to Bt.                  */
static void interface_flux(const oref_pad *P, int k, int i, int j, double *F, double *Ft,
                           double *Bt)
{
    const oref_cfg *c = P->c;
    int nv = nvar(c), mhd = (c->phys == OREF_RMHD);
    int di = (k == 0), dj = (k == 1);
    double alpha[3];
    oref_alpha(c->p, alpha);
    for (int a = 0; a < nv; ++a) F[a] = 0.0;
    *Ft = 0.0;
    *Bt = 0.0;

    /* eq. ECFlux_O2p: sum_n alpha_{p,n} sum_{s=0}^{n-1} F~_k(U_{i-s}, U_{i-s+n}) */
    for (int n = 1; n <= c->p; ++n) {
        double Fs[NVMAX], Fts = 0.0, Bts = 0.0;
        for (int a = 0; a < nv; ++a) Fs[a] = 0.0;
        for (int s = 0; s < n; ++s) {
            int il = i - s * di, jl = j - s * dj;
            int ir = i + (n - s) * di, jr = j + (n - s) * dj;
            double wl[NVMAX], wr[NVMAX], Ml[2][2], Mr[2][2], Mtl[2], Mtr[2];
            pad_prim(P, il, jl, wl);
            pad_prim(P, ir, jr, wr);
            pad_M(P, il, jl, Ml, Mtl);
            pad_M(P, ir, jr, Mr, Mtr);
            /* eq. ECFluxCurv / UFcircle: averaged metrics times U~, F~_j */
            double mt = 0.5 * (Mtl[k] + Mtr[k]);
            double mx = 0.5 * (Ml[k][0] + Mr[k][0]);
            double my = 0.5 * (Ml[k][1] + Mr[k][1]);
            if (mhd) {
                double Ut[8], Ftj[24];
                oref_mhd_ec_flux(c->gamma, wl, wr, Ut, Ftj);
                for (int a = 0; a < 8; ++a) Fs[a] += mt * Ut[a] + mx * Ftj[a] + my * Ftj[8 + a];
                /* eq. BFlux_O2: sum_j 1/4 (M_l + M_r)(B_j,l + B_j,r) */
                Bts += 0.25 * (Ml[k][0] + Mr[k][0]) * (wl[5] + wr[5])
                     + 0.25 * (Ml[k][1] + Mr[k][1]) * (wl[6] + wr[6]);
            } else {
                double Ut[4], F1t[4], F2t[4];
                oref_ec_flux(c->gamma, wl, wr, Ut, F1t, F2t);
                for (int a = 0; a < 4; ++a) Fs[a] += mt * Ut[a] + mx * F1t[a] + my * F2t[a];
            }
            /* eq. MetricsFlux_O2 */
            Fts += 0.5 * (Mtl[k] + Mtr[k]);
        }
        for (int a = 0; a < nv; ++a) F[a] += alpha[n - 1] * Fs[a];
        *Ft += alpha[n - 1] * Fts;
        *Bt += alpha[n - 1] * Bts;
    }
    if (c->w == 0) return;

    /* eq. ESFlux_HO: F^ = F~ - 1/2 D Y <<V~>>, D = lambda^ T^{-1} R(TU). */
    double wL[NVMAX], wR[NVMAX], ML[2][2], MR[2][2], MtL[2], MtR[2];
    pad_prim(P, i, j, wL);
    pad_prim(P, i + di, j + dj, wR);
    pad_M(P, i, j, ML, MtL);
    pad_M(P, i + di, j + dj, MR, MtR);
    /* Reading: interface metrics are the mean of the two node metrics. */
    double nvx = 0.5 * (ML[k][0] + MR[k][0]);
    double nvy = 0.5 * (ML[k][1] + MR[k][1]);
    double jt = 0.5 * (MtL[k] + MtR[k]);
    double Lk = sqrt(nvx * nvx + nvy * nvy);
    /* T_0 rows: the unit normal n (theta is read as the angle of the metric
     * vector, so that the first row is n) and the tangent t = (-n_y, n_x). */
    double nx_ = nvx / Lk, ny_ = nvy / Lk;
    /* Reading: D is evaluated at the interface state built from the averages
     * of the two-point EC flux: rho = {{rho}}^ln, u = {{u}} (u = W v) and
     * p = {{rho}}/{{beta}} (beta = rho/p); for RMHD also B = {{B}}.  (With the
     * arithmetic mean of (rho, u, p) the dissipation R R^T [[V]] turns
     * anti-diffusive when beta jumps by two orders of magnitude across an
     * interface.) */
    double wm[NVMAX], wrot[NVMAX];
    {
        int nvel = mhd ? 3 : 2, ip = mhd ? 4 : 3;
        double v2L = 0.0, v2R = 0.0;
        for (int q = 0; q < nvel; ++q) {
            v2L += wL[1 + q] * wL[1 + q];
            v2R += wR[1 + q] * wR[1 + q];
        }
        double WL = 1.0 / sqrt(1.0 - v2L), WR = 1.0 / sqrt(1.0 - v2R);
        double um[3], W2_m = 1.0;
        for (int q = 0; q < nvel; ++q) {
            um[q] = 0.5 * (WL * wL[1 + q] + WR * wR[1 + q]);
            W2_m += um[q] * um[q];
        }
        double W_m = sqrt(W2_m);
        wm[0] = oref_logmean(wL[0], wR[0]);
        for (int q = 0; q < nvel; ++q) wm[1 + q] = um[q] / W_m;
        wm[ip] = (0.5 * (wL[0] + wR[0])) / (0.5 * (wL[0] / wL[ip] + wR[0] / wR[ip]));
        if (mhd)
            for (int q = 5; q < 8; ++q) wm[q] = 0.5 * (wL[q] + wR[q]);
    }
    rotate(c, nx_, ny_, wm, wrot);
    double lam[NVMAX], R[NVMAX * NVMAX];
    eigen(c, wrot, lam, R);
    /* lambda^ = max_m |J xi_t + L_k lambda_m(TU)| */
    double lhat = 0.0;
    for (int m = 0; m < nv; ++m) {
        double a = fabs(jt + Lk * lam[m]);
        if (a > lhat) lhat = a;
    }
    /* scaled entropy variables V~ = R^T T V on the stencil nodes */
    int lo = (c->w == 5) ? -2 : -1, hi = (c->w == 5) ? 3 : 2;
    double Vt[6][NVMAX];
    double scale[NVMAX];   /* magnitudes forming V~ at nodes 0, 1 */
    for (int m = 0; m < nv; ++m) scale[m] = 0.0;
    for (int q = lo; q <= hi; ++q) {
        double wq[NVMAX], V[NVMAX], TV[NVMAX];
        pad_prim(P, i + q * di, j + q * dj, wq);
        entropy_vars(c, wq, V);
        rotate(c, nx_, ny_, V, TV);
        for (int m = 0; m < nv; ++m) {
            double acc = 0.0;
            for (int a = 0; a < nv; ++a) {
                acc += R[a * nv + m] * TV[a];
                if (q == 0 || q == 1) scale[m] += fabs(R[a * nv + m] * TV[a]);
            }
            Vt[q - lo][m] = acc;
        }
    }
    double z[NVMAX];
    for (int m = 0; m < nv; ++m) {
        double sl[5], sr[5];
        int nw = c->w;
        for (int q = 0; q < nw; ++q) {
            sl[q] = Vt[q][m];                 /* nodes lo .. hi-1 (upwind = left) */
            sr[q] = Vt[(hi - lo) - q][m];     /* nodes hi .. lo+1 (upwind = right) */
        }
        double vminus = oref_weno(nw, c->weno_eps, sl);
        double vplus = oref_weno(nw, c->weno_eps, sr);
        double jw = vplus - vminus;                        /* <<V~>>^WENO */
        double jump = Vt[1 - lo][m] - Vt[0 - lo][m];       /* [[V~]]      */
        /* Reading: a jump within OREF_SIGN_TOL of the magnitudes that form it
         * is rounding noise and has sign 0 (then Y = 0, which keeps the
         * entropy inequality of Thm. 4.1). */
        int sj = fabs(jump) <= OREF_SIGN_TOL * scale[m] ? 0 : sgn(jump);
        double Y = (sgn(jw) == sj) ? 1.0 : 0.0;
        z[m] = Y * jw;
    }
    double d[NVMAX], dr[NVMAX];
    for (int a = 0; a < nv; ++a) {
        double acc = 0.0;
        for (int m = 0; m < nv; ++m) acc += R[a * nv + m] * z[m];
        d[a] = acc;
    }
    /* T^{-1} = T^T: rotate the vector parts back */
    unrotate(c, nx_, ny_, d, dr);
    for (int a = 0; a < nv; ++a) F[a] -= 0.5 * lhat * dr[a];
}

int oref_rhs(const oref_cfg *c, const double *cons, const double *J,
             const double *x, const double *xdot, double *dcons, double *dJ)
{
    int nx = c->nx, ny = c->ny, N = nx * ny, nv = nvar(c);
    oref_pad P;
    int status = build_pad(c, cons, J, x, xdot, &P);
    for (int a = 0; a < nv; ++a)
        for (int id = 0; id < N; ++id) dcons[a * N + id] = 0.0;
    for (int id = 0; id < N; ++id) dJ[id] = 0.0;
    /* eqs. RMHDSemiU_O2p_ES and RMHDSemiJ_O2p_ES (Delta xi_k = 1):
     * flux differences, and for RMHD the Godunov-Powell source
     * -Phi'(V_i)^T sum_k (B~_{i+1/2} - B~_{i-1/2}). */
    #pragma omp parallel for
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int id = j * nx + i;
            double divB = 0.0;
            for (int k = 0; k < 2; ++k) {
                double Fp[NVMAX], Fm[NVMAX], Ftp, Ftm, Btp, Btm;
                interface_flux(&P, k, i, j, Fp, &Ftp, &Btp);
                interface_flux(&P, k, i - (k == 0), j - (k == 1), Fm, &Ftm, &Btm);
                for (int a = 0; a < nv; ++a) dcons[a * N + id] -= Fp[a] - Fm[a];
                dJ[id] -= Ftp - Ftm;
                divB += Btp - Btm;
            }
            if (c->phys == OREF_RMHD) {
                double w[8], Pp[8];
                pad_prim(&P, i, j, w);
                oref_mhd_phiprime(w, Pp);
                for (int a = 0; a < 8; ++a) dcons[a * N + id] -= Pp[a] * divB;
            }
        }
    free_pad(&P);
    return status;
}

/* ------------------------------------------------------------------------ */
int oref_state_prim(const oref_cfg *c, const double *cons, const double *J, double *prim)
{
    int N = c->nx * c->ny, nv = nvar(c), status = 0;
    for (int id = 0; id < N; ++id) {
        double w[NVMAX];
        if (node_prim(c, cons, J, id, w) != 0) status = -1;
        for (int a = 0; a < nv; ++a) prim[a * N + id] = w[a];
    }
    return status;
}

int oref_init_state(const oref_cfg *c, const double *prim, const double *x,
                    double *cons, double *J)
{
    int N = c->nx * c->ny, nv = nvar(c);
    double *m = (double *)malloc(sizeof(double) * 4 * N);
    oref_metrics(c, x, m, J);
    free(m);
    for (int id = 0; id < N; ++id) {
        double w[NVMAX], U[NVMAX];
        for (int a = 0; a < nv; ++a) w[a] = prim[a * N + id];
        p2c(c, w, U);
        for (int a = 0; a < nv; ++a) cons[a * N + id] = J[id] * U[a];
    }
    return 0;
}

/* Speed bounds of every node for eq. cfl: bmin[k][N], bmax[k][N] =
 * L_k lambda_min / J and L_k lambda_max / J, lambda the eigenvalues of the
 * flux Jacobian along the unit metric normal of direction k (L_k its
 * length), i.e. the extreme eigenvalues of d(F_k)/d(JU) on a static mesh. */
static int speed_bounds(const oref_cfg *c, const double *cons, const double *J, const double *x,
                        double *bmin, double *bmax)
{
    int nx = c->nx, ny = c->ny, N = nx * ny, nv = nvar(c), status = 0;
    #pragma omp parallel for reduction(min : status)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int id = j * nx + i;
            double w[NVMAX], M[2][2];
            if (node_prim(c, cons, J, id, w) != 0) status = -1;
            node_metrics(c, x, i, j, M);
            for (int k = 0; k < 2; ++k) {
                double Lk = sqrt(M[k][0] * M[k][0] + M[k][1] * M[k][1]);
                double wr[NVMAX], lam[NVMAX], R[NVMAX * NVMAX];
                rotate(c, M[k][0] / Lk, M[k][1] / Lk, w, wr);
                eigen(c, wr, lam, R);
                double lo = lam[0], hi = lam[0];
                for (int m = 1; m < nv; ++m) {
                    if (lam[m] < lo) lo = lam[m];
                    if (lam[m] > hi) hi = lam[m];
                }
                bmin[k * N + id] = Lk * lo / J[id];
                bmax[k * N + id] = Lk * hi / J[id];
            }
        }
    return status;
}

/* eq. cfl with the mesh velocity in the spectral radius, solved for dt.
 *
 * The spectral radius of d(F_k)/d(JU) at node i is
 *   rho_{k,i} = max_m |(J xi_k)_t + L_k lambda_m| / J_i,
 * with the temporal metric (J xi_k)_t = -xdot . (J xi_k,x) (eq. VCLCoeff) and
 * the mesh velocity xdot = Delta tau d / dt of Sec. 5 (d = x^[mu] - x^n).  So
 *   dt rho_{k,i} = max_m |dt b_{k,i,m} - tau a_{k,i}|,
 *   a = d.(J xi_k,x)/J,  b_m = L_k lambda_m / J,
 * and since max over m of |t b_m - c| for t >= 0 is max(t b_max - c,
 * c - t b_min), eq. cfl, dt sum_k max_i rho_{k,i} = CFL, reads g(dt) = CFL
 * with
 *   g(t) = sum_k max_i max(t bmax_{k,i} - tau a_{k,i}, tau a_{k,i} - t bmin_{k,i}),
 * a convex piecewise-linear function of t (a sum of maxima of lines), with
 * g(0) = C_m = tau sum_k max_i |a_{k,i}| (the displacement's own Courant
 * number) and t S - C_m <= g(t) <= t S + C_m, S = sum_k max_i max(|bmin|,
 * |bmax|) the static radius.  For C_m < CFL the root is unique and lies in
 * [(CFL - C_m)/S, (CFL + C_m)/S].
 *
 * Reading (the paper defines xdot through dt^n and dt^n through xdot):
 *   - dt^n is that root: Newton's method from the right end, each step to
 *     the root of the line that is active at the iterate (the smaller slope
 *     where two lines tie: the left derivative).  A convex function lies
 *     above each such line, so the iterates decrease monotonically to the
 *     root and stop on its piece; the iteration ends once g <= CFL, or once
 *     the Newton step is below 2^-50 t (the root up to rounding).  If
 *     OREF_CFL_NEWTON evaluations do not end it, the safe lower bound
 *     (CFL - C_m)/S is used.
 *   - Delta tau is left as the limiter gave it, unless C_m >= CFL, where no
 *     dt > 0 satisfies eq. cfl: then Delta tau is scaled so that C_m = CFL/2.
 *   - A given dt > 0 is used as is, with the same rule for Delta tau.
 * Arrays [ndir][N]; *tau is the limiter value on entry and the one used on
 * return; *iters (may be NULL) receives the Newton steps taken (-1: the
 * fallback).                                                                 */
double oref_cfl_solve(int ndir, long N, double cfl, const double *a, const double *bmin, const double *bmax,
                      double dt_given, double *tau, int *iters)
{
    double C = 0.0, S = 0.0;
    for (int k = 0; k < ndir; ++k) {
        double amax = 0.0, smax = 0.0;
        for (long i = 0; i < N; ++i) {
            double av = fabs(a[k * N + i]), sv = fmax(fabs(bmin[k * N + i]), fabs(bmax[k * N + i]));
            if (av > amax) amax = av;
            if (sv > smax) smax = sv;
        }
        C += amax;
        S += smax;
    }
    C *= *tau;
    if (C >= cfl) {
        *tau *= 0.5 * cfl / C;
        C = 0.5 * cfl;
    }
    if (iters) *iters = 0;
    if (dt_given > 0.0) return dt_given;
    if (!(C > 0.0)) return cfl / S;
    double t = (cfl + C) / S;
    for (int it = 0; it < OREF_CFL_NEWTON; ++it) {
        double g = 0.0, slope = 0.0;
        for (int k = 0; k < ndir; ++k) {
            double vk = -1.0, sk = 0.0;
            for (long i = 0; i < N; ++i) {
                double ta = *tau * a[k * N + i];
                double up = t * bmax[k * N + i] - ta, dn = ta - t * bmin[k * N + i];
                double v = up > dn ? up : dn;
                double sl = up > dn ? bmax[k * N + i] : (dn > up ? -bmin[k * N + i]
                                                                  : fmin(bmax[k * N + i], -bmin[k * N + i]));
                if (v > vk || (v == vk && sl < sk)) {
                    vk = v;
                    sk = sl;
                }
            }
            g += vk;
            slope += sk;
        }
        if (g <= cfl) {
            if (iters) *iters = it;
            return t;
        }
        if (!(slope > 0.0)) break;
        double step = (g - cfl) / slope;
        if (step <= 0x1p-50 * t) {     /* on the root up to rounding */
            if (iters) *iters = it;
            return t;
        }
        t -= step;
    }
    if (iters) *iters = -1;
    return (cfl - C) / S;
}

/* eq. cfl: dt = CFL / sum_k max_i rho_{k,i}, rho_{k,i} the spectral radius of
 * d(F_k)/d(JU) at node i.  Reading: the static-mesh radius (xdot = 0) is
 * used, rho_{k,i} = L_{k,i} max_m |lambda_m| / J_i, because the mesh velocity
 * of the step is itself defined through dt.                                */
int oref_cfl_dt(const oref_cfg *c, const double *cons, const double *J,
                const double *x, double *dt)
{
    int nx = c->nx, ny = c->ny, nv = nvar(c), status = 0;
    double rmax[2] = {0.0, 0.0};
    #pragma omp parallel for reduction(min : status) reduction(max : rmax[:2])
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int id = j * nx + i;
            double w[NVMAX], M[2][2];
            if (node_prim(c, cons, J, id, w) != 0) status = -1;
            node_metrics(c, x, i, j, M);
            for (int k = 0; k < 2; ++k) {
                double Lk = sqrt(M[k][0] * M[k][0] + M[k][1] * M[k][1]);
                double nx_ = M[k][0] / Lk, ny_ = M[k][1] / Lk;
                double wr[NVMAX], lam[NVMAX], R[NVMAX * NVMAX];
                rotate(c, nx_, ny_, w, wr);
                eigen(c, wr, lam, R);
                double a = 0.0;
                for (int m = 0; m < nv; ++m)
                    if (fabs(lam[m]) > a) a = fabs(lam[m]);
                double r = Lk * a / J[id];
                if (r > rmax[k]) rmax[k] = r;
            }
        }
    *dt = c->cfl / (rmax[0] + rmax[1]);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Sec. 5: adaptive mesh redistribution at t^n, and the step size.
 *   monitor (eq. monitor)  omega = sqrt(1 + alpha |grad sigma| / max |grad sigma|)
 *   low-pass filter        omega <- sum_{j in {-1,0,1}^2} (1/2)^{|j1|+|j2|+2} omega_{i+j}
 *   Jacobi (mu sweeps)     x_i <- sum_k [(w_i + w_{i+e_k}) x_{i+e_k} + (w_i + w_{i-e_k}) x_{i-e_k}]
 *                                 / sum_k [2 w_i + w_{i+e_k} + w_{i-e_k}]
 *   limiter                Delta tau bounds, then xdot = Delta tau (x^[mu] - x^n) / dt.
 * Readings: |grad sigma| by second-order central differences in index space;
 * omega = 1 when max |grad sigma| = 0; the 2D filter exponent is
 * |j1|+|j2|+2 (weights summing to 1, the 2D analogue of the printed 3D
 * filter); nodes on an outflow boundary stay fixed; Delta tau = clip of the
 * bounds to [0, 1]; the neighbour in each bound is along the direction of the
 * coordinate that moves (the printed "(x_1)" read as x_k).
 *
 * Step size (eq. cfl, whose spectral radius includes the temporal metric,
 * i.e. the mesh velocity): see oref_cfl_solve.  *dt_out receives the step. */
/* sigma at node (i, j) of the index space, ghosts included: the inflow
 * state's beyond an inflow end (the data the scheme's fluxes see there), else
 * the boundary-mapped node's */
static double sigma_at(const oref_cfg *c, const double *sig, double sig_in, int i, int j)
{
    if ((c->bc[0] == OREF_INFLOW && i < 0) || (c->bc[1] == OREF_INFLOW && j < 0)) return sig_in;
    return sig[data_index(c, i, j)];
}

int oref_monitor(const oref_cfg *c, const double *cons, const double *J, double *om)
{
    int nx = c->nx, ny = c->ny, N = nx * ny, status = 0;
    double *sig = (double *)malloc(sizeof(double) * N);
    double *lap = (double *)malloc(sizeof(double) * N);
    #pragma omp parallel for reduction(min : status)
    for (int id = 0; id < N; ++id) {
        double w[NVMAX];
        if (node_prim(c, cons, J, id, w) != 0) status = -1;
        sig[id] = (c->monitor == OREF_MONITOR_LNRHO) ? log(w[0]) : w[0];
    }
    double sig_in = (c->monitor == OREF_MONITOR_LNRHO) ? log(c->inflow[0]) : c->inflow[0];
    double gmax = 0.0, lmax = 0.0;
    #pragma omp parallel for reduction(max : gmax, lmax)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double e = sigma_at(c, sig, sig_in, i + 1, j), wv = sigma_at(c, sig, sig_in, i - 1, j);
            double n = sigma_at(c, sig, sig_in, i, j + 1), s = sigma_at(c, sig, sig_in, i, j - 1);
            double gx = 0.5 * (e - wv), gy = 0.5 * (n - s);
            double g = sqrt(gx * gx + gy * gy);
            double l = fabs(e + wv + n + s - 4.0 * sig[j * nx + i]);
            om[j * nx + i] = g;
            lap[j * nx + i] = l;
            if (g > gmax) gmax = g;
            if (l > lmax) lmax = l;
        }
    for (int id = 0; id < N; ++id) {
        double a = 1.0;
        if (gmax > 0.0) a += c->alpha * om[id] / gmax;
        if (lmax > 0.0) a += c->alpha_lap * lap[id] / lmax;
        om[id] = sqrt(a);
    }
    free(sig);
    free(lap);
    return status;
}

/* The low-pass filter of the Sec. 5 remark, applied n times in place:
 * om_i <- sum_{j in {-1,0,1}^2} (1/2)^{|j1|+|j2|+2} om_{i+j}, neighbours
 * through the boundary mapping of the data (periodic wrap or the boundary
 * node's copy). */
void oref_filter(const oref_cfg *c, double *om, int n)
{
    int nx = c->nx, ny = c->ny, N = nx * ny;
    double *om2 = (double *)malloc(sizeof(double) * N);
    for (int f = 0; f < n; ++f) {
        #pragma omp parallel for
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double acc = 0.0;
                for (int b = -1; b <= 1; ++b)
                    for (int a = -1; a <= 1; ++a)
                        acc += ldexp(1.0, -(abs(a) + abs(b) + 2)) * om[data_index(c, i + a, j + b)];
                om2[j * nx + i] = acc;
            }
        memcpy(om, om2, sizeof(double) * N);
    }
    free(om2);
}

/* mu sweeps of the Jacobi iteration of the Sec. 5 mesh equations with the
 * monitor om frozen, from X^[0] = x: each sweep solves, node by node,
 *   sum_k [(om_i + om_{i,k,+1})(X^[nu]_{i,k,+1} - X^[nu+1]_i)
 *          - (om_i + om_{i,k,-1})(X^[nu+1]_i - X^[nu]_{i,k,-1})] = 0
 * for X^[nu+1]_i.  Nodes on a non-periodic end stay fixed; mesh neighbours
 * beyond an end come from the mesh's ghost rule (period shift or linear
 * extrapolation). */
void oref_jacobi(const oref_cfg *c, const double *om, const double *x, int mu, double *X)
{
    int nx = c->nx, ny = c->ny, N = nx * ny;
    double *Xn = (double *)malloc(sizeof(double) * 2 * N);
    memcpy(X, x, sizeof(double) * 2 * N);
    for (int nu = 0; nu < mu; ++nu) {
        #pragma omp parallel for
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int id = j * nx + i;
                int fixed = (c->bc[0] != OREF_PERIODIC && (i == 0 || i == nx - 1)) ||
                            (c->bc[1] != OREF_PERIODIC && (j == 0 || j == ny - 1));
                if (fixed) {
                    Xn[id] = X[id];
                    Xn[N + id] = X[N + id];
                    continue;
                }
                double wi = om[id];
                double we = om[data_index(c, i + 1, j)], ww = om[data_index(c, i - 1, j)];
                double wn = om[data_index(c, i, j + 1)], ws = om[data_index(c, i, j - 1)];
                double den = (2.0 * wi + we + ww) + (2.0 * wi + wn + ws);
                for (int comp = 0; comp < 2; ++comp) {
                    double num = (wi + we) * mesh_value(c, X, comp, i + 1, j, 1)
                               + (wi + ww) * mesh_value(c, X, comp, i - 1, j, 1)
                               + (wi + wn) * mesh_value(c, X, comp, i, j + 1, 1)
                               + (wi + ws) * mesh_value(c, X, comp, i, j - 1, 1);
                    Xn[comp * N + id] = num / den;
                }
            }
        memcpy(X, Xn, sizeof(double) * 2 * N);
    }
    free(Xn);
}

int oref_mesh(const oref_cfg *c, const double *cons, const double *J,
              const double *x, double dt, double *xdot, double *dtau, double *dt_out)
{
    int nx = c->nx, ny = c->ny, N = nx * ny, status = 0;
    if (!c->move_mesh) {
        for (int a = 0; a < 2 * N; ++a) xdot[a] = 0.0;
        if (dtau) *dtau = 0.0;
        if (!(dt > 0.0)) status |= oref_cfl_dt(c, cons, J, x, &dt);
        if (dt_out) *dt_out = dt;
        return status;
    }
    double *om = (double *)malloc(sizeof(double) * N);
    double *X = (double *)malloc(sizeof(double) * 2 * N);
    status |= oref_monitor(c, cons, J, om);
    oref_filter(c, om, c->n_filter);
    oref_jacobi(c, om, x, c->mu, X);
    double tau = 1.0;
    #pragma omp parallel for reduction(min : tau)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int id = j * nx + i;
            for (int k = 0; k < 2; ++k) {
                double d = X[k * N + id] - x[k * N + id];
                int di = (k == 0), dj = (k == 1);
                double b;
                if (d < 0.0) {
                    b = -(x[k * N + id] - mesh_value(c, x, k, i - di, j - dj, 1)) / (2.0 * d);
                } else if (d > 0.0) {
                    b = (mesh_value(c, x, k, i + di, j + dj, 1) - x[k * N + id]) / (2.0 * d);
                } else {
                    continue;
                }
                if (b < tau) tau = b;
            }
        }
    if (tau < 0.0) tau = 0.0;
    /* a_{k,i} = d_i . (J xi_k,x)_i / J_i for the full displacement
     * d = x^[mu] - x^n, and the speed bounds of every node */
    double *am = (double *)malloc(sizeof(double) * 2 * N);
    double *bmin = (double *)malloc(sizeof(double) * 2 * N);
    double *bmax = (double *)malloc(sizeof(double) * 2 * N);
    #pragma omp parallel for
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int id = j * nx + i;
            double M[2][2];
            node_metrics(c, x, i, j, M);
            double d0 = X[id] - x[id], d1 = X[N + id] - x[N + id];
            for (int k = 0; k < 2; ++k) am[k * N + id] = (d0 * M[k][0] + d1 * M[k][1]) / J[id];
        }
    status |= speed_bounds(c, cons, J, x, bmin, bmax);
    dt = oref_cfl_solve(2, N, c->cfl, am, bmin, bmax, dt, &tau, NULL);
    free(am);
    free(bmin);
    free(bmax);
    for (int a = 0; a < 2 * N; ++a) xdot[a] = tau * (X[a] - x[a]) / dt;
    if (dtau) *dtau = tau;
    if (dt_out) *dt_out = dt;
    free(om);
    free(X);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Third-order SSP Runge-Kutta (Prop. 3.2, Sec. 7), applied to (JU, J) and to
 * the mesh dx/dt = xdot with the mesh velocity held for the step:
 *   y1 = y^n + dt L(y^n)
 *   y2 = 3/4 y^n + 1/4 (y1 + dt L(y1))
 *   y^{n+1} = 1/3 y^n + 2/3 (y2 + dt L(y2)).                               */
int oref_rk_step(const oref_cfg *c, double *cons, double *J, double *x,
                 double dt, double *dt_used)
{
    int N = c->nx * c->ny, nv = nvar(c), status = 0;
    double *xdot = (double *)calloc(2 * (size_t)N, sizeof(double));
    double *c1 = (double *)malloc(sizeof(double) * nv * N);
    double *c2 = (double *)malloc(sizeof(double) * nv * N);
    double *J1 = (double *)malloc(sizeof(double) * N);
    double *J2 = (double *)malloc(sizeof(double) * N);
    double *x1 = (double *)malloc(sizeof(double) * 2 * N);
    double *x2 = (double *)malloc(sizeof(double) * 2 * N);
    double *L = (double *)malloc(sizeof(double) * nv * N);
    double *LJ = (double *)malloc(sizeof(double) * N);
    double dtau = 0.0;
    status |= oref_mesh(c, cons, J, x, dt, xdot, &dtau, &dt);

    status |= oref_rhs(c, cons, J, x, xdot, L, LJ);
    for (int a = 0; a < nv * N; ++a) c1[a] = cons[a] + dt * L[a];
    for (int a = 0; a < N; ++a) J1[a] = J[a] + dt * LJ[a];
    for (int a = 0; a < 2 * N; ++a) x1[a] = x[a] + dt * xdot[a];

    status |= oref_rhs(c, c1, J1, x1, xdot, L, LJ);
    for (int a = 0; a < nv * N; ++a) c2[a] = 0.75 * cons[a] + 0.25 * (c1[a] + dt * L[a]);
    for (int a = 0; a < N; ++a) J2[a] = 0.75 * J[a] + 0.25 * (J1[a] + dt * LJ[a]);
    for (int a = 0; a < 2 * N; ++a) x2[a] = 0.75 * x[a] + 0.25 * (x1[a] + dt * xdot[a]);

    status |= oref_rhs(c, c2, J2, x2, xdot, L, LJ);
    for (int a = 0; a < nv * N; ++a) cons[a] = cons[a] / 3.0 + 2.0 / 3.0 * (c2[a] + dt * L[a]);
    for (int a = 0; a < N; ++a) J[a] = J[a] / 3.0 + 2.0 / 3.0 * (J2[a] + dt * LJ[a]);
    for (int a = 0; a < 2 * N; ++a) x[a] = x[a] / 3.0 + 2.0 / 3.0 * (x2[a] + dt * xdot[a]);

    if (dt_used) *dt_used = dt;
    free(xdot); free(c1); free(c2); free(J1); free(J2);
    free(x1); free(x2); free(L); free(LJ);
    return status;
}

/* One SSP-RK3 step with a given mesh velocity xdot [2][N] and step dt (the
 * map whose derivative the adjoint computes: the step's mesh motion and dt
 * held at given values). */
int oref_rk_step_given(const oref_cfg *c, double *cons, double *J, double *x,
                       const double *xdot, double dt)
{
    int N = c->nx * c->ny, nv = nvar(c), status = 0;
    double *c1 = (double *)malloc(sizeof(double) * nv * N);
    double *c2 = (double *)malloc(sizeof(double) * nv * N);
    double *J1 = (double *)malloc(sizeof(double) * N);
    double *J2 = (double *)malloc(sizeof(double) * N);
    double *x1 = (double *)malloc(sizeof(double) * 2 * N);
    double *x2 = (double *)malloc(sizeof(double) * 2 * N);
    double *L = (double *)malloc(sizeof(double) * nv * N);
    double *LJ = (double *)malloc(sizeof(double) * N);
    status |= oref_rhs(c, cons, J, x, xdot, L, LJ);
    for (int a = 0; a < nv * N; ++a) c1[a] = cons[a] + dt * L[a];
    for (int a = 0; a < N; ++a) J1[a] = J[a] + dt * LJ[a];
    for (int a = 0; a < 2 * N; ++a) x1[a] = x[a] + dt * xdot[a];
    status |= oref_rhs(c, c1, J1, x1, xdot, L, LJ);
    for (int a = 0; a < nv * N; ++a) c2[a] = 0.75 * cons[a] + 0.25 * (c1[a] + dt * L[a]);
    for (int a = 0; a < N; ++a) J2[a] = 0.75 * J[a] + 0.25 * (J1[a] + dt * LJ[a]);
    for (int a = 0; a < 2 * N; ++a) x2[a] = 0.75 * x[a] + 0.25 * (x1[a] + dt * xdot[a]);
    status |= oref_rhs(c, c2, J2, x2, xdot, L, LJ);
    for (int a = 0; a < nv * N; ++a) cons[a] = cons[a] / 3.0 + 2.0 / 3.0 * (c2[a] + dt * L[a]);
    for (int a = 0; a < N; ++a) J[a] = J[a] / 3.0 + 2.0 / 3.0 * (J2[a] + dt * LJ[a]);
    for (int a = 0; a < 2 * N; ++a) x[a] = x[a] / 3.0 + 2.0 / 3.0 * (x2[a] + dt * xdot[a]);
    free(c1); free(c2); free(J1); free(J2); free(x1); free(x2); free(L); free(LJ);
    return status;
}

/* Totals: sum_i J_i eta_i (Sec. 6 total entropy, without the 1/N^2),
 * sum_i (J D)_i, sum_i J_i and the semi-discrete entropy production
 * sum_i (V_i . d(JU)_i/dt - phi_i dJ_i/dt), which vanishes for the EC scheme
 * on a periodic grid (Thm. 3.1) and is non-positive for the ES scheme.     */
int oref_totals(const oref_cfg *c, const double *cons, const double *J,
                const double *dcons, const double *dJ, double *out)
{
    int N = c->nx * c->ny, nv = nvar(c), status = 0;
    double S = 0.0, mass = 0.0, vol = 0.0, prod = 0.0;
    for (int id = 0; id < N; ++id) {
        double w[NVMAX];
        if (node_prim(c, cons, J, id, w) != 0) status = -1;
        double eta, phi;
        if (c->phys == OREF_RMHD) {
            double psi[3], Phi;
            eta = oref_mhd_entropy(c->gamma, w);
            oref_mhd_potentials(w, &phi, psi, &Phi);
        } else {
            double psi[2];
            eta = oref_entropy(c->gamma, w);
            oref_potentials(w, &phi, psi);
        }
        S += J[id] * eta;
        mass += cons[id];
        vol += J[id];
        if (dcons && dJ) {
            double V[NVMAX];
            entropy_vars(c, w, V);
            double vd = 0.0;
            for (int a = 0; a < nv; ++a) vd += V[a] * dcons[a * N + id];
            prod += vd - phi * dJ[id];
        }
    }
    out[0] = S;
    out[1] = mass;
    out[2] = vol;
    out[3] = prod;
    return status;
}
