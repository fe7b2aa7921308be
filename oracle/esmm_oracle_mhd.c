/*
 * esmm_oracle_mhd.c -- the pointwise RMHD parts of the plain FP64 CPU oracle
 * (Duan & Tang, arXiv 2107.12027): state conversions, the entropy pair and its
 * potentials with the Godunov-Powell symmetrizer, the two-point EC flux and
 * the scaled eigenvectors of the symmetrized system.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load the oracle; it shares no code with the
 * CUDA library.
 *
 * Primitive state w[8] = (rho, v_1, v_2, v_3, p, B_1, B_2, B_3); conservative
 * U[8] = (D, m_1, m_2, m_3, E, B_1, B_2, B_3) (eq. RMHDdiv2).  Auxiliary
 * quantities: W = 1/sqrt(1 - |v|^2), u = W v, b^0 = W (v.B),
 * b = B/W + b^0 v (spatial part of the magnetic four-vector),
 * |b|^2 = b^alpha b_alpha = |B|^2/W^2 + (v.B)^2, beta = rho/p.
 */
#include "esmm_oracle.h"

#include <complex.h>
#include <math.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------------ */
/* eq. RMHDdiv2: D = rho W, m = (rho h W^2 + |B|^2) v - (v.B) B,
 * E = rho h W^2 - p_t + |B|^2, p_t = p + |b|^2/2, h = 1 + Gamma/(Gamma-1) p/rho
 * (ideal gas, eq. EOS).                                                     */
void oref_mhd_prim2cons(double gamma, const double *w, double *U)
{
    double rho = w[0], p = w[4];
    const double *v = w + 1, *B = w + 5;
    double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    double W2 = 1.0 / (1.0 - v2);
    double W = sqrt(W2);
    double vB = v[0] * B[0] + v[1] * B[1] + v[2] * B[2];
    double B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    double bb = B2 / W2 + vB * vB;
    double rhoh = rho + gamma / (gamma - 1.0) * p;
    U[0] = rho * W;
    for (int k = 0; k < 3; ++k) U[1 + k] = (rhoh * W2 + B2) * v[k] - vB * B[k];
    U[4] = rhoh * W2 - (p + 0.5 * bb) + B2;
    for (int k = 0; k < 3; ++k) U[5 + k] = B[k];
}

/* eq. RMHDdiv2: F_d = (D v_d, m v_d - B_d (B/W^2 + (v.B) v) + p_t e_d, m_d,
 * v_d B - B_d v). */
void oref_mhd_flux(double gamma, const double *w, int dir, double *F)
{
    double U[8];
    oref_mhd_prim2cons(gamma, w, U);
    const double *v = w + 1, *B = w + 5;
    double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    double W2 = 1.0 / (1.0 - v2);
    double vB = v[0] * B[0] + v[1] * B[1] + v[2] * B[2];
    double B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    double pt = w[4] + 0.5 * (B2 / W2 + vB * vB);
    F[0] = U[0] * v[dir];
    for (int k = 0; k < 3; ++k)
        F[1 + k] = U[1 + k] * v[dir] - B[dir] * (B[k] / W2 + vB * v[k]) + (k == dir ? pt : 0.0);
    F[4] = U[1 + dir];
    for (int k = 0; k < 3; ++k) F[5 + k] = v[dir] * B[k] - B[dir] * v[k];
}

/* Conservative -> primitive recovery (Sec. 1 names only "a nonlinear
 * algebraic equation").  Reading: Newton's method on Z = rho h W^2 with a
 * bisection safeguard.  With S = m.B, the momentum relation gives
 *   v.B = S/Z,  |v|^2(Z) = (|m|^2 + (2Z + |B|^2) S^2/Z^2) / (Z + |B|^2)^2,
 *   p(Z) = (Gamma-1)/Gamma (Z/W^2 - D/W),
 * and the energy relation is the residual
 *   f(Z) = Z - p(Z) + |B|^2 (1 + |v|^2)/2 - S^2/(2 Z^2) - E.
 * f > 0 at Z = Gamma E (there Z - p >= Z/Gamma = E), and a trial Z with
 * |v|^2(Z) >= 1 lies below the root, so [0, Gamma E] brackets it.  Stops when
 * a step changes Z by at most 1e-15 (E + Z), or at an iterate where
 * |f| <= 2e-15 (E + Z), f's rounding level (the open bracket would reject
 * that root's tiny steps and bisect).  Returns 0, -1 (non-admissible
 * input or result) or -2 (no convergence).                                 */
int oref_mhd_cons2prim(double gamma, const double *U, double *w, int *iters)
{
    double D = U[0], E = U[4];
    const double *m = U + 1, *B = U + 5;
    double m2 = m[0] * m[0] + m[1] * m[1] + m[2] * m[2];
    double B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    double S = m[0] * B[0] + m[1] * B[1] + m[2] * B[2];
    double S2 = S * S;
    double g = (gamma - 1.0) / gamma;
    if (!(D > 0.0) || !(E > 0.0)) return -1;
    double lo = 0.0, hi = gamma * E;
    double Z = 0.5 * (lo + hi);
    int it, ok = 0;
    for (it = 1; it <= 300; ++it) {
        double ZB = Z + B2;
        double N = m2 + (2.0 * Z + B2) * S2 / (Z * Z);
        double v2 = N / (ZB * ZB);
        double Zn;
        if (!(v2 < 1.0)) {
            lo = Z;
            Zn = 0.5 * (lo + hi);
        } else {
            double iW2 = 1.0 - v2, iW = sqrt(iW2);
            double p = g * (Z * iW2 - D * iW);
            double f = Z - p + 0.5 * B2 * (1.0 + v2) - 0.5 * S2 / (Z * Z) - E;
            double dN = -2.0 * S2 / (Z * Z) - 2.0 * B2 * S2 / (Z * Z * Z);
            double dv2 = dN / (ZB * ZB) - 2.0 * N / (ZB * ZB * ZB);
            double dp = g * (iW2 - Z * dv2 + 0.5 * D * dv2 / iW);
            double df = 1.0 - dp + 0.5 * B2 * dv2 + S2 / (Z * Z * Z);
            if (fabs(f) <= 2.0e-15 * (E + Z)) { /* residual at rounding level */
                ok = 1;
                break;
            }
            Zn = Z;                         /* f = 0: Z is a root */
            if (f != 0.0) {
                if (f < 0.0) lo = Z; else hi = Z;
                Zn = Z - f / df;
                if (!(Zn > lo && Zn < hi)) Zn = 0.5 * (lo + hi);
            }
        }
        if (fabs(Zn - Z) <= 1.0e-15 * (E + Zn)) {
            Z = Zn;
            ok = 1;
            break;
        }
        Z = Zn;
    }
    if (iters) *iters = it;
    double ZB = Z + B2;
    double v2 = (m2 + (2.0 * Z + B2) * S2 / (Z * Z)) / (ZB * ZB);
    if (!(v2 < 1.0)) return -1;
    double iW2 = 1.0 - v2, iW = sqrt(iW2);
    double vB = S / Z;
    w[0] = D * iW;
    for (int k = 0; k < 3; ++k) w[1 + k] = (m[k] + vB * B[k]) / ZB;
    w[4] = g * (Z * iW2 - D * iW);
    for (int k = 0; k < 3; ++k) w[5 + k] = B[k];
    if (!(w[4] > 0.0)) return -1;
    return ok ? 0 : -2;
}

/* ------------------------------------------------------------------------ */
/* eq. EntropyPair: eta = -rho W s/(Gamma-1), s = ln(p/rho^Gamma). */
double oref_mhd_entropy(double gamma, const double *w)
{
    double v2 = w[1] * w[1] + w[2] * w[2] + w[3] * w[3];
    double W = 1.0 / sqrt(1.0 - v2);
    double s = log(w[4]) - gamma * log(w[0]);
    return -w[0] * W * s / (gamma - 1.0);
}

/* Sec. 2, explicit entropy variables:
 *   V = ((Gamma - s)/(Gamma-1) + rho/p, rho W v/p, -rho W/p,
 *        rho (B + W^2 v (v.B))/(p W)),
 * the last block being beta b.                                              */
void oref_mhd_entropy_vars(double gamma, const double *w, double *V)
{
    double rho = w[0], p = w[4];
    const double *v = w + 1, *B = w + 5;
    double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    double W = 1.0 / sqrt(1.0 - v2);
    double vB = v[0] * B[0] + v[1] * B[1] + v[2] * B[2];
    double s = log(p) - gamma * log(rho);
    double beta = rho / p;
    V[0] = (gamma - s) / (gamma - 1.0) + beta;
    for (int k = 0; k < 3; ++k) V[1 + k] = beta * W * v[k];
    V[4] = -beta * W;
    for (int k = 0; k < 3; ++k) V[5 + k] = beta * (B[k] + W * W * v[k] * vB) / W;
}

/* eq. Phi and eq. EntropyPotential:
 *   Phi = rho W (v.B)/p,
 *   phi = rho W + rho W |b|^2/(2p),  psi_k = rho v_k W + rho v_k W |b|^2/(2p). */
void oref_mhd_potentials(const double *w, double *phi, double *psi, double *Phi)
{
    double rho = w[0], p = w[4];
    const double *v = w + 1, *B = w + 5;
    double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    double W2 = 1.0 / (1.0 - v2), W = sqrt(W2);
    double vB = v[0] * B[0] + v[1] * B[1] + v[2] * B[2];
    double B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    double bb = B2 / W2 + vB * vB;
    double f = rho * W * (1.0 + bb / (2.0 * p));
    *phi = f;
    for (int k = 0; k < 3; ++k) psi[k] = f * v[k];
    *Phi = rho * W * vB / p;
}

/* eq. Phi: Phi'(V) = (0, B/W^2 + v (v.B), v.B, v). */
void oref_mhd_phiprime(const double *w, double *P)
{
    const double *v = w + 1, *B = w + 5;
    double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    double iW2 = 1.0 - v2;
    double vB = v[0] * B[0] + v[1] * B[1] + v[2] * B[2];
    P[0] = 0.0;
    for (int k = 0; k < 3; ++k) P[1 + k] = B[k] * iW2 + v[k] * vB;
    P[4] = vB;
    for (int k = 0; k < 3; ++k) P[5 + k] = v[k];
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1, the two-point parts of the EC flux, with
 *   [[V]]^T U~ = [[phi]],   [[V]]^T F~_j = [[psi_j]] - {{B_j}} [[Phi]].
 * Means: {{a}} = (a_l + a_r)/2, a^ln = [[a]]/[[ln a]].
 *
 * U~ is the paper's U~^RMHD.  Reading: in R_1 the sum runs over k = 1..3
 * (the printed k = 1..2 drops the third component) and its magnetic term is
 * 1/2 {{W (b^k)^2}} (printed 1/2 {{W}}{{(b^k)^2}}, which misses the EC
 * condition by exactly (1/8)[[beta]][[W]][[|b|^2]]; the product mean is what
 * the coefficient matching gives, by the same rule that yields the printed
 * {{W (b^0)^2}}).
 *
 * F~_j is not printed (the paper cites it).  Reading: the same coefficient
 * matching, with the jumps of the entropy variables written in those of
 * (rho, beta, u_k, b_k),
 *   [[V_1]] = [[rho]]/rho^ln + alpha_0 [[beta]],
 *   [[beta u_k]] = {{beta}}[[u_k]] + {{u_k}}[[beta]],
 *   [[-beta W]] = -{{beta}}[[W]] - {{W}}[[beta]],  [[W]] = sum_k {{u_k}}[[u_k]]/{{W}},
 *   [[beta b_k]] = {{beta}}[[b_k]] + {{b_k}}[[beta]],
 * and the right-hand side expanded exactly by the product rule
 * [[ab]] = {{a}}[[b]] + {{b}}[[a]] with c = W b^0 = u.b:
 *   [[rho u_j]]            = {{rho}}[[u_j]] + {{u_j}}[[rho]],
 *   [[beta u_j (b^k)^2]]   = {{u_j (b^k)^2}}[[beta]]
 *                            + {{beta}}({{u_j}} 2{{b_k}}[[b_k]] + {{(b^k)^2}}[[u_j]]),
 *   [[beta u_j (b^0)^2]]   = {{u_j (b^0)^2}}[[beta]] + {{beta}}[[v_j (W (b^0)^2)]],
 *   [[v_j X]] = {{v_j}}[[X]] + {{X}}[[v_j]], [[v_j]] = ([[u_j]] - {{v_j}}[[W]])/{{W}},
 *   [[W (b^0)^2]]          = (2{{c}}[[c]] - {{W (b^0)^2}}[[W]])/{{W}},
 *   [[Phi]] = [[beta b^0]] = {{b^0}}[[beta]] + {{beta}}([[c]] - {{b^0}}[[W]])/{{W}},
 *   [[c]] = sum_k {{u_k}}[[b_k]] + {{b_k}}[[u_k]].
 * Matching the coefficients of [[rho]], [[u_k]], [[b_k]], [[beta]] gives
 *   F~_D = rho^ln r_rho,  F~_{B_k} = r_{b_k}/{{beta}},
 *   F~_E = {{W}} (alpha_0 F~_D + sum_k {{u_k}} r_{u_k}/{{beta}}
 *                 + sum_k {{b_k}} F~_{B_k} - r_beta) / Lambda,
 *   F~_{m_k} = r_{u_k}/{{beta}} + {{u_k}} F~_E/{{W}},
 *   Lambda = {{W}}^2 - sum_k {{u_k}}^2,  alpha_0 = 1 + 1/((Gamma-1) beta^ln),
 * with r_q the coefficient of [[q]] in [[psi_j]] - {{B_j}}[[Phi]].  At
 * b = 0 both reduce to the RHD fluxes.                                      */
typedef struct {
    double rho, beta, W, u[3], v[3], b[3], b0, B[3];
} mhd_aux;

static void mhd_aux_of(const double *w, mhd_aux *a)
{
    const double *v = w + 1, *B = w + 5;
    double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    double W = 1.0 / sqrt(1.0 - v2);
    double vB = v[0] * B[0] + v[1] * B[1] + v[2] * B[2];
    a->rho = w[0];
    a->beta = w[0] / w[4];
    a->W = W;
    a->b0 = W * vB;
    for (int k = 0; k < 3; ++k) {
        a->v[k] = v[k];
        a->u[k] = W * v[k];
        a->b[k] = B[k] / W + a->b0 * v[k];
        a->B[k] = B[k];
    }
}

void oref_mhd_ec_flux(double gamma, const double *wl, const double *wr,
                      double *Ut, double *Ft)
{
    mhd_aux L, R;
    mhd_aux_of(wl, &L);
    mhd_aux_of(wr, &R);
#define MEAN(e_l, e_r) (0.5 * ((e_l) + (e_r)))
    double rho_ln = oref_logmean(L.rho, R.rho);
    double beta_ln = oref_logmean(L.beta, R.beta);
    double rho_m = MEAN(L.rho, R.rho);
    double beta_m = MEAN(L.beta, R.beta);
    double W_m = MEAN(L.W, R.W);
    double u_m[3], b_m[3], bsq_m[3], Wbsq_m[3];
    for (int k = 0; k < 3; ++k) {
        u_m[k] = MEAN(L.u[k], R.u[k]);
        b_m[k] = MEAN(L.b[k], R.b[k]);
        bsq_m[k] = MEAN(L.b[k] * L.b[k], R.b[k] * R.b[k]);
        Wbsq_m[k] = MEAN(L.W * L.b[k] * L.b[k], R.W * R.b[k] * R.b[k]);
    }
    double c_m = MEAN(L.W * L.b0, R.W * R.b0);                 /* {{W b^0}}     */
    double Wb0sq_m = MEAN(L.W * L.b0 * L.b0, R.W * R.b0 * R.b0); /* {{W (b^0)^2}} */
    double b0_m = MEAN(L.b0, R.b0);
    double usq = u_m[0] * u_m[0] + u_m[1] * u_m[1] + u_m[2] * u_m[2];
    double Lam = W_m * W_m - usq;
    double alpha0 = 1.0 + 1.0 / (gamma - 1.0) / beta_ln;

    /* U~ in the paper's notation */
    {
        double alpha1 = rho_m + 0.5 * beta_m * (bsq_m[0] + bsq_m[1] + bsq_m[2])
                      + 0.5 * beta_m * Wb0sq_m / W_m;
        double Dcal = beta_m * Lam / W_m;
        double U1 = rho_ln * W_m;
        double UB[3], Rk[3];
        for (int k = 0; k < 3; ++k) UB[k] = (W_m * W_m * b_m[k] - c_m * u_m[k]) / W_m;
        double R1 = -alpha0 * U1 - 0.5 * Wb0sq_m;
        for (int k = 0; k < 3; ++k) R1 += 0.5 * Wbsq_m[k] - b_m[k] * UB[k];
        for (int k = 0; k < 3; ++k) Rk[k] = (alpha1 * u_m[k] - beta_m * c_m * b_m[k]) / W_m;
        double U5 = (u_m[0] * Rk[0] + u_m[1] * Rk[1] + u_m[2] * Rk[2] - beta_m * R1) / Dcal;
        Ut[0] = U1;
        for (int k = 0; k < 3; ++k) Ut[1 + k] = u_m[k] * U5 / W_m + Rk[k] / beta_m;
        Ut[4] = U5;
        for (int k = 0; k < 3; ++k) Ut[5 + k] = UB[k];
    }

    /* F~_j, j = 1..3 */
    for (int j = 0; j < 3; ++j) {
        double *F = Ft + 8 * j;
        double ujbsq_m = 0.0;
        for (int k = 0; k < 3; ++k)
            ujbsq_m += MEAN(L.u[j] * L.b[k] * L.b[k], R.u[j] * R.b[k] * R.b[k]);
        double ujb0sq_m = MEAN(L.u[j] * L.b0 * L.b0, R.u[j] * R.b0 * R.b0);
        double vj_m = MEAN(L.v[j], R.v[j]);
        double Bj_m = MEAN(L.B[j], R.B[j]);
        double r_rho = u_m[j], r_beta = 0.0, r_u[3] = {0.0, 0.0, 0.0}, r_b[3];
        double cW = 0.0;   /* coefficient of [[W]] */
        double cc = 0.0;   /* coefficient of [[c]] */
        /* [[rho u_j]] */
        r_u[j] += rho_m;
        /* (1/2) sum_k [[beta u_j (b^k)^2]] */
        r_beta += 0.5 * ujbsq_m;
        r_u[j] += 0.5 * beta_m * (bsq_m[0] + bsq_m[1] + bsq_m[2]);
        for (int k = 0; k < 3; ++k) r_b[k] = beta_m * u_m[j] * b_m[k];
        /* -(1/2) [[beta u_j (b^0)^2]] */
        r_beta -= 0.5 * ujb0sq_m;
        cc -= beta_m * vj_m * c_m / W_m;
        cW += 0.5 * beta_m * vj_m * Wb0sq_m / W_m;
        r_u[j] -= 0.5 * beta_m * Wb0sq_m / W_m;
        cW += 0.5 * beta_m * Wb0sq_m * vj_m / W_m;
        /* -{{B_j}} [[Phi]] */
        r_beta -= Bj_m * b0_m;
        cc -= Bj_m * beta_m / W_m;
        cW += Bj_m * beta_m * b0_m / W_m;
        /* distribute [[W]] and [[c]] */
        for (int k = 0; k < 3; ++k) {
            r_u[k] += cW * u_m[k] / W_m + cc * b_m[k];
            r_b[k] += cc * u_m[k];
        }
        F[0] = rho_ln * r_rho;
        for (int k = 0; k < 3; ++k) F[5 + k] = r_b[k] / beta_m;
        double acc = alpha0 * F[0] - r_beta;
        for (int k = 0; k < 3; ++k) acc += u_m[k] * r_u[k] / beta_m + b_m[k] * F[5 + k];
        F[4] = W_m * acc / Lam;
        for (int k = 0; k < 3; ++k) F[1 + k] = r_u[k] / beta_m + u_m[k] * F[4] / W_m;
    }
#undef MEAN
}

/* ------------------------------------------------------------------------ */
/* Sec. 4: scaled eigenvectors R of the symmetrized x_1-flux Jacobian with
 * dU/dV = R R^T, at a primitive state w already rotated so that the interface
 * normal is e_1 (the paper cites their formulas).
 *
 * Reading, a construction that is exact up to rounding and deterministic:
 *  1. Jacobians by the complex step (exact to rounding): JU = dU/dw,
 *     JV = dV/dw, JF = dF_1/dw, and the Godunov-Powell column: the source
 *     -Phi'(V)^T dB_1/dx contributes Phi'(V)^T dB_1 to the quasi-linear
 *     flux differential, so dF~ = JF dw + Phi' dw_{B_1}.
 *  2. Two bilinear forms on primitive perturbations: <a, b> = (JU a).(JV b)
 *     (symmetric positive definite: it is (JV a)^T dU/dV (JV b)), and
 *     k(a, b) = (JV a).(dF~ b) (symmetric: the symmetrized Jacobian).  A wave
 *     of speed lam is a perturbation with k(., a) = lam <., a>; its column of
 *     R is JU a with <a, a> = 1, so the columns satisfy R R^T = dU/dV.
 *  3. Two waves of speed v_1 are known in closed form: the entropy wave
 *     a_rho = e_rho, and the divergence wave a_div with dB = e_1 - v_1 v
 *     (no other component).  Both are orthogonal in <.,.>.
 *  4. The other six waves (fast, Alfven, slow, each +-) span the <.,.>
 *     complement of those two: y_a = e_a minus its projections on a_rho and
 *     a_div for a = v_1, v_2, v_3, p, B_2, B_3.  With G = <y_a, y_b> = L L^T
 *     (Cholesky) and K = k(y_a, y_b), the symmetric C = L^{-1} K L^{-T} is
 *     diagonalized by cyclic Jacobi rotations (row order, until the squared
 *     off-diagonal falls below 1e-30 of the squared diagonal, at most 50
 *     sweeps).
 *  5. Degenerate speeds (B_t = 0, B_n = 0 and near them) leave the basis of
 *     an eigenspace to rounding, and the WENO reconstruction and the sign
 *     switch Y do depend on that basis.  So the sorted speeds are grouped in
 *     clusters of consecutive gaps below OREF_MHD_CLUSTER_TOL, and each
 *     cluster gets a canonical basis: Gram-Schmidt, in index order, of the
 *     coordinate vectors e_1..e_6 of the C-space projected onto the
 *     cluster's span, taking a projected vector when its remaining squared
 *     norm is at least 1/8 (for a k-dimensional span the squared norms of
 *     the six projections sum to k, so k of them are always taken).  This
 *     depends only on the span, so it is reproducible, and it is continuous
 *     in the span away from the 1/8 threshold: a choice by largest norm
 *     would switch on the exact ties that symmetric states (B along n, gas
 *     at rest) create, and the dissipation with it.
 *  6. Column order: a_rho, a_div, then the six in ascending speed.  (Order and
 *     sign of the columns do not change the dissipation.)
 * lam[8] gets the speeds, R[8*8] row-major (row = component, column = wave).*/
#define OREF_MHD_CLUSTER_TOL 1.0e-5

static void mhd_UFV_c(double gamma, const cplx *w, cplx *U, cplx *F, cplx *V)
{
    cplx rho = w[0], p = w[4];
    const cplx *v = w + 1, *B = w + 5;
    cplx v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    cplx W2 = 1.0 / (1.0 - v2);
    cplx W = csqrt(W2);
    cplx vB = v[0] * B[0] + v[1] * B[1] + v[2] * B[2];
    cplx B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    cplx bb = B2 / W2 + vB * vB;
    cplx rhoh = rho + gamma / (gamma - 1.0) * p;
    cplx pt = p + 0.5 * bb;
    U[0] = rho * W;
    for (int k = 0; k < 3; ++k) U[1 + k] = (rhoh * W2 + B2) * v[k] - vB * B[k];
    U[4] = rhoh * W2 - pt + B2;
    for (int k = 0; k < 3; ++k) U[5 + k] = B[k];
    F[0] = U[0] * v[0];
    for (int k = 0; k < 3; ++k)
        F[1 + k] = U[1 + k] * v[0] - B[0] * (B[k] / W2 + vB * v[k]) + (k == 0 ? pt : 0.0);
    F[4] = U[1];
    for (int k = 0; k < 3; ++k) F[5 + k] = v[0] * B[k] - B[0] * v[k];
    cplx s = clog(p) - gamma * clog(rho);
    cplx beta = rho / p;
    V[0] = (gamma - s) / (gamma - 1.0) + beta;
    for (int k = 0; k < 3; ++k) V[1 + k] = beta * W * v[k];
    V[4] = -beta * W;
    for (int k = 0; k < 3; ++k) V[5 + k] = beta * (B[k] + W2 * v[k] * vB) / W;
}

/* JU, JV, JF as [8][8] row-major (row = output, column = primitive). */
static void mhd_jacobians(double gamma, const double *w, double *JU, double *JV, double *JF)
{
    const double h = 1.0e-30;
    for (int c = 0; c < 8; ++c) {
        cplx wc[8], U[8], F[8], V[8];
        for (int a = 0; a < 8; ++a) wc[a] = w[a];
        wc[c] += h * I;
        mhd_UFV_c(gamma, wc, U, F, V);
        for (int r = 0; r < 8; ++r) {
            JU[r * 8 + c] = cimag(U[r]) / h;
            JV[r * 8 + c] = cimag(V[r]) / h;
            JF[r * 8 + c] = cimag(F[r]) / h;
        }
    }
}

static void matvec8(const double *A, const double *x, double *y)
{
    for (int r = 0; r < 8; ++r) {
        double acc = 0.0;
        for (int c = 0; c < 8; ++c) acc += A[r * 8 + c] * x[c];
        y[r] = acc;
    }
}

static double dot8(const double *a, const double *b)
{
    double acc = 0.0;
    for (int r = 0; r < 8; ++r) acc += a[r] * b[r];
    return acc;
}

void oref_mhd_eigen(double gamma, const double *w, double *lam, double *R)
{
    double JU[64], JV[64], JF[64], Pp[8];
    mhd_jacobians(gamma, w, JU, JV, JF);
    oref_mhd_phiprime(w, Pp);
    const double *v = w + 1;

    /* images of a perturbation a: JU a, JV a and the symmetrized JF a + Phi' a_5 */
    double a_rho[8] = {1, 0, 0, 0, 0, 0, 0, 0};
    double a_div[8] = {0, 0, 0, 0, 0, 1.0 - v[0] * v[0], -v[0] * v[1], -v[0] * v[2]};
    double Ur[8], Vr[8], Ud[8], Vd[8];
    matvec8(JU, a_rho, Ur);
    matvec8(JV, a_rho, Vr);
    matvec8(JU, a_div, Ud);
    matvec8(JV, a_div, Vd);
    double n_rho = dot8(Ur, Vr), n_div = dot8(Ud, Vd);

    /* complement basis y_a and their images */
    static const int comp[6] = {1, 2, 3, 4, 6, 7};
    double y[6][8], Uy[6][8], Vy[6][8], Fy[6][8];
    for (int a = 0; a < 6; ++a) {
        double e[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        e[comp[a]] = 1.0;
        double Ue[8];
        matvec8(JU, e, Ue);
        double c_rho = dot8(Ue, Vr) / n_rho;    /* <e, a_rho>/<a_rho, a_rho> */
        double c_div = dot8(Ue, Vd) / n_div;
        for (int r = 0; r < 8; ++r) y[a][r] = e[r] - c_rho * a_rho[r] - c_div * a_div[r];
        matvec8(JU, y[a], Uy[a]);
        matvec8(JV, y[a], Vy[a]);
        matvec8(JF, y[a], Fy[a]);
        for (int r = 0; r < 8; ++r) Fy[a][r] += Pp[r] * y[a][5];
    }
    double Gm[6][6], Km[6][6];
    for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) {
            Gm[a][b] = dot8(Uy[a], Vy[b]);
            Km[a][b] = dot8(Vy[a], Fy[b]);
        }
    /* symmetrize the rounding of the two forms */
    for (int a = 0; a < 6; ++a)
        for (int b = 0; b < a; ++b) {
            double g = 0.5 * (Gm[a][b] + Gm[b][a]), k = 0.5 * (Km[a][b] + Km[b][a]);
            Gm[a][b] = Gm[b][a] = g;
            Km[a][b] = Km[b][a] = k;
        }
    /* Cholesky G = L L^T */
    double Lc[6][6];
    memset(Lc, 0, sizeof Lc);
    for (int j = 0; j < 6; ++j) {
        double d = Gm[j][j];
        for (int k = 0; k < j; ++k) d -= Lc[j][k] * Lc[j][k];
        Lc[j][j] = sqrt(d);
        for (int i = j + 1; i < 6; ++i) {
            double s = Gm[i][j];
            for (int k = 0; k < j; ++k) s -= Lc[i][k] * Lc[j][k];
            Lc[i][j] = s / Lc[j][j];
        }
    }
    /* C = L^{-1} K L^{-T}: X = L^{-1} K (forward substitution on columns),
     * then C = L^{-1} X^T. */
    double X[6][6], C[6][6];
    for (int c = 0; c < 6; ++c)
        for (int i = 0; i < 6; ++i) {
            double s = Km[i][c];
            for (int k = 0; k < i; ++k) s -= Lc[i][k] * X[k][c];
            X[i][c] = s / Lc[i][i];
        }
    for (int c = 0; c < 6; ++c)
        for (int i = 0; i < 6; ++i) {
            double s = X[c][i];
            for (int k = 0; k < i; ++k) s -= Lc[i][k] * C[k][c];
            C[i][c] = s / Lc[i][i];
        }
    for (int a = 0; a < 6; ++a)
        for (int b = 0; b < a; ++b) C[a][b] = C[b][a] = 0.5 * (C[a][b] + C[b][a]);
    /* cyclic Jacobi */
    double Q[6][6];
    for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) Q[a][b] = (a == b) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 50; ++sweep) {
        double off = 0.0, dg = 0.0;
        for (int a = 0; a < 6; ++a) {
            dg += C[a][a] * C[a][a];
            for (int b = a + 1; b < 6; ++b) off += C[a][b] * C[a][b];
        }
        if (off <= 1.0e-30 * dg) break;
        for (int p = 0; p < 5; ++p)
            for (int q = p + 1; q < 6; ++q) {
                if (C[p][q] == 0.0) continue;
                double theta = (C[q][q] - C[p][p]) / (2.0 * C[p][q]);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < 6; ++k) {          /* columns p, q */
                    double ckp = C[k][p], ckq = C[k][q];
                    C[k][p] = cs * ckp - sn * ckq;
                    C[k][q] = sn * ckp + cs * ckq;
                }
                for (int k = 0; k < 6; ++k) {          /* rows p, q */
                    double cpk = C[p][k], cqk = C[q][k];
                    C[p][k] = cs * cpk - sn * cqk;
                    C[q][k] = sn * cpk + cs * cqk;
                }
                for (int k = 0; k < 6; ++k) {
                    double qkp = Q[k][p], qkq = Q[k][q];
                    Q[k][p] = cs * qkp - sn * qkq;
                    Q[k][q] = sn * qkp + cs * qkq;
                }
            }
    }
    /* sort ascending (stable selection on the diagonal) */
    int ord[6] = {0, 1, 2, 3, 4, 5};
    for (int a = 0; a < 6; ++a)
        for (int b = a + 1; b < 6; ++b)
            if (C[ord[b]][ord[b]] < C[ord[a]][ord[a]]) {
                int t = ord[a];
                ord[a] = ord[b];
                ord[b] = t;
            }
    double mu[6], E6[6][6];   /* E6[.][m]: C-space eigenvector m */
    for (int m = 0; m < 6; ++m) {
        mu[m] = C[ord[m]][ord[m]];
        for (int r = 0; r < 6; ++r) E6[r][m] = Q[r][ord[m]];
    }
    /* canonical bases of clusters */
    int start = 0;
    while (start < 6) {
        int end = start + 1;
        while (end < 6 && mu[end] - mu[end - 1] < OREF_MHD_CLUSTER_TOL) ++end;
        int k = end - start;
        if (k > 1) {
            /* z_i = coordinates of P e_i in the cluster basis = row i of E6 */
            double z[6][6], basis[6][6];
            for (int i = 0; i < 6; ++i)
                for (int c = 0; c < k; ++c) z[i][c] = E6[i][start + c];
            int nt = 0;
            for (int i = 0; i < 6 && nt < k; ++i) {
                double n2 = 0.0;
                for (int c = 0; c < k; ++c) n2 += z[i][c] * z[i][c];
                if (!(n2 >= 0.125)) continue;
                double nrm = sqrt(n2);
                for (int c = 0; c < k; ++c) basis[nt][c] = z[i][c] / nrm;
                for (int ii = i + 1; ii < 6; ++ii) {
                    double pr = 0.0;
                    for (int c = 0; c < k; ++c) pr += z[ii][c] * basis[nt][c];
                    for (int c = 0; c < k; ++c) z[ii][c] -= pr * basis[nt][c];
                }
                ++nt;
            }
            if (nt < k) {   /* only for non-finite input: keep the Jacobi basis */
                start = end;
                continue;
            }
            double newE[6][6];
            for (int t = 0; t < k; ++t)
                for (int r = 0; r < 6; ++r) {
                    double acc = 0.0;
                    for (int c = 0; c < k; ++c) acc += E6[r][start + c] * basis[t][c];
                    newE[r][t] = acc;
                }
            for (int t = 0; t < k; ++t)
                for (int r = 0; r < 6; ++r) E6[r][start + t] = newE[r][t];
        }
        start = end;
    }
    /* columns: a_rho, a_div, then the six */
    double srho = 1.0 / sqrt(n_rho), sdiv = 1.0 / sqrt(n_div);
    for (int r = 0; r < 8; ++r) {
        R[r * 8 + 0] = Ur[r] * srho;
        R[r * 8 + 1] = Ud[r] * sdiv;
    }
    lam[0] = v[0];
    lam[1] = v[0];
    for (int m = 0; m < 6; ++m) {
        /* coefficients in the y basis: s = L^{-T} e (back substitution) */
        double s[6];
        for (int i = 5; i >= 0; --i) {
            double acc = E6[i][m];
            for (int k = i + 1; k < 6; ++k) acc -= Lc[k][i] * s[k];
            s[i] = acc / Lc[i][i];
        }
        for (int r = 0; r < 8; ++r) {
            double acc = 0.0;
            for (int a = 0; a < 6; ++a) acc += s[a] * Uy[a][r];
            R[r * 8 + 2 + m] = acc;
        }
        lam[2 + m] = mu[m];
    }
}
