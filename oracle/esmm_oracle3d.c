/*
 * esmm_oracle3d.c -- the 3D RMHD grid parts of the plain FP64 CPU oracle
 * (Duan & Tang, arXiv 2107.12027): nested conservative metrics, the
 * semi-discrete ES scheme with the Godunov-Powell source on a moving
 * curvilinear mesh, the CFL step, the 3D mesh redistribution and SSP-RK3.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load the oracle; it shares no code with the
 * CUDA library.  The pointwise RMHD parts are those of esmm_oracle_mhd.c.
 *
 * Conventions: nodes (i, j, k), i fastest; N = nx ny nz;
 * index = (k ny + j) nx + i; prim[8][N], cons[8][N] = J U, J[N], x[3][N],
 * xdot[3][N]; computational coordinates are node indices.
 */
#include "esmm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define G3 3   /* ghost layers of the padded node data */
#define NV3 8
#define SIGN_TOL3 1.0e-10

static int wrap3(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }
static int fdiv3(int a, int n) { return (a >= 0) ? a / n : -((-a + n - 1) / n); }
static int clamp3(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }

static int ext(const oref3_cfg *c, int d) { return d == 0 ? c->nx : (d == 1 ? c->ny : c->nz); }

/* data ghosts: periodic wrap or zero-gradient copy, per direction */
static long data_index3(const oref3_cfg *c, int i, int j, int k)
{
    int ii = c->bc[0] == OREF_PERIODIC ? wrap3(i, c->nx) : clamp3(i, 0, c->nx - 1);
    int jj = c->bc[1] == OREF_PERIODIC ? wrap3(j, c->ny) : clamp3(j, 0, c->ny - 1);
    int kk = c->bc[2] == OREF_PERIODIC ? wrap3(k, c->nz) : clamp3(k, 0, c->nz - 1);
    return ((long)kk * c->ny + jj) * c->nx + ii;
}

/* mesh ghosts: periodic wrap plus the period (shift = 1, coordinates only)
 * or linear extrapolation of the two nodes next to the boundary, applied
 * direction by direction (d = 2, then 1, then 0). */
static double mesh3_dir(const oref3_cfg *c, const double *a, int comp, int idx[3], int d, int shift)
{
    if (d < 0) {
        long N = (long)c->nx * c->ny * c->nz;
        return a[comp * N + ((long)idx[2] * c->ny + idx[1]) * c->nx + idx[0]];
    }
    int n = ext(c, d), m = idx[d];
    if (c->bc[d] == OREF_PERIODIC) {
        double s = (shift && comp == d) ? fdiv3(m, n) * c->period[d] : 0.0;
        idx[d] = wrap3(m, n);
        double v = mesh3_dir(c, a, comp, idx, d - 1, shift) + s;
        idx[d] = m;
        return v;
    }
    if (m >= 0 && m <= n - 1) return mesh3_dir(c, a, comp, idx, d - 1, shift);
    int b0 = m < 0 ? 0 : n - 1, b1 = m < 0 ? 1 : n - 2;
    idx[d] = b0;
    double v0 = mesh3_dir(c, a, comp, idx, d - 1, shift);
    idx[d] = b1;
    double v1 = mesh3_dir(c, a, comp, idx, d - 1, shift);
    idx[d] = m;
    double off = m < 0 ? (double)(-m) : (double)(m - (n - 1));
    return v0 + off * (v0 - v1);
}

static double mesh3(const oref3_cfg *c, const double *a, int comp, int i, int j, int k, int shift)
{
    int idx[3] = {i, j, k};
    return mesh3_dir(c, a, comp, idx, 2, shift);
}

/* ------------------------------------------------------------------------ */
/* eq. SCLCoeff (the 3D CMM): with (k, k1, k2) and (j, j1, j2) cyclic,
 *   (J xi_k/x_j) = delta_{k2}[ delta_{k1}[x_{j1}] x_{j2} ]
 *                - delta_{k1}[ delta_{k2}[x_{j1}] x_{j2} ],
 * delta_d[a]_i = 1/2 sum_n alpha_{p,n} (a_{i,d,+n} - a_{i,d,-n}).          */
static void shifted(int i, int j, int k, int d, int s, int *o)
{
    o[0] = i + (d == 0) * s;
    o[1] = j + (d == 1) * s;
    o[2] = k + (d == 2) * s;
}

static double delta_x(const oref3_cfg *c, const double *x, int comp, int i, int j, int k, int d)
{
    double alpha[3];
    oref_alpha(c->p, alpha);
    double s = 0.0;
    for (int n = 1; n <= c->p; ++n) {
        int a[3], b[3];
        shifted(i, j, k, d, n, a);
        shifted(i, j, k, d, -n, b);
        s += 0.5 * alpha[n - 1] * (mesh3(c, x, comp, a[0], a[1], a[2], 1) - mesh3(c, x, comp, b[0], b[1], b[2], 1));
    }
    return s;
}

/* delta_{d_out}[ delta_{d_in}[x_{ja}] x_{jb} ] */
static double nested(const oref3_cfg *c, const double *x, int d_out, int d_in, int ja, int jb, int i, int j, int k)
{
    double alpha[3];
    oref_alpha(c->p, alpha);
    double s = 0.0;
    for (int n = 1; n <= c->p; ++n) {
        int a[3], b[3];
        shifted(i, j, k, d_out, n, a);
        shifted(i, j, k, d_out, -n, b);
        double fa = delta_x(c, x, ja, a[0], a[1], a[2], d_in) * mesh3(c, x, jb, a[0], a[1], a[2], 1);
        double fb = delta_x(c, x, ja, b[0], b[1], b[2], d_in) * mesh3(c, x, jb, b[0], b[1], b[2], 1);
        s += 0.5 * alpha[n - 1] * (fa - fb);
    }
    return s;
}

/* M[k][j] = J d xi_k/d x_j at node (i, j, k) */
static void node_metrics3(const oref3_cfg *c, const double *x, int i, int j, int k, double M[3][3])
{
    for (int kk = 0; kk < 3; ++kk) {
        int k1 = (kk + 1) % 3, k2 = (kk + 2) % 3;
        for (int jj = 0; jj < 3; ++jj) {
            int j1 = (jj + 1) % 3, j2 = (jj + 2) % 3;
            M[kk][jj] = nested(c, x, k2, k1, j1, j2, i, j, k) - nested(c, x, k1, k2, j1, j2, i, j, k);
        }
    }
}

void oref3_metrics(const oref3_cfg *c, const double *x, double *m, double *J0)
{
    long N = (long)c->nx * c->ny * c->nz;
    #pragma omp parallel for
    for (int k = 0; k < c->nz; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                long id = ((long)k * c->ny + j) * c->nx + i;
                double M[3][3];
                node_metrics3(c, x, i, j, k, M);
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) m[(a * 3 + b) * N + id] = M[a][b];
                if (J0) {
                    /* Reading: J0 = det(delta_k[x_j]), as in 2D. */
                    double D[3][3];
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b) D[a][b] = delta_x(c, x, b, i, j, k, a);
                    J0[id] = D[0][0] * (D[1][1] * D[2][2] - D[1][2] * D[2][1])
                           - D[0][1] * (D[1][0] * D[2][2] - D[1][2] * D[2][0])
                           + D[0][2] * (D[1][0] * D[2][1] - D[1][1] * D[2][0]);
                }
            }
}

/* ------------------------------------------------------------------------ */
typedef struct {
    const oref3_cfg *c;
    int px, py, pz;
    long S;
    double *prim;   /* [8][S] */
    double *M;      /* [9][S] */
    double *Mt;     /* [3][S] */
} pad3;

static long pidx3(const pad3 *P, int i, int j, int k)
{
    return ((long)(k + G3) * P->py + (j + G3)) * P->px + (i + G3);
}

static int node_prim3(const oref3_cfg *c, const double *cons, const double *J, long id, double *w)
{
    long N = (long)c->nx * c->ny * c->nz;
    double U[8];
    for (int a = 0; a < 8; ++a) U[a] = cons[a * N + id] / J[id];
    return oref_mhd_cons2prim(c->gamma, U, w, NULL);
}

static int build_pad3(const oref3_cfg *c, const double *cons, const double *J, const double *x,
                      const double *xdot, pad3 *P)
{
    long N = (long)c->nx * c->ny * c->nz;
    P->c = c;
    P->px = c->nx + 2 * G3;
    P->py = c->ny + 2 * G3;
    P->pz = c->nz + 2 * G3;
    P->S = (long)P->px * P->py * P->pz;
    P->prim = (double *)malloc(sizeof(double) * 8 * P->S);
    P->M = (double *)malloc(sizeof(double) * 9 * P->S);
    P->Mt = (double *)malloc(sizeof(double) * 3 * P->S);
    double *w = (double *)malloc(sizeof(double) * 8 * N);
    int status = 0;
    #pragma omp parallel for reduction(min : status)
    for (long id = 0; id < N; ++id) {
        double wi[8];
        if (node_prim3(c, cons, J, id, wi) != 0) status = -1;
        for (int a = 0; a < 8; ++a) w[a * N + id] = wi[a];
    }
    #pragma omp parallel for
    for (int k = -G3; k < c->nz + G3; ++k)
        for (int j = -G3; j < c->ny + G3; ++j)
            for (int i = -G3; i < c->nx + G3; ++i) {
                long id = pidx3(P, i, j, k), src = data_index3(c, i, j, k);
                int in = (c->bc[0] == OREF_INFLOW && i < 0) || (c->bc[1] == OREF_INFLOW && j < 0) ||
                         (c->bc[2] == OREF_INFLOW && k < 0);
                for (int a = 0; a < 8; ++a) P->prim[a * P->S + id] = in ? c->inflow[a] : w[a * N + src];
                double M[3][3];
                node_metrics3(c, x, i, j, k, M);
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) P->M[(a * 3 + b) * P->S + id] = M[a][b];
                /* eq. VCLCoeff */
                double xd[3];
                for (int b = 0; b < 3; ++b) xd[b] = mesh3(c, xdot, b, i, j, k, 0);
                for (int a = 0; a < 3; ++a)
                    P->Mt[a * P->S + id] = -(xd[0] * M[a][0] + xd[1] * M[a][1] + xd[2] * M[a][2]);
            }
    free(w);
    return status;
}

static void free_pad3(pad3 *P)
{
    free(P->prim);
    free(P->M);
    free(P->Mt);
}

static void pget3(const pad3 *P, int i, int j, int k, double *w, double M[3][3], double Mt[3])
{
    long id = pidx3(P, i, j, k);
    if (w)
        for (int a = 0; a < 8; ++a) w[a] = P->prim[a * P->S + id];
    if (M)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) M[a][b] = P->M[(a * 3 + b) * P->S + id];
    if (Mt)
        for (int a = 0; a < 3; ++a) Mt[a] = P->Mt[a * P->S + id];
}

static int sgn3(double a) { return (a > 0.0) - (a < 0.0); }

/* Sec. 4 rotation T_0 for the unit normal n: rows
 *   (cos phi cos theta, cos phi sin theta, sin phi), (-sin theta, cos theta, 0),
 *   (-sin phi cos theta, -sin phi sin theta, cos phi),
 * theta = atan2(n_2, n_1) (reading: the angle of the metric vector; theta = 0
 * when n_1 = n_2 = 0), phi = atan2(n_3, sqrt(n_1^2 + n_2^2)).               */
static void frame3(const double n[3], double T[3][3])
{
    double r = sqrt(n[0] * n[0] + n[1] * n[1]);
    /* theta is 0/0 for a normal along x_3; below 1e-12 the x_1-x_2 part is
     * rounding noise of the metrics and theta = 0 is taken */
    int pole = r <= 1.0e-12;
    double ct = pole ? 1.0 : n[0] / r, st = pole ? 0.0 : n[1] / r;
    double cp = r, sp = n[2];
    T[0][0] = cp * ct; T[0][1] = cp * st; T[0][2] = sp;
    T[1][0] = -st;     T[1][1] = ct;      T[1][2] = 0.0;
    T[2][0] = -sp * ct; T[2][1] = -sp * st; T[2][2] = cp;
}

/* Reading: the tangential axes of T_0 are then turned about n so that the
 * first lies along the tangential magnetic field of the state w (along the
 * tangential velocity when |B_t| <= 1e-10 max(1, |B|); unchanged when also
 * |v_t| <= 1e-10, c = 1).  The thresholds are absolute so that a field or a
 * velocity that is zero up to rounding (a gas at rest, a symmetry plane) does
 * not orient the frame.
 * The paper's theta, phi fix them by the coordinate axes, and the
 * characteristic split of degenerate waves (and, at a normal along x_3,
 * rounding noise in theta) would then depend on the coordinates; aligned
 * with B_t the dissipation is invariant under rotations about n. */
static void align3(double T[3][3], const double *w)
{
    double b1 = T[1][0] * w[5] + T[1][1] * w[6] + T[1][2] * w[7];
    double b2 = T[2][0] * w[5] + T[2][1] * w[6] + T[2][2] * w[7];
    double B2 = w[5] * w[5] + w[6] * w[6] + w[7] * w[7];
    double t2 = b1 * b1 + b2 * b2;
    if (!(t2 > 1.0e-20 * (1.0 + B2))) {
        b1 = T[1][0] * w[1] + T[1][1] * w[2] + T[1][2] * w[3];
        b2 = T[2][0] * w[1] + T[2][1] * w[2] + T[2][2] * w[3];
        t2 = b1 * b1 + b2 * b2;
        if (!(t2 > 1.0e-20)) return;
    }
    double tn = sqrt(t2), c = b1 / tn, s = b2 / tn;
    for (int q = 0; q < 3; ++q) {
        double a1 = T[1][q], a2 = T[2][q];
        T[1][q] = c * a1 + s * a2;
        T[2][q] = -s * a1 + c * a2;
    }
}

static void rot3(const double T[3][3], const double *a, double *r)
{
    r[0] = a[0];
    r[4] = a[4];
    for (int q = 0; q < 3; ++q) {
        r[1 + q] = T[q][0] * a[1] + T[q][1] * a[2] + T[q][2] * a[3];
        r[5 + q] = T[q][0] * a[5] + T[q][1] * a[6] + T[q][2] * a[7];
    }
}

static void unrot3(const double T[3][3], const double *r, double *a)
{
    a[0] = r[0];
    a[4] = r[4];
    for (int q = 0; q < 3; ++q) {
        a[1 + q] = T[0][q] * r[1] + T[1][q] * r[2] + T[2][q] * r[3];
        a[5 + q] = T[0][q] * r[5] + T[1][q] * r[6] + T[2][q] * r[7];
    }
}

/* ES interface flux between node (i, j, k) and its neighbour in direction d
 * (eq. ESFlux_HO): F[8], the metric flux Ft and the magnetic flux Bt. */
static void iface3(const pad3 *P, int d, int i, int j, int k, double *F, double *Ft, double *Bt)
{
    const oref3_cfg *c = P->c;
    int di = d == 0, dj = d == 1, dk = d == 2;
    double alpha[3];
    oref_alpha(c->p, alpha);
    for (int a = 0; a < 8; ++a) F[a] = 0.0;
    *Ft = 0.0;
    *Bt = 0.0;
    /* eq. ECFlux_O2p, eq. BFlux_O2p, eq. MetricsFlux_O2p */
    for (int n = 1; n <= c->p; ++n) {
        double Fs[8] = {0, 0, 0, 0, 0, 0, 0, 0}, Fts = 0.0, Bts = 0.0;
        for (int s = 0; s < n; ++s) {
            double wl[8], wr[8], Ml[3][3], Mr[3][3], Mtl[3], Mtr[3];
            pget3(P, i - s * di, j - s * dj, k - s * dk, wl, Ml, Mtl);
            pget3(P, i + (n - s) * di, j + (n - s) * dj, k + (n - s) * dk, wr, Mr, Mtr);
            double Ut[8], Ftj[24];
            oref_mhd_ec_flux(c->gamma, wl, wr, Ut, Ftj);
            double mt = 0.5 * (Mtl[d] + Mtr[d]);
            double m[3];
            for (int q = 0; q < 3; ++q) m[q] = 0.5 * (Ml[d][q] + Mr[d][q]);
            for (int a = 0; a < 8; ++a)
                Fs[a] += mt * Ut[a] + m[0] * Ftj[a] + m[1] * Ftj[8 + a] + m[2] * Ftj[16 + a];
            Fts += 0.5 * (Mtl[d] + Mtr[d]);
            for (int q = 0; q < 3; ++q) Bts += 0.25 * (Ml[d][q] + Mr[d][q]) * (wl[5 + q] + wr[5 + q]);
        }
        for (int a = 0; a < 8; ++a) F[a] += alpha[n - 1] * Fs[a];
        *Ft += alpha[n - 1] * Fts;
        *Bt += alpha[n - 1] * Bts;
    }
    if (c->w == 0) return;

    double wL[8], wR[8], ML[3][3], MR[3][3], MtL[3], MtR[3];
    pget3(P, i, j, k, wL, ML, MtL);
    pget3(P, i + di, j + dj, k + dk, wR, MR, MtR);
    double nv[3], nn[3], T[3][3];
    for (int q = 0; q < 3; ++q) nv[q] = 0.5 * (ML[d][q] + MR[d][q]);
    double jt = 0.5 * (MtL[d] + MtR[d]);
    double Lk = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
    for (int q = 0; q < 3; ++q) nn[q] = nv[q] / Lk;
    frame3(nn, T);
    /* interface state: rho^ln, {{u}}, {{rho}}/{{beta}}, {{B}} */
    double wm[8], wrot[8];
    {
        double WL = 1.0 / sqrt(1.0 - (wL[1] * wL[1] + wL[2] * wL[2] + wL[3] * wL[3]));
        double WR = 1.0 / sqrt(1.0 - (wR[1] * wR[1] + wR[2] * wR[2] + wR[3] * wR[3]));
        double um[3], W2 = 1.0;
        for (int q = 0; q < 3; ++q) {
            um[q] = 0.5 * (WL * wL[1 + q] + WR * wR[1 + q]);
            W2 += um[q] * um[q];
        }
        double Wm = sqrt(W2);
        wm[0] = oref_logmean(wL[0], wR[0]);
        for (int q = 0; q < 3; ++q) wm[1 + q] = um[q] / Wm;
        wm[4] = (0.5 * (wL[0] + wR[0])) / (0.5 * (wL[0] / wL[4] + wR[0] / wR[4]));
        for (int q = 5; q < 8; ++q) wm[q] = 0.5 * (wL[q] + wR[q]);
    }
    align3(T, wm);
    rot3(T, wm, wrot);
    double lam[8], R[64];
    oref_mhd_eigen(c->gamma, wrot, lam, R);
    double lhat = 0.0;
    for (int m = 0; m < 8; ++m) {
        double a = fabs(jt + Lk * lam[m]);
        if (a > lhat) lhat = a;
    }
    int lo = (c->w == 5) ? -2 : -1, hi = (c->w == 5) ? 3 : 2;
    double Vt[6][8], scale[8];
    for (int m = 0; m < 8; ++m) scale[m] = 0.0;
    for (int q = lo; q <= hi; ++q) {
        double wq[8], V[8], TV[8];
        pget3(P, i + q * di, j + q * dj, k + q * dk, wq, NULL, NULL);
        oref_mhd_entropy_vars(c->gamma, wq, V);
        rot3(T, V, TV);
        for (int m = 0; m < 8; ++m) {
            double acc = 0.0;
            for (int a = 0; a < 8; ++a) {
                acc += R[a * 8 + m] * TV[a];
                if (q == 0 || q == 1) scale[m] += fabs(R[a * 8 + m] * TV[a]);
            }
            Vt[q - lo][m] = acc;
        }
    }
    double z[8];
    for (int m = 0; m < 8; ++m) {
        double sl[5], sr[5];
        for (int q = 0; q < c->w; ++q) {
            sl[q] = Vt[q][m];
            sr[q] = Vt[(hi - lo) - q][m];
        }
        double jw = oref_weno(c->w, c->weno_eps, sr) - oref_weno(c->w, c->weno_eps, sl);
        double jump = Vt[1 - lo][m] - Vt[0 - lo][m];
        int sj = fabs(jump) <= SIGN_TOL3 * scale[m] ? 0 : sgn3(jump);
        z[m] = (sgn3(jw) == sj) ? jw : 0.0;
    }
    double dd[8], dr[8];
    for (int a = 0; a < 8; ++a) {
        double acc = 0.0;
        for (int m = 0; m < 8; ++m) acc += R[a * 8 + m] * z[m];
        dd[a] = acc;
    }
    unrot3(T, dd, dr);
    for (int a = 0; a < 8; ++a) F[a] -= 0.5 * lhat * dr[a];
}

int oref3_rhs(const oref3_cfg *c, const double *cons, const double *J, const double *x,
              const double *xdot, double *dcons, double *dJ)
{
    long N = (long)c->nx * c->ny * c->nz;
    pad3 P;
    int status = build_pad3(c, cons, J, x, xdot, &P);
    for (long a = 0; a < 8 * N; ++a) dcons[a] = 0.0;
    for (long a = 0; a < N; ++a) dJ[a] = 0.0;
    /* eqs. RMHDSemiU_O2p_ES / RMHDSemiJ_O2p_ES with the Powell source */
    #pragma omp parallel for
    for (int k = 0; k < c->nz; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                long id = ((long)k * c->ny + j) * c->nx + i;
                double divB = 0.0;
                for (int d = 0; d < 3; ++d) {
                    double Fp[8], Fm[8], Ftp, Ftm, Btp, Btm;
                    iface3(&P, d, i, j, k, Fp, &Ftp, &Btp);
                    iface3(&P, d, i - (d == 0), j - (d == 1), k - (d == 2), Fm, &Ftm, &Btm);
                    for (int a = 0; a < 8; ++a) dcons[a * N + id] -= Fp[a] - Fm[a];
                    dJ[id] -= Ftp - Ftm;
                    divB += Btp - Btm;
                }
                double w[8], Pp[8];
                pget3(&P, i, j, k, w, NULL, NULL);
                oref_mhd_phiprime(w, Pp);
                for (int a = 0; a < 8; ++a) dcons[a * N + id] -= Pp[a] * divB;
            }
    free_pad3(&P);
    return status;
}

int oref3_init_state(const oref3_cfg *c, const double *prim, const double *x, double *cons, double *J)
{
    long N = (long)c->nx * c->ny * c->nz;
    double *m = (double *)malloc(sizeof(double) * 9 * N);
    oref3_metrics(c, x, m, J);
    free(m);
    for (long id = 0; id < N; ++id) {
        double w[8], U[8];
        for (int a = 0; a < 8; ++a) w[a] = prim[a * N + id];
        oref_mhd_prim2cons(c->gamma, w, U);
        for (int a = 0; a < 8; ++a) cons[a * N + id] = J[id] * U[a];
    }
    return 0;
}

int oref3_state_prim(const oref3_cfg *c, const double *cons, const double *J, double *prim)
{
    long N = (long)c->nx * c->ny * c->nz;
    int status = 0;
    for (long id = 0; id < N; ++id) {
        double w[8];
        if (node_prim3(c, cons, J, id, w) != 0) status = -1;
        for (int a = 0; a < 8; ++a) prim[a * N + id] = w[a];
    }
    return status;
}

/* eq. cfl with the static-mesh spectral radius (as in 2D) */
int oref3_cfl_dt(const oref3_cfg *c, const double *cons, const double *J, const double *x, double *dt)
{
    int status = 0;
    double rmax[3] = {0.0, 0.0, 0.0};
    #pragma omp parallel for reduction(min : status) reduction(max : rmax[:3])
    for (int k = 0; k < c->nz; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                long id = ((long)k * c->ny + j) * c->nx + i;
                double w[8], M[3][3];
                if (node_prim3(c, cons, J, id, w) != 0) status = -1;
                node_metrics3(c, x, i, j, k, M);
                for (int d = 0; d < 3; ++d) {
                    double Lk = sqrt(M[d][0] * M[d][0] + M[d][1] * M[d][1] + M[d][2] * M[d][2]);
                    double nn[3] = {M[d][0] / Lk, M[d][1] / Lk, M[d][2] / Lk}, T[3][3], wr[8], lam[8], R[64];
                    frame3(nn, T);
                    rot3(T, w, wr);
                    oref_mhd_eigen(c->gamma, wr, lam, R);
                    double a = 0.0;
                    for (int m = 0; m < 8; ++m)
                        if (fabs(lam[m]) > a) a = fabs(lam[m]);
                    double r = Lk * a / J[id];
                    if (r > rmax[d]) rmax[d] = r;
                }
            }
    *dt = c->cfl / (rmax[0] + rmax[1] + rmax[2]);
    return status;
}

/* Speed bounds of every node for eq. cfl (the 3D form of the 2D oracle's
 * speed_bounds): L_k lambda_min / J and L_k lambda_max / J per direction. */
static int speed_bounds3(const oref3_cfg *c, const double *cons, const double *J, const double *x,
                         double *bmin, double *bmax)
{
    long N = (long)c->nx * c->ny * c->nz;
    int status = 0;
    #pragma omp parallel for reduction(min : status)
    for (int k = 0; k < c->nz; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                long id = ((long)k * c->ny + j) * c->nx + i;
                double w[8], M[3][3];
                if (node_prim3(c, cons, J, id, w) != 0) status = -1;
                node_metrics3(c, x, i, j, k, M);
                for (int d = 0; d < 3; ++d) {
                    double Lk = sqrt(M[d][0] * M[d][0] + M[d][1] * M[d][1] + M[d][2] * M[d][2]);
                    double nn[3] = {M[d][0] / Lk, M[d][1] / Lk, M[d][2] / Lk}, T[3][3], wr[8], lam[8], R[64];
                    frame3(nn, T);
                    rot3(T, w, wr);
                    oref_mhd_eigen(c->gamma, wr, lam, R);
                    double lo = lam[0], hi = lam[0];
                    for (int m = 1; m < 8; ++m) {
                        if (lam[m] < lo) lo = lam[m];
                        if (lam[m] > hi) hi = lam[m];
                    }
                    bmin[d * N + id] = Lk * lo / J[id];
                    bmax[d * N + id] = Lk * hi / J[id];
                }
            }
    return status;
}

/* Sec. 5 in 3D: monitor, the 27-point low-pass filter with weights
 * (1/2)^{|j1|+|j2|+|j3|+3}, mu Jacobi sweeps with omega frozen, the movement
 * limiter over the three directions, xdot = Delta tau (x^[mu] - x^n)/dt.
 * Readings as in 2D (central |grad sigma| in index space, fixed outflow
 * boundary nodes, "(x_1)" read as x_k).                                     */
/* Sec. 5 monitor (and the Laplacian term of the 3D vortex example), before
 * the low-pass filter; the 3D form of oref_monitor. */
/* sigma at a node of the index space, ghosts included (see sigma_at of the
 * 2D oracle) */
static double sigma_at3(const oref3_cfg *c, const double *sig, double sig_in, int i, int j, int k)
{
    if ((c->bc[0] == OREF_INFLOW && i < 0) || (c->bc[1] == OREF_INFLOW && j < 0) ||
        (c->bc[2] == OREF_INFLOW && k < 0))
        return sig_in;
    return sig[data_index3(c, i, j, k)];
}

int oref3_monitor(const oref3_cfg *c, const double *cons, const double *J, double *om)
{
    long N = (long)c->nx * c->ny * c->nz;
    int status = 0;
    double *sig = (double *)malloc(sizeof(double) * N);
    double *lap = (double *)malloc(sizeof(double) * N);
    #pragma omp parallel for reduction(min : status)
    for (long id = 0; id < N; ++id) {
        double w[8];
        if (node_prim3(c, cons, J, id, w) != 0) status = -1;
        sig[id] = (c->monitor == OREF_MONITOR_LNRHO) ? log(w[0]) : w[0];
    }
    double sig_in = (c->monitor == OREF_MONITOR_LNRHO) ? log(c->inflow[0]) : c->inflow[0];
    double gmax = 0.0, lmax = 0.0;
    #pragma omp parallel for reduction(max : gmax, lmax)
    for (int k = 0; k < c->nz; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                long id = ((long)k * c->ny + j) * c->nx + i;
                double xp = sigma_at3(c, sig, sig_in, i + 1, j, k), xm = sigma_at3(c, sig, sig_in, i - 1, j, k);
                double yp = sigma_at3(c, sig, sig_in, i, j + 1, k), ym = sigma_at3(c, sig, sig_in, i, j - 1, k);
                double zp = sigma_at3(c, sig, sig_in, i, j, k + 1), zm = sigma_at3(c, sig, sig_in, i, j, k - 1);
                double gx = 0.5 * (xp - xm), gy = 0.5 * (yp - ym), gz = 0.5 * (zp - zm);
                double g = sqrt(gx * gx + gy * gy + gz * gz);
                double l = fabs(xp + xm + yp + ym + zp + zm - 6.0 * sig[id]);
                om[id] = g;
                lap[id] = l;
                if (g > gmax) gmax = g;
                if (l > lmax) lmax = l;
            }
    for (long id = 0; id < N; ++id) {
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
 * om_i <- sum_{j in {-1,0,1}^3} (1/2)^{|j1|+|j2|+|j3|+3} om_{i+j}, neighbours
 * through the boundary mapping of the data. */
void oref3_filter(const oref3_cfg *c, double *om, int n)
{
    long N = (long)c->nx * c->ny * c->nz;
    double *om2 = (double *)malloc(sizeof(double) * N);
    for (int f = 0; f < n; ++f) {
        #pragma omp parallel for
        for (int k = 0; k < c->nz; ++k)
            for (int j = 0; j < c->ny; ++j)
                for (int i = 0; i < c->nx; ++i) {
                    double acc = 0.0;
                    for (int cc = -1; cc <= 1; ++cc)
                        for (int b = -1; b <= 1; ++b)
                            for (int a = -1; a <= 1; ++a)
                                acc += ldexp(1.0, -(abs(a) + abs(b) + abs(cc) + 3)) *
                                       om[data_index3(c, i + a, j + b, k + cc)];
                    om2[((long)k * c->ny + j) * c->nx + i] = acc;
                }
        memcpy(om, om2, sizeof(double) * N);
    }
    free(om2);
}

/* mu sweeps of the Sec. 5 Jacobi iteration with the monitor om frozen, from
 * X^[0] = x (the three-direction form of the 2D sweep: each node solves
 * sum_k [(om_i + om_{i,k,+1})(X_{i,k,+1} - X_i) - (om_i + om_{i,k,-1})(X_i -
 * X_{i,k,-1})] = 0 with the neighbours of the previous sweep); nodes on a
 * non-periodic face stay fixed. */
void oref3_jacobi(const oref3_cfg *c, const double *om, const double *x, int mu, double *X)
{
    long N = (long)c->nx * c->ny * c->nz;
    double *Xn = (double *)malloc(sizeof(double) * 3 * N);
    memcpy(X, x, sizeof(double) * 3 * N);
    for (int nu = 0; nu < mu; ++nu) {
        #pragma omp parallel for
        for (int k = 0; k < c->nz; ++k)
            for (int j = 0; j < c->ny; ++j)
                for (int i = 0; i < c->nx; ++i) {
                    long id = ((long)k * c->ny + j) * c->nx + i;
                    int fixed = (c->bc[0] != OREF_PERIODIC && (i == 0 || i == c->nx - 1)) ||
                                (c->bc[1] != OREF_PERIODIC && (j == 0 || j == c->ny - 1)) ||
                                (c->bc[2] != OREF_PERIODIC && (k == 0 || k == c->nz - 1));
                    if (fixed) {
                        for (int comp = 0; comp < 3; ++comp) Xn[comp * N + id] = X[comp * N + id];
                        continue;
                    }
                    double wi = om[id];
                    double wp[3], wmn[3];
                    wp[0] = om[data_index3(c, i + 1, j, k)];
                    wmn[0] = om[data_index3(c, i - 1, j, k)];
                    wp[1] = om[data_index3(c, i, j + 1, k)];
                    wmn[1] = om[data_index3(c, i, j - 1, k)];
                    wp[2] = om[data_index3(c, i, j, k + 1)];
                    wmn[2] = om[data_index3(c, i, j, k - 1)];
                    double den = 0.0;
                    for (int d = 0; d < 3; ++d) den += 2.0 * wi + wp[d] + wmn[d];
                    for (int comp = 0; comp < 3; ++comp) {
                        double num = 0.0;
                        for (int d = 0; d < 3; ++d) {
                            int a[3], b[3];
                            shifted(i, j, k, d, 1, a);
                            shifted(i, j, k, d, -1, b);
                            num += (wi + wp[d]) * mesh3(c, X, comp, a[0], a[1], a[2], 1) +
                                   (wi + wmn[d]) * mesh3(c, X, comp, b[0], b[1], b[2], 1);
                        }
                        Xn[comp * N + id] = num / den;
                    }
                }
        memcpy(X, Xn, sizeof(double) * 3 * N);
    }
    free(Xn);
}

int oref3_mesh(const oref3_cfg *c, const double *cons, const double *J, const double *x, double dt,
               double *xdot, double *dtau, double *dt_out)
{
    long N = (long)c->nx * c->ny * c->nz;
    int status = 0;
    if (!c->move_mesh) {
        for (long a = 0; a < 3 * N; ++a) xdot[a] = 0.0;
        if (dtau) *dtau = 0.0;
        if (!(dt > 0.0)) status |= oref3_cfl_dt(c, cons, J, x, &dt);
        if (dt_out) *dt_out = dt;
        return status;
    }
    double *om = (double *)malloc(sizeof(double) * N);
    double *X = (double *)malloc(sizeof(double) * 3 * N);
    status |= oref3_monitor(c, cons, J, om);
    oref3_filter(c, om, c->n_filter);
    oref3_jacobi(c, om, x, c->mu, X);
    double tau = 1.0;
    #pragma omp parallel for reduction(min : tau)
    for (int k = 0; k < c->nz; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                long id = ((long)k * c->ny + j) * c->nx + i;
                for (int d = 0; d < 3; ++d) {
                    double dd = X[d * N + id] - x[d * N + id];
                    int a[3];
                    double b;
                    if (dd < 0.0) {
                        shifted(i, j, k, d, -1, a);
                        b = -(x[d * N + id] - mesh3(c, x, d, a[0], a[1], a[2], 1)) / (2.0 * dd);
                    } else if (dd > 0.0) {
                        shifted(i, j, k, d, 1, a);
                        b = (mesh3(c, x, d, a[0], a[1], a[2], 1) - x[d * N + id]) / (2.0 * dd);
                    } else {
                        continue;
                    }
                    if (b < tau) tau = b;
                }
            }
    if (tau < 0.0) tau = 0.0;
    /* the step of eq. cfl with the mesh velocity in the spectral radius
     * (oref_cfl_solve): the displacement terms and the speed bounds */
    double *am = (double *)malloc(sizeof(double) * 3 * N);
    double *bmin = (double *)malloc(sizeof(double) * 3 * N);
    double *bmax = (double *)malloc(sizeof(double) * 3 * N);
    #pragma omp parallel for
    for (int k = 0; k < c->nz; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                long id = ((long)k * c->ny + j) * c->nx + i;
                double M[3][3];
                node_metrics3(c, x, i, j, k, M);
                double dd[3] = {X[id] - x[id], X[N + id] - x[N + id], X[2 * N + id] - x[2 * N + id]};
                for (int d = 0; d < 3; ++d)
                    am[d * N + id] = (dd[0] * M[d][0] + dd[1] * M[d][1] + dd[2] * M[d][2]) / J[id];
            }
    status |= speed_bounds3(c, cons, J, x, bmin, bmax);
    dt = oref_cfl_solve(3, N, c->cfl, am, bmin, bmax, dt, &tau, NULL);
    free(am);
    free(bmin);
    free(bmax);
    for (long a = 0; a < 3 * N; ++a) xdot[a] = tau * (X[a] - x[a]) / dt;
    if (dtau) *dtau = tau;
    if (dt_out) *dt_out = dt;
    free(om);
    free(X);
    return status;
}

/* SSP-RK3 (as in 2D) on (cons, J) and the mesh with a given mesh velocity
 * xdot [3][N] and step dt, both held for the step: the map the adjoint
 * differentiates. */
int oref3_rk_step_given(const oref3_cfg *c, double *cons, double *J, double *x, const double *xdot, double dt)
{
    long N = (long)c->nx * c->ny * c->nz;
    int status = 0;
    double *c1 = (double *)malloc(sizeof(double) * 8 * N), *c2 = (double *)malloc(sizeof(double) * 8 * N);
    double *J1 = (double *)malloc(sizeof(double) * N), *J2 = (double *)malloc(sizeof(double) * N);
    double *x1 = (double *)malloc(sizeof(double) * 3 * N), *x2 = (double *)malloc(sizeof(double) * 3 * N);
    double *L = (double *)malloc(sizeof(double) * 8 * N), *LJ = (double *)malloc(sizeof(double) * N);
    status |= oref3_rhs(c, cons, J, x, xdot, L, LJ);
    for (long a = 0; a < 8 * N; ++a) c1[a] = cons[a] + dt * L[a];
    for (long a = 0; a < N; ++a) J1[a] = J[a] + dt * LJ[a];
    for (long a = 0; a < 3 * N; ++a) x1[a] = x[a] + dt * xdot[a];
    status |= oref3_rhs(c, c1, J1, x1, xdot, L, LJ);
    for (long a = 0; a < 8 * N; ++a) c2[a] = 0.75 * cons[a] + 0.25 * (c1[a] + dt * L[a]);
    for (long a = 0; a < N; ++a) J2[a] = 0.75 * J[a] + 0.25 * (J1[a] + dt * LJ[a]);
    for (long a = 0; a < 3 * N; ++a) x2[a] = 0.75 * x[a] + 0.25 * (x1[a] + dt * xdot[a]);
    status |= oref3_rhs(c, c2, J2, x2, xdot, L, LJ);
    for (long a = 0; a < 8 * N; ++a) cons[a] = cons[a] / 3.0 + 2.0 / 3.0 * (c2[a] + dt * L[a]);
    for (long a = 0; a < N; ++a) J[a] = J[a] / 3.0 + 2.0 / 3.0 * (J2[a] + dt * LJ[a]);
    for (long a = 0; a < 3 * N; ++a) x[a] = x[a] / 3.0 + 2.0 / 3.0 * (x2[a] + dt * xdot[a]);
    free(c1); free(c2); free(J1); free(J2); free(x1); free(x2); free(L); free(LJ);
    return status;
}

/* SSP-RK3 (as in 2D) on (cons, J) and the mesh with xdot held for the step */
int oref3_rk_step(const oref3_cfg *c, double *cons, double *J, double *x, double dt, double *dt_used)
{
    long N = (long)c->nx * c->ny * c->nz;
    int status = 0;
    double *xdot = (double *)calloc(3 * (size_t)N, sizeof(double));
    status |= oref3_mesh(c, cons, J, x, dt, xdot, NULL, &dt);
    status |= oref3_rk_step_given(c, cons, J, x, xdot, dt);
    if (dt_used) *dt_used = dt;
    free(xdot);
    return status;
}

/* totals: sum J eta, sum J D, sum J, and the semi-discrete entropy
 * production sum (V . dcons - phi dJ) when dcons, dJ are given */
int oref3_totals(const oref3_cfg *c, const double *cons, const double *J, const double *dcons,
                 const double *dJ, double *out)
{
    long N = (long)c->nx * c->ny * c->nz;
    int status = 0;
    double S = 0.0, mass = 0.0, vol = 0.0, prod = 0.0;
    for (long id = 0; id < N; ++id) {
        double w[8];
        if (node_prim3(c, cons, J, id, w) != 0) status = -1;
        double phi, psi[3], Phi;
        oref_mhd_potentials(w, &phi, psi, &Phi);
        S += J[id] * oref_mhd_entropy(c->gamma, w);
        mass += cons[id];
        vol += J[id];
        if (dcons && dJ) {
            double V[8];
            oref_mhd_entropy_vars(c->gamma, w, V);
            double vd = 0.0;
            for (int a = 0; a < 8; ++a) vd += V[a] * dcons[a * N + id];
            prod += vd - phi * dJ[id];
        }
    }
    out[0] = S;
    out[1] = mass;
    out[2] = vol;
    out[3] = prod;
    return status;
}
