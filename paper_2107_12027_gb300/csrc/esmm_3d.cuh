// esmm_3d.cuh -- device arithmetic of the 3D RMHD path shared by the forward
// kernels (esmm_3d.cu, esmm_3d_iface.cu) and the adjoint (esmm_3d_adjoint.cu):
// the padded 3D grid, boundary mapping, nested conservative metrics (eq.
// SCLCoeff), the Sec. 4 rotation with its tangential alignment, the node loads
// and the interface-flux kernel template.
#pragma once

#include "esmm_mhd.cuh"

namespace esmm {
namespace d3 {

struct Geom3 {
    int n[3];
    int pd[3];
    long long P, N;
    int bc[3];
    double per[3];
};

// node data fields (FP64, padded grid)
enum {
    F_RHO = 0, F_P, F_BETA, F_U0, F_U1, F_U2, F_W, F_LNR, F_LNB, F_B0, F_B1, F_B2,
    F_M = 12,      // 9 spatial metrics M[k][j] = J d xi_k / d x_j at F_M + 3k + j
    F_MT = 21,     // 3 temporal metrics J d xi_k / dt
    NQ3 = 24
};
constexpr int NF3 = 10;     // per direction and padded node: F[8], metric flux, B~
constexpr int NR3 = 9;      // reduction slots: grad, tau, radius[3], mesh Courant[3], Laplacian

__host__ __device__ __forceinline__ long long pidx3(const Geom3 &g, int i, int j, int k)
{
    return ((long long)(k + GH) * g.pd[1] + (j + GH)) * g.pd[0] + (i + GH);
}

__device__ __forceinline__ long long data_src3(const Geom3 &g, int i, int j, int k)
{
    int ii = g.bc[0] == 0 ? wrapi(i, g.n[0]) : clampi(i, 0, g.n[0] - 1);
    int jj = g.bc[1] == 0 ? wrapi(j, g.n[1]) : clampi(j, 0, g.n[1] - 1);
    int kk = g.bc[2] == 0 ? wrapi(k, g.n[2]) : clampi(k, 0, g.n[2] - 1);
    return ((long long)kk * g.n[1] + jj) * g.n[0] + ii;
}

// Boundary-mapped mesh value, one direction at a time (2, then 1, then 0):
// periodic wrap plus the period for the coordinate along that direction
// (shift = 1), or linear extrapolation of the two nodes next to the boundary.
__device__ __forceinline__ double mesh_d0(const Geom3 &g, const double *a, int comp, int i, int j, int k, int shift)
{
    const double *row = a + (long long)comp * g.N + ((long long)k * g.n[1] + j) * g.n[0];
    int n = g.n[0];
    if (g.bc[0] == 0) {
        double s = (shift && comp == 0) ? floordivi(i, n) * g.per[0] : 0.0;
        return row[wrapi(i, n)] + s;
    }
    if (i < 0) { double v0 = row[0], v1 = row[1]; return v0 + (double)(-i) * (v0 - v1); }
    if (i > n - 1) { double v0 = row[n - 1], v1 = row[n - 2]; return v0 + (double)(i - (n - 1)) * (v0 - v1); }
    return row[i];
}

__device__ __forceinline__ double mesh_d1(const Geom3 &g, const double *a, int comp, int i, int j, int k, int shift)
{
    int n = g.n[1];
    if (g.bc[1] == 0) {
        double s = (shift && comp == 1) ? floordivi(j, n) * g.per[1] : 0.0;
        return mesh_d0(g, a, comp, i, wrapi(j, n), k, shift) + s;
    }
    if (j >= 0 && j <= n - 1) return mesh_d0(g, a, comp, i, j, k, shift);
    int b0 = j < 0 ? 0 : n - 1, b1 = j < 0 ? 1 : n - 2;
    double v0 = mesh_d0(g, a, comp, i, b0, k, shift), v1 = mesh_d0(g, a, comp, i, b1, k, shift);
    double off = j < 0 ? (double)(-j) : (double)(j - (n - 1));
    return v0 + off * (v0 - v1);
}

__device__ __forceinline__ double mesh3_at(const Geom3 &g, const double *a, int comp, int i, int j, int k, int shift)
{
    int n = g.n[2];
    if (g.bc[2] == 0) {
        double s = (shift && comp == 2) ? floordivi(k, n) * g.per[2] : 0.0;
        return mesh_d1(g, a, comp, i, j, wrapi(k, n), shift) + s;
    }
    if (k >= 0 && k <= n - 1) return mesh_d1(g, a, comp, i, j, k, shift);
    int b0 = k < 0 ? 0 : n - 1, b1 = k < 0 ? 1 : n - 2;
    double v0 = mesh_d1(g, a, comp, i, j, b0, shift), v1 = mesh_d1(g, a, comp, i, j, b1, shift);
    double off = k < 0 ? (double)(-k) : (double)(k - (n - 1));
    return v0 + off * (v0 - v1);
}

template <int P> __device__ __forceinline__ constexpr double alpha3(int n)
{
    return P == 1 ? 1.0 : (P == 2 ? (n == 1 ? 4.0 / 3.0 : -1.0 / 6.0) : (n == 1 ? 1.5 : (n == 2 ? -0.3 : 1.0 / 30.0)));
}

__device__ __forceinline__ void step3(int i, int j, int k, int d, int s, int &a, int &b, int &c)
{
    a = i + (d == 0) * s;
    b = j + (d == 1) * s;
    c = k + (d == 2) * s;
}

// delta_d[x_comp] at (i, j, k)
template <int P>
__device__ __forceinline__ double delta_x3(const Geom3 &g, const double *x, int comp, int i, int j, int k, int d)
{
    double s = 0.0;
#pragma unroll
    for (int n = 1; n <= P; ++n) {
        int a0, a1, a2, b0, b1, b2;
        step3(i, j, k, d, n, a0, a1, a2);
        step3(i, j, k, d, -n, b0, b1, b2);
        s += 0.5 * alpha3<P>(n) * (mesh3_at(g, x, comp, a0, a1, a2, 1) - mesh3_at(g, x, comp, b0, b1, b2, 1));
    }
    return s;
}

// Sec. 4 rotation for the unit normal n (rows n, t1, t2; theta = 0 when the
// x_1-x_2 part of n is below 1e-12), then turned about n so that t1 lies
// along the tangential B of the state w (along the tangential v when
// |B_t| <= 1e-10 max(1, |B|); unchanged when also |v_t| <= 1e-10, c = 1;
// absolute thresholds, so that rounding noise in a field or velocity that
// vanishes does not orient the frame).
__device__ __forceinline__ void frame3(const double n[3], double T[3][3])
{
    double r = sqrt(n[0] * n[0] + n[1] * n[1]);
    bool pole = r <= 1.0e-12;
    double ct = pole ? 1.0 : n[0] / r, st = pole ? 0.0 : n[1] / r;
    double cp = r, sp = n[2];
    T[0][0] = cp * ct; T[0][1] = cp * st; T[0][2] = sp;
    T[1][0] = -st;     T[1][1] = ct;      T[1][2] = 0.0;
    T[2][0] = -sp * ct; T[2][1] = -sp * st; T[2][2] = cp;
}

__device__ __forceinline__ void align3(double T[3][3], const double w[8])
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
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        double a1 = T[1][q], a2 = T[2][q];
        T[1][q] = c * a1 + s * a2;
        T[2][q] = -s * a1 + c * a2;
    }
}

__device__ __forceinline__ void rot3(const double T[3][3], const double *a, double *r)
{
    r[0] = a[0];
    r[4] = a[4];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        r[1 + q] = T[q][0] * a[1] + T[q][1] * a[2] + T[q][2] * a[3];
        r[5 + q] = T[q][0] * a[5] + T[q][1] * a[6] + T[q][2] * a[7];
    }
}

__device__ __forceinline__ void unrot3(const double T[3][3], const double *r, double *a)
{
    a[0] = r[0];
    a[4] = r[4];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        a[1 + q] = T[0][q] * r[1] + T[1][q] * r[2] + T[2][q] * r[3];
        a[5 + q] = T[0][q] * r[5] + T[1][q] * r[6] + T[2][q] * r[7];
    }
}

__device__ __forceinline__ NodeM load3(const double *__restrict__ q, long long P, long long c)
{
    NodeM v;
    v.rho = q[F_RHO * P + c];
    v.beta = q[F_BETA * P + c];
    v.lnr = q[F_LNR * P + c];
    v.lnb = q[F_LNB * P + c];
    v.r = v.rho;
    v.b = v.beta;
    v.W = q[F_W * P + c];
    v.u[0] = q[F_U0 * P + c];
    v.u[1] = q[F_U1 * P + c];
    v.u[2] = q[F_U2 * P + c];
    v.B[0] = q[F_B0 * P + c];
    v.B[1] = q[F_B1 * P + c];
    v.B[2] = q[F_B2 * P + c];
    return v;
}

__device__ __forceinline__ void node_V3(const double *__restrict__ q, long long P, long long c, double c1g, double ig,
                                        double V[8])
{
    double beta = q[F_BETA * P + c], W = q[F_W * P + c];
    double u0 = q[F_U0 * P + c], u1 = q[F_U1 * P + c], u2 = q[F_U2 * P + c];
    double B0 = q[F_B0 * P + c], B1 = q[F_B1 * P + c], B2 = q[F_B2 * P + c];
    double b0 = u0 * B0 + u1 * B1 + u2 * B2;
    double bW = beta / W;
    V[0] = c1g + q[F_LNR * P + c] + ig * q[F_LNB * P + c] + beta;
    V[1] = beta * u0;
    V[2] = beta * u1;
    V[3] = beta * u2;
    V[4] = -beta * W;
    V[5] = bW * (B0 + b0 * u0);
    V[6] = bW * (B1 + b0 * u1);
    V[7] = bW * (B2 + b0 * u2);
}

// ES interface flux (eq. ESFlux_HO) between node L (index -1 .. n_d - 1 along
// the sweep) and L + 1, every line of the other two indices.
template <int P, int WW>
__global__ void __launch_bounds__(128) k3_iface(Geom3 g, Phys ph, const double *__restrict__ q,
                                                double *__restrict__ iflux, int dir)
{
    const int nd = g.n[dir];
    const int oa = dir == 0 ? 1 : 0, ob = dir == 2 ? 1 : 2;
    const long long count = (long long)(nd + 1) * g.n[oa] * g.n[ob];
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= count) return;
    int c3[3];
    c3[dir] = (int)(idx % (nd + 1)) - 1;
    c3[oa] = (int)((idx / (nd + 1)) % g.n[oa]);
    c3[ob] = (int)(idx / ((long long)(nd + 1) * g.n[oa]));
    const long long c0 = pidx3(g, c3[0], c3[1], c3[2]);
    const long long sd = dir == 0 ? 1 : (dir == 1 ? (long long)g.pd[0] : (long long)g.pd[0] * g.pd[1]);
    const double *Mt = q + (F_MT + dir) * g.P;
    const double *Md = q + (F_M + 3 * dir) * g.P;   // M[dir][0..2] at Md + q' P
    const double gm1inv = 1.0 / (ph.gamma - 1.0);
    double F[8] = {0, 0, 0, 0, 0, 0, 0, 0}, Ft = 0.0, Bt = 0.0;
#pragma unroll
    for (int n = 1; n <= P; ++n) {
        double Fs[8] = {0, 0, 0, 0, 0, 0, 0, 0}, Fts = 0.0, Bts = 0.0;
#pragma unroll
        for (int s = 0; s < n; ++s) {
            const long long cl = c0 - s * sd, cr = cl + n * sd;
            NodeM l = load3(q, g.P, cl), r = load3(q, g.P, cr);
            double mm[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) mm[a] = 0.5 * (Md[a * g.P + cl] + Md[a * g.P + cr]);
            double out[8];
            ec_pair_mhd<3>(l, r, gm1inv, ph.ln_thr, 0.5 * (Mt[cl] + Mt[cr]), mm, out);
#pragma unroll
            for (int a = 0; a < 8; ++a) Fs[a] += out[a];
            Fts += 0.5 * (Mt[cl] + Mt[cr]);
#pragma unroll
            for (int a = 0; a < 3; ++a) Bts += 0.5 * mm[a] * (l.B[a] + r.B[a]);
        }
        const double an = ph.alpha[n - 1];
#pragma unroll
        for (int a = 0; a < 8; ++a) F[a] += an * Fs[a];
        Ft += an * Fts;
        Bt += an * Bts;
    }
    if (WW > 0) {
        constexpr int NS = WW + 1, OFF = (WW - 1) / 2;
        const long long c1 = c0 + sd;
        double nv[3], nn[3], T[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a) nv[a] = 0.5 * (Md[a * g.P + c0] + Md[a * g.P + c1]);
        const double jt = 0.5 * (Mt[c0] + Mt[c1]);
        const double Lk = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) nn[a] = nv[a] / Lk;
        frame3(nn, T);
        double wm[8], wrot[8];
        {
            double rho, irho;
            logmean<double, double>(q[F_RHO * g.P + c0], q[F_RHO * g.P + c1], q[F_LNR * g.P + c0],
                                    q[F_LNR * g.P + c1], ph.ln_thr, rho, irho);
            double um[3], W2 = 1.0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                um[a] = 0.5 * (q[(F_U0 + a) * g.P + c0] + q[(F_U0 + a) * g.P + c1]);
                W2 += um[a] * um[a];
            }
            double W = sqrt(W2);
            wm[0] = rho;
#pragma unroll
            for (int a = 0; a < 3; ++a) wm[1 + a] = um[a] / W;
            wm[4] = (q[F_RHO * g.P + c0] + q[F_RHO * g.P + c1]) / (q[F_BETA * g.P + c0] + q[F_BETA * g.P + c1]);
#pragma unroll
            for (int a = 0; a < 3; ++a) wm[5 + a] = 0.5 * (q[(F_B0 + a) * g.P + c0] + q[(F_B0 + a) * g.P + c1]);
        }
        align3(T, wm);
        rot3(T, wm, wrot);
        double lam[8], R[8][8];
        eigen_mhd(ph.gamma, wrot, lam, R, true);
        double lhat = 0.0;
#pragma unroll
        for (int m = 0; m < 8; ++m) lhat = fmax(lhat, fabs(jt + Lk * lam[m]));
        const double ig = gm1inv, c1g = ph.gamma * gm1inv;
        double Vt[NS][8], scale[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) scale[m] = 0.0;
        for (int kk = 0; kk < NS; ++kk) {
            double V[8], TV[8];
            node_V3(q, g.P, c0 + (kk - OFF) * sd, c1g, ig, V);
            rot3(T, V, TV);
            for (int m = 0; m < 8; ++m) {
                double acc = 0.0;
                for (int a = 0; a < 8; ++a) {
                    double t = R[a][m] * TV[a];
                    acc += t;
                    if (kk == OFF || kk == OFF + 1) scale[m] += fabs(t);
                }
                Vt[kk][m] = acc;
            }
        }
        double z[8];
        for (int m = 0; m < 8; ++m) {
            double vminus, vplus;
            if (WW == 5)
                weno5_lr<double>(Vt[0][m], Vt[1][m], Vt[2][m], Vt[3][m], Vt[4][m], Vt[5][m], ph.eps, vminus, vplus);
            else
                weno3_lr<double>(Vt[0][m], Vt[1][m], Vt[2][m], Vt[3][m], ph.eps, vminus, vplus);
            double jw = vplus - vminus;
            double jump = Vt[OFF + 1][m] - Vt[OFF][m];
            int sj = fabs(jump) <= ph.sign_tol * scale[m] ? 0 : sgn_d(jump);
            z[m] = (sgn_d(jw) == sj) ? jw : 0.0;
        }
        double d[8], dr[8];
        for (int a = 0; a < 8; ++a) {
            double acc = 0.0;
            for (int m = 0; m < 8; ++m) acc += R[a][m] * z[m];
            d[a] = acc;
        }
        unrot3(T, d, dr);
        const double hl = 0.5 * lhat;
#pragma unroll
        for (int a = 0; a < 8; ++a) F[a] -= hl * dr[a];
    }
    double *out = iflux + (long long)(dir * NF3) * g.P + c0;
#pragma unroll
    for (int a = 0; a < 8; ++a) out[a * g.P] = F[a];
    out[8 * g.P] = Ft;
    out[9 * g.P] = Bt;
}

// launch of the interface kernel of one direction (esmm_3d_iface.cu)
void launch3_iface(const Geom3 &g, const Phys &ph, int p, int w, const double *q, double *iflux, int dir,
                   unsigned nb, cudaStream_t st);

// adjoint kernels (esmm_3d_adjoint.cu): node-quantity adjoints lamq[11][P]
// from the pair and interface passes, then the node pass into lam [8][N]
void launch3_pairs_vjp(const Geom3 &g, const Phys &ph, const double *q, const double *mu, double *lamq, int dir,
                       cudaStream_t st);
void launch3_iface_vjp(const Geom3 &g, const Phys &ph, const double *q, const double *mu, double *lamq, int dir,
                       cudaStream_t st);
void launch3_node_vjp(const Geom3 &g, double gam, const double *q, const double *lamq, const double *iflux,
                      const double *mu, const double *J, double *lam, cudaStream_t st);
void launch3_prim_grad(const Geom3 &g, double gam, const double *cons, const double *J, const double *lam,
                       double *out, int *status, cudaStream_t st);
void launch3_lincomb(long long n, double a, const double *x, double b, const double *y, double *out,
                     cudaStream_t st);

}  // namespace d3
}  // namespace esmm
