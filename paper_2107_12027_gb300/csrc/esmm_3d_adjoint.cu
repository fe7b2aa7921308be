// esmm_3d_adjoint.cu -- vector-Jacobian products of the 3D RMHD right-hand
// side (the 3D form of esmm_mhd_adjoint.cu; the step adjoint around it is in
// esmm_3d.cu).
//
// Same map and conventions as in 2D: mesh velocity and step held at their
// recorded values, Y and the lambda^ maximum frozen at their forward
// selection.  Three sweep directions; the metric vector of an interface has
// three components, and the rotation T of Sec. 4 is turned about the normal
// to the tangential B of the interface state (or its tangential v), so the
// dissipation also depends on the state through that angle phi:
//   dT/dphi takes the tangential rows (t1, t2) to (t2, -t1),
//   phi = atan2(t2.B, t1.B) with (t1, t2) the rows before the turn,
// and the adjoint adds d(objective)/d(phi) d(phi)/d(interface state).
#include "esmm_3d.cuh"

namespace esmm {
namespace d3 {

namespace {

enum { A_RHO = 0, A_BETA, A_LNR, A_LNB, A_W, A_U0, A_U1, A_U2, A_B0, A_B1, A_B2, NQN };

__device__ __forceinline__ bool inside3(const Geom3 &g, const int c[3])
{
    return c[0] >= 0 && c[0] < g.n[0] && c[1] >= 0 && c[1] < g.n[1] && c[2] >= 0 && c[2] < g.n[2];
}

__device__ __forceinline__ long long nid3(const Geom3 &g, const int c[3])
{
    return ((long long)c[2] * g.n[1] + c[1]) * g.n[0] + c[0];
}

// mu_i . Phi'(w_i) at an interior node; 0 outside
__device__ double mu_phi3(const Geom3 &g, const double *__restrict__ q, const double *__restrict__ mu, const int c[3])
{
    if (!inside3(g, c)) return 0.0;
    const long long p = pidx3(g, c[0], c[1], c[2]), id = nid3(g, c);
    const double iW = 1.0 / q[F_W * g.P + p];
    double w[8] = {0.0, q[F_U0 * g.P + p] * iW, q[F_U1 * g.P + p] * iW, q[F_U2 * g.P + p] * iW, 0.0,
                   q[F_B0 * g.P + p], q[F_B1 * g.P + p], q[F_B2 * g.P + p]};
    double Pp[8];
    mhd_phiprime(w, Pp);
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a) s += mu[a * g.N + id] * Pp[a];
    return s;
}

// adjoints of the interface between node c and its neighbour along dir
__device__ void lambda_face3(const Geom3 &g, const double *__restrict__ q, const double *__restrict__ mu,
                             const int c[3], int dir, double lf[8], double &lb)
{
    int c1[3] = {c[0], c[1], c[2]};
    c1[dir] += 1;
    const bool a = inside3(g, c), b = inside3(g, c1);
    const long long ia = nid3(g, c), ib = nid3(g, c1);
#pragma unroll
    for (int k = 0; k < 8; ++k) lf[k] = (b ? mu[k * g.N + ib] : 0.0) - (a ? mu[k * g.N + ia] : 0.0);
    lb = mu_phi3(g, q, mu, c1) - mu_phi3(g, q, mu, c);
}

__device__ __forceinline__ NodeMT<dual> load3_dual(const double *__restrict__ q, long long P, long long c)
{
    NodeMT<dual> v;
    v.rho = dual(q[F_RHO * P + c]);
    v.beta = dual(q[F_BETA * P + c]);
    v.lnr = dual(q[F_LNR * P + c]);
    v.lnb = dual(q[F_LNB * P + c]);
    v.r = v.rho;
    v.b = v.beta;
    v.W = dual(q[F_W * P + c]);
    for (int a = 0; a < 3; ++a) {
        v.u[a] = dual(q[(F_U0 + a) * P + c]);
        v.B[a] = dual(q[(F_B0 + a) * P + c]);
    }
    return v;
}

__device__ __forceinline__ void seed3(NodeMT<dual> &v, int k)
{
    switch (k) {
    case A_RHO: v.rho.d = 1.0; v.r.d = 1.0; break;
    case A_BETA: v.beta.d = 1.0; v.b.d = 1.0; break;
    case A_LNR: v.lnr.d = 1.0; break;
    case A_LNB: v.lnb.d = 1.0; break;
    case A_W: v.W.d = 1.0; break;
    case A_U0: case A_U1: case A_U2: v.u[k - A_U0].d = 1.0; break;
    default: v.B[k - A_B0].d = 1.0; break;
    }
}

__device__ __forceinline__ void addq(double *lamq, long long P, int k, long long c, double v)
{
    if (v != 0.0) atomicAdd(lamq + k * P + c, v);
}

__device__ __forceinline__ void sweep_index(const Geom3 &g, int dir, int nd, int ext, long long idx, int c3[3])
{
    const int oa = dir == 0 ? 1 : 0, ob = dir == 2 ? 1 : 2;
    c3[dir] = (int)(idx % (nd + ext)) - ext;
    c3[oa] = (int)((idx / (nd + ext)) % g.n[oa]);
    c3[ob] = (int)(idx / ((long long)(nd + ext) * g.n[oa]));
}

// Pairs (A, A + n), A in [-P, n_dir - 1] along dir: enter the interfaces
// A + s (s < n) with weight alpha_{p,n} (eq. ECFlux_O2p, eq. BFlux_O2p).
template <int P>
__global__ void __launch_bounds__(128) k3_pairs_vjp(Geom3 g, Phys ph, const double *__restrict__ q,
                                                    const double *__restrict__ mu, double *__restrict__ lamq, int dir)
{
    const int nd = g.n[dir];
    const int oa = dir == 0 ? 1 : 0, ob = dir == 2 ? 1 : 2;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)(nd + P) * g.n[oa] * g.n[ob]) return;
    int c3[3];
    sweep_index(g, dir, nd, P, idx, c3);
    const long long c0 = pidx3(g, c3[0], c3[1], c3[2]);
    const long long sd = dir == 0 ? 1 : (dir == 1 ? (long long)g.pd[0] : (long long)g.pd[0] * g.pd[1]);
    const double *Mt = q + (F_MT + dir) * g.P;
    const double *Md = q + (F_M + 3 * dir) * g.P;
    const dual gm1inv = dual(1.0 / (ph.gamma - 1.0));
    const int A = c3[dir];
    for (int n = 1; n <= P; ++n) {
        double lp[8] = {0, 0, 0, 0, 0, 0, 0, 0}, lbs = 0.0;
        for (int s = 0; s < n; ++s) {
            int cl[3] = {c3[0], c3[1], c3[2]};
            cl[dir] = A + s;
            if (cl[dir] < -1 || cl[dir] > nd - 1) continue;
            double lf[8], lb;
            lambda_face3(g, q, mu, cl, dir, lf, lb);
#pragma unroll
            for (int a = 0; a < 8; ++a) lp[a] += lf[a];
            lbs += lb;
        }
        const double an = ph.alpha[n - 1];
        bool any = lbs != 0.0;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            lp[a] *= an;
            any = any || lp[a] != 0.0;
        }
        lbs *= an;
        if (!any) continue;
        const long long cr = c0 + n * sd;
        double mmv[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) mmv[a] = 0.5 * (Md[a * g.P + c0] + Md[a * g.P + cr]);
        // B~ of the pair: 1/2 sum_a mm_a (B_a,l + B_a,r)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            addq(lamq, g.P, A_B0 + a, c0, lbs * 0.5 * mmv[a]);
            addq(lamq, g.P, A_B0 + a, cr, lbs * 0.5 * mmv[a]);
        }
        const dual mt = dual(0.5 * (Mt[c0] + Mt[cr]));
        const dual mm[3] = {dual(mmv[0]), dual(mmv[1]), dual(mmv[2])};
        for (int side = 0; side < 2; ++side)
            for (int k = 0; k < NQN; ++k) {
                NodeMT<dual> l = load3_dual(q, g.P, c0), r = load3_dual(q, g.P, cr);
                seed3(side ? r : l, k);
                dual out[8];
                ec_pair_mhd<3, dual>(l, r, gm1inv, ph.ln_thr, mt, mm, out);
                double gsum = 0.0;
#pragma unroll
                for (int a = 0; a < 8; ++a) gsum += lp[a] * out[a].d;
                addq(lamq, g.P, k, side ? cr : c0, gsum);
            }
    }
}

// rotation by the tangential angle: (r_2, r_3) -> (r_3, -r_2) for the vector
// parts 1..3 and 5..7 of an 8-vector in the rotated frame
__device__ __forceinline__ void dphi8(const double r[8], double d[8])
{
    d[0] = 0.0; d[1] = 0.0; d[2] = r[3]; d[3] = -r[2];
    d[4] = 0.0; d[5] = 0.0; d[6] = r[7]; d[7] = -r[6];
}

template <int WW>
__global__ void __launch_bounds__(128) k3_iface_vjp(Geom3 g, Phys ph, const double *__restrict__ q,
                                                    const double *__restrict__ mu, double *__restrict__ lamq, int dir)
{
    constexpr int NS = WW + 1, OFF = (WW - 1) / 2;
    const int nd = g.n[dir];
    const int oa = dir == 0 ? 1 : 0, ob = dir == 2 ? 1 : 2;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)(nd + 1) * g.n[oa] * g.n[ob]) return;
    int c3[3];
    sweep_index(g, dir, nd, 1, idx, c3);
    double lf[8], lbdummy;
    lambda_face3(g, q, mu, c3, dir, lf, lbdummy);
    bool any = false;
#pragma unroll
    for (int a = 0; a < 8; ++a) any = any || lf[a] != 0.0;
    if (!any) return;
    const long long c0 = pidx3(g, c3[0], c3[1], c3[2]);
    const long long sd = dir == 0 ? 1 : (dir == 1 ? (long long)g.pd[0] : (long long)g.pd[0] * g.pd[1]);
    const long long c1 = c0 + sd;
    const double *Mt = q + (F_MT + dir) * g.P;
    const double *Md = q + (F_M + 3 * dir) * g.P;
    double nv[3], nn[3], T0[3][3], T[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) nv[a] = 0.5 * (Md[a * g.P + c0] + Md[a * g.P + c1]);
    const double jt = 0.5 * (Mt[c0] + Mt[c1]);
    const double Lk = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) nn[a] = nv[a] / Lk;
    frame3(nn, T0);
    const double r0 = q[F_RHO * g.P + c0], r1 = q[F_RHO * g.P + c1];
    const double l0 = q[F_LNR * g.P + c0], l1 = q[F_LNR * g.P + c1];
    const double b0 = q[F_BETA * g.P + c0], b1 = q[F_BETA * g.P + c1];
    double um[3], wm[8], wrot[8];
    {
        double rho, irho;
        logmean<double, double>(r0, r1, l0, l1, ph.ln_thr, rho, irho);
        double W2 = 1.0;
        for (int a = 0; a < 3; ++a) {
            um[a] = 0.5 * (q[(F_U0 + a) * g.P + c0] + q[(F_U0 + a) * g.P + c1]);
            W2 += um[a] * um[a];
        }
        const double W = sqrt(W2);
        wm[0] = rho;
        for (int a = 0; a < 3; ++a) wm[1 + a] = um[a] / W;
        wm[4] = (r0 + r1) / (b0 + b1);
        for (int a = 0; a < 3; ++a) wm[5 + a] = 0.5 * (q[(F_B0 + a) * g.P + c0] + q[(F_B0 + a) * g.P + c1]);
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) T[a][b] = T0[a][b];
    align3(T, wm);
    // which quantity turned the frame (as align3 decides): 1 = B, 2 = v, 0 = none
    int mode = 0, fo = 5;
    double tb1, tb2, tt2;
    {
        const double B2 = wm[5] * wm[5] + wm[6] * wm[6] + wm[7] * wm[7];
        tb1 = T0[1][0] * wm[5] + T0[1][1] * wm[6] + T0[1][2] * wm[7];
        tb2 = T0[2][0] * wm[5] + T0[2][1] * wm[6] + T0[2][2] * wm[7];
        tt2 = tb1 * tb1 + tb2 * tb2;
        if (tt2 > 1.0e-20 * (1.0 + B2)) mode = 1;
        else {
            fo = 1;
            tb1 = T0[1][0] * wm[1] + T0[1][1] * wm[2] + T0[1][2] * wm[3];
            tb2 = T0[2][0] * wm[1] + T0[2][1] * wm[2] + T0[2][2] * wm[3];
            tt2 = tb1 * tb1 + tb2 * tb2;
            if (tt2 > 1.0e-20) mode = 2;
        }
    }
    rot3(T, wm, wrot);
    double lam[8], R[8][8];
    eigen_mhd<double>(ph.gamma, wrot, lam, R, true);
    double lhat = 0.0;
    int msel = 0;
    for (int m = 0; m < 8; ++m) {
        const double v = fabs(jt + Lk * lam[m]);
        if (v > lhat) { lhat = v; msel = m; }
    }
    const double sg = (jt + Lk * lam[msel]) >= 0.0 ? 1.0 : -1.0;
    const double ig = 1.0 / (ph.gamma - 1.0), c1g = ph.gamma * ig;
    double TV[NS][8], Vt[NS][8], scale[8];
    for (int m = 0; m < 8; ++m) scale[m] = 0.0;
    for (int k = 0; k < NS; ++k) {
        double V[8];
        node_V3(q, g.P, c0 + (k - OFF) * sd, c1g, ig, V);
        rot3(T, V, TV[k]);
        for (int m = 0; m < 8; ++m) {
            double acc = 0.0;
            for (int a = 0; a < 8; ++a) {
                const double t = R[a][m] * TV[k][a];
                acc += t;
                if (k == OFF || k == OFF + 1) scale[m] += fabs(t);
            }
            Vt[k][m] = acc;
        }
    }
    double z[8];
    bool ym[8];
    for (int m = 0; m < 8; ++m) {
        double vminus, vplus;
        if (WW == 5)
            weno5_lr<double>(Vt[0][m], Vt[1][m], Vt[2][m], Vt[3][m], Vt[4][m], Vt[5][m], ph.eps, vminus, vplus);
        else
            weno3_lr<double>(Vt[0][m], Vt[1][m], Vt[2][m], Vt[3][m], ph.eps, vminus, vplus);
        const double jw = vplus - vminus;
        const double jump = Vt[OFF + 1][m] - Vt[OFF][m];
        const int sj = fabs(jump) <= ph.sign_tol * scale[m] ? 0 : sgn_d(jump);
        ym[m] = sgn_d(jw) == sj;
        z[m] = ym[m] ? jw : 0.0;
    }
    // reverse: objective contribution -hl lrot . (R z), lrot = rot3(T, lambda_F)
    double lrot[8];
    rot3(T, lf, lrot);
    const double hl = 0.5 * lhat;
    double zeta = 0.0, qm[8], Rz[8];
    for (int b = 0; b < 8; ++b) {
        double a = 0.0;
        for (int m = 0; m < 8; ++m) a += R[b][m] * z[m];
        Rz[b] = a;
    }
    for (int m = 0; m < 8; ++m) {
        double a = 0.0;
        for (int b = 0; b < 8; ++b) a += R[b][m] * lrot[b];
        qm[m] = -hl * a;
        zeta += a * z[m];
    }
    double lVt[NS][8];
    const dual epsd = dual(ph.eps);
    for (int k = 0; k < NS; ++k) {
        dual s[NS];
        for (int m = 0; m < 8; ++m) {
            for (int kk = 0; kk < NS; ++kk) s[kk] = dual(Vt[kk][m], kk == k ? 1.0 : 0.0);
            dual vminus, vplus;
            if (WW == 5)
                weno5_lr<dual>(s[0], s[1], s[2], s[3], s[4], s[5], epsd, vminus, vplus);
            else
                weno3_lr<dual>(s[0], s[1], s[2], s[3], epsd, vminus, vplus);
            lVt[k][m] = ym[m] ? qm[m] * (vplus.d - vminus.d) : 0.0;
        }
    }
    // stencil nodes
    for (int k = 0; k < NS; ++k) {
        double lT[8], lV[8];
        for (int b = 0; b < 8; ++b) {
            double a = 0.0;
            for (int m = 0; m < 8; ++m) a += R[b][m] * lVt[k][m];
            lT[b] = a;
        }
        unrot3(T, lT, lV);
        const long long ck = c0 + (k - OFF) * sd;
        const double beta = q[F_BETA * g.P + ck], W = q[F_W * g.P + ck];
        const double u[3] = {q[F_U0 * g.P + ck], q[F_U1 * g.P + ck], q[F_U2 * g.P + ck]};
        const double B[3] = {q[F_B0 * g.P + ck], q[F_B1 * g.P + ck], q[F_B2 * g.P + ck]};
        const double bb0 = u[0] * B[0] + u[1] * B[1] + u[2] * B[2];
        const double bW = beta / W;
        double lbeta = lV[0] - lV[4] * W, lW = -lV[4] * beta;
        double lu[3] = {0, 0, 0}, lB[3] = {0, 0, 0};
        for (int jj = 0; jj < 3; ++jj) {
            const double bj = B[jj] + bb0 * u[jj];
            lbeta += lV[1 + jj] * u[jj] + lV[5 + jj] * bj / W;
            lW -= lV[5 + jj] * bW * bj / W;
            lu[jj] += lV[1 + jj] * beta;
            for (int l = 0; l < 3; ++l) {
                lu[l] += lV[5 + jj] * bW * ((jj == l ? bb0 : 0.0) + u[jj] * B[l]);
                lB[l] += lV[5 + jj] * bW * ((jj == l ? 1.0 : 0.0) + u[jj] * u[l]);
            }
        }
        addq(lamq, g.P, A_LNR, ck, lV[0]);
        addq(lamq, g.P, A_LNB, ck, lV[0] * ig);
        addq(lamq, g.P, A_BETA, ck, lbeta);
        addq(lamq, g.P, A_W, ck, lW);
        for (int l = 0; l < 3; ++l) {
            addq(lamq, g.P, A_U0 + l, ck, lu[l]);
            addq(lamq, g.P, A_B0 + l, ck, lB[l]);
        }
    }
    // interface state, through the eigen-system
    double Rbar[8][8];
    for (int b = 0; b < 8; ++b)
        for (int m = 0; m < 8; ++m) {
            double a = -hl * lrot[b] * z[m];
            for (int k = 0; k < NS; ++k) a += lVt[k][m] * TV[k][b];
            Rbar[b][m] = a;
        }
    double gw[8];
    for (int a = 0; a < 8; ++a) {
        dual wd[8], lamd[8], Rd[8][8];
        for (int k = 0; k < 8; ++k) wd[k] = dual(wrot[k], k == a ? 1.0 : 0.0);
        eigen_mhd<dual>(ph.gamma, wd, lamd, Rd, true);
        double acc = -0.5 * sg * Lk * lamd[msel].d * zeta;
        for (int b = 0; b < 8; ++b)
            for (int m = 0; m < 8; ++m) acc += Rbar[b][m] * Rd[b][m].d;
        gw[a] = acc;
    }
    double gwm[8];
    unrot3(T, gw, gwm);
    // ... and through the frame's angle
    if (mode) {
        double d8[8], gphi = 0.0;
        dphi8(lrot, d8);
        for (int b = 0; b < 8; ++b) gphi -= hl * d8[b] * Rz[b];
        dphi8(wrot, d8);
        for (int a = 0; a < 8; ++a) gphi += gw[a] * d8[a];
        for (int k = 0; k < NS; ++k) {
            dphi8(TV[k], d8);
            for (int m = 0; m < 8; ++m) {
                double dv = 0.0;
                for (int b = 0; b < 8; ++b) dv += R[b][m] * d8[b];
                gphi += lVt[k][m] * dv;
            }
        }
        // phi = atan2(tb2, tb1), tb_i = (row i of the unturned frame) . (B or v)
        for (int qq = 0; qq < 3; ++qq) gwm[fo + qq] += gphi * (tb1 * T0[2][qq] - tb2 * T0[1][qq]) / tt2;
    }
    // wm[0] = {{rho}}^ln from (rho, ln rho) of both nodes
    for (int s = 0; s < 4; ++s) {
        dual a0 = dual(r0), a1 = dual(r1), f0 = dual(l0), f1 = dual(l1);
        if (s == 0) a0.d = 1.0;
        if (s == 1) a1.d = 1.0;
        if (s == 2) f0.d = 1.0;
        if (s == 3) f1.d = 1.0;
        dual rho, irho;
        logmean<dual, dual>(a0, a1, f0, f1, ph.ln_thr, rho, irho);
        addq(lamq, g.P, s < 2 ? A_RHO : A_LNR, (s % 2) ? c1 : c0, gwm[0] * rho.d);
    }
    {
        const double W2 = 1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2];
        const double W = sqrt(W2);
        for (int l = 0; l < 3; ++l) {
            double a = 0.0;
            for (int k = 0; k < 3; ++k) a += gwm[1 + k] * ((k == l ? 1.0 : 0.0) - um[k] * um[l] / W2) / W;
            addq(lamq, g.P, A_U0 + l, c0, 0.5 * a);
            addq(lamq, g.P, A_U0 + l, c1, 0.5 * a);
        }
        const double ib = 1.0 / (b0 + b1);
        addq(lamq, g.P, A_RHO, c0, gwm[4] * ib);
        addq(lamq, g.P, A_RHO, c1, gwm[4] * ib);
        addq(lamq, g.P, A_BETA, c0, -gwm[4] * wm[4] * ib);
        addq(lamq, g.P, A_BETA, c1, -gwm[4] * wm[4] * ib);
        for (int k = 0; k < 3; ++k) {
            addq(lamq, g.P, A_B0 + k, c0, 0.5 * gwm[5 + k]);
            addq(lamq, g.P, A_B0 + k, c1, 0.5 * gwm[5 + k]);
        }
    }
}

__device__ void dUdw3(double gam, const double w[8], double A[8][8])
{
    for (int c = 0; c < 8; ++c) {
        dual wd[8], U[8], F[8], V[8];
        for (int k = 0; k < 8; ++k) wd[k] = dual(w[k], k == c ? 1.0 : 0.0);
        mhd_UFV<dual>(gam, wd, U, F, V);
        for (int r = 0; r < 8; ++r) A[r][c] = U[r].d;
    }
}

__device__ void solve_t8_3(const double A[8][8], const double b[8], double x[8])
{
    double M[8][9];
    for (int r = 0; r < 8; ++r) {
        for (int c = 0; c < 8; ++c) M[r][c] = A[c][r];
        M[r][8] = b[r];
    }
    for (int c = 0; c < 8; ++c) {
        int piv = c;
        for (int r = c + 1; r < 8; ++r)
            if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
        if (piv != c)
            for (int k = 0; k < 9; ++k) { double t = M[c][k]; M[c][k] = M[piv][k]; M[piv][k] = t; }
        for (int r = c + 1; r < 8; ++r) {
            const double f = M[r][c] / M[c][c];
            for (int k = c; k < 9; ++k) M[r][k] -= f * M[c][k];
        }
    }
    for (int r = 7; r >= 0; --r) {
        double acc = M[r][8];
        for (int k = r + 1; k < 8; ++k) acc -= M[r][k] * x[k];
        x[r] = acc / M[r][r];
    }
}

// per padded node: node-quantity adjoints (+ the Powell term of interior
// nodes) -> primitives -> recovery adjoint -> lambda_cons of the source node
__global__ void k3_node_vjp(Geom3 g, double gam, const double *__restrict__ q, const double *__restrict__ lamq,
                            const double *__restrict__ fl, const double *__restrict__ mu,
                            const double *__restrict__ J, double *__restrict__ lam)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.P) return;
    const int c3[3] = {(int)(t % g.pd[0]) - GH, (int)((t / g.pd[0]) % g.pd[1]) - GH,
                       (int)(t / ((long long)g.pd[0] * g.pd[1])) - GH};
    double lq[NQN];
    bool any = false;
    for (int k = 0; k < NQN; ++k) {
        lq[k] = lamq[k * g.P + t];
        any = any || lq[k] != 0.0;
    }
    const bool interior = inside3(g, c3);
    if (!any && !interior) return;
    const double rho = q[F_RHO * g.P + t], p = q[F_P * g.P + t], W = q[F_W * g.P + t];
    const double v[3] = {q[F_U0 * g.P + t] / W, q[F_U1 * g.P + t] / W, q[F_U2 * g.P + t] / W};
    const double B[3] = {q[F_B0 * g.P + t], q[F_B1 * g.P + t], q[F_B2 * g.P + t]};
    double lw[8];
    lw[0] = lq[A_RHO] + lq[A_BETA] / p + (lq[A_LNR] + lq[A_LNB]) / rho;
    lw[4] = -lq[A_BETA] * rho / (p * p) - lq[A_LNB] / p;
    const double W3 = W * W * W;
    for (int k = 0; k < 3; ++k) {
        double a = lq[A_W] * W3 * v[k];
        for (int jj = 0; jj < 3; ++jj) a += lq[A_U0 + jj] * ((jj == k ? W : 0.0) + v[jj] * W3 * v[k]);
        lw[1 + k] = a;
        lw[5 + k] = lq[A_B0 + k];
    }
    if (interior) {
        const long long id = nid3(g, c3);
        const long long sdd[3] = {1, (long long)g.pd[0], (long long)g.pd[0] * g.pd[1]};
        double L9 = 0.0;
        for (int d = 0; d < 3; ++d) {
            const double *f = fl + (long long)(d * NF3 + 9) * g.P;
            L9 -= f[t] - f[t - sdd[d]];
        }
        double cP[8];
        for (int a = 0; a < 8; ++a) cP[a] = mu[a * g.N + id] * L9;
        const double iW2 = 1.0 - (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        const double vB = v[0] * B[0] + v[1] * B[1] + v[2] * B[2];
        for (int k = 0; k < 3; ++k) {
            double av = cP[4] * B[k] + cP[5 + k], aB = cP[4] * v[k];
            for (int jj = 0; jj < 3; ++jj) {
                av += cP[1 + jj] * (-2.0 * B[jj] * v[k] + (jj == k ? vB : 0.0) + v[jj] * B[k]);
                aB += cP[1 + jj] * ((jj == k ? iW2 : 0.0) + v[jj] * v[k]);
            }
            lw[1 + k] += av;
            lw[5 + k] += aB;
        }
    }
    const double w[8] = {rho, v[0], v[1], v[2], p, B[0], B[1], B[2]};
    double A[8][8], x[8];
    dUdw3(gam, w, A);
    solve_t8_3(A, lw, x);
    const long long src = data_src3(g, c3[0], c3[1], c3[2]);
    const double iJ = 1.0 / J[src];
    for (int a = 0; a < 8; ++a)
        if (x[a] != 0.0) atomicAdd(lam + a * g.N + src, x[a] * iJ);
}

__global__ void k3_prim_grad(Geom3 g, double gam, const double *__restrict__ cons, const double *__restrict__ J,
                             const double *__restrict__ lam, double *__restrict__ out, int *__restrict__ status)
{
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    const double iJ = 1.0 / J[id];
    double U[8], w[8], Z;
    for (int a = 0; a < 8; ++a) U[a] = cons[a * g.N + id] * iJ;
    if (cons2prim_mhd(gam, U, -1.0, w, Z)) atomicAdd(status, 1);
    double A[8][8];
    dUdw3(gam, w, A);
    for (int c = 0; c < 8; ++c) {
        double acc = 0.0;
        for (int r = 0; r < 8; ++r) acc += A[r][c] * lam[r * g.N + id];
        out[c * g.N + id] = J[id] * acc;
    }
}

__global__ void k3_lincomb(long long n, double a, const double *__restrict__ x, double b, const double *__restrict__ y,
                           double *__restrict__ out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a * x[i] + (y ? b * y[i] : 0.0);
}

inline unsigned nbk(long long n, int bs = 128) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

void launch3_pairs_vjp(const Geom3 &g, const Phys &ph, const double *q, const double *mu, double *lamq, int dir,
                       cudaStream_t st)
{
    const int oa = dir == 0 ? 1 : 0, ob = dir == 2 ? 1 : 2;
    const unsigned nb = nbk((long long)(g.n[dir] + ph.p) * g.n[oa] * g.n[ob]);
    if (ph.p == 1) k3_pairs_vjp<1><<<nb, 128, 0, st>>>(g, ph, q, mu, lamq, dir);
    else if (ph.p == 2) k3_pairs_vjp<2><<<nb, 128, 0, st>>>(g, ph, q, mu, lamq, dir);
    else k3_pairs_vjp<3><<<nb, 128, 0, st>>>(g, ph, q, mu, lamq, dir);
}

void launch3_iface_vjp(const Geom3 &g, const Phys &ph, const double *q, const double *mu, double *lamq, int dir,
                       cudaStream_t st)
{
    const int oa = dir == 0 ? 1 : 0, ob = dir == 2 ? 1 : 2;
    const unsigned nb = nbk((long long)(g.n[dir] + 1) * g.n[oa] * g.n[ob]);
    if (ph.w == 5) k3_iface_vjp<5><<<nb, 128, 0, st>>>(g, ph, q, mu, lamq, dir);
    else if (ph.w == 3) k3_iface_vjp<3><<<nb, 128, 0, st>>>(g, ph, q, mu, lamq, dir);
}

void launch3_node_vjp(const Geom3 &g, double gam, const double *q, const double *lamq, const double *iflux,
                      const double *mu, const double *J, double *lam, cudaStream_t st)
{
    k3_node_vjp<<<nbk(g.P), 128, 0, st>>>(g, gam, q, lamq, iflux, mu, J, lam);
}

void launch3_prim_grad(const Geom3 &g, double gam, const double *cons, const double *J, const double *lam,
                       double *out, int *status, cudaStream_t st)
{
    k3_prim_grad<<<nbk(g.N), 128, 0, st>>>(g, gam, cons, J, lam, out, status);
}

void launch3_lincomb(long long n, double a, const double *x, double b, const double *y, double *out, cudaStream_t st)
{
    k3_lincomb<<<nbk(n, 256), 256, 0, st>>>(n, a, x, b, y, out);
}

}  // namespace d3
}  // namespace esmm
