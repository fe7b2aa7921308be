// esmm_mhd_adjoint.cu -- vector-Jacobian products of the 2D RMHD right-hand
// side (the adjoint form on RMHD grids; the step adjoint around it is the one
// of esmm_api.cu), and the eigen-system entry point esmm_mhd_eigen.
//
// As for RHD (esmm_adjoint.cu), a time step is differentiated with its mesh
// velocity and step held at their recorded values, and with the sign switch
// Y and the lambda^ maximum frozen at their forward selection, so J and the
// metrics do not depend on the state.  With mu the adjoint of d(JU)/dt at the
// interior nodes (eq. RMHDSemiU_O2p_ES):
//   lambda_F = mu_{L+1} - mu_L for the interface fluxes, and
//   lambda_B = mu_{L+1}.Phi'_{L+1} - mu_L.Phi'_L for the magnetic flux B~ of
//   the Powell source;
//   per node pair: dual numbers seeded at one of 11 node quantities give the
//   two-point flux's Jacobian-vector products;
//   per interface: a reverse sweep of the dissipation (WENO weights through
//   dual numbers per stencil position, Y frozen), and the eigen-system's
//   tangent along each of the 8 interface-state directions (eigen_mhd<dual>:
//   perturbation theory on the Jacobi result, cluster spans kept);
//   per node: the Powell term's own dependence on v and B, the chain rule to
//   the primitives w, and the implicit-function adjoint of the Newton
//   recovery, lambda_U = (dU/dw)^-T lambda_w; lambda_cons += lambda_U / J.
// Node-quantity adjoints are accumulated with atomics in lamq[11][P] on the
// padded grid; ghost nodes fold into their source node in the node pass.
#include "esmm_launch.h"
#include "esmm_mhd.cuh"

namespace esmm {

namespace {

enum { A_RHO = 0, A_BETA, A_LNR, A_LNB, A_W, A_U0, A_U1, A_U2, A_B0, A_B1, A_B2, NQN };

__device__ __forceinline__ bool inside(const Geom &g, int i, int j)
{
    return i >= 0 && i < g.nx && j >= 0 && j < g.ny;
}

// mu_i . Phi'(w_i) at node (i, j); 0 outside the interior
__device__ double mu_phi(const Geom &g, const double *__restrict__ q, const double *__restrict__ mu, int i, int j)
{
    if (!inside(g, i, j)) return 0.0;
    const long long c = pidx(g, i, j), id = (long long)j * g.nx + i;
    const double iW = 1.0 / q[Q_W * g.P + c];
    double w[8] = {0.0, q[Q_UX * g.P + c] * iW, q[Q_UY * g.P + c] * iW, q[QM_UZ * g.P + c] * iW, 0.0,
                   q[QM_B1 * g.P + c], q[QM_B2 * g.P + c], q[QM_B3 * g.P + c]};
    double Pp[8];
    mhd_phiprime(w, Pp);
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a) s += mu[a * g.N + id] * Pp[a];
    return s;
}

// adjoints of the interface between (i, j) and its neighbour along dir
__device__ void lambda_face_mhd(const Geom &g, const double *__restrict__ q, const double *__restrict__ mu, int i,
                                int j, int dir, double lf[8], double &lb)
{
    const int i1 = i + (dir == 0), j1 = j + (dir == 1);
    const bool a = inside(g, i, j), b = inside(g, i1, j1);
    const long long ia = (long long)j * g.nx + i, ib = (long long)j1 * g.nx + i1;
#pragma unroll
    for (int k = 0; k < 8; ++k) lf[k] = (b ? mu[k * g.N + ib] : 0.0) - (a ? mu[k * g.N + ia] : 0.0);
    lb = mu_phi(g, q, mu, i1, j1) - mu_phi(g, q, mu, i, j);
}

__device__ __forceinline__ void seed_m(NodeMT<dual> &v, int k)
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

__device__ __forceinline__ void add_q(double *lamq, long long P, int k, long long c, double v)
{
    if (v != 0.0) atomicAdd(lamq + k * P + c, v);
}

// Pairs (A, A + n), A in [-P, n_dir - 1]: the pair enters the interfaces
// L = A + s (s < n) with weight alpha_{p,n} (eq. ECFlux_O2p, eq. BFlux_O2p).
template <int P>
__global__ void __launch_bounds__(128) k_pairs_vjp_mhd(ProbArg pa, Phys ph, const double *__restrict__ q,
                                                       const double *__restrict__ mu, double *__restrict__ lamq,
                                                       int dir)
{
    ProbDesc D;
    long long lb_;
    locate(pa, D, lb_);
    const Geom &g = D.g;
    const int nd = dir == 0 ? g.nx : g.ny, no = dir == 0 ? g.ny : g.nx;
    const long long idx = lb_ * blockDim.x + threadIdx.x;
    if (idx >= (long long)(nd + P) * no) return;
    int i, j;
    if (dir == 0) { j = (int)(idx / (nd + P)); i = (int)(idx % (nd + P)) - P; }
    else { i = (int)(idx % no); j = (int)(idx / no) - P; }
    const long long c0 = pidx(g, i, j);
    const long long sd = dir == 0 ? 1 : g.px;
    const double *Mt = q + (Q_MT0 + dir) * g.P;
    const double *Mx = q + (Q_M00 + 2 * dir) * g.P;
    const double *My = q + (Q_M01 + 2 * dir) * g.P;
    const dual gm1inv = dual(1.0 / (ph.gamma - 1.0));
    const int A = dir == 0 ? i : j;
    for (int n = 1; n <= P; ++n) {
        double lp[8] = {0, 0, 0, 0, 0, 0, 0, 0}, lbs = 0.0;
        for (int s = 0; s < n; ++s) {
            const int L = A + s;
            if (L < -1 || L > nd - 1) continue;
            double lf[8], lb;
            lambda_face_mhd(g, q, mu, dir == 0 ? L : i, dir == 0 ? j : L, dir, lf, lb);
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
        // B~ of the pair: 1/4 (Mx_l + Mx_r)(B1_l + B1_r) + 1/4 (My_l + My_r)(B2_l + B2_r)
        const double bx = 0.25 * (Mx[c0] + Mx[cr]), by = 0.25 * (My[c0] + My[cr]);
        add_q(lamq, g.P, A_B0, c0, lbs * bx);
        add_q(lamq, g.P, A_B0, cr, lbs * bx);
        add_q(lamq, g.P, A_B1, c0, lbs * by);
        add_q(lamq, g.P, A_B1, cr, lbs * by);
        const dual mt = dual(0.5 * (Mt[c0] + Mt[cr]));
        const dual mm[3] = {dual(0.5 * (Mx[c0] + Mx[cr])), dual(0.5 * (My[c0] + My[cr])), dual(0.0)};
        for (int side = 0; side < 2; ++side)
            for (int k = 0; k < NQN; ++k) {
                NodeMT<dual> l = load_node_m<dual>(q, g.P, c0), r = load_node_m<dual>(q, g.P, cr);
                seed_m(side ? r : l, k);
                dual out[8];
                ec_pair_mhd<2, dual>(l, r, gm1inv, ph.ln_thr, mt, mm, out);
                double gsum = 0.0;
#pragma unroll
                for (int a = 0; a < 8; ++a) gsum += lp[a] * out[a].d;
                add_q(lamq, g.P, k, side ? cr : c0, gsum);
            }
    }
}

// The ES dissipation of one interface (eq. ESFlux_HO; F = F_EC - diss), in
// reverse: its adjoint with respect to the stencil nodes' entropy variables
// and to the interface state (through the eigen-system's tangents).
template <int WW>
__global__ void __launch_bounds__(128) k_iface_vjp_mhd(ProbArg pa, Phys ph, const double *__restrict__ q,
                                                       const double *__restrict__ mu, double *__restrict__ lamq,
                                                       int dir)
{
    constexpr int NS = WW + 1, OFF = (WW - 1) / 2;
    ProbDesc D;
    long long lb_;
    locate(pa, D, lb_);
    const Geom &g = D.g;
    const int nd = dir == 0 ? g.nx : g.ny, no = dir == 0 ? g.ny : g.nx;
    const long long idx = lb_ * blockDim.x + threadIdx.x;
    if (idx >= (long long)(nd + 1) * no) return;
    int i, j;
    if (dir == 0) { j = (int)(idx / (nd + 1)); i = (int)(idx % (nd + 1)) - 1; }
    else { i = (int)(idx % no); j = (int)(idx / no) - 1; }
    double lf[8], lbdummy;
    lambda_face_mhd(g, q, mu, i, j, dir, lf, lbdummy);
    bool any = false;
#pragma unroll
    for (int a = 0; a < 8; ++a) any = any || lf[a] != 0.0;
    if (!any) return;
    const long long c0 = pidx(g, i, j);
    const long long sd = dir == 0 ? 1 : g.px;
    const long long c1 = c0 + sd;
    const double *Mt = q + (Q_MT0 + dir) * g.P;
    const double *Mx = q + (Q_M00 + 2 * dir) * g.P;
    const double *My = q + (Q_M01 + 2 * dir) * g.P;
    const double nvx = 0.5 * (Mx[c0] + Mx[c1]), nvy = 0.5 * (My[c0] + My[c1]);
    const double jt = 0.5 * (Mt[c0] + Mt[c1]);
    const double Lk = sqrt(nvx * nvx + nvy * nvy);
    const double nx = nvx / Lk, ny = nvy / Lk;
    // forward: interface state, eigen-system, projections, WENO, Y
    const double r0 = q[Q_RHO * g.P + c0], r1 = q[Q_RHO * g.P + c1];
    const double l0 = q[Q_LNR * g.P + c0], l1 = q[Q_LNR * g.P + c1];
    const double b0 = q[Q_BETA * g.P + c0], b1 = q[Q_BETA * g.P + c1];
    double um[3], wm[8], wrot[8];
    {
        double rho, irho;
        logmean<double, double>(r0, r1, l0, l1, ph.ln_thr, rho, irho);
        um[0] = 0.5 * (q[Q_UX * g.P + c0] + q[Q_UX * g.P + c1]);
        um[1] = 0.5 * (q[Q_UY * g.P + c0] + q[Q_UY * g.P + c1]);
        um[2] = 0.5 * (q[QM_UZ * g.P + c0] + q[QM_UZ * g.P + c1]);
        const double W = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
        wm[0] = rho;
        for (int k = 0; k < 3; ++k) wm[1 + k] = um[k] / W;
        wm[4] = (r0 + r1) / (b0 + b1);
        wm[5] = 0.5 * (q[QM_B1 * g.P + c0] + q[QM_B1 * g.P + c1]);
        wm[6] = 0.5 * (q[QM_B2 * g.P + c0] + q[QM_B2 * g.P + c1]);
        wm[7] = 0.5 * (q[QM_B3 * g.P + c0] + q[QM_B3 * g.P + c1]);
        wrot[0] = wm[0];
        wrot[1] = nx * wm[1] + ny * wm[2];
        wrot[2] = -ny * wm[1] + nx * wm[2];
        wrot[3] = wm[3];
        wrot[4] = wm[4];
        wrot[5] = nx * wm[5] + ny * wm[6];
        wrot[6] = -ny * wm[5] + nx * wm[6];
        wrot[7] = wm[7];
    }
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
        node_V_mhd<double>(q, g.P, c0 + (k - OFF) * sd, c1g, ig, V);
        TV[k][0] = V[0];
        TV[k][1] = nx * V[1] + ny * V[2];
        TV[k][2] = -ny * V[1] + nx * V[2];
        TV[k][3] = V[3];
        TV[k][4] = V[4];
        TV[k][5] = nx * V[5] + ny * V[6];
        TV[k][6] = -ny * V[5] + nx * V[6];
        TV[k][7] = V[7];
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
    // reverse: objective contribution -hl lrot . (R z), lrot = T lambda_F
    double lrot[8] = {lf[0], nx * lf[1] + ny * lf[2], -ny * lf[1] + nx * lf[2], lf[3],
                      lf[4], nx * lf[5] + ny * lf[6], -ny * lf[5] + nx * lf[6], lf[7]};
    const double hl = 0.5 * lhat;
    double zeta = 0.0, qm[8];
    for (int m = 0; m < 8; ++m) {
        double a = 0.0;
        for (int b = 0; b < 8; ++b) a += R[b][m] * lrot[b];
        qm[m] = -hl * a;
        zeta += a * z[m];
    }
    // WENO partials d z_m / d Vt[k][m] (the fields are independent, so one
    // dual pass per stencil position serves all eight)
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
    // stencil nodes: lambda of V_k, then of the node quantities V depends on
    for (int k = 0; k < NS; ++k) {
        double lT[8];
        for (int b = 0; b < 8; ++b) {
            double a = 0.0;
            for (int m = 0; m < 8; ++m) a += R[b][m] * lVt[k][m];
            lT[b] = a;
        }
        const double lV[8] = {lT[0], nx * lT[1] - ny * lT[2], ny * lT[1] + nx * lT[2], lT[3],
                              lT[4], nx * lT[5] - ny * lT[6], ny * lT[5] + nx * lT[6], lT[7]};
        const long long ck = c0 + (k - OFF) * sd;
        const double beta = q[Q_BETA * g.P + ck], W = q[Q_W * g.P + ck];
        const double u[3] = {q[Q_UX * g.P + ck], q[Q_UY * g.P + ck], q[QM_UZ * g.P + ck]};
        const double B[3] = {q[QM_B1 * g.P + ck], q[QM_B2 * g.P + ck], q[QM_B3 * g.P + ck]};
        const double bb0 = u[0] * B[0] + u[1] * B[1] + u[2] * B[2];
        const double bW = beta / W;
        // V0 = c1g + ln rho + ig ln beta + beta, V_{1+j} = beta u_j, V4 = -beta W,
        // V_{5+j} = (beta/W)(B_j + b0 u_j), b0 = u.B
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
        add_q(lamq, g.P, A_LNR, ck, lV[0]);
        add_q(lamq, g.P, A_LNB, ck, lV[0] * ig);
        add_q(lamq, g.P, A_BETA, ck, lbeta);
        add_q(lamq, g.P, A_W, ck, lW);
        for (int l = 0; l < 3; ++l) {
            add_q(lamq, g.P, A_U0 + l, ck, lu[l]);
            add_q(lamq, g.P, A_B0 + l, ck, lB[l]);
        }
    }
    // interface state: tangents of (lam, R) along each rotated-state direction
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
    // wrot = T wm
    const double gm_[8] = {gw[0], nx * gw[1] - ny * gw[2], ny * gw[1] + nx * gw[2], gw[3],
                           gw[4], nx * gw[5] - ny * gw[6], ny * gw[5] + nx * gw[6], gw[7]};
    // wm[0] = {{rho}}^ln from (rho, ln rho) of both nodes
    for (int s = 0; s < 4; ++s) {
        dual a0 = dual(r0), a1 = dual(r1), f0 = dual(l0), f1 = dual(l1);
        if (s == 0) a0.d = 1.0;
        if (s == 1) a1.d = 1.0;
        if (s == 2) f0.d = 1.0;
        if (s == 3) f1.d = 1.0;
        dual rho, irho;
        logmean<dual, dual>(a0, a1, f0, f1, ph.ln_thr, rho, irho);
        add_q(lamq, g.P, s < 2 ? A_RHO : A_LNR, (s % 2) ? c1 : c0, gm_[0] * rho.d);
    }
    // wm[1+k] = um_k / W(um), um = (u_0 + u_1)/2
    {
        const double W2 = 1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2];
        const double W = sqrt(W2);
        for (int l = 0; l < 3; ++l) {
            double a = 0.0;
            for (int k = 0; k < 3; ++k) a += gm_[1 + k] * ((k == l ? 1.0 : 0.0) - um[k] * um[l] / W2) / W;
            add_q(lamq, g.P, A_U0 + l, c0, 0.5 * a);
            add_q(lamq, g.P, A_U0 + l, c1, 0.5 * a);
        }
    }
    // wm[4] = (rho_0 + rho_1)/(beta_0 + beta_1), wm[5+k] = (B_0 + B_1)/2
    {
        const double ib = 1.0 / (b0 + b1);
        add_q(lamq, g.P, A_RHO, c0, gm_[4] * ib);
        add_q(lamq, g.P, A_RHO, c1, gm_[4] * ib);
        add_q(lamq, g.P, A_BETA, c0, -gm_[4] * wm[4] * ib);
        add_q(lamq, g.P, A_BETA, c1, -gm_[4] * wm[4] * ib);
        for (int k = 0; k < 3; ++k) {
            add_q(lamq, g.P, A_B0 + k, c0, 0.5 * gm_[5 + k]);
            add_q(lamq, g.P, A_B0 + k, c1, 0.5 * gm_[5 + k]);
        }
    }
}

// dU/dw at the primitive state w (column c = derivative along w_c)
__device__ void dUdw_mhd(double gam, const double w[8], double A[8][8])
{
    for (int c = 0; c < 8; ++c) {
        dual wd[8], U[8], F[8], V[8];
        for (int k = 0; k < 8; ++k) wd[k] = dual(w[k], k == c ? 1.0 : 0.0);
        mhd_UFV<dual>(gam, wd, U, F, V);
        for (int r = 0; r < 8; ++r) A[r][c] = U[r].d;
    }
}

// x with A^T x = b (Gaussian elimination, partial pivoting)
__device__ void solve_t8(const double A[8][8], const double b[8], double x[8])
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

// Per padded node: node-quantity adjoints -> primitives (with the Powell
// term of interior nodes) -> recovery adjoint -> lambda_cons of the source node.
__global__ void k_node_vjp_mhd(ProbArg pa, double gam, const double *__restrict__ q, const double *__restrict__ lamq,
                               const double *__restrict__ fl, const double *__restrict__ mu,
                               const double *__restrict__ J, double *__restrict__ lam)
{
    ProbDesc D;
    long long lb_;
    locate(pa, D, lb_);
    const Geom &g = D.g;
    const long long t = lb_ * blockDim.x + threadIdx.x;
    if (t >= g.P) return;
    const int I = (int)(t % g.px) - GH, Jn = (int)(t / g.px) - GH;
    double lq[NQN];
    bool any = false;
    for (int k = 0; k < NQN; ++k) {
        lq[k] = lamq[k * g.P + t];
        any = any || lq[k] != 0.0;
    }
    const bool interior = inside(g, I, Jn);
    if (!any && !interior) return;
    const double rho = q[Q_RHO * g.P + t], p = q[Q_P * g.P + t], W = q[Q_W * g.P + t];
    const double v[3] = {q[Q_UX * g.P + t] / W, q[Q_UY * g.P + t] / W, q[QM_UZ * g.P + t] / W};
    const double B[3] = {q[QM_B1 * g.P + t], q[QM_B2 * g.P + t], q[QM_B3 * g.P + t]};
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
        // Powell source Phi'(w_i) * L9_i, L9 = -div B~ (eq. RMHDSemiU_O2p_ES)
        const long long id = (long long)Jn * g.nx + I;
        const double *f0 = fl + 9 * g.P, *f1 = fl + (NFM + 9) * g.P;
        const double L9 = -((f0[t] - f0[t - 1]) + (f1[t] - f1[t - g.px]));
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
    dUdw_mhd(gam, w, A);
    solve_t8(A, lw, x);
    const long long src = data_src(g, I, Jn);
    const double iJ = 1.0 / J[src];
    for (int a = 0; a < 8; ++a)
        if (x[a] != 0.0) atomicAdd(lam + a * g.N + src, x[a] * iJ);
}

// gradient with respect to the initial primitives: cons = J U(w), so
// lambda_w = J (dU/dw)^T lambda_cons
__global__ void k_prim_grad_mhd(ProbArg pa, double gam, const double *__restrict__ cons,
                                const double *__restrict__ J, const double *__restrict__ lam,
                                double *__restrict__ out, int *__restrict__ status)
{
    ProbDesc D;
    long long lb_;
    locate(pa, D, lb_);
    const Geom &g = D.g;
    const long long id = lb_ * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    const double iJ = 1.0 / J[id];
    double U[8], w[8], Z;
    for (int a = 0; a < 8; ++a) U[a] = cons[a * g.N + id] * iJ;
    if (cons2prim_mhd(gam, U, -1.0, w, Z)) atomicAdd(status, 1);
    double A[8][8];
    dUdw_mhd(gam, w, A);
    for (int c = 0; c < 8; ++c) {
        double acc = 0.0;
        for (int r = 0; r < 8; ++r) acc += A[r][c] * lam[r * g.N + id];
        out[c * g.N + id] = J[id] * acc;
    }
}

// one state per thread: (lam, R) and, with dw, their tangents
__global__ void k_eigen_mhd(double gam, int n, const double *__restrict__ w, const double *__restrict__ dw,
                            double *__restrict__ lam, double *__restrict__ R, double *__restrict__ dlam,
                            double *__restrict__ dR)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    if (!dw) {
        double wk[8], l[8], Rk[8][8];
        for (int a = 0; a < 8; ++a) wk[a] = w[8 * k + a];
        eigen_mhd<double>(gam, wk, l, Rk, true);
        for (int a = 0; a < 8; ++a) {
            lam[8 * k + a] = l[a];
            for (int b = 0; b < 8; ++b) R[64 * k + 8 * a + b] = Rk[a][b];
        }
        return;
    }
    dual wk[8], l[8], Rk[8][8];
    for (int a = 0; a < 8; ++a) wk[a] = dual(w[8 * k + a], dw[8 * k + a]);
    eigen_mhd<dual>(gam, wk, l, Rk, true);
    for (int a = 0; a < 8; ++a) {
        lam[8 * k + a] = l[a].v;
        dlam[8 * k + a] = l[a].d;
        for (int b = 0; b < 8; ++b) {
            R[64 * k + 8 * a + b] = Rk[a][b].v;
            dR[64 * k + 8 * a + b] = Rk[a][b].d;
        }
    }
}

}  // namespace

int mhd_eigen_host(double gam, int n, const double *w, const double *dw, double *lam, double *R, double *dlam,
                   double *dR)
{
    const size_t d = sizeof(double), nn = (size_t)n;
    double *b = nullptr;
    if (cudaMalloc((void **)&b, nn * (8 + 8 + 8 + 64 + 8 + 64) * d) != cudaSuccess) return 1;
    double *dw_ = b, *w_ = dw_ + 8 * nn, *l_ = w_ + 8 * nn, *R_ = l_ + 8 * nn, *dl_ = R_ + 64 * nn;
    double *dR_ = dl_ + 8 * nn;
    cudaError_t e = cudaMemcpy(w_, w, 8 * nn * d, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && dw) e = cudaMemcpy(dw_, dw, 8 * nn * d, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_eigen_mhd<<<(n + 63) / 64, 64>>>(gam, n, w_, dw ? dw_ : nullptr, l_, R_, dl_, dR_);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(lam, l_, 8 * nn * d, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(R, R_, 64 * nn * d, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && dw) e = cudaMemcpy(dlam, dl_, 8 * nn * d, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && dw) e = cudaMemcpy(dR, dR_, 64 * nn * d, cudaMemcpyDeviceToHost);
    cudaFree(b);
    return e == cudaSuccess ? 0 : 1;
}

void launch_pairs_vjp_mhd(const LaunchDom &L, const Phys &ph, const double *q, const double *mu, double *lamq,
                          int dir, cudaStream_t st)
{
    if (ph.p == 1) k_pairs_vjp_mhd<1><<<L.nblk, L.bs, 0, st>>>(L.pa, ph, q, mu, lamq, dir);
    else if (ph.p == 2) k_pairs_vjp_mhd<2><<<L.nblk, L.bs, 0, st>>>(L.pa, ph, q, mu, lamq, dir);
    else k_pairs_vjp_mhd<3><<<L.nblk, L.bs, 0, st>>>(L.pa, ph, q, mu, lamq, dir);
}

void launch_iface_vjp_mhd(const LaunchDom &L, const Phys &ph, const double *q, const double *mu, double *lamq,
                          int dir, cudaStream_t st)
{
    if (ph.w == 5) k_iface_vjp_mhd<5><<<L.nblk, L.bs, 0, st>>>(L.pa, ph, q, mu, lamq, dir);
    else if (ph.w == 3) k_iface_vjp_mhd<3><<<L.nblk, L.bs, 0, st>>>(L.pa, ph, q, mu, lamq, dir);
}

void launch_node_vjp_mhd(const LaunchDom &L, double gam, const double *q, const double *lamq, const double *iflux,
                         const double *mu, const double *J, double *lam, cudaStream_t st)
{
    k_node_vjp_mhd<<<L.nblk, L.bs, 0, st>>>(L.pa, gam, q, lamq, iflux, mu, J, lam);
}

void launch_prim_grad_mhd(const LaunchDom &L, double gam, const double *cons, const double *J, const double *lam,
                          double *out, int *status, cudaStream_t st)
{
    k_prim_grad_mhd<<<L.nblk, L.bs, 0, st>>>(L.pa, gam, cons, J, lam, out, status);
}

}  // namespace esmm
