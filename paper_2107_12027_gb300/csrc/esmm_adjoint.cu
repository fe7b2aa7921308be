// esmm_adjoint.cu -- vector-Jacobian products of the right-hand side and of
// the SSP-RK3 step (gradients of a final-time functional
// with respect to the initial data).
//
// The map differentiated is one time step with its mesh velocity xdot and
// time step dt held at their recorded values (the mesh monitor's maximum and
// the movement limiter's minimum are not differentiable), and with the sign
// switch Y and the lambda^ maximum frozen at their forward selection.  With
// xdot fixed the metrics and J are independent of the state, so the adjoint
// runs through the conserved state only:
//   mu (adjoint of dU/dt)  ->  lambda_F = mu_{L+1} - mu_L per interface
//   -> per pair / per interface: local Jacobian-vector products by dual
//      numbers seeded at one node quantity at a time (EC pair fluxes: log
//      means and averages; ES dissipation: eigenvectors, WENO weights)
//   -> per node: gather, chain rule to the primitives, and the implicit-
//      function adjoint of the Newton recovery, lambda_U = (dU/dw)^-T lambda_w
//   -> lambda_cons += lambda_U / J (ghost nodes add into their source node).
#include <cuda_runtime.h>

#include "esmm_flux.cuh"

namespace esmm {

namespace {

constexpr int NQA = 7;      // adjoint node quantities: beta, u_x, u_y, W, ln rho, ln beta, rho
constexpr int NSMAX = 6;    // stencil nodes of WENO5

__device__ __forceinline__ double mu_at(const Geom &g, const double *mu, int i, int j, int a)
{
    if (i < 0 || i >= g.nx || j < 0 || j >= g.ny) return 0.0;
    return mu[(long long)a * g.N + (long long)j * g.nx + i];
}

// lambda_F of the interface whose left node is (i, j) in direction dir
__device__ __forceinline__ void lambda_face(const Geom &g, const double *mu, int i, int j, int dir, double lf[4])
{
    int i1 = i + (dir == 0), j1 = j + (dir == 1);
#pragma unroll
    for (int a = 0; a < 4; ++a) lf[a] = mu_at(g, mu, i1, j1, a) - mu_at(g, mu, i, j, a);
}

__device__ __forceinline__ void seed_node(NodeV<dual> &v, int jq)
{
    switch (jq) {
    case 0: v.beta.d = 1.0; v.b.d = 1.0; break;
    case 1: v.ux.d = 1.0; break;
    case 2: v.uy.d = 1.0; break;
    case 3: v.W.d = 1.0; break;
    case 4: v.lnr.d = 1.0; break;
    case 5: v.lnb.d = 1.0; break;
    default: v.rho.d = 1.0; v.r.d = 1.0; break;
    }
}

__device__ __forceinline__ NodeV<dual> node_dual(const Geom &g, const double *q, long long c)
{
    NodeV<dual> v;
    v.rho = dual(q[Q_RHO * g.P + c]);
    v.beta = dual(q[Q_BETA * g.P + c]);
    v.lnr = dual(q[Q_LNR * g.P + c]);
    v.lnb = dual(q[Q_LNB * g.P + c]);
    v.r = v.rho;
    v.b = v.beta;
    v.ux = dual(q[Q_UX * g.P + c]);
    v.uy = dual(q[Q_UY * g.P + c]);
    v.W = dual(q[Q_W * g.P + c]);
    return v;
}

// Adjoint contributions of the pair fluxes anchored at A: the pair (A, A+n)
// enters the interfaces A + s (s < n) with weight alpha_{p,n}, so its adjoint
// is alpha_n sum_s lambda_F(A + s); its derivative with respect to the 7
// quantities of either node follows from dual evaluation.
template <int P>
__global__ void __launch_bounds__(128) k_pairs_vjp(ProbArg pa, Phys ph, const double *__restrict__ q,
                                                   const double *__restrict__ mu, double *__restrict__ Gp, int dir)
{
    ProbDesc D;
    long long lb;
    locate(pa, D, lb);
    const Geom &g = D.g;
    q += (long long)NQ * D.op;
    mu += 4 * D.on;
    Gp += (long long)2 * PMAX * 2 * NQA * D.op;
    const int nd = dir == 0 ? g.nx : g.ny, no = dir == 0 ? g.ny : g.nx;
    const long long idx = lb * blockDim.x + threadIdx.x;
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
        double lp[4] = {0.0, 0.0, 0.0, 0.0};
        for (int s = 0; s < n; ++s) {
            int L = A + s;
            if (L < -1 || L > nd - 1) continue;
            double lf[4];
            lambda_face(g, mu, dir == 0 ? L : i, dir == 0 ? j : L, dir, lf);
#pragma unroll
            for (int a = 0; a < 4; ++a) lp[a] += lf[a];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) lp[a] *= ph.alpha[n - 1];
        const long long cr = c0 + n * sd;
        const dual mt = dual(0.5 * (Mt[c0] + Mt[cr])), mx = dual(0.5 * (Mx[c0] + Mx[cr])),
                   my = dual(0.5 * (My[c0] + My[cr]));
        for (int side = 0; side < 2; ++side)
            for (int jq = 0; jq < NQA; ++jq) {
                NodeV<dual> l = node_dual(g, q, c0), r = node_dual(g, q, cr);
                seed_node(side == 0 ? l : r, jq);
                dual out[4];
                ec_pair<dual>(l, r, mt, mx, my, gm1inv, ph.ln_thr, out);
                double gsum = 0.0;
#pragma unroll
                for (int a = 0; a < 4; ++a) gsum += lp[a] * out[a].d;
                Gp[((((long long)dir * PMAX + (n - 1)) * 2 + side) * NQA + jq) * g.P + c0] = gsum;
            }
    }
}

// Adjoint contributions of the ES dissipation at one interface: F = F_EC -
// diss, so d(lambda_F . F)/d(input) = -lambda_F . d diss/d(input).
template <int WW>
__global__ void __launch_bounds__(128) k_iface_vjp(ProbArg pa, Phys ph, const double *__restrict__ q,
                                                   const double *__restrict__ mu, double *__restrict__ G, int dir)
{
    constexpr int NS = WW + 1, OFF = (WW - 1) / 2;
    ProbDesc D;
    long long lb;
    locate(pa, D, lb);
    const Geom &g = D.g;
    q += (long long)NQ * D.op;
    mu += 4 * D.on;
    G += (long long)2 * NSMAX * NQA * D.op;
    const int nd = dir == 0 ? g.nx : g.ny, no = dir == 0 ? g.ny : g.nx;
    const long long idx = lb * blockDim.x + threadIdx.x;
    if (idx >= (long long)(nd + 1) * no) return;
    int i, j;
    if (dir == 0) { j = (int)(idx / (nd + 1)); i = (int)(idx % (nd + 1)) - 1; }
    else { i = (int)(idx % no); j = (int)(idx / no) - 1; }
    const long long c0 = pidx(g, i, j);
    const long long sd = dir == 0 ? 1 : g.px;
    const long long c1 = c0 + sd;
    double lf[4];
    lambda_face(g, mu, i, j, dir, lf);
    const double *Mt = q + (Q_MT0 + dir) * g.P;
    const double *Mx = q + (Q_M00 + 2 * dir) * g.P;
    const double *My = q + (Q_M01 + 2 * dir) * g.P;
    const dual nvx = dual(0.5 * (Mx[c0] + Mx[c1])), nvy = dual(0.5 * (My[c0] + My[c1]));
    const dual jt = dual(0.5 * (Mt[c0] + Mt[c1]));
    const int fld[6] = {Q_BETA, Q_UX, Q_UY, Q_W, Q_LNR, Q_LNB};
    for (int k = 0; k < NS; ++k)
        for (int jq = 0; jq < NQA; ++jq) {
            if (jq == 6 && k != OFF && k != OFF + 1) continue;   // rho enters at the interface nodes only
            dual st[NS][6];
            for (int kk = 0; kk < NS; ++kk)
                for (int f = 0; f < 6; ++f) st[kk][f] = dual(q[fld[f] * g.P + c0 + (kk - OFF) * sd]);
            dual r0 = dual(q[Q_RHO * g.P + c0]), r1 = dual(q[Q_RHO * g.P + c1]);
            dual l0 = dual(q[Q_LNR * g.P + c0]), l1 = dual(q[Q_LNR * g.P + c1]);
            if (jq < 6) st[k][jq].d = 1.0;
            if (jq == 4 && k == OFF) l0.d = 1.0;
            if (jq == 4 && k == OFF + 1) l1.d = 1.0;
            if (jq == 6) (k == OFF ? r0 : r1).d = 1.0;
            dual diss[4];
            ArrStencil<dual, NS> acc{st};
            es_dissipation<dual, dual, WW>(nvx, nvy, jt, r0, r1, l0, l1, r0, r1, acc, ph, diss);
            double gsum = 0.0;
#pragma unroll
            for (int a = 0; a < 4; ++a) gsum -= lf[a] * diss[a].d;
            G[(((long long)dir * NSMAX + k) * NQA + jq) * g.P + c0] = gsum;
        }
}

// Per padded node: gather the pair and interface contributions, chain them to
// the primitives w = (rho, v_x, v_y, p), apply the recovery's adjoint
// lambda_U = (dU/dw)^-T lambda_w and add lambda_U / J into the source node.
__global__ void k_node_vjp(ProbArg pa, double gam, int p, int ww, const double *__restrict__ q,
                           const double *__restrict__ G, const double *__restrict__ Gp,
                           const double *__restrict__ J, double *__restrict__ lam)
{
    ProbDesc D;
    long long lb;
    locate(pa, D, lb);
    const Geom &g = D.g;
    long long t = lb * blockDim.x + threadIdx.x;
    if (t >= g.P) return;
    q += (long long)NQ * D.op;
    G += (long long)2 * NSMAX * NQA * D.op;
    Gp += (long long)2 * PMAX * 2 * NQA * D.op;
    J += D.on;
    lam += 4 * D.on;
    const int I = (int)(t % g.px) - GH, Jn = (int)(t / g.px) - GH;
    double lq[NQA] = {0, 0, 0, 0, 0, 0, 0};
    const int NS = ww + 1, OFF = (ww - 1) / 2;
    for (int dir = 0; dir < 2; ++dir) {
        const int nd = dir == 0 ? g.nx : g.ny, no = dir == 0 ? g.ny : g.nx;
        const int pos = dir == 0 ? I : Jn, line = dir == 0 ? Jn : I;
        if (line < 0 || line >= no) continue;
        auto cidx = [&](int a) { return dir == 0 ? pidx(g, a, line) : pidx(g, line, a); };
        if (ww > 0)
            for (int k = 0; k < NS; ++k) {
                int L = pos - (k - OFF);
                if (L < -1 || L > nd - 1) continue;
                long long cl = cidx(L);
                for (int jq = 0; jq < NQA; ++jq) lq[jq] += G[(((long long)dir * NSMAX + k) * NQA + jq) * g.P + cl];
            }
        for (int n = 1; n <= p; ++n)
            for (int side = 0; side < 2; ++side) {
                int A = pos - side * n;
                if (A < -p || A > nd - 1) continue;
                long long ca = cidx(A);
                for (int jq = 0; jq < NQA; ++jq)
                    lq[jq] += Gp[((((long long)dir * PMAX + (n - 1)) * 2 + side) * NQA + jq) * g.P + ca];
            }
    }
    // node quantities -> primitives
    double rho = q[Q_RHO * g.P + t], pr = q[Q_P * g.P + t], W = q[Q_W * g.P + t];
    double vx = q[Q_UX * g.P + t] / W, vy = q[Q_UY * g.P + t] / W;
    double W3 = W * W * W;
    double lw[4];
    lw[0] = lq[6] + lq[0] / pr + (lq[4] + lq[5]) / rho;
    lw[3] = -lq[0] * rho / (pr * pr) - lq[5] / pr;
    lw[1] = lq[1] * (W + vx * W3 * vx) + lq[2] * (vy * W3 * vx) + lq[3] * (W3 * vx);
    lw[2] = lq[1] * (vx * W3 * vy) + lq[2] * (W + vy * W3 * vy) + lq[3] * (W3 * vy);
    // dU/dw (rows D, m_x, m_y, E; columns rho, v_x, v_y, p)
    double g1 = gam / (gam - 1.0), rh = rho + g1 * pr, W2 = W * W, W4 = W2 * W2;
    double A[4][4] = {
        {W, rho * W3 * vx, rho * W3 * vy, 0.0},
        {W2 * vx, rh * (2.0 * W4 * vx * vx + W2), rh * 2.0 * W4 * vy * vx, g1 * W2 * vx},
        {W2 * vy, rh * 2.0 * W4 * vx * vy, rh * (2.0 * W4 * vy * vy + W2), g1 * W2 * vy},
        {W2, rh * 2.0 * W4 * vx, rh * 2.0 * W4 * vy, g1 * W2 - 1.0}};
    // solve A^T x = lw (Gaussian elimination with partial pivoting on M = A^T)
    double M[4][5];
    for (int r = 0; r < 4; ++r) {
        for (int c = 0; c < 4; ++c) M[r][c] = A[c][r];
        M[r][4] = lw[r];
    }
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int r = c + 1; r < 4; ++r)
            if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
        if (piv != c)
            for (int k = 0; k < 5; ++k) { double tmp = M[c][k]; M[c][k] = M[piv][k]; M[piv][k] = tmp; }
        for (int r = c + 1; r < 4; ++r) {
            double f = M[r][c] / M[c][c];
            for (int k = c; k < 5; ++k) M[r][k] -= f * M[c][k];
        }
    }
    double xs[4];
    for (int r = 3; r >= 0; --r) {
        double acc = M[r][4];
        for (int k = r + 1; k < 4; ++k) acc -= M[r][k] * xs[k];
        xs[r] = acc / M[r][r];
    }
    long long src = data_src(g, I, Jn);
    double iJ = 1.0 / J[src];
    for (int a = 0; a < 4; ++a)
        if (xs[a] != 0.0) atomicAdd(lam + a * g.N + src, xs[a] * iJ);
}

// out = a x + b y over n values
__global__ void k_lincomb(long long n, double a, const double *__restrict__ x, double b, const double *__restrict__ y,
                          double *__restrict__ out)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a * x[i] + (y ? b * y[i] : 0.0);
}

// gradient with respect to the initial primitives: cons = J U(w), so
// lambda_w = J (dU/dw)^T lambda_cons
__global__ void k_prim_grad(ProbArg pa, double gam, const double *__restrict__ cons, const double *__restrict__ J,
                            const double *__restrict__ lam, double *__restrict__ out)
{
    ProbDesc D;
    long long lb;
    locate(pa, D, lb);
    const Geom &g = D.g;
    long long id = lb * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    cons += 4 * D.on;
    J += D.on;
    lam += 4 * D.on;
    out += 4 * D.on;
    double iJ = 1.0 / J[id];
    double rho, vx, vy, pr, W;
    cons2prim(gam, cons[id] * iJ, cons[g.N + id] * iJ, cons[2 * g.N + id] * iJ, cons[3 * g.N + id] * iJ, -1.0, rho,
              vx, vy, pr, W);
    double g1 = gam / (gam - 1.0), rh = rho + g1 * pr, W2 = W * W, W3 = W2 * W, W4 = W2 * W2;
    double A[4][4] = {
        {W, rho * W3 * vx, rho * W3 * vy, 0.0},
        {W2 * vx, rh * (2.0 * W4 * vx * vx + W2), rh * 2.0 * W4 * vy * vx, g1 * W2 * vx},
        {W2 * vy, rh * 2.0 * W4 * vx * vy, rh * (2.0 * W4 * vy * vy + W2), g1 * W2 * vy},
        {W2, rh * 2.0 * W4 * vx, rh * 2.0 * W4 * vy, g1 * W2 - 1.0}};
    for (int c = 0; c < 4; ++c) {
        double acc = 0.0;
        for (int r = 0; r < 4; ++r) acc += A[r][c] * lam[r * g.N + id];
        out[c * g.N + id] = J[id] * acc;
    }
}

}  // namespace

void launch_pairs_vjp(const LaunchDom &L, const Phys &ph, const double *q, const double *mu, double *Gp, int dir,
                      cudaStream_t st)
{
    if (ph.p == 1) k_pairs_vjp<1><<<L.nblk, L.bs, 0, st>>>(L.pa, ph, q, mu, Gp, dir);
    else if (ph.p == 2) k_pairs_vjp<2><<<L.nblk, L.bs, 0, st>>>(L.pa, ph, q, mu, Gp, dir);
    else k_pairs_vjp<3><<<L.nblk, L.bs, 0, st>>>(L.pa, ph, q, mu, Gp, dir);
}

void launch_iface_vjp(const LaunchDom &L, const Phys &ph, const double *q, const double *mu, double *G, int dir,
                      cudaStream_t st)
{
    if (ph.w == 5) k_iface_vjp<5><<<L.nblk, L.bs, 0, st>>>(L.pa, ph, q, mu, G, dir);
    else if (ph.w == 3) k_iface_vjp<3><<<L.nblk, L.bs, 0, st>>>(L.pa, ph, q, mu, G, dir);
}

void launch_node_vjp(const LaunchDom &L, double gam, int p, int w, const double *q, const double *G,
                     const double *Gp, const double *J, double *lam, cudaStream_t st)
{
    k_node_vjp<<<L.nblk, L.bs, 0, st>>>(L.pa, gam, p, w, q, G, Gp, J, lam);
}

void launch_lincomb(long long n, double a, const double *x, double b, const double *y, double *out, cudaStream_t st)
{
    k_lincomb<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, a, x, b, y, out);
}

void launch_prim_grad(const LaunchDom &L, double gam, const double *cons, const double *J, const double *lam,
                      double *out, cudaStream_t st)
{
    k_prim_grad<<<L.nblk, L.bs, 0, st>>>(L.pa, gam, cons, J, lam, out);
}

}  // namespace esmm
