// esmm_kernels.cuh -- the per-node, update, CFL, mesh-redistribution, state
// and totals kernels (the flux kernels are in esmm_flux.cuh).  Every kernel
// takes a ProbArg: one problem by value, or a batch of problems addressed
// through a block -> (problem, tile) map; pointers are the bases of the
// concatenated arrays and each kernel offsets them to its problem's slice.
//
// Scheme: Duan & Tang, arXiv 2107.12027 (2D RHD: B = 0).
#pragma once

#include "esmm_device.cuh"
#include "esmm_reduce.cuh"

namespace esmm {

// ---------------------------------------------------------------------------
// alpha_{p,n} of eq. HOCoeff as compile-time constants
template <int P> __device__ __forceinline__ constexpr double alpha_c(int n)
{
    return P == 1 ? 1.0
                  : (P == 2 ? (n == 1 ? 4.0 / 3.0 : -1.0 / 6.0)
                            : (n == 1 ? 1.5 : (n == 2 ? -0.3 : 1.0 / 30.0)));
}

// The four differences delta_xi[x], delta_xi[y], delta_eta[x], delta_eta[y]
// (eq. SCLCoeff / App. B) at node (I, J) of the padded grid.  Nodes whose
// stencil stays inside the mesh read it directly; the others go through the
// boundary mapping.
template <int P>
__device__ __forceinline__ void mesh_deltas(const Geom &g, const double *__restrict__ x, int I, int J,
                                            double &dxi_x, double &dxi_y, double &deta_x, double &deta_y)
{
    dxi_x = dxi_y = deta_x = deta_y = 0.0;
    if (I - P >= 0 && I + P < g.nx && J - P >= 0 && J + P < g.ny) {
        const double *X = x, *Y = x + g.N;
        const long long c = (long long)J * g.nx + I;
#pragma unroll
        for (int n = 1; n <= P; ++n) {
            const double a = 0.5 * alpha_c<P>(n);
            const long long s = (long long)n * g.nx;
            dxi_x += a * (X[c + n] - X[c - n]);
            dxi_y += a * (Y[c + n] - Y[c - n]);
            deta_x += a * (X[c + s] - X[c - s]);
            deta_y += a * (Y[c + s] - Y[c - s]);
        }
        return;
    }
#pragma unroll
    for (int n = 1; n <= P; ++n) {
        const double a = 0.5 * alpha_c<P>(n);
        dxi_x += a * (mesh_at(g, x, I + n, J, 0, 1) - mesh_at(g, x, I - n, J, 0, 1));
        dxi_y += a * (mesh_at(g, x, I + n, J, 1, 1) - mesh_at(g, x, I - n, J, 1, 1));
        deta_x += a * (mesh_at(g, x, I, J + n, 0, 1) - mesh_at(g, x, I, J - n, 0, 1));
        deta_y += a * (mesh_at(g, x, I, J + n, 1, 1) - mesh_at(g, x, I, J - n, 1, 1));
    }
}

// Per padded node: primitive recovery (FP64 Newton, warm-started from pg_in
// when given), W, u = W v, beta = rho/p, ln rho, ln beta, the CMM metrics and
// the temporal metrics J xi_k,t = -xdot . (J xi_k,x) (eq. VCLCoeff).  Ghost
// nodes take the data of their boundary source node and metrics of the
// boundary-mapped mesh, so the flux kernels need no boundary logic.  With
// q32 (the mixed form) the node also writes the FP32 copies the flux kernels
// read; with f32_logs (the mixed form's scheme passes) ln rho and ln beta are
// FP32 logarithms: in that form they enter only FP32 arithmetic and the log
// mean's jump outside its near-equal branch, while the totals take a pass
// with FP64 logarithms.  gg = (Gamma - 1)/Gamma comes with the launch.
template <int P>
__global__ void k_node(ProbArg pa, double gam, double gg, const double *__restrict__ cons,
                       const double *__restrict__ J, const double *__restrict__ x, const double *__restrict__ xdot,
                       const double *__restrict__ pg_in, double *__restrict__ pg_out, double *__restrict__ q,
                       int *__restrict__ status, float *__restrict__ q32, const double *__restrict__ inflow,
                       int f32_logs = 0)
{
    ProbDesc D;
    long long lb;
    locate(pa, D, lb);
    const Geom &g = D.g;
    long long t = lb * blockDim.x + threadIdx.x;
    if (t >= g.P) return;
    cons += 4 * D.on;
    J += D.on;
    x += 2 * D.on;
    if (xdot) xdot += 2 * D.on;
    if (pg_in) pg_in += D.on;
    if (pg_out) pg_out += D.on;
    q += (long long)NQ * D.op;
    int I = (int)(t % g.px) - GH, Jn = (int)(t / g.px) - GH;
    long long src = data_src(g, I, Jn);
    double iJ = __drcp_rn(J[src]);
    double Dd = cons[src] * iJ, mx = cons[g.N + src] * iJ, my = cons[2 * g.N + src] * iJ,
           E = cons[3 * g.N + src] * iJ;
    double rho, vx, vy, p, W;
    int st;
    if (inflow && ((g.bc0 == 2 && I < 0) || (g.bc1 == 2 && Jn < 0))) {
        // a ghost beyond an inflow end: the given state
        rho = inflow[0]; vx = inflow[1]; vy = inflow[2]; p = inflow[3];
        W = rsqrt(1.0 - (vx * vx + vy * vy));
        st = 0;
    } else {
        st = cons2prim_gg(gam, gg, Dd, mx, my, E, pg_in ? pg_in[src] : -1.0, rho, vx, vy, p, W);
    }
    bool interior = I >= 0 && I < g.nx && Jn >= 0 && Jn < g.ny;
    if (interior) {
        if (st) atomicAdd(status, 1);
        if (pg_out) pg_out[src] = p;
    }
    double beta = rho * __drcp_rn(p);
    q[Q_RHO * g.P + t] = rho;
    q[Q_P * g.P + t] = p;
    q[Q_BETA * g.P + t] = beta;
    q[Q_UX * g.P + t] = W * vx;
    q[Q_UY * g.P + t] = W * vy;
    q[Q_W * g.P + t] = W;
    float lr32 = 0.0f, lb32 = 0.0f;
    if (f32_logs) {
        lr32 = logf(d2f_int(rho));
        lb32 = logf(d2f_int(beta));
        q[Q_LNR * g.P + t] = f2d_int(lr32);
        q[Q_LNB * g.P + t] = f2d_int(lb32);
    } else {
        q[Q_LNR * g.P + t] = log(rho);
        q[Q_LNB * g.P + t] = log(beta);
    }
    double dxi_x, dxi_y, deta_x, deta_y;
    mesh_deltas<P>(g, x, I, Jn, dxi_x, dxi_y, deta_x, deta_y);
    double M00 = deta_y, M01 = -deta_x, M10 = -dxi_y, M11 = dxi_x;
    q[Q_M00 * g.P + t] = M00;
    q[Q_M01 * g.P + t] = M01;
    q[Q_M10 * g.P + t] = M10;
    q[Q_M11 * g.P + t] = M11;
    double xd = 0.0, yd = 0.0;
    if (xdot) { xd = mesh_at(g, xdot, I, Jn, 0, 0); yd = mesh_at(g, xdot, I, Jn, 1, 0); }
    const double MT0 = -(xd * M00 + yd * M01), MT1 = -(xd * M10 + yd * M11);
    q[Q_MT0 * g.P + t] = MT0;
    q[Q_MT1 * g.P + t] = MT1;
    if (q32) {
        q32 += (long long)NQ32 * D.op;
        q32[Q32_R * g.P + t] = d2f_int(rho);
        q32[Q32_B * g.P + t] = d2f_int(beta);
        q32[Q32_UX * g.P + t] = d2f_int(W * vx);
        q32[Q32_UY * g.P + t] = d2f_int(W * vy);
        q32[Q32_W * g.P + t] = d2f_int(W);
        q32[Q32_LNR * g.P + t] = f32_logs ? lr32 : d2f_int(q[Q_LNR * g.P + t]);
        q32[Q32_LNB * g.P + t] = f32_logs ? lb32 : d2f_int(q[Q_LNB * g.P + t]);
        q32[Q32_M00 * g.P + t] = d2f_int(M00);
        q32[Q32_M01 * g.P + t] = d2f_int(M01);
        q32[Q32_M10 * g.P + t] = d2f_int(M10);
        q32[Q32_M11 * g.P + t] = d2f_int(M11);
        q32[Q32_MT0 * g.P + t] = d2f_int(MT0);
        q32[Q32_MT1 * g.P + t] = d2f_int(MT1);
    }
}

// temporal metrics only (the spatial ones and the state are unchanged), and
// their FP32 copies when q32 is given
__global__ void k_tmetric(ProbArg pa, const double *__restrict__ xdot, double *__restrict__ q,
                          float *__restrict__ q32 = nullptr)
{
    ProbDesc D;
    long long lb;
    locate(pa, D, lb);
    const Geom &g = D.g;
    long long t = lb * blockDim.x + threadIdx.x;
    if (t >= g.P) return;
    xdot += 2 * D.on;
    q += (long long)NQ * D.op;
    int I = (int)(t % g.px) - GH, Jn = (int)(t / g.px) - GH;
    double xd = mesh_at(g, xdot, I, Jn, 0, 0), yd = mesh_at(g, xdot, I, Jn, 1, 0);
    const double MT0 = -(xd * q[Q_M00 * g.P + t] + yd * q[Q_M01 * g.P + t]);
    const double MT1 = -(xd * q[Q_M10 * g.P + t] + yd * q[Q_M11 * g.P + t]);
    q[Q_MT0 * g.P + t] = MT0;
    q[Q_MT1 * g.P + t] = MT1;
    if (q32) {
        q32 += (long long)NQ32 * D.op;
        q32[Q32_MT0 * g.P + t] = d2f_int(MT0);
        q32[Q32_MT1 * g.P + t] = d2f_int(MT1);
    }
}

// d/dt = -sum_k (F_k(i + 1/2) - F_k(i - 1/2)) (eqs. RMHDSemiU_O2p_ES,
// RMHDSemiJ_O2p_ES); written out (dcons != NULL) or combined into the SSP-RK3
// stage  y_o = A y_n + B (y_s + dt L)  of (cons, J) and of the mesh x with
// velocity xdot, dt the problem's step.
template <typename R>
__global__ void k_update(ProbArg pa, const R *__restrict__ fl, double *__restrict__ dcons, double *__restrict__ dJ,
                         const double *__restrict__ cn, const double *__restrict__ Jn_,
                         const double *__restrict__ xn, const double *__restrict__ cs,
                         const double *__restrict__ Js, const double *__restrict__ xs,
                         const double *__restrict__ xdot, double A, double B,
                         const double *__restrict__ dt_dev, double *__restrict__ co, double *__restrict__ Jo,
                         double *__restrict__ xo)
{
    ProbDesc D;
    long long lb;
    int b = locate(pa, D, lb);
    const Geom &g = D.g;
    long long id = lb * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    fl += (long long)2 * 5 * D.op;
    int i = (int)(id % g.nx), j = (int)(id / g.nx);
    long long c = pidx(g, i, j);
    const R *f0 = fl, *f1 = fl + 5 * g.P;
    double L[5];
#pragma unroll
    for (int a = 0; a < 5; ++a) {
        // the differences in the fluxes' own precision (an FP32 difference
        // of two FP32 fluxes is exact when they are within a factor 2 and
        // rounds once otherwise), summed in FP64
        R d0 = f0[a * g.P + c] - f0[a * g.P + c - 1];
        R d1 = f1[a * g.P + c] - f1[a * g.P + c - g.px];
        L[a] = -(to_f64(d0) + to_f64(d1));
    }
    if (dcons) {
        dcons += 4 * D.on;
        dJ += D.on;
#pragma unroll
        for (int a = 0; a < 4; ++a) dcons[a * g.N + id] = L[a];
        dJ[id] = L[4];
        return;
    }
    cn += 4 * D.on; cs += 4 * D.on; co += 4 * D.on;
    Jn_ += D.on; Js += D.on; Jo += D.on;
    xn += 2 * D.on; xs += 2 * D.on; xo += 2 * D.on; xdot += 2 * D.on;
    double dt = dt_dev[b];
#pragma unroll
    for (int a = 0; a < 4; ++a) co[a * g.N + id] = A * cn[a * g.N + id] + B * (cs[a * g.N + id] + dt * L[a]);
    Jo[id] = A * Jn_[id] + B * (Js[id] + dt * L[4]);
    xo[id] = A * xn[id] + B * (xs[id] + dt * xdot[id]);
    xo[g.N + id] = A * xn[g.N + id] + B * (xs[g.N + id] + dt * xdot[g.N + id]);
}

// the spectral radius of k_cfl in FP32 (mixed form): with p = rho/beta,
// c^2 = Gamma p / (rho h) = Gamma / (beta + Gamma/(Gamma-1))
__device__ __forceinline__ void cfl_f32(const ProbArg &pa, float gam, const float *__restrict__ q32,
                                        const double *__restrict__ J, unsigned long long *red, double *cflb)
{
    ProbDesc D;
    long long lb;
    int b = locate(pa, D, lb);
    const Geom &g = D.g;
    long long id = lb * blockDim.x + threadIdx.x;
    q32 += (long long)NQ32 * D.op;
    J += D.on;
    if (cflb) cflb += 6 * D.on;
    double r[2] = {0.0, 0.0};
    if (id < g.N) {
        int i = (int)(id % g.nx), j = (int)(id / g.nx);
        long long c = pidx(g, i, j);
        float W = q32[Q32_W * g.P + c], beta = q32[Q32_B * g.P + c];
        float iW = __frcp_rn(W);
        float vx = q32[Q32_UX * g.P + c] * iW, vy = q32[Q32_UY * g.P + c] * iW;
        float v2 = vx * vx + vy * vy;
        float c2 = gam * __frcp_rn(beta + gam / (gam - 1.0f)), cs = sqrtf(c2);
        float iJ = __frcp_rn(d2f_int(J[id]));
        float iden = __frcp_rn(1.0f - v2 * c2);
        for (int k = 0; k < 2; ++k) {
            float mx = q32[(Q32_M00 + 2 * k) * g.P + c], my = q32[(Q32_M01 + 2 * k) * g.P + c];
            float n2 = mx * mx + my * my, iL = rsqrtf(n2), Lk = n2 * iL;
            float vn = (mx * vx + my * vy) * iL;
            float disc = sqrtf(fmaxf((1.0f - v2) * (1.0f - v2 * c2 - vn * vn * (1.0f - c2)), 0.0f));
            float lm = (vn * (1.0f - c2) - cs * disc) * iden, lp = (vn * (1.0f - c2) + cs * disc) * iden;
            r[k] = owned_row(g, j) ? f2d_int(Lk * fmaxf(fabsf(lm), fabsf(lp)) * iJ) : 0.0;
            if (cflb) {
                cflb[(2 + k) * g.N + id] = f2d_int(Lk * lm * iJ);
                cflb[(4 + k) * g.N + id] = f2d_int(Lk * lp * iJ);
            }
        }
    }
    for (int k = 0; k < 2; ++k) {
        double m = block_reduce<0>(r[k]);
        if (threadIdx.x == 0) atomic_max_nonneg(red + (long long)NRED * b + 2 + k, m);
    }
}


// spectral radius rho_k = L_k max |lambda_+-| / J at every node (eq. cfl,
// static mesh), reduced to a per-problem maximum per direction; with cflb
// (the moving-mesh step) also the speed bounds L_k lambda_-/J and
// L_k lambda_+/J of every node into its rows 2 + k and 4 + k
// gg = Gamma/(Gamma - 1) comes with the launch
__global__ void k_cfl(ProbArg pa, double gam, double gg, const double *__restrict__ q, const double *__restrict__ J,
                      unsigned long long *red, const float *__restrict__ q32, double *__restrict__ cflb)
{
    if (q32) {   // the mixed form: the same speeds in FP32 from the FP32 node copies
        cfl_f32(pa, (float)gam, q32, J, red, cflb);
        return;
    }
    ProbDesc D;
    long long lb;
    int b = locate(pa, D, lb);
    const Geom &g = D.g;
    long long id = lb * blockDim.x + threadIdx.x;
    q += (long long)NQ * D.op;
    J += D.on;
    if (cflb) cflb += 6 * D.on;
    double r[2] = {0.0, 0.0};
    if (id < g.N) {
        int i = (int)(id % g.nx), j = (int)(id / g.nx);
        long long c = pidx(g, i, j);
        double rho = q[Q_RHO * g.P + c], p = q[Q_P * g.P + c], W = q[Q_W * g.P + c];
        double iW = __drcp_rn(W);
        double vx = q[Q_UX * g.P + c] * iW, vy = q[Q_UY * g.P + c] * iW;
        double v2 = vx * vx + vy * vy;
        double rh = rho + p * gg;
        double c2 = gam * p * __drcp_rn(rh), cs = sqrt(c2);
        double iJ = __drcp_rn(J[id]);
        const double iden = __drcp_rn(1.0 - v2 * c2);   // the same for both directions
        for (int k = 0; k < 2; ++k) {
            double mx = q[(Q_M00 + 2 * k) * g.P + c], my = q[(Q_M01 + 2 * k) * g.P + c];
            const double n2 = mx * mx + my * my, iL = rsqrt(n2), Lk = n2 * iL;
            double vn = (mx * vx + my * vy) * iL;
            double disc = sqrt((1.0 - v2) * (1.0 - v2 * c2 - vn * vn * (1.0 - c2)));
            double lm = (vn * (1.0 - c2) - cs * disc) * iden, lp = (vn * (1.0 - c2) + cs * disc) * iden;
            r[k] = owned_row(g, j) ? Lk * fmax(fabs(lm), fabs(lp)) * iJ : 0.0;
            if (cflb) {
                cflb[(2 + k) * g.N + id] = Lk * lm * iJ;
                cflb[(4 + k) * g.N + id] = Lk * lp * iJ;
            }
        }
    }
    for (int k = 0; k < 2; ++k) {
        double m = block_reduce<0>(r[k]);
        if (threadIdx.x == 0) atomic_max_nonneg(red + (long long)NRED * b + 2 + k, m);
    }
}

__global__ void k_red_init(int nprob, unsigned long long *red)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nprob) return;
    red[NRED * b + 0] = 0ull;
    red[NRED * b + 1] = (unsigned long long)__double_as_longlong(1.0);
    red[NRED * b + 2] = 0ull;
    red[NRED * b + 3] = 0ull;
    red[NRED * b + 4] = 0ull;
    red[NRED * b + 5] = 0ull;
    red[NRED * b + 6] = 0ull;
    red[NRED * b + 7] = 0ull;
}

// Set-up of each problem's step (eq. cfl with the mesh velocity in the
// spectral radius, esmm_reduce.cuh dt_setup): slots 4, 5 hold A_k = max_i
// |a_{k,i}|, slots 2, 3 the static radius per direction, slot 1 the limiter
// Delta tau (written back, scaled where C_m >= CFL).  Without mesh motion
// C_m = 0 and dt = CFL / sum_k max rho_k.
__global__ void k_dt(int nprob, double cfl, double dt_fixed, unsigned long long *red, DtSolve *ds, double *dt_dev)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nprob) return;
    unsigned long long *r = red + (long long)NRED * b;
    double tau = bits_to_double(r[1]);
    dt_setup(ds + b, cfl, dt_fixed, bits_to_double(r[4]) + bits_to_double(r[5]),
             bits_to_double(r[2]) + bits_to_double(r[3]), &tau, dt_dev + b);
    r[1] = (unsigned long long)__double_as_longlong(tau);
}

// One Newton evaluation of the step solve (esmm_reduce.cuh) over the nodes
// of every problem still solving: cflb rows 0, 1 hold a_{k,i}, rows 2..5 the
// speed bounds (per problem at 6 D.on).  part: [blocks][2][2].  A block
// covers blockDim.x * DT_NPT nodes.
__global__ void k_dt_newton(ProbArg pa, double cfl, const double *__restrict__ cflb,
                            const unsigned long long *red, DtSolve *ds, double *part, double *dt_dev,
                            double *vs_out)
{
    ProbDesc D;
    long long lb;
    int b = locate(pa, D, lb);
    const Geom &g = D.g;
    DtSolve *S = ds + b;
    __shared__ double t_sh, tau_sh;
    __shared__ int skip;
    if (threadIdx.x == 0) {
        skip = S->done;
        t_sh = S->t;
        tau_sh = bits_to_double(red[(long long)NRED * b + 1]);
    }
    __syncthreads();
    if (skip) return;
    cflb += 6 * D.on;
    unsigned long long v[2] = {0ull, 0ull}, sl[2] = {~0ull, ~0ull};
    // DT_NPT nodes per thread, consecutive threads on consecutive nodes
    const long long base = lb * blockDim.x * DT_NPT + threadIdx.x;
    for (int r = 0; r < DT_NPT; ++r) {
        const long long id = base + (long long)r * blockDim.x;
        if (id < g.N && owned_row(g, (int)(id / g.nx)))
            for (int k = 0; k < 2; ++k) {
                unsigned long long vk, sk;
                cfl_line(t_sh, tau_sh * cflb[k * g.N + id], cflb[(2 + k) * g.N + id], cflb[(4 + k) * g.N + id],
                         vk, sk);
                vs_take(v[k], sl[k], vk, sk);
            }
    }
    const long long nb = (g.N + (long long)blockDim.x * DT_NPT - 1) / ((long long)blockDim.x * DT_NPT);
    dt_newton_block<2>(S, v, sl, blockIdx.x, (long long)blockIdx.x - lb, nb, (unsigned long long *)part, cfl,
                       dt_dev + b, vs_out);
}

__global__ void k_time(int nprob, const double *dt_dev, double *t_dev)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nprob) t_dev[b] += dt_dev[b];
}

// ---- Sec. 5 mesh redistribution ---------------------------------------------
// |grad_xi sigma| (max to slot 0) and, with_lap, |lap_xi sigma| (max to slot 6)
__global__ void k_mesh_grad(ProbArg pa, int lnrho, int with_lap, const double *__restrict__ q,
                            double *__restrict__ grad, double *__restrict__ lap, unsigned long long *red)
{
    ProbDesc D;
    long long lb;
    int b = locate(pa, D, lb);
    const Geom &g = D.g;
    long long id = lb * blockDim.x + threadIdx.x;
    q += (long long)NQ * D.op;
    grad += D.on;
    lap += D.on;
    double gv = 0.0, lv = 0.0;
    if (id < g.N) {
        int i = (int)(id % g.nx), j = (int)(id / g.nx);
        long long c = pidx(g, i, j);
        const double *s = q + (lnrho ? Q_LNR : Q_RHO) * g.P;
        double e = s[c + 1], w = s[c - 1], n = s[c + g.px], so = s[c - g.px];
        double gx = 0.5 * (e - w);
        double gy = 0.5 * (n - so);
        gv = sqrt(gx * gx + gy * gy);
        grad[id] = gv;
        if (with_lap) {
            lv = fabs(e + w + n + so - 4.0 * s[c]);
            lap[id] = lv;
        }
        if (!owned_row(g, j)) gv = lv = 0.0;
    }
    double m = block_reduce<0>(gv);
    if (threadIdx.x == 0) atomic_max_nonneg(red + (long long)NRED * b, m);
    if (with_lap) {
        double ml = block_reduce<0>(lv);
        if (threadIdx.x == 0) atomic_max_nonneg(red + (long long)NRED * b + 6, ml);
    }
}

__global__ void k_mesh_omega(ProbArg pa, double alpha, double alpha_lap, const double *__restrict__ grad,
                             const double *__restrict__ lap, const unsigned long long *red, double *__restrict__ om)
{
    ProbDesc D;
    long long lb;
    int b = locate(pa, D, lb);
    const Geom &g = D.g;
    long long id = lb * blockDim.x + threadIdx.x;
    // alpha / max, once per block
    __shared__ double sc[2];
    if (threadIdx.x == 0) {
        double gmax = bits_to_double(red[(long long)NRED * b]);
        double lmax = bits_to_double(red[(long long)NRED * b + 6]);
        sc[0] = gmax > 0.0 ? alpha / gmax : 0.0;
        sc[1] = (alpha_lap > 0.0 && lmax > 0.0) ? alpha_lap / lmax : 0.0;
    }
    __syncthreads();
    if (id >= g.N) return;
    double a = 1.0 + sc[0] * grad[D.on + id];
    if (sc[1] > 0.0) a += sc[1] * lap[D.on + id];
    om[D.on + id] = sqrt(a);
}

// omega <- sum_{a,b in {-1,0,1}} 2^-(|a|+|b|+2) omega_{i+a, j+b}
__global__ void k_mesh_filter(ProbArg pa, const double *__restrict__ om, double *__restrict__ om2)
{
    ProbDesc D;
    long long lb;
    locate(pa, D, lb);
    const Geom &g = D.g;
    long long id = lb * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    om += D.on;
    om2 += D.on;
    int i = (int)(id % g.nx), j = (int)(id / g.nx);
    double acc = 0.0;
    const bool inner = i > 0 && i < g.nx - 1 && j > 0 && j < g.ny - 1;
    for (int bb = -1; bb <= 1; ++bb)
        for (int a = -1; a <= 1; ++a) {
            double wgt = (a == 0 && bb == 0) ? 0.25 : ((a == 0 || bb == 0) ? 0.125 : 0.0625);
            acc += wgt * om[inner ? id + bb * g.nx + a : data_src(g, i + a, j + bb)];
        }
    om2[id] = acc;
}

// The weights of the Jacobi iteration of the Winslow mesh equations with
// omega frozen: X_i <- sum_k c_k X_k over the four neighbours (E, W, N, S),
// c_k = (omega_i + omega_k) / sum_k' (omega_i + omega_k').  Computed once per
// redistribution (the sweeps then take four FMAs per component).
__global__ void k_mesh_weights(ProbArg pa, const double *__restrict__ om, double *__restrict__ cw)
{
    ProbDesc D;
    long long lb;
    locate(pa, D, lb);
    const Geom &g = D.g;
    long long id = lb * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    om += D.on;
    cw += 4 * D.on;
    int i = (int)(id % g.nx), j = (int)(id / g.nx);
    double wi = om[id];
    double we = om[data_src(g, i + 1, j)], ww = om[data_src(g, i - 1, j)];
    double wn = om[data_src(g, i, j + 1)], ws = om[data_src(g, i, j - 1)];
    double iden = __drcp_rn((2.0 * wi + we + ww) + (2.0 * wi + wn + ws));
    cw[id] = (wi + we) * iden;
    cw[g.N + id] = (wi + ww) * iden;
    cw[2 * g.N + id] = (wi + wn) * iden;
    cw[3 * g.N + id] = (wi + ws) * iden;
}

// mesh_at with the shift for coordinates, out of line (edge paths)
__device__ __noinline__ double mesh_edge(const Geom &g, const double *__restrict__ x, int i, int j, int comp)
{
    return mesh_at(g, x, i, j, comp, 1);
}

// ---- the Jacobi sweeps, temporally blocked ---------------------------------
// The iteration X_i <- sum_k c_k X_k (k_mesh_weights) written for the
// displacement D = X - x^n, which starts at 0:
//   D_i <- sum_k c_k D_k + r_i,   r_i = sum_k c_k x^n_k - x^n_i,
// the same iterates in exact arithmetic, with D free of the positions'
// magnitude (so T = float keeps the displacement to FP32 relative precision
// in the mixed form).  A block owns a TX x TY tile and iterates nsw <= SB
// sweeps on the tile plus an SB-wide halo in shared memory (the valid region
// shrinks by one node per sweep), then writes the tile: one launch for SB
// sweeps.  The weights and r come per node from k_mesh_wr, in T; halo nodes
// across a periodic end take their source node's (D, the weights and r do
// not depend on the period's shift); nodes across an outflow or inflow end
// are read only by fixed boundary nodes and are held at 0.
constexpr int MT_TX = 32, MT_TY = 16, MT_THREADS = 256;

template <typename T, int SB>
constexpr size_t mesh_sweeps_smem()
{
    return (size_t)(10 * sizeof(T) + 1) * (MT_TX + 2 * SB) * (MT_TY + 2 * SB);
}

template <typename T, int SB>
__global__ void __launch_bounds__(MT_THREADS) k_mesh_sweeps(ProbArg pa, const T *__restrict__ wr,
                                                            const T *__restrict__ Din, T *__restrict__ Dout,
                                                            int nsw)
{
    constexpr int RX = MT_TX + 2 * SB, RY = MT_TY + 2 * SB, RN = RX * RY;
    extern __shared__ __align__(16) unsigned char mt_smem[];
    T *sD = reinterpret_cast<T *>(mt_smem);      // [2 buffers][2 components][RN]
    T *sW = sD + 4 * RN;                         // [4][RN]  c_E, c_W, c_N, c_S
    T *sR = sW + 4 * RN;                         // [2][RN]  r
    unsigned char *sF = reinterpret_cast<unsigned char *>(sR + 2 * RN);   // [RN] node held
    ProbDesc D;
    long long lb;
    locate(pa, D, lb);
    const Geom &g = D.g;
    wr += 6 * D.on;
    if (Din) Din += 2 * D.on;
    Dout += 2 * D.on;
    const int ntx = (g.nx + MT_TX - 1) / MT_TX;
    const int ti = (int)(lb % ntx) * MT_TX, tj = (int)(lb / ntx) * MT_TY;
    for (int r = threadIdx.x; r < RN; r += blockDim.x) {
        const int gi = ti - SB + r % RX, gj = tj - SB + r / RX;
        const bool outx = gi < 0 || gi >= g.nx, outy = gj < 0 || gj >= g.ny;
        if ((outx && g.bc0 != 0) || (outy && g.bc1 != 0)) {
            sF[r] = 1;
            for (int a = 0; a < 4; ++a) sW[a * RN + r] = (T)0;
            for (int c = 0; c < 2; ++c) { sD[c * RN + r] = (T)0; sD[(2 + c) * RN + r] = (T)0; sR[c * RN + r] = (T)0; }
            continue;
        }
        const int si = outx ? wrapi(gi, g.nx) : gi, sj = outy ? wrapi(gj, g.ny) : gj;
        const long long id = (long long)sj * g.nx + si;
        const bool fixed = (g.bc0 != 0 && (si == 0 || si == g.nx - 1)) || (g.bc1 != 0 && (sj == 0 || sj == g.ny - 1));
        sF[r] = fixed;
#pragma unroll
        for (int a = 0; a < 4; ++a) sW[a * RN + r] = wr[a * g.N + id];
        for (int c = 0; c < 2; ++c) {
            sR[c * RN + r] = wr[(4 + c) * g.N + id];   // 0 at a fixed node
            sD[c * RN + r] = Din ? Din[c * g.N + id] : (T)0;
        }
    }
    __syncthreads();
    int cur = 0;
    for (int s = 0; s < nsw; ++s) {
        const T *Dc = sD + cur * 2 * RN;
        T *Dn = sD + (cur ^ 1) * 2 * RN;
        for (int r = threadIdx.x; r < RN; r += blockDim.x) {
            const int li = r % RX, lj = r / RX;
            if (li <= s || li >= RX - 1 - s || lj <= s || lj >= RY - 1 - s) continue;
            for (int c = 0; c < 2; ++c) {
                const T *d = Dc + c * RN;
                Dn[c * RN + r] = sF[r] ? d[r]
                                       : sW[r] * d[r + 1] + sW[RN + r] * d[r - 1] + sW[2 * RN + r] * d[r + RX] +
                                             sW[3 * RN + r] * d[r - RX] + sR[c * RN + r];
            }
        }
        __syncthreads();
        cur ^= 1;
    }
    const T *Df = sD + cur * 2 * RN;
    for (int r = threadIdx.x; r < MT_TX * MT_TY; r += blockDim.x) {
        const int gi = ti + r % MT_TX, gj = tj + r / MT_TX;
        if (gi >= g.nx || gj >= g.ny) continue;
        const int rr = (r / MT_TX + SB) * RX + (r % MT_TX + SB);
        const long long id = (long long)gj * g.nx + gi;
        Dout[id] = Df[rr];
        Dout[g.N + id] = Df[RN + rr];
    }
}

// The same iteration one sweep per launch, for the FP64 form (where the
// blocked kernel's halo work would cost FP64 issue slots): the residual r
// once per redistribution, then D_i <- sum_k c_k D_k + r_i.  D needs no ghost
// arithmetic: it is shift-free across a periodic end and 0 at held nodes,
// and nodes next to an outflow end read only the held boundary nodes.
// The blocked sweeps' inputs in working type T, once per node: wr[0..3] the
// Jacobi weights c_E, c_W, c_N, c_S and wr[4..5] the residual of k_mesh_resid
// (FP64 arithmetic, then rounded), so that the sweep kernel's halo nodes,
// each staged by several tiles, only load them.  A ghost beyond a periodic
// end takes its source node's values.
template <typename T>
__global__ void k_mesh_wr(ProbArg pa, const double *__restrict__ x, const double *__restrict__ cw,
                          T *__restrict__ wr)
{
    ProbDesc D;
    long long lb;
    locate(pa, D, lb);
    const Geom &g = D.g;
    long long id = lb * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    x += 2 * D.on;
    cw += 4 * D.on;
    wr += 6 * D.on;
    int i = (int)(id % g.nx), j = (int)(id / g.nx);
    bool fixed = (g.bc0 != 0 && (i == 0 || i == g.nx - 1)) || (g.bc1 != 0 && (j == 0 || j == g.ny - 1));
    const double ce = cw[id], cwe = cw[g.N + id], cn = cw[2 * g.N + id], cs = cw[3 * g.N + id];
    wr[id] = from_f64<T>(ce);
    wr[g.N + id] = from_f64<T>(cwe);
    wr[2 * g.N + id] = from_f64<T>(cn);
    wr[3 * g.N + id] = from_f64<T>(cs);
    const bool inner = i > 0 && i < g.nx - 1 && j > 0 && j < g.ny - 1;
    for (int c = 0; c < 2; ++c) {
        double r = 0.0;
        if (!fixed) {
            const double *a = x + c * g.N;
            const double xe = inner ? a[id + 1] : mesh_edge(g, x, i + 1, j, c);
            const double xw = inner ? a[id - 1] : mesh_edge(g, x, i - 1, j, c);
            const double xn = inner ? a[id + g.nx] : mesh_edge(g, x, i, j + 1, c);
            const double xs = inner ? a[id - g.nx] : mesh_edge(g, x, i, j - 1, c);
            r = ce * xe + cwe * xw + cn * xn + cs * xs - a[id];
        }
        wr[(4 + c) * g.N + id] = from_f64<T>(r);
    }
}

__global__ void k_mesh_resid(ProbArg pa, const double *__restrict__ x, const double *__restrict__ cw,
                             double *__restrict__ rs)
{
    ProbDesc D;
    long long lb;
    locate(pa, D, lb);
    const Geom &g = D.g;
    long long id = lb * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    x += 2 * D.on;
    cw += 4 * D.on;
    rs += 2 * D.on;
    int i = (int)(id % g.nx), j = (int)(id / g.nx);
    bool fixed = (g.bc0 != 0 && (i == 0 || i == g.nx - 1)) || (g.bc1 != 0 && (j == 0 || j == g.ny - 1));
    const double ce = cw[id], cwe = cw[g.N + id], cn = cw[2 * g.N + id], cs = cw[3 * g.N + id];
    const bool inner = i > 0 && i < g.nx - 1 && j > 0 && j < g.ny - 1;
    for (int c = 0; c < 2; ++c) {
        double r = 0.0;
        if (!fixed) {
            const double *a = x + c * g.N;
            const double xe = inner ? a[id + 1] : mesh_edge(g, x, i + 1, j, c);
            const double xw = inner ? a[id - 1] : mesh_edge(g, x, i - 1, j, c);
            const double xn = inner ? a[id + g.nx] : mesh_edge(g, x, i, j + 1, c);
            const double xs = inner ? a[id - g.nx] : mesh_edge(g, x, i, j - 1, c);
            r = ce * xe + cwe * xw + cn * xn + cs * xs - a[id];
        }
        rs[c * g.N + id] = r;
    }
}

__global__ void k_mesh_sweep(ProbArg pa, const double *__restrict__ cw, const double *__restrict__ rs,
                             const double *__restrict__ Din, double *__restrict__ Dout)
{
    ProbDesc D;
    long long lb;
    locate(pa, D, lb);
    const Geom &g = D.g;
    long long id = lb * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    cw += 4 * D.on;
    rs += 2 * D.on;
    Dout += 2 * D.on;
    int i = (int)(id % g.nx), j = (int)(id / g.nx);
    bool fixed = (g.bc0 != 0 && (i == 0 || i == g.nx - 1)) || (g.bc1 != 0 && (j == 0 || j == g.ny - 1));
    if (!Din || fixed) {        // the first sweep from D = 0, and held nodes
        for (int c = 0; c < 2; ++c) Dout[c * g.N + id] = fixed ? 0.0 : rs[c * g.N + id];
        return;
    }
    Din += 2 * D.on;
    const long long e = i == g.nx - 1 ? id - (g.nx - 1) : id + 1, w = i == 0 ? id + (g.nx - 1) : id - 1;
    const long long n = j == g.ny - 1 ? id - (long long)(g.ny - 1) * g.nx : id + g.nx;
    const long long s = j == 0 ? id + (long long)(g.ny - 1) * g.nx : id - g.nx;
    const double ce = cw[id], cwe = cw[g.N + id], cn = cw[2 * g.N + id], cs = cw[3 * g.N + id];
    for (int c = 0; c < 2; ++c) {
        const double *d = Din + c * g.N;
        Dout[c * g.N + id] = ce * d[e] + cwe * d[w] + cn * d[n] + cs * d[s] + rs[c * g.N + id];
    }
}

// movement limiter: Delta tau = min over nodes and directions of half the
// neighbour spacing over the displacement toward it, clipped to [0, 1]; and
// the displacement's Courant terms a_k = d.(J xi_k,x)/J per node (into cflb
// rows 0, 1) and their maximum modulus per direction (the node metrics of x^n
// in q, J of the state)
// (Dd: the displacement x^[mu] - x^n of k_mesh_sweeps)
template <typename T>
__global__ void k_mesh_tau(ProbArg pa, const double *__restrict__ x, const T *__restrict__ Dd,
                           const double *__restrict__ q, const double *__restrict__ J, unsigned long long *red,
                           double *__restrict__ cflb)
{
    ProbDesc D;
    long long lb;
    int b = locate(pa, D, lb);
    const Geom &g = D.g;
    long long id = lb * blockDim.x + threadIdx.x;
    x += 2 * D.on;
    Dd += 2 * D.on;
    J += D.on;
    q += (long long)NQ * D.op;
    double tau = 1.0, cm[2] = {0.0, 0.0};
    if (id < g.N) {
        int i = (int)(id % g.nx), j = (int)(id / g.nx);
        double dd[2];
        for (int k = 0; k < 2; ++k) {
            double d = to_f64(Dd[k * g.N + id]);
            dd[k] = d;
            int di = k == 0, dj = k == 1;
            const bool inner = k == 0 ? (i > 0 && i < g.nx - 1) : (j > 0 && j < g.ny - 1);
            const long long step = k == 0 ? 1 : g.nx;
            double bnd = 1.0;
            if (d != 0.0) {
                const double xi = x[k * g.N + id];
                const double xb = inner ? x[k * g.N + id + (d < 0.0 ? -step : step)]
                                        : mesh_edge(g, x, d < 0.0 ? i - di : i + di, d < 0.0 ? j - dj : j + dj, k);
                bnd = (xb - xi) * __drcp_rn(2.0 * d);
            }
            tau = fmin(tau, bnd);
        }
        tau = fmax(tau, 0.0);
        long long c = pidx(g, i, j);
        double iJ = __drcp_rn(J[id]);
        const bool own = owned_row(g, j);
        for (int k = 0; k < 2; ++k) {
            const double ak = (dd[0] * q[(Q_M00 + 2 * k) * g.P + c] + dd[1] * q[(Q_M01 + 2 * k) * g.P + c]) * iJ;
            cm[k] = own ? fabs(ak) : 0.0;
            cflb[6 * D.on + k * g.N + id] = ak;
        }
        if (!own) tau = 1.0;
    }
    double m = block_reduce<1>(tau);
    if (threadIdx.x == 0) atomic_min_nonneg(red + (long long)NRED * b + 1, m);
    for (int k = 0; k < 2; ++k) {
        double mk = block_reduce<0>(cm[k]);
        if (threadIdx.x == 0) atomic_max_nonneg(red + (long long)NRED * b + 4 + k, mk);
    }
}

// xdot = Delta tau (x^[mu] - x^n) / dt (over 2 N values per problem; Dd the
// displacement x^[mu] - x^n)
template <typename T>
__global__ void k_mesh_xdot(ProbArg pa, const T *__restrict__ Dd, const unsigned long long *red,
                            const double *__restrict__ dt_dev, double *__restrict__ xdot)
{
    ProbDesc D;
    long long lb;
    int b = locate(pa, D, lb);
    const Geom &g = D.g;
    long long id = lb * blockDim.x + threadIdx.x;
    __shared__ double s;
    // a step of 0 (a NaN spectral radius) leaves the mesh where it is
    if (threadIdx.x == 0) s = dt_dev[b] > 0.0 ? bits_to_double(red[(long long)NRED * b + 1]) / dt_dev[b] : 0.0;
    __syncthreads();
    if (id >= 2 * g.N) return;
    long long o = 2 * D.on + id;
    xdot[o] = s * to_f64(Dd[o]);
}

// ---- state set-up and read-out ------------------------------------------------
// initial J (reading: the determinant of the metric differences) and
// cons = J U(prim); counts non-admissible states or tangled cells in status[1]
template <int P>
__global__ void k_init_state(ProbArg pa, double gam, const double *__restrict__ prim,
                             const double *__restrict__ x, double *__restrict__ cons, double *__restrict__ J,
                             int *status)
{
    ProbDesc D;
    long long lb;
    locate(pa, D, lb);
    const Geom &g = D.g;
    long long id = lb * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    prim += 4 * D.on;
    x += 2 * D.on;
    cons += 4 * D.on;
    J += D.on;
    int i = (int)(id % g.nx), j = (int)(id / g.nx);
    double dxi_x, dxi_y, deta_x, deta_y;
    mesh_deltas<P>(g, x, i, j, dxi_x, dxi_y, deta_x, deta_y);
    double J0 = dxi_x * deta_y - deta_x * dxi_y;
    double rho = prim[id], vx = prim[g.N + id], vy = prim[2 * g.N + id], p = prim[3 * g.N + id];
    double v2 = vx * vx + vy * vy;
    if (!(rho > 0.0) || !(p > 0.0) || !(v2 < 1.0) || !(J0 > 0.0)) atomicAdd(status + 1, 1);
    double W = 1.0 / sqrt(1.0 - v2);
    double h = 1.0 + gam * p / ((gam - 1.0) * rho);
    double rhW2 = rho * h * W * W;
    J[id] = J0;
    cons[id] = J0 * (rho * W);
    cons[g.N + id] = J0 * (rhW2 * vx);
    cons[2 * g.N + id] = J0 * (rhW2 * vy);
    cons[3 * g.N + id] = J0 * (rhW2 - p);
}

__global__ void k_prim_out(ProbArg pa, double gam, const double *__restrict__ cons, const double *__restrict__ J,
                           double *__restrict__ prim, int *status)
{
    ProbDesc D;
    long long lb;
    locate(pa, D, lb);
    const Geom &g = D.g;
    long long id = lb * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    cons += 4 * D.on;
    J += D.on;
    prim += 4 * D.on;
    double iJ = 1.0 / J[id];
    double rho, vx, vy, p, W;
    int st = cons2prim(gam, cons[id] * iJ, cons[g.N + id] * iJ, cons[2 * g.N + id] * iJ, cons[3 * g.N + id] * iJ,
                       -1.0, rho, vx, vy, p, W);
    if (st) atomicAdd(status, 1);
    prim[id] = rho;
    prim[g.N + id] = vx;
    prim[2 * g.N + id] = vy;
    prim[3 * g.N + id] = p;
}

// totals: per-block partial sums of (J eta, J D, J) ...
__global__ void k_totals(ProbArg pa, double gam, const double *__restrict__ q, const double *__restrict__ cons,
                         const double *__restrict__ J, double *__restrict__ partials)
{
    ProbDesc D;
    long long lb;
    locate(pa, D, lb);
    const Geom &g = D.g;
    long long id = lb * blockDim.x + threadIdx.x;
    q += (long long)NQ * D.op;
    cons += 4 * D.on;
    J += D.on;
    double v[3] = {0.0, 0.0, 0.0};
    if (id < g.N) {
        int i = (int)(id % g.nx), j = (int)(id / g.nx);
        long long c = pidx(g, i, j);
        double rho = q[Q_RHO * g.P + c], W = q[Q_W * g.P + c];
        double lnr = q[Q_LNR * g.P + c], lnb = q[Q_LNB * g.P + c];
        double s = (lnr - lnb) - gam * lnr;        // ln(p / rho^Gamma)
        if (owned_row(g, j)) {
            v[0] = J[id] * (-rho * W * s / (gam - 1.0));
            v[1] = cons[id];
            v[2] = J[id];
        }
    }
    for (int k = 0; k < 3; ++k) {
        double s = block_reduce<2>(v[k]);
        if (threadIdx.x == 0) partials[(long long)blockIdx.x * 3 + k] = s;
    }
}

// ... then a fixed-order sum per problem (deterministic): one thread per
// (problem, quantity) walks the blocks of its problem
__global__ void k_totals_final(int nprob, int nb, const int2 *__restrict__ tiles, const double *__restrict__ partials,
                               double *__restrict__ out)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * nprob) return;
    int b = t / 3, k = t % 3;
    double s = 0.0;
    for (int blk = 0; blk < nb; ++blk)
        if (!tiles || tiles[blk].x == b) s += partials[(long long)blk * 3 + k];
    out[t] = s;
}

}  // namespace esmm
