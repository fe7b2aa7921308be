// esmm_api.cu -- grid handle, per-node / update / CFL / mesh / totals kernels
// and the C ABI declared in include/esmm.h.
//
// One right-hand-side evaluation (eqs. RMHDSemiU_O2p_ES / RMHDSemiJ_O2p_ES of
// Duan & Tang, arXiv 2107.12027, with B = 0) is four kinds of launch:
//   k_node   per padded node: primitive recovery (FP64 Newton), W, u, beta,
//            ln rho, ln beta, CMM metrics (eq. SCLCoeff / App. B) and
//            temporal metrics (eq. VCLCoeff), with the boundary conditions
//            applied by index mapping (ghost layers of width 3);
//   k_pairs  per direction: every two-point EC flux once (esmm_flux.cuh);
//   k_iface  per direction: the ES interface flux (esmm_flux.cuh);
//   k_update per node: flux differences, written as d/dt or fused with the
//            SSP-RK3 combination of the stage.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <mutex>
#include <utility>
#include <vector>

#include "esmm.h"
#include "esmm_device.cuh"
#include "esmm_launch.h"

using namespace esmm;

struct esmm_grid {
    int dev;
    Geom g;
    double lo[2], hi[2];
    double gamma;
    int p, w;
    esmm_params prm;
    cudaStream_t st;
    int has_state;
    int xdot_zero;            // the grid's xdot buffer is known to be zero
    // state y^n = (cons, J, x), mesh velocity, stage buffers
    double *cons, *J, *x, *xdot;
    double *c1, *J1, *x1, *c2, *J2, *x2;
    // right-hand-side work arrays
    double *q;                // [NQ][P]
    double *pg[2];            // pressure warm starts (ping-pong) [N]
    int pgi;
    void *pairs;              // [2][PMAX][4][P] of the working precision
    void *iflux;              // [2][5][P] of the working precision
    double *in_cons, *in_J, *in_x, *in_xdot, *out_dc, *out_dJ;  // host-mode staging
    // mesh redistribution
    double *grad, *om, *om2, *X, *Xn;
    unsigned long long *red;  // [0] max |grad sigma|, [1] Delta tau (min), [2..3] max rho_k
    double *dt_dev, *t_dev;
    double *partials;         // totals: per-block partial sums
    int *status;              // [0] failed primitive recoveries
    double *pin;              // pinned host scalars
    char msg[256];
    // profiling: launches per kind, CUDA events around the kinds in prof_mask
    int prof_mask;
    long long launches[ESMM_NKINDS];
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> *ev;   // [ESMM_NKINDS]
    std::vector<cudaEvent_t> *pool;
};

namespace {

constexpr int BS = 256;

inline unsigned nblk(long long n, int bs = BS) { return (unsigned)((n + bs - 1) / bs); }

cudaEvent_t pool_get(esmm_grid *g)
{
    if (!g->pool->empty()) {
        cudaEvent_t e = g->pool->back();
        g->pool->pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Counts one launch of a kind and, when the kind is profiled, brackets the
// launches issued during its lifetime with CUDA events on the grid's stream.
struct Prof {
    esmm_grid *g;
    int kind;
    cudaEvent_t a = nullptr;
    Prof(esmm_grid *g_, int kind_, int n = 1) : g(g_), kind(kind_)
    {
        g->launches[kind] += n;
        if (g->prof_mask & (1 << kind)) {
            a = pool_get(g);
            cudaEventRecord(a, g->st);
        }
    }
    ~Prof()
    {
        if (a) {
            cudaEvent_t b = pool_get(g);
            cudaEventRecord(b, g->st);
            g->ev[kind].push_back({a, b});
        }
    }
};

// ---------------------------------------------------------------------------
// block reductions (warp shuffles, then one value per warp through shared memory)
__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_min(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// op: 0 max, 1 min, 2 sum; result valid in thread 0
template <int OP>
__device__ double block_reduce(double v)
{
    __shared__ double sh[32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = OP == 0 ? warp_max(v) : (OP == 1 ? warp_min(v) : warp_sum(v));
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    if (wid == 0) {
        double init = OP == 0 ? 0.0 : (OP == 1 ? 1.0e300 : 0.0);
        v = lane < nw ? sh[lane] : init;
        v = OP == 0 ? warp_max(v) : (OP == 1 ? warp_min(v) : warp_sum(v));
    }
    return v;
}

// Non-negative doubles order like their bit patterns, so the global max/min
// of such values is an integer atomic on the bits.
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *a, double v)
{
    atomicMax(a, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ void atomic_min_nonneg(unsigned long long *a, double v)
{
    atomicMin(a, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ double bits_to_double(unsigned long long b) { return __longlong_as_double((long long)b); }

// ---------------------------------------------------------------------------
struct MetricCoef { double a[PMAX]; int p; };

// delta_k[a] = 1/2 sum_n alpha_{p,n} (a_{+n} - a_{-n}) of a mesh coordinate
__device__ __forceinline__ double delta_mesh(const Geom &g, const MetricCoef &mc, const double *x,
                                             int i, int j, int comp, int k)
{
    double d = 0.0;
    for (int n = 1; n <= mc.p; ++n) {
        double ap = k == 0 ? mesh_at(g, x, i + n, j, comp, 1) : mesh_at(g, x, i, j + n, comp, 1);
        double am = k == 0 ? mesh_at(g, x, i - n, j, comp, 1) : mesh_at(g, x, i, j - n, comp, 1);
        d += 0.5 * mc.a[n - 1] * (ap - am);
    }
    return d;
}

// alpha_{p,n} of eq. HOCoeff as compile-time constants
template <int P> __device__ __forceinline__ constexpr double alpha_c(int n)
{
    return P == 1 ? 1.0
                  : (P == 2 ? (n == 1 ? 4.0 / 3.0 : -1.0 / 6.0)
                            : (n == 1 ? 1.5 : (n == 2 ? -0.3 : 1.0 / 30.0)));
}

// The four differences delta_xi[x], delta_xi[y], delta_eta[x], delta_eta[y]
// at node (I, J) of the padded grid.  Nodes whose stencil stays inside the
// mesh read it directly; the others go through the boundary mapping.
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

template <int P>
__global__ void k_node(Geom g, double gam, const double *__restrict__ cons, const double *__restrict__ J,
                       const double *__restrict__ x, const double *__restrict__ xdot,
                       const double *__restrict__ pg_in, double *__restrict__ pg_out, double *__restrict__ q,
                       int *__restrict__ status)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.P) return;
    int I = (int)(t % g.px) - GH, Jn = (int)(t / g.px) - GH;
    long long src = data_src(g, I, Jn);
    double iJ = __drcp_rn(J[src]);
    double D = cons[src] * iJ, mx = cons[g.N + src] * iJ, my = cons[2 * g.N + src] * iJ,
           E = cons[3 * g.N + src] * iJ;
    double rho, vx, vy, p;
    int st = cons2prim(gam, D, mx, my, E, pg_in ? pg_in[src] : -1.0, rho, vx, vy, p);
    bool interior = I >= 0 && I < g.nx && Jn >= 0 && Jn < g.ny;
    if (interior) {
        if (st) atomicAdd(status, 1);
        if (pg_out) pg_out[src] = p;
    }
    double W = rsqrt(1.0 - (vx * vx + vy * vy));
    double beta = rho * __drcp_rn(p);
    q[Q_RHO * g.P + t] = rho;
    q[Q_P * g.P + t] = p;
    q[Q_BETA * g.P + t] = beta;
    q[Q_UX * g.P + t] = W * vx;
    q[Q_UY * g.P + t] = W * vy;
    q[Q_W * g.P + t] = W;
    q[Q_LNR * g.P + t] = log(rho);
    q[Q_LNB * g.P + t] = log(beta);
    // App. B with index-space computational coordinates
    double dxi_x, dxi_y, deta_x, deta_y;
    mesh_deltas<P>(g, x, I, Jn, dxi_x, dxi_y, deta_x, deta_y);
    double M00 = deta_y, M01 = -deta_x, M10 = -dxi_y, M11 = dxi_x;
    q[Q_M00 * g.P + t] = M00;
    q[Q_M01 * g.P + t] = M01;
    q[Q_M10 * g.P + t] = M10;
    q[Q_M11 * g.P + t] = M11;
    double xd = 0.0, yd = 0.0;
    if (xdot) { xd = mesh_at(g, xdot, I, Jn, 0, 0); yd = mesh_at(g, xdot, I, Jn, 1, 0); }
    q[Q_MT0 * g.P + t] = -(xd * M00 + yd * M01);
    q[Q_MT1 * g.P + t] = -(xd * M10 + yd * M11);
}

void launch_node(int p, const Geom &G, double gam, const double *cons, const double *J, const double *x, const double *xdot, const double *pg_in, double *pg_out, double *q, int *status, cudaStream_t st)
{
    const unsigned nb = (unsigned)((G.P + 255) / 256);
    if (p == 1) k_node<1><<<nb, 256, 0, st>>>(G, gam, cons, J, x, xdot, pg_in, pg_out, q, status);
    else if (p == 2) k_node<2><<<nb, 256, 0, st>>>(G, gam, cons, J, x, xdot, pg_in, pg_out, q, status);
    else k_node<3><<<nb, 256, 0, st>>>(G, gam, cons, J, x, xdot, pg_in, pg_out, q, status);
}

// temporal metrics only (the spatial ones and the state are unchanged)
__global__ void k_tmetric(Geom g, const double *__restrict__ xdot, double *__restrict__ q)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.P) return;
    int I = (int)(t % g.px) - GH, Jn = (int)(t / g.px) - GH;
    double xd = mesh_at(g, xdot, I, Jn, 0, 0), yd = mesh_at(g, xdot, I, Jn, 1, 0);
    q[Q_MT0 * g.P + t] = -(xd * q[Q_M00 * g.P + t] + yd * q[Q_M01 * g.P + t]);
    q[Q_MT1 * g.P + t] = -(xd * q[Q_M10 * g.P + t] + yd * q[Q_M11 * g.P + t]);
}

// d/dt = -sum_k (F_k(i + 1/2) - F_k(i - 1/2)); written out (dcons != NULL) or
// combined into the SSP-RK3 stage  y_o = A y_n + B (y_s + dt L)  of (cons, J)
// and of the mesh x with velocity xdot.
template <typename R>
__global__ void k_update(Geom g, const R *__restrict__ fl, double *__restrict__ dcons, double *__restrict__ dJ,
                         const double *__restrict__ cn, const double *__restrict__ Jn_,
                         const double *__restrict__ xn, const double *__restrict__ cs,
                         const double *__restrict__ Js, const double *__restrict__ xs,
                         const double *__restrict__ xdot, double A, double B,
                         const double *__restrict__ dt_dev, double *__restrict__ co, double *__restrict__ Jo,
                         double *__restrict__ xo)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    int i = (int)(id % g.nx), j = (int)(id / g.nx);
    long long c = pidx(g, i, j);
    const R *f0 = fl, *f1 = fl + 5 * g.P;
    double L[5];
#pragma unroll
    for (int a = 0; a < 5; ++a) {
        double d0 = (double)f0[a * g.P + c] - (double)f0[a * g.P + c - 1];
        double d1 = (double)f1[a * g.P + c] - (double)f1[a * g.P + c - g.px];
        L[a] = -(d0 + d1);
    }
    if (dcons) {
#pragma unroll
        for (int a = 0; a < 4; ++a) dcons[a * g.N + id] = L[a];
        dJ[id] = L[4];
        return;
    }
    double dt = *dt_dev;
#pragma unroll
    for (int a = 0; a < 4; ++a) co[a * g.N + id] = A * cn[a * g.N + id] + B * (cs[a * g.N + id] + dt * L[a]);
    Jo[id] = A * Jn_[id] + B * (Js[id] + dt * L[4]);
    xo[id] = A * xn[id] + B * (xs[id] + dt * xdot[id]);
    xo[g.N + id] = A * xn[g.N + id] + B * (xs[g.N + id] + dt * xdot[g.N + id]);
}

// spectral radius rho_k = L_k max |lambda_+-| / J at every node (static mesh)
__global__ void k_cfl(Geom g, double gam, const double *__restrict__ q, const double *__restrict__ J,
                      unsigned long long *red)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double r[2] = {0.0, 0.0};
    if (id < g.N) {
        int i = (int)(id % g.nx), j = (int)(id / g.nx);
        long long c = pidx(g, i, j);
        double rho = q[Q_RHO * g.P + c], p = q[Q_P * g.P + c], W = q[Q_W * g.P + c];
        double vx = q[Q_UX * g.P + c] / W, vy = q[Q_UY * g.P + c] / W;
        double v2 = vx * vx + vy * vy;
        double rh = rho + gam * p / (gam - 1.0);
        double c2 = gam * p / rh, cs = sqrt(c2);
        for (int k = 0; k < 2; ++k) {
            double mx = q[(Q_M00 + 2 * k) * g.P + c], my = q[(Q_M01 + 2 * k) * g.P + c];
            double Lk = sqrt(mx * mx + my * my);
            double vn = (mx * vx + my * vy) / Lk;
            double disc = sqrt((1.0 - v2) * (1.0 - v2 * c2 - vn * vn * (1.0 - c2)));
            double den = 1.0 - v2 * c2;
            double lm = (vn * (1.0 - c2) - cs * disc) / den, lp = (vn * (1.0 - c2) + cs * disc) / den;
            r[k] = Lk * fmax(fabs(lm), fabs(lp)) / J[id];
        }
    }
    for (int k = 0; k < 2; ++k) {
        double m = block_reduce<0>(r[k]);
        if (threadIdx.x == 0) atomic_max_nonneg(red + 2 + k, m);
        __syncthreads();
    }
}

__global__ void k_red_init(unsigned long long *red)
{
    red[0] = 0ull;
    red[1] = (unsigned long long)__double_as_longlong(1.0);
    red[2] = 0ull;
    red[3] = 0ull;
}

__global__ void k_dt(double cfl, double dt_fixed, const unsigned long long *red, double *dt_dev)
{
    dt_dev[0] = dt_fixed > 0.0 ? dt_fixed : cfl / (bits_to_double(red[2]) + bits_to_double(red[3]));
}

__global__ void k_time(const double *dt_dev, double *t_dev) { t_dev[0] += dt_dev[0]; }

// ---- Sec. 5 mesh redistribution -------------------------------------------
__global__ void k_mesh_grad(Geom g, int lnrho, const double *__restrict__ q, double *__restrict__ grad,
                            unsigned long long *red)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double gv = 0.0;
    if (id < g.N) {
        int i = (int)(id % g.nx), j = (int)(id / g.nx);
        long long c = pidx(g, i, j);
        const double *s = q + (lnrho ? Q_LNR : Q_RHO) * g.P;
        double gx = 0.5 * (s[c + 1] - s[c - 1]);
        double gy = 0.5 * (s[c + g.px] - s[c - g.px]);
        gv = sqrt(gx * gx + gy * gy);
        grad[id] = gv;
    }
    double m = block_reduce<0>(gv);
    if (threadIdx.x == 0) atomic_max_nonneg(red, m);
}

__global__ void k_mesh_omega(Geom g, double alpha, const double *__restrict__ grad,
                             const unsigned long long *red, double *__restrict__ om)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    double gmax = bits_to_double(red[0]);
    om[id] = gmax > 0.0 ? sqrt(1.0 + alpha * grad[id] / gmax) : 1.0;
}

// omega <- sum_{a,b in {-1,0,1}} 2^-(|a|+|b|+2) omega_{i+a, j+b}
__global__ void k_mesh_filter(Geom g, const double *__restrict__ om, double *__restrict__ om2)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    int i = (int)(id % g.nx), j = (int)(id / g.nx);
    double acc = 0.0;
    for (int b = -1; b <= 1; ++b)
        for (int a = -1; a <= 1; ++a) {
            double wgt = (a == 0 && b == 0) ? 0.25 : ((a == 0 || b == 0) ? 0.125 : 0.0625);
            acc += wgt * om[data_src(g, i + a, j + b)];
        }
    om2[id] = acc;
}

// one Jacobi sweep of the Winslow mesh equations with omega frozen
__global__ void k_mesh_jacobi(Geom g, const double *__restrict__ om, const double *__restrict__ X,
                              double *__restrict__ Xn)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    int i = (int)(id % g.nx), j = (int)(id / g.nx);
    bool fixed = (g.bc0 == 1 && (i == 0 || i == g.nx - 1)) || (g.bc1 == 1 && (j == 0 || j == g.ny - 1));
    if (fixed) {
        Xn[id] = X[id];
        Xn[g.N + id] = X[g.N + id];
        return;
    }
    double wi = om[id];
    double we = om[data_src(g, i + 1, j)], ww = om[data_src(g, i - 1, j)];
    double wn = om[data_src(g, i, j + 1)], ws = om[data_src(g, i, j - 1)];
    double den = (2.0 * wi + we + ww) + (2.0 * wi + wn + ws);
    for (int comp = 0; comp < 2; ++comp) {
        double num = (wi + we) * mesh_at(g, X, i + 1, j, comp, 1) + (wi + ww) * mesh_at(g, X, i - 1, j, comp, 1) +
                     (wi + wn) * mesh_at(g, X, i, j + 1, comp, 1) + (wi + ws) * mesh_at(g, X, i, j - 1, comp, 1);
        Xn[comp * g.N + id] = num / den;
    }
}

// movement limiter: Delta tau = min over nodes and directions of half the
// neighbour spacing over the displacement toward it, clipped to [0, 1]
__global__ void k_mesh_tau(Geom g, const double *__restrict__ x, const double *__restrict__ X,
                           unsigned long long *red)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double tau = 1.0;
    if (id < g.N) {
        int i = (int)(id % g.nx), j = (int)(id / g.nx);
        for (int k = 0; k < 2; ++k) {
            double d = X[k * g.N + id] - x[k * g.N + id];
            int di = k == 0, dj = k == 1;
            double b = 1.0;
            if (d < 0.0) b = -(x[k * g.N + id] - mesh_at(g, x, i - di, j - dj, k, 1)) / (2.0 * d);
            else if (d > 0.0) b = (mesh_at(g, x, i + di, j + dj, k, 1) - x[k * g.N + id]) / (2.0 * d);
            tau = fmin(tau, b);
        }
        tau = fmax(tau, 0.0);
    }
    double m = block_reduce<1>(tau);
    if (threadIdx.x == 0) atomic_min_nonneg(red + 1, m);
}

__global__ void k_mesh_xdot(Geom g, const double *__restrict__ x, const double *__restrict__ X,
                            const unsigned long long *red, const double *__restrict__ dt_dev,
                            double *__restrict__ xdot)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= 2 * g.N) return;
    double tau = bits_to_double(red[1]);
    xdot[id] = tau * (X[id] - x[id]) / dt_dev[0];
}

// ---- state set-up and read-out ----------------------------------------------
__global__ void k_init_state(Geom g, double gam, MetricCoef mc, const double *__restrict__ prim,
                             const double *__restrict__ x, double *__restrict__ cons, double *__restrict__ J,
                             int *status)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    int i = (int)(id % g.nx), j = (int)(id / g.nx);
    double J0 = delta_mesh(g, mc, x, i, j, 0, 0) * delta_mesh(g, mc, x, i, j, 1, 1) -
                delta_mesh(g, mc, x, i, j, 0, 1) * delta_mesh(g, mc, x, i, j, 1, 0);
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

__global__ void k_prim_out(Geom g, double gam, const double *__restrict__ cons, const double *__restrict__ J,
                           double *__restrict__ prim, int *status)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    double iJ = 1.0 / J[id];
    double rho, vx, vy, p;
    int st = cons2prim(gam, cons[id] * iJ, cons[g.N + id] * iJ, cons[2 * g.N + id] * iJ, cons[3 * g.N + id] * iJ,
                       -1.0, rho, vx, vy, p);
    if (st) atomicAdd(status, 1);
    prim[id] = rho;
    prim[g.N + id] = vx;
    prim[2 * g.N + id] = vy;
    prim[3 * g.N + id] = p;
}

// totals: per-block partial sums of (J eta, J D, J), then a fixed-order sum
__global__ void k_totals(Geom g, double gam, const double *__restrict__ q, const double *__restrict__ cons,
                         const double *__restrict__ J, double *__restrict__ partials)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double v[3] = {0.0, 0.0, 0.0};
    if (id < g.N) {
        int i = (int)(id % g.nx), j = (int)(id / g.nx);
        long long c = pidx(g, i, j);
        double rho = q[Q_RHO * g.P + c], W = q[Q_W * g.P + c];
        double lnr = q[Q_LNR * g.P + c], lnb = q[Q_LNB * g.P + c];
        double s = (lnr - lnb) - gam * lnr;        // ln(p / rho^Gamma)
        v[0] = J[id] * (-rho * W * s / (gam - 1.0));
        v[1] = cons[id];
        v[2] = J[id];
    }
    for (int k = 0; k < 3; ++k) {
        double s = block_reduce<2>(v[k]);
        if (threadIdx.x == 0) partials[(long long)blockIdx.x * 3 + k] = s;
        __syncthreads();
    }
}

__global__ void k_totals_final(int nb, const double *__restrict__ partials, double *__restrict__ out)
{
    int k = threadIdx.x;
    if (k >= 3) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partials[(long long)b * 3 + k];
    out[k] = s;
}

// ---------------------------------------------------------------------------
int fail(esmm_grid *g, int code, const char *what, cudaError_t e = cudaSuccess)
{
    if (g) {
        if (e != cudaSuccess) snprintf(g->msg, sizeof g->msg, "%s: %s", what, cudaGetErrorString(e));
        else snprintf(g->msg, sizeof g->msg, "%s", what);
    }
    return code;
}

#define CK(call)                                                     \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return fail(g, ESMM_ERR_CUDA, #call, e_); \
    } while (0)

MetricCoef metric_coef(const esmm_grid *g)
{
    MetricCoef mc;
    mc.p = g->p;
    if (g->p == 1) { mc.a[0] = 1.0; mc.a[1] = 0.0; mc.a[2] = 0.0; }
    else if (g->p == 2) { mc.a[0] = 4.0 / 3.0; mc.a[1] = -1.0 / 6.0; mc.a[2] = 0.0; }
    else { mc.a[0] = 3.0 / 2.0; mc.a[1] = -3.0 / 10.0; mc.a[2] = 1.0 / 30.0; }
    return mc;
}

Phys phys(const esmm_grid *g)
{
    Phys ph;
    MetricCoef mc = metric_coef(g);
    ph.gamma = g->gamma;
    ph.eps = g->prm.weno_eps;
    // FP64: switch to the series below 1e-4 (its dropped term is < 1e-17);
    // FP32 bulk: below 1e-2, where the FP32 quotient would lose ~6 digits.
    ph.ln_thr = g->prm.precision == ESMM_MIXED ? 1.0e-2 : 1.0e-4;
    // sign switch: rounding noise of the projected jump (FP64 / FP32 bulk)
    ph.sign_tol = g->prm.precision == ESMM_MIXED ? 1.0e-5 : 1.0e-10;
    for (int n = 0; n < PMAX; ++n) ph.alpha[n] = mc.a[n];
    ph.p = g->p;
    ph.w = g->w;
    return ph;
}

// node pass + both sweeps + update.  xdot may be NULL (static mesh); warm
// selects the pressure warm start of the grid.
int rhs_core(esmm_grid *g, const double *cons, const double *J, const double *x, const double *xdot, bool warm,
             bool node_done)
{
    const Geom &G = g->g;
    if (!node_done) {
        const double *pin = warm ? g->pg[g->pgi] : nullptr;
        double *pout = warm ? g->pg[1 - g->pgi] : nullptr;
        {
            Prof pr_(g, ESMM_KIND_NODE);
            launch_node(g->p, G, g->gamma, cons, J, x, xdot, pin, pout, g->q, g->status, g->st);
        }
        if (warm) g->pgi = 1 - g->pgi;
    }
    Phys ph = phys(g);
    bool f32 = g->prm.precision == ESMM_MIXED;
    for (int dir = 0; dir < 2; ++dir) {
        if (f32) {
            {
                Prof pr_(g, ESMM_KIND_PAIRS);
                launch_pairs_f32(G, ph, g->q, g->pairs, dir, g->st);
            }
            {
                Prof pr_(g, ESMM_KIND_IFACE);
                launch_iface_f32(G, ph, g->q, g->pairs, g->iflux, dir, g->st);
            }
        } else {
            {
                Prof pr_(g, ESMM_KIND_PAIRS);
                launch_pairs_f64(G, ph, g->q, g->pairs, dir, g->st);
            }
            {
                Prof pr_(g, ESMM_KIND_IFACE);
                launch_iface_f64(G, ph, g->q, g->pairs, g->iflux, dir, g->st);
            }
        }
    }
    CK(cudaGetLastError());
    return ESMM_OK;
}

template <typename R>
void launch_update(esmm_grid *g, double *dcons, double *dJ, const double *cn, const double *Jn,
                   const double *xn, const double *cs, const double *Js, const double *xs, const double *xdot,
                   double A, double B, double *co, double *Jo, double *xo)
{
    const Geom &G = g->g;
    {
        Prof pr_(g, ESMM_KIND_UPDATE);
        k_update<R><<<nblk(G.N), BS, 0, g->st>>>(G, (const R *)g->iflux, dcons, dJ, cn, Jn, xn, cs, Js, xs, xdot, A, B,
                                                 g->dt_dev, co, Jo, xo);
    }
}

void update(esmm_grid *g, double *dcons, double *dJ, const double *cn, const double *Jn, const double *xn,
            const double *cs, const double *Js, const double *xs, const double *xdot, double A, double B,
            double *co, double *Jo, double *xo)
{
    if (g->prm.precision == ESMM_MIXED)
        launch_update<float>(g, dcons, dJ, cn, Jn, xn, cs, Js, xs, xdot, A, B, co, Jo, xo);
    else
        launch_update<double>(g, dcons, dJ, cn, Jn, xn, cs, Js, xs, xdot, A, B, co, Jo, xo);
}

// dt of the step into dt_dev; requires g->q of the state with a static mesh
int step_dt(esmm_grid *g, double dt)
{
    const Geom &G = g->g;
    if (!(dt > 0.0)) { Prof pr_(g, ESMM_KIND_OTHER); k_cfl<<<nblk(G.N), BS, 0, g->st>>>(G, g->gamma, g->q, g->J, g->red); }
    {
        Prof pr_(g, ESMM_KIND_OTHER);
        k_dt<<<1, 1, 0, g->st>>>(g->prm.cfl, dt, g->red, g->dt_dev);
    }
    CK(cudaGetLastError());
    return ESMM_OK;
}

// mesh velocity of the step into g->xdot; requires g->q of the state and dt_dev
int mesh_core(esmm_grid *g)
{
    const Geom &G = g->g;
    if (!g->prm.move_mesh) {
        if (!g->xdot_zero) {
            CK(cudaMemsetAsync(g->xdot, 0, sizeof(double) * 2 * G.N, g->st));
            g->xdot_zero = 1;
        }
        return ESMM_OK;
    }
    g->xdot_zero = 0;
    {
        Prof pr_(g, ESMM_KIND_MESH);
        k_mesh_grad<<<nblk(G.N), BS, 0, g->st>>>(G, g->prm.monitor == ESMM_MONITOR_LNRHO, g->q, g->grad, g->red);
    }
    {
        Prof pr_(g, ESMM_KIND_MESH);
        k_mesh_omega<<<nblk(G.N), BS, 0, g->st>>>(G, g->prm.alpha, g->grad, g->red, g->om);
    }
    for (int f = 0; f < g->prm.n_filter; ++f) {
        {
            Prof pr_(g, ESMM_KIND_MESH);
            k_mesh_filter<<<nblk(G.N), BS, 0, g->st>>>(G, g->om, g->om2);
        }
        double *t = g->om; g->om = g->om2; g->om2 = t;
    }
    const double *src = g->x;
    for (int nu = 0; nu < g->prm.mu; ++nu) {
        double *dst = (nu % 2 == 0) ? g->X : g->Xn;
        {
            Prof pr_(g, ESMM_KIND_MESH);
            k_mesh_jacobi<<<nblk(G.N), BS, 0, g->st>>>(G, g->om, src, dst);
        }
        src = dst;
    }
    {
        Prof pr_(g, ESMM_KIND_MESH);
        k_mesh_tau<<<nblk(G.N), BS, 0, g->st>>>(G, g->x, src, g->red);
    }
    {
        Prof pr_(g, ESMM_KIND_MESH);
        k_mesh_xdot<<<nblk(2 * G.N), BS, 0, g->st>>>(G, g->x, src, g->red, g->dt_dev, g->xdot);
    }
    CK(cudaGetLastError());
    return ESMM_OK;
}

int rk_step_async(esmm_grid *g, double dt)
{
    const Geom &G = g->g;
    int rc;
    // state's node data with a static mesh: CFL step and monitor (Sec. 5)
    {
        Prof pr_(g, ESMM_KIND_NODE);
        launch_node(g->p, G, g->gamma, g->cons, g->J, g->x, nullptr, g->pg[g->pgi], g->pg[1 - g->pgi], g->q, g->status, g->st);
    }
    g->pgi = 1 - g->pgi;
    {
        Prof pr_(g, ESMM_KIND_OTHER);
        k_red_init<<<1, 1, 0, g->st>>>(g->red);
    }
    if ((rc = step_dt(g, dt))) return rc;
    if ((rc = mesh_core(g))) return rc;
    // stage 1: y1 = y^n + dt L(y^n); only the temporal metrics change
    {
        Prof pr_(g, ESMM_KIND_NODE);
        k_tmetric<<<nblk(G.P), BS, 0, g->st>>>(G, g->xdot, g->q);
    }
    if ((rc = rhs_core(g, g->cons, g->J, g->x, g->xdot, true, true))) return rc;
    update(g, nullptr, nullptr, g->cons, g->J, g->x, g->cons, g->J, g->x, g->xdot, 0.0, 1.0, g->c1, g->J1, g->x1);
    // stage 2: y2 = 3/4 y^n + 1/4 (y1 + dt L(y1))
    if ((rc = rhs_core(g, g->c1, g->J1, g->x1, g->xdot, true, false))) return rc;
    update(g, nullptr, nullptr, g->cons, g->J, g->x, g->c1, g->J1, g->x1, g->xdot, 0.75, 0.25, g->c2, g->J2, g->x2);
    // stage 3: y^{n+1} = 1/3 y^n + 2/3 (y2 + dt L(y2)), in place
    if ((rc = rhs_core(g, g->c2, g->J2, g->x2, g->xdot, true, false))) return rc;
    update(g, nullptr, nullptr, g->cons, g->J, g->x, g->c2, g->J2, g->x2, g->xdot, 1.0 / 3.0, 2.0 / 3.0, g->cons,
           g->J, g->x);
    {
        Prof pr_(g, ESMM_KIND_OTHER);
        k_time<<<1, 1, 0, g->st>>>(g->dt_dev, g->t_dev);
    }
    CK(cudaGetLastError());
    return ESMM_OK;
}

int check_c2p(esmm_grid *g)
{
    int h[2];
    CK(cudaMemcpyAsync(h, g->status, sizeof h, cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    if (h[0] > 0) {
        CK(cudaMemsetAsync(g->status, 0, sizeof(int), g->st));
        snprintf(g->msg, sizeof g->msg, "primitive recovery failed at %d node(s)", h[0]);
        return ESMM_ERR_C2P;
    }
    return ESMM_OK;
}

void free_all(esmm_grid *g)
{
    double **bufs[] = {&g->cons, &g->J, &g->x, &g->xdot, &g->c1, &g->J1, &g->x1, &g->c2, &g->J2, &g->x2,
                       &g->q, &g->pg[0], &g->pg[1], &g->in_cons, &g->in_J, &g->in_x, &g->in_xdot,
                       &g->out_dc, &g->out_dJ, &g->grad, &g->om, &g->om2, &g->X, &g->Xn, &g->dt_dev,
                       &g->t_dev, &g->partials};
    for (double **b : bufs)
        if (*b) { cudaFree(*b); *b = nullptr; }
    if (g->pairs) cudaFree(g->pairs);
    if (g->iflux) cudaFree(g->iflux);
    if (g->red) cudaFree(g->red);
    if (g->status) cudaFree(g->status);
    if (g->pin) cudaFreeHost(g->pin);
    if (g->ev) {
        for (int k = 0; k < ESMM_NKINDS; ++k)
            for (auto &pr : g->ev[k]) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
        delete[] g->ev;
        g->ev = nullptr;
    }
    if (g->pool) {
        for (cudaEvent_t e : *g->pool) cudaEventDestroy(e);
        delete g->pool;
        g->pool = nullptr;
    }
    g->pairs = g->iflux = nullptr;
    g->red = nullptr;
    g->status = nullptr;
    g->pin = nullptr;
}

int copy_in(esmm_grid *g, double *dst, const double *src, size_t n, int mem)
{
    CK(cudaMemcpyAsync(dst, src, n * sizeof(double),
                       mem == ESMM_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g->st));
    return ESMM_OK;
}

int copy_out(esmm_grid *g, double *dst, const double *src, size_t n, int mem)
{
    CK(cudaMemcpyAsync(dst, src, n * sizeof(double),
                       mem == ESMM_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->st));
    return ESMM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Allocation-free right-hand side (esmm_rhs_static).
//
// Its scratch lives in one file-scope device array: per padded node the NQ
// node arrays, the pair fluxes [2][PMAX][4] and the interface fluxes [2][5]
// (48 doubles), then two status ints.  Every GPU that loads the library holds
// this array until the process exits.  Host code only ever passes the
// device address obtained from cudaGetSymbolAddress: in host code the
// array's name is a host-side stand-in, not a device address.
constexpr long long STATIC_PER_NODE = NQ + 2 * PMAX * 4 + 2 * 5;
constexpr long long STATIC_DOUBLES = STATIC_PER_NODE * ESMM_STATIC_MAX_PADDED_NODES + 32;
static __device__ __align__(256) double esmm_static_scratch[STATIC_DOUBLES];

namespace {
constexpr int STATIC_MAX_DEVICES = 64;
std::mutex static_mu;
double *static_ptr[STATIC_MAX_DEVICES];     // device address per device, set once

// Device address of the scratch on the current device (set-up on the first
// call per device, with that device current).
cudaError_t static_scratch(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= STATIC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(static_mu);
    if (!static_ptr[dev]) {
        double *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, esmm_static_scratch);
        if (e != cudaSuccess) return e;
        static_ptr[dev] = p;
    }
    *out = static_ptr[dev];
    return cudaSuccess;
}
}  // namespace

// ===========================================================================
extern "C" {

const char *esmm_version(void) { return "esmm 0.1 (2D RHD, sm_103a)"; }

int esmm_grid_create(esmm_grid **out, int dim, const int n[3], const double lo[3], const double hi[3], int phys,
                     const int bc[3], void *stream)
{
    esmm_grid *g = nullptr;
    if (!out || !n || !lo || !hi || !bc) return ESMM_ERR_ARG;
    *out = nullptr;
    if (dim != 2 || phys != ESMM_RHD) return ESMM_ERR_ARG;
    for (int k = 0; k < 2; ++k) {
        if (n[k] < 4 || n[k] > (1 << 15)) return ESMM_ERR_ARG;
        if (bc[k] != ESMM_PERIODIC && bc[k] != ESMM_OUTFLOW) return ESMM_ERR_ARG;
        if (!(hi[k] > lo[k])) return ESMM_ERR_ARG;
    }
    g = new (std::nothrow) esmm_grid;
    if (!g) return ESMM_ERR_ARG;
    memset(g, 0, sizeof *g);
    g->ev = new (std::nothrow) std::vector<std::pair<cudaEvent_t, cudaEvent_t>>[ESMM_NKINDS];
    g->pool = new (std::nothrow) std::vector<cudaEvent_t>;
    if (!g->ev || !g->pool || cudaGetDevice(&g->dev) != cudaSuccess) {
        free_all(g);
        delete g;
        return ESMM_ERR_CUDA;
    }
    g->st = (cudaStream_t)stream;
    Geom &G = g->g;
    G.nx = n[0];
    G.ny = n[1];
    G.px = G.nx + 2 * GH;
    G.py = G.ny + 2 * GH;
    G.P = (long long)G.px * G.py;
    G.N = (long long)G.nx * G.ny;
    G.bc0 = bc[0];
    G.bc1 = bc[1];
    G.per0 = hi[0] - lo[0];
    G.per1 = hi[1] - lo[1];
    for (int k = 0; k < 2; ++k) { g->lo[k] = lo[k]; g->hi[k] = hi[k]; }
    g->gamma = 5.0 / 3.0;
    g->p = 2;
    g->w = 5;
    g->prm.cfl = 0.4;
    g->prm.weno_eps = 1e-6;
    g->prm.monitor = ESMM_MONITOR_LNRHO;
    g->prm.alpha = 20.0;
    g->prm.n_filter = 4;
    g->prm.mu = 10;
    g->prm.move_mesh = 1;
    g->prm.precision = ESMM_FP64;

    size_t N = (size_t)G.N, P = (size_t)G.P, d = sizeof(double);
    struct { double **p; size_t n; } al[] = {
        {&g->cons, 4 * N}, {&g->J, N}, {&g->x, 2 * N}, {&g->xdot, 2 * N}, {&g->c1, 4 * N}, {&g->J1, N},
        {&g->x1, 2 * N}, {&g->c2, 4 * N}, {&g->J2, N}, {&g->x2, 2 * N}, {&g->q, (size_t)NQ * P},
        {&g->pg[0], N}, {&g->pg[1], N}, {&g->in_cons, 4 * N}, {&g->in_J, N}, {&g->in_x, 2 * N},
        {&g->in_xdot, 2 * N}, {&g->out_dc, 4 * N}, {&g->out_dJ, N}, {&g->grad, N}, {&g->om, N}, {&g->om2, N},
        {&g->X, 2 * N}, {&g->Xn, 2 * N}, {&g->dt_dev, 1}, {&g->t_dev, 1}, {&g->partials, 3 * (N / BS + 2)}};
    for (auto &a : al) {
        cudaError_t e = cudaMalloc((void **)a.p, a.n * d);
        if (e != cudaSuccess) { free_all(g); delete g; return ESMM_ERR_CUDA; }
    }
    if (cudaMalloc(&g->pairs, (size_t)2 * PMAX * 4 * P * d) != cudaSuccess ||
        cudaMalloc(&g->iflux, (size_t)2 * 5 * P * d) != cudaSuccess ||
        cudaMalloc((void **)&g->red, 8 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc((void **)&g->status, 2 * sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void **)&g->pin, 16 * sizeof(double)) != cudaSuccess) {
        free_all(g);
        delete g;
        return ESMM_ERR_CUDA;
    }
    // initial (cold) pressure guesses: the bracket midpoint
    if (cudaMemsetAsync(g->pg[0], 0xff, N * d, g->st) != cudaSuccess ||
        cudaMemsetAsync(g->pg[1], 0xff, N * d, g->st) != cudaSuccess ||
        cudaMemsetAsync(g->status, 0, 2 * sizeof(int), g->st) != cudaSuccess ||
        cudaMemsetAsync(g->t_dev, 0, d, g->st) != cudaSuccess ||
        cudaStreamSynchronize(g->st) != cudaSuccess) {
        free_all(g);
        delete g;
        return ESMM_ERR_CUDA;
    }
    *out = g;
    return ESMM_OK;
}

int esmm_grid_destroy(esmm_grid *g)
{
    if (!g) return ESMM_ERR_ARG;
    cudaStreamSynchronize(g->st);
    free_all(g);
    delete g;
    return ESMM_OK;
}

int esmm_set_stream(esmm_grid *g, void *stream)
{
    if (!g) return ESMM_ERR_ARG;
    CK(cudaStreamSynchronize(g->st));
    g->st = (cudaStream_t)stream;
    return ESMM_OK;
}

int esmm_set_eos(esmm_grid *g, double gamma)
{
    if (!g || !(gamma > 1.0 && gamma <= 2.0)) return fail(g, ESMM_ERR_ARG, "Gamma must be in (1, 2]");
    g->gamma = gamma;
    return ESMM_OK;
}

int esmm_set_order(esmm_grid *g, int p, int w)
{
    if (!g || p < 1 || p > PMAX || !(w == 0 || w == 3 || w == 5))
        return fail(g, ESMM_ERR_ARG, "p must be 1..3 and w one of 0, 3, 5");
    g->p = p;
    g->w = w;
    return ESMM_OK;
}

int esmm_set_params(esmm_grid *g, const esmm_params *prm)
{
    if (!g || !prm) return ESMM_ERR_ARG;
    if (!(prm->cfl > 0.0) || !(prm->weno_eps > 0.0) || !(prm->alpha >= 0.0) || prm->n_filter < 0 ||
        prm->mu < 0 || (prm->precision != ESMM_FP64 && prm->precision != ESMM_MIXED) ||
        (prm->monitor != ESMM_MONITOR_RHO && prm->monitor != ESMM_MONITOR_LNRHO))
        return fail(g, ESMM_ERR_ARG, "invalid parameter");
    g->prm = *prm;
    return ESMM_OK;
}

int esmm_get_params(const esmm_grid *g, esmm_params *prm)
{
    if (!g || !prm) return ESMM_ERR_ARG;
    *prm = g->prm;
    return ESMM_OK;
}

int esmm_state_set(esmm_grid *g, const double *prim, const double *x, int mem)
{
    if (!g || !prim) return ESMM_ERR_ARG;
    const Geom &G = g->g;
    size_t N = (size_t)G.N;
    if (x) {
        int rc = copy_in(g, g->x, x, 2 * N, mem);
        if (rc) return rc;
    } else {
        double *hx = (double *)malloc(2 * N * sizeof(double));
        if (!hx) return ESMM_ERR_ARG;
        for (int j = 0; j < G.ny; ++j)
            for (int i = 0; i < G.nx; ++i) {
                int nx_ = G.bc0 == ESMM_PERIODIC ? G.nx : G.nx - 1;
                int ny_ = G.bc1 == ESMM_PERIODIC ? G.ny : G.ny - 1;
                hx[(size_t)j * G.nx + i] = g->lo[0] + (g->hi[0] - g->lo[0]) * i / nx_;
                hx[N + (size_t)j * G.nx + i] = g->lo[1] + (g->hi[1] - g->lo[1]) * j / ny_;
            }
        cudaError_t e = cudaMemcpyAsync(g->x, hx, 2 * N * sizeof(double), cudaMemcpyHostToDevice, g->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
        free(hx);
        if (e != cudaSuccess) return fail(g, ESMM_ERR_CUDA, "mesh upload", e);
    }
    int rc = copy_in(g, g->in_cons, prim, 4 * N, mem);
    if (rc) return rc;
    CK(cudaMemsetAsync(g->status, 0, 2 * sizeof(int), g->st));
    {
        Prof pr_(g, ESMM_KIND_NODE);
        k_init_state<<<nblk(G.N), BS, 0, g->st>>>(G, g->gamma, metric_coef(g), g->in_cons, g->x, g->cons, g->J,
                                                  g->status);
    }
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(g->xdot, 0, 2 * N * sizeof(double), g->st));
    CK(cudaMemsetAsync(g->pg[0], 0xff, N * sizeof(double), g->st));
    CK(cudaMemsetAsync(g->pg[1], 0xff, N * sizeof(double), g->st));
    CK(cudaMemsetAsync(g->t_dev, 0, sizeof(double), g->st));
    int h[2];
    CK(cudaMemcpyAsync(h, g->status, sizeof h, cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    g->xdot_zero = 1;
    if (h[1] > 0) {
        CK(cudaMemsetAsync(g->status, 0, 2 * sizeof(int), g->st));
        g->has_state = 0;
        return fail(g, ESMM_ERR_ARG, "non-admissible initial state or tangled mesh");
    }
    g->has_state = 1;
    return ESMM_OK;
}

int esmm_state_set_cons(esmm_grid *g, const double *cons, const double *J, const double *x, double t, int mem)
{
    if (!g || !cons || !J || !x) return ESMM_ERR_ARG;
    size_t N = (size_t)g->g.N;
    int rc;
    if ((rc = copy_in(g, g->cons, cons, 4 * N, mem)) || (rc = copy_in(g, g->J, J, N, mem)) ||
        (rc = copy_in(g, g->x, x, 2 * N, mem)))
        return rc;
    g->pin[0] = t;
    CK(cudaMemcpyAsync(g->t_dev, g->pin, sizeof(double), cudaMemcpyHostToDevice, g->st));
    CK(cudaMemsetAsync(g->xdot, 0, 2 * N * sizeof(double), g->st));
    CK(cudaMemsetAsync(g->pg[0], 0xff, N * sizeof(double), g->st));
    CK(cudaMemsetAsync(g->pg[1], 0xff, N * sizeof(double), g->st));
    CK(cudaStreamSynchronize(g->st));
    g->xdot_zero = 1;
    g->has_state = 1;
    return ESMM_OK;
}

int esmm_state_get(esmm_grid *g, int what, double *out, int mem)
{
    if (!g || !out) return ESMM_ERR_ARG;
    if (!g->has_state) return fail(g, ESMM_ERR_STATE, "no state");
    size_t N = (size_t)g->g.N;
    int rc = ESMM_OK;
    switch (what) {
    case ESMM_GET_PRIM:
        {
            Prof pr_(g, ESMM_KIND_NODE);
            k_prim_out<<<nblk(g->g.N), BS, 0, g->st>>>(g->g, g->gamma, g->cons, g->J, g->out_dc, g->status);
        }
        CK(cudaGetLastError());
        rc = copy_out(g, out, g->out_dc, 4 * N, mem);
        break;
    case ESMM_GET_CONS: rc = copy_out(g, out, g->cons, 4 * N, mem); break;
    case ESMM_GET_J: rc = copy_out(g, out, g->J, N, mem); break;
    case ESMM_GET_X: rc = copy_out(g, out, g->x, 2 * N, mem); break;
    case ESMM_GET_XDOT: rc = copy_out(g, out, g->xdot, 2 * N, mem); break;
    default: return fail(g, ESMM_ERR_ARG, "unknown field");
    }
    if (rc) return rc;
    CK(cudaStreamSynchronize(g->st));
    if (what == ESMM_GET_PRIM) return check_c2p(g);
    return ESMM_OK;
}

int esmm_get_time(esmm_grid *g, double *t)
{
    if (!g || !t) return ESMM_ERR_ARG;
    CK(cudaMemcpyAsync(g->pin, g->t_dev, sizeof(double), cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    *t = g->pin[0];
    return ESMM_OK;
}

int esmm_rhs(esmm_grid *g, const double *cons, const double *J, const double *x, const double *xdot,
             double *dcons, double *dJ, int mem)
{
    if (!g || !cons || !J || !x || !dcons || !dJ) return ESMM_ERR_ARG;
    size_t N = (size_t)g->g.N;
    int rc;
    if (mem == ESMM_MEM_HOST) {
        if ((rc = copy_in(g, g->in_cons, cons, 4 * N, mem)) || (rc = copy_in(g, g->in_J, J, N, mem)) ||
            (rc = copy_in(g, g->in_x, x, 2 * N, mem)))
            return rc;
        if (xdot && (rc = copy_in(g, g->in_xdot, xdot, 2 * N, mem))) return rc;
        cons = g->in_cons;
        J = g->in_J;
        x = g->in_x;
        xdot = xdot ? g->in_xdot : nullptr;
    }
    if ((rc = rhs_core(g, cons, J, x, xdot, false, false))) return rc;
    double *dc = mem == ESMM_MEM_HOST ? g->out_dc : dcons;
    double *dj = mem == ESMM_MEM_HOST ? g->out_dJ : dJ;
    update(g, dc, dj, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, 0.0, nullptr, nullptr,
           nullptr);
    CK(cudaGetLastError());
    if (mem == ESMM_MEM_HOST) {
        if ((rc = copy_out(g, dcons, g->out_dc, 4 * N, mem)) || (rc = copy_out(g, dJ, g->out_dJ, N, mem)))
            return rc;
        CK(cudaStreamSynchronize(g->st));
        return check_c2p(g);
    }
    return ESMM_OK;
}

int esmm_cfl_dt(esmm_grid *g, double *dt)
{
    if (!g || !dt) return ESMM_ERR_ARG;
    if (!g->has_state) return fail(g, ESMM_ERR_STATE, "no state");
    const Geom &G = g->g;
    {
        Prof pr_(g, ESMM_KIND_NODE);
        launch_node(g->p, G, g->gamma, g->cons, g->J, g->x, nullptr, nullptr, nullptr, g->q, g->status, g->st);
    }
    {
        Prof pr_(g, ESMM_KIND_OTHER);
        k_red_init<<<1, 1, 0, g->st>>>(g->red);
    }
    int rc = step_dt(g, 0.0);
    if (rc) return rc;
    CK(cudaMemcpyAsync(g->pin, g->dt_dev, sizeof(double), cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    *dt = g->pin[0];
    return check_c2p(g);
}

int esmm_mesh_redistribute(esmm_grid *g, double dt, double *xdot, double *dtau, int mem)
{
    if (!g) return ESMM_ERR_ARG;
    if (!g->has_state) return fail(g, ESMM_ERR_STATE, "no state");
    const Geom &G = g->g;
    {
        Prof pr_(g, ESMM_KIND_NODE);
        launch_node(g->p, G, g->gamma, g->cons, g->J, g->x, nullptr, nullptr, nullptr, g->q, g->status, g->st);
    }
    {
        Prof pr_(g, ESMM_KIND_OTHER);
        k_red_init<<<1, 1, 0, g->st>>>(g->red);
    }
    int rc;
    if ((rc = step_dt(g, dt)) || (rc = mesh_core(g))) return rc;
    if (xdot && (rc = copy_out(g, xdot, g->xdot, 2 * (size_t)G.N, mem))) return rc;
    CK(cudaMemcpyAsync(g->pin, g->red + 1, sizeof(double), cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    if (dtau) *dtau = g->prm.move_mesh ? g->pin[0] : 0.0;
    return check_c2p(g);
}

int esmm_rk_step(esmm_grid *g, double dt, double *dt_used)
{
    if (!g) return ESMM_ERR_ARG;
    if (!g->has_state) return fail(g, ESMM_ERR_STATE, "no state");
    int rc = rk_step_async(g, dt);
    if (rc) return rc;
    if (dt_used) {
        CK(cudaMemcpyAsync(g->pin, g->dt_dev, sizeof(double), cudaMemcpyDeviceToHost, g->st));
        CK(cudaStreamSynchronize(g->st));
        *dt_used = g->pin[0];
        return check_c2p(g);
    }
    return ESMM_OK;
}

int esmm_advance(esmm_grid *g, int nsteps, double dt)
{
    if (!g || nsteps < 0) return ESMM_ERR_ARG;
    if (!g->has_state) return fail(g, ESMM_ERR_STATE, "no state");
    for (int s = 0; s < nsteps; ++s) {
        int rc = rk_step_async(g, dt);
        if (rc) return rc;
    }
    return ESMM_OK;
}

int esmm_totals(esmm_grid *g, double out[3])
{
    if (!g || !out) return ESMM_ERR_ARG;
    if (!g->has_state) return fail(g, ESMM_ERR_STATE, "no state");
    const Geom &G = g->g;
    {
        Prof pr_(g, ESMM_KIND_NODE);
        launch_node(g->p, G, g->gamma, g->cons, g->J, g->x, nullptr, nullptr, nullptr, g->q, g->status, g->st);
    }
    int nb = (int)nblk(G.N);
    {
        Prof pr_(g, ESMM_KIND_OTHER);
        k_totals<<<nb, BS, 0, g->st>>>(G, g->gamma, g->q, g->cons, g->J, g->partials);
    }
    {
        Prof pr_(g, ESMM_KIND_OTHER);
        k_totals_final<<<1, 32, 0, g->st>>>(nb, g->partials, g->out_dJ);
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(g->pin, g->out_dJ, 3 * sizeof(double), cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    for (int k = 0; k < 3; ++k) out[k] = g->pin[k];
    return check_c2p(g);
}

int esmm_rhs_static(int nx, int ny, const int bc[2], const double lo[2], const double hi[2], double gamma, int p,
                    int w, const double *cons, const double *J, const double *x, const double *xdot, double *dcons,
                    double *dJ, void *stream)
{
    if (!bc || !lo || !hi || !cons || !J || !x || !dcons || !dJ) return ESMM_ERR_ARG;
    if (nx < 4 || ny < 4 || (long long)(nx + 2 * GH) * (ny + 2 * GH) > ESMM_STATIC_MAX_PADDED_NODES)
        return ESMM_ERR_ARG;
    for (int k = 0; k < 2; ++k)
        if ((bc[k] != ESMM_PERIODIC && bc[k] != ESMM_OUTFLOW) || !(hi[k] > lo[k])) return ESMM_ERR_ARG;
    if (!(gamma > 1.0 && gamma <= 2.0) || p < 1 || p > PMAX || !(w == 0 || w == 3 || w == 5)) return ESMM_ERR_ARG;
    double *scratch = nullptr;
    if (static_scratch(&scratch) != cudaSuccess) return ESMM_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    Geom G;
    G.nx = nx;
    G.ny = ny;
    G.px = nx + 2 * GH;
    G.py = ny + 2 * GH;
    G.P = (long long)G.px * G.py;
    G.N = (long long)nx * ny;
    G.bc0 = bc[0];
    G.bc1 = bc[1];
    G.per0 = hi[0] - lo[0];
    G.per1 = hi[1] - lo[1];
    MetricCoef mc;
    mc.p = p;
    mc.a[0] = p == 1 ? 1.0 : (p == 2 ? 4.0 / 3.0 : 3.0 / 2.0);
    mc.a[1] = p == 1 ? 0.0 : (p == 2 ? -1.0 / 6.0 : -3.0 / 10.0);
    mc.a[2] = p == 3 ? 1.0 / 30.0 : 0.0;
    Phys ph;
    ph.gamma = gamma;
    ph.eps = 1e-6;
    ph.ln_thr = 1.0e-4;
    ph.sign_tol = 1.0e-10;
    for (int n = 0; n < PMAX; ++n) ph.alpha[n] = mc.a[n];
    ph.p = p;
    ph.w = w;
    // carve the scratch: node arrays, pair fluxes, interface fluxes, status
    double *q = scratch;
    double *pairs = q + (long long)NQ * G.P;
    double *iflux = pairs + (long long)2 * PMAX * 4 * G.P;
    int *status = (int *)(scratch + STATIC_PER_NODE * ESMM_STATIC_MAX_PADDED_NODES);
    if (cudaMemsetAsync(status, 0, 2 * sizeof(int), st) != cudaSuccess) return ESMM_ERR_CUDA;
    launch_node(p, G, gamma, cons, J, x, xdot, nullptr, nullptr, q, status, st);
    for (int dir = 0; dir < 2; ++dir) {
        launch_pairs_f64(G, ph, q, pairs, dir, st);
        launch_iface_f64(G, ph, q, pairs, iflux, dir, st);
    }
    k_update<double><<<nblk(G.N), BS, 0, st>>>(G, iflux, dcons, dJ, nullptr, nullptr, nullptr, nullptr, nullptr,
                                               nullptr, nullptr, 0.0, 0.0, nullptr, nullptr, nullptr, nullptr);
    return cudaGetLastError() == cudaSuccess ? ESMM_OK : ESMM_ERR_CUDA;
}

int esmm_profile(esmm_grid *g, int mask)
{
    if (!g || mask < 0 || mask >= (1 << ESMM_NKINDS)) return ESMM_ERR_ARG;
    CK(cudaStreamSynchronize(g->st));
    for (int k = 0; k < ESMM_NKINDS; ++k) {
        for (auto &pr : g->ev[k]) { g->pool->push_back(pr.first); g->pool->push_back(pr.second); }
        g->ev[k].clear();
        g->launches[k] = 0;
    }
    g->prof_mask = mask;
    return ESMM_OK;
}

int esmm_profile_read(esmm_grid *g, double ms[ESMM_NKINDS], long long launches[ESMM_NKINDS],
                      long long timed[ESMM_NKINDS])
{
    if (!g) return ESMM_ERR_ARG;
    CK(cudaStreamSynchronize(g->st));
    for (int k = 0; k < ESMM_NKINDS; ++k) {
        double acc = 0.0;
        for (auto &pr : g->ev[k]) {
            float t = 0.0f;
            CK(cudaEventElapsedTime(&t, pr.first, pr.second));
            acc += t;
        }
        if (ms) ms[k] = acc;
        if (launches) launches[k] = g->launches[k];
        if (timed) timed[k] = (long long)g->ev[k].size();
    }
    return ESMM_OK;
}

int esmm_last_error(esmm_grid *g, int *n_c2p_fail, char *msg, int len)
{
    if (!g) return ESMM_ERR_ARG;
    int h[2] = {0, 0};
    CK(cudaMemcpyAsync(h, g->status, sizeof h, cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    CK(cudaMemsetAsync(g->status, 0, sizeof(int), g->st));
    CK(cudaStreamSynchronize(g->st));
    if (n_c2p_fail) *n_c2p_fail = h[0];
    if (msg && len > 0) {
        strncpy(msg, g->msg, (size_t)len - 1);
        msg[len - 1] = '\0';
    }
    return ESMM_OK;
}

}  // extern "C"
