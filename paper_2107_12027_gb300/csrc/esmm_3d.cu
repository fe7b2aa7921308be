// esmm_3d.cu -- the 3D RMHD path (Duan & Tang, arXiv 2107.12027): nested
// conservative metrics (eq. SCLCoeff), the ES interface flux with the
// Godunov-Powell source on a moving curvilinear mesh, the CFL step with the
// mesh velocity, the 3D mesh redistribution (Sec. 5) and SSP-RK3, behind the
// esmm3_* functions that the C ABI dispatches to for dim = 3 grids.
//
// Layout: nodes (i, j, k), i fastest, N = nx ny nz; node data on the padded
// grid (n + 2 GH per direction), NQ3 fields per padded node.  Single problems.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "esmm.h"
#include "esmm_3d.h"
#include "esmm_3d.cuh"
#include "esmm_reduce.cuh"

namespace esmm {
namespace d3 {

// ---------------------------------------------------------------------------
// The metrics of eq. SCLCoeff in two passes.  k3_dx stores, on the grid
// extended by HE = GH + PMAX nodes per side, the boundary-mapped mesh x[3]
// and its first differences delta_d[x_c] (at 3 + 3 d + c); k3_node then forms
// M[k][j] = delta_{k2}[delta_{k1}[x_{j1}] x_{j2}] - delta_{k1}[delta_{k2}[x_{j1}] x_{j2}]
// from those values at +-n along k2 and k1 (eq. SCLCoeff's nested central
// differences, evaluated once per difference instead of once per use).
constexpr int HE = GH + PMAX;
constexpr int NXE = 12;

__host__ __device__ __forceinline__ long long eidx3(const Geom3 &g, int i, int j, int k)
{
    return ((long long)(k + HE) * (g.n[1] + 2 * HE) + (j + HE)) * (g.n[0] + 2 * HE) + (i + HE);
}

__host__ __device__ __forceinline__ long long ext_count3(const Geom3 &g)
{
    return (long long)(g.n[0] + 2 * HE) * (g.n[1] + 2 * HE) * (g.n[2] + 2 * HE);
}

template <int P>
__global__ void k3_dx(Geom3 g, const double *__restrict__ x, double *__restrict__ xe)
{
    const long long E = ext_count3(g);
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= E) return;
    const int e0 = g.n[0] + 2 * HE, e1 = g.n[1] + 2 * HE;
    const int I = (int)(t % e0) - HE, Jn = (int)((t / e0) % e1) - HE, K = (int)(t / ((long long)e0 * e1)) - HE;
#pragma unroll
    for (int c = 0; c < 3; ++c) xe[c * E + t] = mesh3_at(g, x, c, I, Jn, K, 1);
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int c = 0; c < 3; ++c) xe[(3 + 3 * d + c) * E + t] = delta_x3<P>(g, x, c, I, Jn, K, d);
}

// nested3 from the stored differences
template <int P>
__device__ __forceinline__ double nested_e3(const Geom3 &g, const double *__restrict__ xe, long long E, int d_out,
                                            int d_in, int ja, int jb, int i, int j, int k)
{
    double s = 0.0;
#pragma unroll
    for (int n = 1; n <= P; ++n) {
        int a0, a1, a2, b0, b1, b2;
        step3(i, j, k, d_out, n, a0, a1, a2);
        step3(i, j, k, d_out, -n, b0, b1, b2);
        const long long ea = eidx3(g, a0, a1, a2), eb = eidx3(g, b0, b1, b2);
        const double *Dd = xe + (3 + 3 * d_in + ja) * E, *X = xe + jb * E;
        double fa = Dd[ea] * X[ea];
        double fb = Dd[eb] * X[eb];
        s += 0.5 * alpha3<P>(n) * (fa - fb);
    }
    return s;
}

template <int P>
__global__ void k3_node(Geom3 g, double gam, const double *__restrict__ cons, const double *__restrict__ J,
                        const double *__restrict__ xe, const double *__restrict__ xdot,
                        const double *__restrict__ zg_in, double *__restrict__ zg_out, double *__restrict__ q,
                        int *__restrict__ status, const double *__restrict__ inflow)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.P) return;
    int I = (int)(t % g.pd[0]) - GH;
    int Jn = (int)((t / g.pd[0]) % g.pd[1]) - GH;
    int K = (int)(t / ((long long)g.pd[0] * g.pd[1])) - GH;
    long long src = data_src3(g, I, Jn, K);
    double iJ = 1.0 / J[src];
    double U[8], w[8], Z;
#pragma unroll
    for (int a = 0; a < 8; ++a) U[a] = cons[a * g.N + src] * iJ;
    int st = 0;
    if (inflow && ((g.bc[0] == 2 && I < 0) || (g.bc[1] == 2 && Jn < 0) || (g.bc[2] == 2 && K < 0))) {
        // a ghost beyond an inflow end: the given state
        for (int a = 0; a < 8; ++a) w[a] = inflow[a];
        Z = 0.0;
    } else {
        st = cons2prim_mhd(gam, U, zg_in ? zg_in[src] : -1.0, w, Z);
    }
    bool interior = I >= 0 && I < g.n[0] && Jn >= 0 && Jn < g.n[1] && K >= 0 && K < g.n[2];
    if (interior) {
        if (st) atomicAdd(status, 1);
        if (zg_out) zg_out[src] = Z;
    }
    double W = 1.0 / sqrt(1.0 - (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]));
    double beta = w[0] / w[4];
    q[F_RHO * g.P + t] = w[0];
    q[F_P * g.P + t] = w[4];
    q[F_BETA * g.P + t] = beta;
    q[F_U0 * g.P + t] = W * w[1];
    q[F_U1 * g.P + t] = W * w[2];
    q[F_U2 * g.P + t] = W * w[3];
    q[F_W * g.P + t] = W;
    q[F_LNR * g.P + t] = log(w[0]);
    q[F_LNB * g.P + t] = log(beta);
    q[F_B0 * g.P + t] = w[5];
    q[F_B1 * g.P + t] = w[6];
    q[F_B2 * g.P + t] = w[7];
    double M[3][3];
    {
        const long long E = ext_count3(g);
#pragma unroll 1
        for (int kk = 0; kk < 3; ++kk) {
            const int k1 = (kk + 1) % 3, k2 = (kk + 2) % 3;
#pragma unroll 1
            for (int jj = 0; jj < 3; ++jj) {
                const int j1 = (jj + 1) % 3, j2 = (jj + 2) % 3;
                M[kk][jj] = nested_e3<P>(g, xe, E, k2, k1, j1, j2, I, Jn, K) -
                            nested_e3<P>(g, xe, E, k1, k2, j1, j2, I, Jn, K);
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) q[(F_M + 3 * a + b) * g.P + t] = M[a][b];
    double xd[3] = {0.0, 0.0, 0.0};
    if (xdot)
        for (int b = 0; b < 3; ++b) xd[b] = mesh3_at(g, xdot, b, I, Jn, K, 0);
#pragma unroll
    for (int a = 0; a < 3; ++a) q[(F_MT + a) * g.P + t] = -(xd[0] * M[a][0] + xd[1] * M[a][1] + xd[2] * M[a][2]);
}

__global__ void k3_tmetric(Geom3 g, const double *__restrict__ xdot, double *__restrict__ q)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.P) return;
    int I = (int)(t % g.pd[0]) - GH;
    int Jn = (int)((t / g.pd[0]) % g.pd[1]) - GH;
    int K = (int)(t / ((long long)g.pd[0] * g.pd[1])) - GH;
    double xd[3];
    for (int b = 0; b < 3; ++b) xd[b] = mesh3_at(g, xdot, b, I, Jn, K, 0);
    for (int a = 0; a < 3; ++a)
        q[(F_MT + a) * g.P + t] = -(xd[0] * q[(F_M + 3 * a) * g.P + t] + xd[1] * q[(F_M + 3 * a + 1) * g.P + t] +
                                    xd[2] * q[(F_M + 3 * a + 2) * g.P + t]);
}

// flux differences over the three directions, the Powell source, written out
// or fused with the SSP-RK3 stage y_o = A y_n + B (y_s + dt L)
__global__ void k3_update(Geom3 g, const double *__restrict__ q, const double *__restrict__ fl,
                          double *__restrict__ dcons, double *__restrict__ dJ, const double *__restrict__ cn,
                          const double *__restrict__ Jn_, const double *__restrict__ xn,
                          const double *__restrict__ cs, const double *__restrict__ Js,
                          const double *__restrict__ xs, const double *__restrict__ xdot, double A, double B,
                          const double *__restrict__ dt_dev, double *__restrict__ co, double *__restrict__ Jo,
                          double *__restrict__ xo)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    int i = (int)(id % g.n[0]), j = (int)((id / g.n[0]) % g.n[1]), k = (int)(id / ((long long)g.n[0] * g.n[1]));
    long long c = pidx3(g, i, j, k);
    const long long sd[3] = {1, (long long)g.pd[0], (long long)g.pd[0] * g.pd[1]};
    double L[10];
#pragma unroll
    for (int a = 0; a < 10; ++a) {
        double s = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double *f = fl + (long long)(d * NF3 + a) * g.P;
            s += f[c] - f[c - sd[d]];
        }
        L[a] = -s;
    }
    double iW = 1.0 / q[F_W * g.P + c];
    double w[8];
    w[1] = q[F_U0 * g.P + c] * iW;
    w[2] = q[F_U1 * g.P + c] * iW;
    w[3] = q[F_U2 * g.P + c] * iW;
    w[5] = q[F_B0 * g.P + c];
    w[6] = q[F_B1 * g.P + c];
    w[7] = q[F_B2 * g.P + c];
    double Pp[8];
    mhd_phiprime(w, Pp);
#pragma unroll
    for (int a = 0; a < 8; ++a) L[a] += Pp[a] * L[9];
    if (dcons) {
#pragma unroll
        for (int a = 0; a < 8; ++a) dcons[a * g.N + id] = L[a];
        dJ[id] = L[8];
        return;
    }
    double dt = dt_dev[0];
#pragma unroll
    for (int a = 0; a < 8; ++a) co[a * g.N + id] = A * cn[a * g.N + id] + B * (cs[a * g.N + id] + dt * L[a]);
    Jo[id] = A * Jn_[id] + B * (Js[id] + dt * L[8]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
        xo[a * g.N + id] = A * xn[a * g.N + id] + B * (xs[a * g.N + id] + dt * xdot[a * g.N + id]);
}

// static spectral radius per direction (eq. cfl); with cflb (the moving-mesh
// step) also the speed bounds L_k lambda_min/J and L_k lambda_max/J of every
// node into its rows 3 + d and 6 + d
__global__ void k3_cfl(Geom3 g, double gam, const double *__restrict__ q, const double *__restrict__ J,
                       unsigned long long *red, double *__restrict__ cflb)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double r[3] = {0.0, 0.0, 0.0};
    if (id < g.N) {
        int i = (int)(id % g.n[0]), j = (int)((id / g.n[0]) % g.n[1]), k = (int)(id / ((long long)g.n[0] * g.n[1]));
        long long c = pidx3(g, i, j, k);
        double iW = 1.0 / q[F_W * g.P + c];
        double w[8] = {q[F_RHO * g.P + c], q[F_U0 * g.P + c] * iW, q[F_U1 * g.P + c] * iW, q[F_U2 * g.P + c] * iW,
                       q[F_P * g.P + c], q[F_B0 * g.P + c], q[F_B1 * g.P + c], q[F_B2 * g.P + c]};
        double iJ = 1.0 / J[id];
        for (int d = 0; d < 3; ++d) {
            double m[3];
            for (int a = 0; a < 3; ++a) m[a] = q[(F_M + 3 * d + a) * g.P + c];
            double Lk = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
            double nn[3] = {m[0] / Lk, m[1] / Lk, m[2] / Lk}, T[3][3], wr[8], lam[8], R[8][8];
            frame3(nn, T);
            rot3(T, w, wr);
            eigen_mhd(gam, wr, lam, R, false);
            double a = 0.0, lo = lam[0], hi = lam[0];
            for (int mm = 0; mm < 8; ++mm) {
                a = fmax(a, fabs(lam[mm]));
                lo = fmin(lo, lam[mm]);
                hi = fmax(hi, lam[mm]);
            }
            r[d] = Lk * a * iJ;
            if (cflb) {
                cflb[(3 + d) * g.N + id] = Lk * lo * iJ;
                cflb[(6 + d) * g.N + id] = Lk * hi * iJ;
            }
        }
    }
    for (int d = 0; d < 3; ++d) {
        double m = block_reduce<0>(r[d]);
        if (threadIdx.x == 0) atomic_max_nonneg(red + 2 + d, m);
    }
}

__global__ void k3_red_init(unsigned long long *red)
{
    int t = threadIdx.x;
    if (t < NR3) red[t] = t == 1 ? (unsigned long long)__double_as_longlong(1.0) : 0ull;
}

// set-up of the step solve of eq. cfl with the mesh velocity (the 2D rule
// over three directions, esmm_reduce.cuh dt_setup): slots 5..7 hold A_d,
// slots 2..4 the static radius, slot 1 the limiter (written back)
__global__ void k3_dt(double cfl, double dt_fixed, unsigned long long *red, DtSolve *ds, double *dt_dev)
{
    if (threadIdx.x || blockIdx.x) return;
    double tau = bits_to_double(red[1]);
    dt_setup(ds, cfl, dt_fixed, bits_to_double(red[5]) + bits_to_double(red[6]) + bits_to_double(red[7]),
             bits_to_double(red[2]) + bits_to_double(red[3]) + bits_to_double(red[4]), &tau, dt_dev);
    red[1] = (unsigned long long)__double_as_longlong(tau);
}

// one Newton evaluation of the step solve over all nodes: cflb rows 0..2
// hold a_d, rows 3..8 the speed bounds; part [blocks][3][2]
__global__ void k3_dt_newton(Geom3 g, double cfl, const double *__restrict__ cflb, const unsigned long long *red,
                             DtSolve *ds, double *part, double *dt_dev)
{
    __shared__ double t_sh, tau_sh;
    __shared__ int skip;
    if (threadIdx.x == 0) {
        skip = ds->done;
        t_sh = ds->t;
        tau_sh = bits_to_double(red[1]);
    }
    __syncthreads();
    if (skip) return;
    unsigned long long v[3] = {0ull, 0ull, 0ull}, sl[3] = {~0ull, ~0ull, ~0ull};
    const long long base = (long long)blockIdx.x * blockDim.x * DT_NPT + threadIdx.x;
    for (int r = 0; r < DT_NPT; ++r) {
        const long long id = base + (long long)r * blockDim.x;
        if (id < g.N)
            for (int d = 0; d < 3; ++d) {
                unsigned long long vk, sk;
                cfl_line(t_sh, tau_sh * cflb[d * g.N + id], cflb[(3 + d) * g.N + id], cflb[(6 + d) * g.N + id], vk,
                         sk);
                vs_take(v[d], sl[d], vk, sk);
            }
    }
    dt_newton_block<3>(ds, v, sl, blockIdx.x, 0, gridDim.x, (unsigned long long *)part, cfl, dt_dev);
}

__global__ void k3_time(const double *dt_dev, double *t_dev)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) t_dev[0] += dt_dev[0];
}

// ---- Sec. 5 in 3D ------------------------------------------------------------
__global__ void k3_mesh_grad(Geom3 g, int lnrho, int with_lap, const double *__restrict__ q,
                             double *__restrict__ grad, double *__restrict__ lap, unsigned long long *red)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double gv = 0.0, lv = 0.0;
    if (id < g.N) {
        int i = (int)(id % g.n[0]), j = (int)((id / g.n[0]) % g.n[1]), k = (int)(id / ((long long)g.n[0] * g.n[1]));
        long long c = pidx3(g, i, j, k);
        const double *s = q + (lnrho ? F_LNR : F_RHO) * g.P;
        long long sy = g.pd[0], sz = (long long)g.pd[0] * g.pd[1];
        double xp = s[c + 1], xm = s[c - 1], yp = s[c + sy], ym = s[c - sy], zp = s[c + sz], zm = s[c - sz];
        double gx = 0.5 * (xp - xm);
        double gy = 0.5 * (yp - ym);
        double gz = 0.5 * (zp - zm);
        gv = sqrt(gx * gx + gy * gy + gz * gz);
        grad[id] = gv;
        if (with_lap) {
            lv = fabs(xp + xm + yp + ym + zp + zm - 6.0 * s[c]);
            lap[id] = lv;
        }
    }
    double m = block_reduce<0>(gv);
    if (threadIdx.x == 0) atomic_max_nonneg(red, m);
    if (with_lap) {
        double ml = block_reduce<0>(lv);
        if (threadIdx.x == 0) atomic_max_nonneg(red + 8, ml);
    }
}

__global__ void k3_mesh_omega(Geom3 g, double alpha, double alpha_lap, const double *__restrict__ grad,
                              const double *__restrict__ lap, const unsigned long long *red, double *__restrict__ om)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    double gmax = bits_to_double(red[0]);
    double a = 1.0;
    if (gmax > 0.0) a += alpha * grad[id] / gmax;
    if (alpha_lap > 0.0) {
        double lmax = bits_to_double(red[8]);
        if (lmax > 0.0) a += alpha_lap * lap[id] / lmax;
    }
    om[id] = sqrt(a);
}

// omega <- sum_{a,b,c in {-1,0,1}} 2^-(|a|+|b|+|c|+3) omega_{i+a, j+b, k+c}
__global__ void k3_mesh_filter(Geom3 g, const double *__restrict__ om, double *__restrict__ om2)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    int i = (int)(id % g.n[0]), j = (int)((id / g.n[0]) % g.n[1]), k = (int)(id / ((long long)g.n[0] * g.n[1]));
    double acc = 0.0;
    for (int cc = -1; cc <= 1; ++cc)
        for (int bb = -1; bb <= 1; ++bb)
            for (int a = -1; a <= 1; ++a) {
                int e = (a != 0) + (bb != 0) + (cc != 0) + 3;
                acc += ldexp(1.0, -e) * om[data_src3(g, i + a, j + bb, k + cc)];
            }
    om2[id] = acc;
}

__global__ void k3_mesh_jacobi(Geom3 g, const double *__restrict__ om, const double *__restrict__ X,
                               double *__restrict__ Xn)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    int i = (int)(id % g.n[0]), j = (int)((id / g.n[0]) % g.n[1]), k = (int)(id / ((long long)g.n[0] * g.n[1]));
    bool fixed = (g.bc[0] != 0 && (i == 0 || i == g.n[0] - 1)) || (g.bc[1] != 0 && (j == 0 || j == g.n[1] - 1)) ||
                 (g.bc[2] != 0 && (k == 0 || k == g.n[2] - 1));
    if (fixed) {
        for (int comp = 0; comp < 3; ++comp) Xn[comp * g.N + id] = X[comp * g.N + id];
        return;
    }
    double wi = om[id];
    double wp[3] = {om[data_src3(g, i + 1, j, k)], om[data_src3(g, i, j + 1, k)], om[data_src3(g, i, j, k + 1)]};
    double wm[3] = {om[data_src3(g, i - 1, j, k)], om[data_src3(g, i, j - 1, k)], om[data_src3(g, i, j, k - 1)]};
    double den = 0.0;
    for (int d = 0; d < 3; ++d) den += 2.0 * wi + wp[d] + wm[d];
    for (int comp = 0; comp < 3; ++comp) {
        double num = 0.0;
        for (int d = 0; d < 3; ++d) {
            int a0, a1, a2, b0, b1, b2;
            step3(i, j, k, d, 1, a0, a1, a2);
            step3(i, j, k, d, -1, b0, b1, b2);
            num += (wi + wp[d]) * mesh3_at(g, X, comp, a0, a1, a2, 1) + (wi + wm[d]) * mesh3_at(g, X, comp, b0, b1, b2, 1);
        }
        Xn[comp * g.N + id] = num / den;
    }
}

// limiter (half the neighbour spacing toward the displacement, three
// directions) and the displacement's Courant number per direction
__global__ void k3_mesh_tau(Geom3 g, const double *__restrict__ x, const double *__restrict__ X,
                            const double *__restrict__ q, const double *__restrict__ J, unsigned long long *red,
                            double *__restrict__ cflb)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double tau = 1.0, cm[3] = {0.0, 0.0, 0.0};
    if (id < g.N) {
        int i = (int)(id % g.n[0]), j = (int)((id / g.n[0]) % g.n[1]), k = (int)(id / ((long long)g.n[0] * g.n[1]));
        double dd[3];
        for (int d = 0; d < 3; ++d) {
            double dv = X[d * g.N + id] - x[d * g.N + id];
            dd[d] = dv;
            double bnd = 1.0;
            int a0, a1, a2;
            if (dv < 0.0) {
                step3(i, j, k, d, -1, a0, a1, a2);
                bnd = -(x[d * g.N + id] - mesh3_at(g, x, d, a0, a1, a2, 1)) / (2.0 * dv);
            } else if (dv > 0.0) {
                step3(i, j, k, d, 1, a0, a1, a2);
                bnd = (mesh3_at(g, x, d, a0, a1, a2, 1) - x[d * g.N + id]) / (2.0 * dv);
            }
            tau = fmin(tau, bnd);
        }
        tau = fmax(tau, 0.0);
        long long c = pidx3(g, i, j, k);
        double iJ = 1.0 / J[id];
        for (int d = 0; d < 3; ++d) {
            const double ad = (dd[0] * q[(F_M + 3 * d) * g.P + c] + dd[1] * q[(F_M + 3 * d + 1) * g.P + c] +
                               dd[2] * q[(F_M + 3 * d + 2) * g.P + c]) * iJ;
            cm[d] = fabs(ad);
            cflb[d * g.N + id] = ad;
        }
    }
    double m = block_reduce<1>(tau);
    if (threadIdx.x == 0) atomic_min_nonneg(red + 1, m);
    for (int d = 0; d < 3; ++d) {
        double mk = block_reduce<0>(cm[d]);
        if (threadIdx.x == 0) atomic_max_nonneg(red + 5 + d, mk);
    }
}

__global__ void k3_mesh_xdot(Geom3 g, const double *__restrict__ x, const double *__restrict__ X,
                             const unsigned long long *red, const double *__restrict__ dt_dev, double *__restrict__ xdot)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= 3 * g.N) return;
    // a step of 0 (a NaN spectral radius) leaves the mesh where it is
    xdot[id] = dt_dev[0] > 0.0 ? bits_to_double(red[1]) * (X[id] - x[id]) / dt_dev[0] : 0.0;
}

// initial J = det(delta_k[x_j]) and cons = J U(prim)
template <int P>
__global__ void k3_init(Geom3 g, double gam, const double *__restrict__ prim, const double *__restrict__ x,
                        double *__restrict__ cons, double *__restrict__ J, int *status)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    int i = (int)(id % g.n[0]), j = (int)((id / g.n[0]) % g.n[1]), k = (int)(id / ((long long)g.n[0] * g.n[1]));
    double D[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) D[a][b] = delta_x3<P>(g, x, b, i, j, k, a);
    double J0 = D[0][0] * (D[1][1] * D[2][2] - D[1][2] * D[2][1]) - D[0][1] * (D[1][0] * D[2][2] - D[1][2] * D[2][0]) +
                D[0][2] * (D[1][0] * D[2][1] - D[1][1] * D[2][0]);
    double w[8], U[8], F[8], V[8];
    for (int a = 0; a < 8; ++a) w[a] = prim[a * g.N + id];
    double v2 = w[1] * w[1] + w[2] * w[2] + w[3] * w[3];
    if (!(w[0] > 0.0) || !(w[4] > 0.0) || !(v2 < 1.0) || !(J0 > 0.0)) {
        atomicAdd(status + 1, 1);
        w[0] = 1.0; w[4] = 1.0; w[1] = w[2] = w[3] = 0.0;
    }
    mhd_UFV<double>(gam, w, U, F, V);
    J[id] = J0;
    for (int a = 0; a < 8; ++a) cons[a * g.N + id] = J0 * U[a];
}

__global__ void k3_prim_out(Geom3 g, double gam, const double *__restrict__ cons, const double *__restrict__ J,
                            double *__restrict__ prim, int *status)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    double iJ = 1.0 / J[id];
    double U[8], w[8], Z;
    for (int a = 0; a < 8; ++a) U[a] = cons[a * g.N + id] * iJ;
    if (cons2prim_mhd(gam, U, -1.0, w, Z)) atomicAdd(status, 1);
    for (int a = 0; a < 8; ++a) prim[a * g.N + id] = w[a];
}

// totals: per-block partial sums of (J eta, J D, J), then a fixed-order sum
__global__ void k3_totals(Geom3 g, double gam, const double *__restrict__ q, const double *__restrict__ cons,
                          const double *__restrict__ J, double *__restrict__ partials)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double v[3] = {0.0, 0.0, 0.0};
    if (id < g.N) {
        int i = (int)(id % g.n[0]), j = (int)((id / g.n[0]) % g.n[1]), k = (int)(id / ((long long)g.n[0] * g.n[1]));
        long long c = pidx3(g, i, j, k);
        double rho = q[F_RHO * g.P + c], W = q[F_W * g.P + c];
        double lnr = q[F_LNR * g.P + c], lnb = q[F_LNB * g.P + c];
        double s = (lnr - lnb) - gam * lnr;
        v[0] = J[id] * (-rho * W * s / (gam - 1.0));
        v[1] = cons[id];
        v[2] = J[id];
    }
    for (int a = 0; a < 3; ++a) {
        double s = block_reduce<2>(v[a]);
        if (threadIdx.x == 0) partials[(long long)blockIdx.x * 3 + a] = s;
    }
}

__global__ void k3_totals_final(int nb, const double *__restrict__ partials, double *__restrict__ out)
{
    int t = threadIdx.x;
    if (t >= 3) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partials[(long long)b * 3 + t];
    out[t] = s;
}

}  // namespace d3
}  // namespace esmm

// ===========================================================================
using namespace esmm;
using namespace esmm::d3;

struct esmm3 {
    Geom3 g;
    double lo[3], hi[3];
    double gamma;
    int p, w;
    esmm_params prm;
    cudaStream_t st;
    int has_state, xdot_zero;
    int needs_inflow, has_inflow;
    double *inflow_dev;        // [8] primitive inflow state (ESMM_INFLOW ends)
    double *cons, *J, *x, *xdot, *c1, *J1, *x1, *c2, *J2, *x2;
    double *q, *zg[3], *iflux, *out_dc, *out_dJ, *in_cons, *in_J, *in_x, *in_xdot;
    double *grad, *om, *om2, *X, *Xn, *dt_dev, *t_dev, *partials, *tot;
    double *cflb, *npart;      // the step solve: [9][N] a_d, bmin_d, bmax_d; [blocks][3][2] partials
    DtSolve *ds;
    unsigned long long *red;
    int *status;
    double *pin;
    char msg[256];
    long long launches;
    // profiling: launches per kind, CUDA events around the kinds in prof_mask
    long long nl[ESMM_NKINDS];
    int prof_mask;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> *ev;   // [ESMM_NKINDS]
    // adjoint: per-step checkpoints [cons 8N | J N | x 3N | xdot 3N], steps,
    // adjoint state buffers and the node-quantity adjoints lamq[11][P]
    std::vector<double *> *ck;
    std::vector<double> *ck_dt;
    int ck_n;
    double *lam_a, *lam_b, *lam_c, *lam_v, *lamq;
    double *xe;   // the mesh and its first differences on the extended grid (k3_dx)
};

namespace {

constexpr int BS3 = 128;
inline unsigned nb3(long long n, int bs = BS3) { return (unsigned)((n + bs - 1) / bs); }

int fail3(esmm3 *g, int code, const char *what, cudaError_t e = cudaSuccess)
{
    if (e != cudaSuccess) snprintf(g->msg, sizeof g->msg, "%s: %s", what, cudaGetErrorString(e));
    else snprintf(g->msg, sizeof g->msg, "%s", what);
    return code;
}

// counts n launches of one kind; times them (one event pair) when the kind is
// in the profile mask
struct Prof3 {
    esmm3 *g;
    int kind;
    cudaEvent_t a = nullptr;
    Prof3(esmm3 *g_, int kind_, int n = 1) : g(g_), kind(kind_)
    {
        g->launches += n;
        g->nl[kind] += n;
        if (g->ev && (g->prof_mask & (1 << kind)) && cudaEventCreate(&a) == cudaSuccess) cudaEventRecord(a, g->st);
    }
    ~Prof3()
    {
        cudaEvent_t b;
        if (a && cudaEventCreate(&b) == cudaSuccess) {
            cudaEventRecord(b, g->st);
            g->ev[kind].push_back({a, b});
        }
    }
};

void prof_clear3(esmm3 *g)
{
    if (!g->ev) return;
    for (int k = 0; k < ESMM_NKINDS; ++k) {
        for (auto &pr : g->ev[k]) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
        g->ev[k].clear();
    }
}

#define CK3(call)                                                          \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return fail3(g, ESMM_ERR_CUDA, #call, e_);  \
    } while (0)

Phys phys3(const esmm3 *g)
{
    Phys ph;
    ph.gamma = g->gamma;
    ph.eps = g->prm.weno_eps;
    ph.gm1i = 1.0 / (g->gamma - 1.0);
    ph.ln_thr = 1.0e-4;
    ph.sign_tol = 1.0e-10;
    double a[3][3] = {{1.0, 0.0, 0.0}, {4.0 / 3.0, -1.0 / 6.0, 0.0}, {1.5, -0.3, 1.0 / 30.0}};
    for (int n = 0; n < PMAX; ++n) ph.alpha[n] = a[g->p - 1][n];
    ph.p = g->p;
    ph.w = g->w;
    return ph;
}

void node3(esmm3 *g, const double *cons, const double *J, const double *x, const double *xdot, const double *zi,
           double *zo)
{
    unsigned nb = nb3(g->g.P), nbe = nb3(ext_count3(g->g));
    Prof3 pr_(g, ESMM_KIND_NODE, 2);
    double *xe = g->xe;
    const double *in = g->has_inflow ? g->inflow_dev : nullptr;
    if (g->p == 1) {
        k3_dx<1><<<nbe, BS3, 0, g->st>>>(g->g, x, xe);
        k3_node<1><<<nb, BS3, 0, g->st>>>(g->g, g->gamma, cons, J, xe, xdot, zi, zo, g->q, g->status, in);
    } else if (g->p == 2) {
        k3_dx<2><<<nbe, BS3, 0, g->st>>>(g->g, x, xe);
        k3_node<2><<<nb, BS3, 0, g->st>>>(g->g, g->gamma, cons, J, xe, xdot, zi, zo, g->q, g->status, in);
    } else {
        k3_dx<3><<<nbe, BS3, 0, g->st>>>(g->g, x, xe);
        k3_node<3><<<nb, BS3, 0, g->st>>>(g->g, g->gamma, cons, J, xe, xdot, zi, zo, g->q, g->status, in);
    }
}

void fluxes3(esmm3 *g)
{
    Phys ph = phys3(g);
    for (int dir = 0; dir < 3; ++dir) {
        int oa = dir == 0 ? 1 : 0, ob = dir == 2 ? 1 : 2;
        long long count = (long long)(g->g.n[dir] + 1) * g->g.n[oa] * g->g.n[ob];
        unsigned nb = nb3(count, 128);
        Prof3 pr_(g, ESMM_KIND_IFACE);
        launch3_iface(g->g, ph, g->p, g->w, g->q, g->iflux, dir, nb, g->st);
    }
}

void update3(esmm3 *g, double *dc, double *dJ, const double *cn, const double *Jn, const double *xn, const double *cs,
             const double *Js, const double *xs, double A, double B, double *co, double *Jo, double *xo)
{
    Prof3 pr_(g, ESMM_KIND_UPDATE);
    k3_update<<<nb3(g->g.N), BS3, 0, g->st>>>(g->g, g->q, g->iflux, dc, dJ, cn, Jn, xn, cs, Js, xs, g->xdot, A, B,
                                              g->dt_dev, co, Jo, xo);
}

int mesh_and_dt3(esmm3 *g, double dt)
{
    unsigned nb = nb3(g->g.N);
    {
        Prof3 pr_(g, ESMM_KIND_OTHER, dt > 0.0 ? 1 : 2);
        k3_red_init<<<1, 32, 0, g->st>>>(g->red);
        if (!(dt > 0.0))
            k3_cfl<<<nb, BS3, 0, g->st>>>(g->g, g->gamma, g->q, g->J, g->red, g->prm.move_mesh ? g->cflb : nullptr);
    }
    if (!g->prm.move_mesh) {
        Prof3 pr_(g, ESMM_KIND_OTHER);
        k3_dt<<<1, 32, 0, g->st>>>(g->prm.cfl, dt, g->red, g->ds, g->dt_dev);
        if (!g->xdot_zero) {
            CK3(cudaMemsetAsync(g->xdot, 0, 3 * g->g.N * sizeof(double), g->st));
            g->xdot_zero = 1;
        }
        return ESMM_OK;
    }
    g->xdot_zero = 0;
    const double *src = g->x;
    {
        Prof3 pr_(g, ESMM_KIND_MESH, 3 + g->prm.n_filter + g->prm.mu);
        // the Laplacian goes to om2, which the filter overwrites only after k3_mesh_omega
        k3_mesh_grad<<<nb, BS3, 0, g->st>>>(g->g, g->prm.monitor == ESMM_MONITOR_LNRHO, g->prm.alpha_lap > 0.0,
                                            g->q, g->grad, g->om2, g->red);
        k3_mesh_omega<<<nb, BS3, 0, g->st>>>(g->g, g->prm.alpha, g->prm.alpha_lap, g->grad, g->om2, g->red, g->om);
        double *om = g->om, *om2 = g->om2;
        for (int f = 0; f < g->prm.n_filter; ++f) {
            k3_mesh_filter<<<nb, BS3, 0, g->st>>>(g->g, om, om2);
            std::swap(om, om2);
        }
        for (int nu = 0; nu < g->prm.mu; ++nu) {
            double *dst = (nu % 2 == 0) ? g->X : g->Xn;
            k3_mesh_jacobi<<<nb, BS3, 0, g->st>>>(g->g, om, src, dst);
            src = dst;
        }
        k3_mesh_tau<<<nb, BS3, 0, g->st>>>(g->g, g->x, src, g->q, g->J, g->red, g->cflb);
    }
    {
        Prof3 pr_(g, ESMM_KIND_OTHER, dt > 0.0 ? 1 : 1 + DT_NEWTON);
        k3_dt<<<1, 32, 0, g->st>>>(g->prm.cfl, dt, g->red, g->ds, g->dt_dev);
        if (!(dt > 0.0))
            for (int it = 0; it < DT_NEWTON; ++it)
                k3_dt_newton<<<nb3(g->g.N, BS3 * DT_NPT), BS3, 0, g->st>>>(g->g, g->prm.cfl, g->cflb, g->red, g->ds,
                                                                          g->npart, g->dt_dev);
    }
    Prof3 pr_(g, ESMM_KIND_MESH);
    k3_mesh_xdot<<<nb3(3 * g->g.N), BS3, 0, g->st>>>(g->g, g->x, src, g->red, g->dt_dev, g->xdot);
    return ESMM_OK;
}

int stages3(esmm3 *g)
{
    fluxes3(g);
    update3(g, nullptr, nullptr, g->cons, g->J, g->x, g->cons, g->J, g->x, 0.0, 1.0, g->c1, g->J1, g->x1);
    node3(g, g->c1, g->J1, g->x1, g->xdot, g->zg[1], g->zg[2]);
    fluxes3(g);
    update3(g, nullptr, nullptr, g->cons, g->J, g->x, g->c1, g->J1, g->x1, 0.75, 0.25, g->c2, g->J2, g->x2);
    node3(g, g->c2, g->J2, g->x2, g->xdot, g->zg[2], g->zg[0]);
    fluxes3(g);
    update3(g, nullptr, nullptr, g->cons, g->J, g->x, g->c2, g->J2, g->x2, 1.0 / 3.0, 2.0 / 3.0, g->cons, g->J, g->x);
    Prof3 pr_(g, ESMM_KIND_OTHER);
    k3_time<<<1, 32, 0, g->st>>>(g->dt_dev, g->t_dev);
    CK3(cudaGetLastError());
    return ESMM_OK;
}

int check3(esmm3 *g)
{
    int h[2];
    CK3(cudaMemcpyAsync(h, g->status, sizeof h, cudaMemcpyDeviceToHost, g->st));
    CK3(cudaStreamSynchronize(g->st));
    if (h[0] > 0) {
        CK3(cudaMemsetAsync(g->status, 0, sizeof(int), g->st));
        snprintf(g->msg, sizeof g->msg, "primitive recovery failed at %d node(s)", h[0]);
        return ESMM_ERR_C2P;
    }
    return ESMM_OK;
}

int copy3(esmm3 *g, double *dst, const double *src, size_t n, int mem, bool in)
{
    cudaMemcpyKind k = mem == ESMM_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                              : (in ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost);
    CK3(cudaMemcpyAsync(dst, src, n * sizeof(double), k, g->st));
    return ESMM_OK;
}

void free3(esmm3 *g)
{
    double **b[] = {&g->cons, &g->J, &g->x, &g->xdot, &g->c1, &g->J1, &g->x1, &g->c2, &g->J2, &g->x2, &g->q,
                    &g->zg[0], &g->zg[1], &g->zg[2], &g->iflux, &g->out_dc, &g->out_dJ, &g->in_cons, &g->in_J,
                    &g->in_x, &g->in_xdot, &g->grad, &g->om, &g->om2, &g->X, &g->Xn, &g->dt_dev, &g->t_dev,
                    &g->partials, &g->tot, &g->lam_a, &g->lam_b, &g->lam_c, &g->lam_v, &g->lamq, &g->xe,
                    &g->inflow_dev, &g->cflb, &g->npart};
    for (double **p : b)
        if (*p) { cudaFree(*p); *p = nullptr; }
    if (g->ck) {
        for (double *c : *g->ck) cudaFree(c);
        delete g->ck;
        g->ck = nullptr;
    }
    delete g->ck_dt;
    g->ck_dt = nullptr;
    if (g->red) cudaFree(g->red);
    if (g->ds) cudaFree(g->ds);
    g->ds = nullptr;
    if (g->status) cudaFree(g->status);
    if (g->pin) cudaFreeHost(g->pin);
}

// ---- adjoint -------------------------------------------------------------------
int adj_alloc3(esmm3 *g)
{
    size_t N = (size_t)g->g.N, P = (size_t)g->g.P, d = sizeof(double);
    double **b[] = {&g->lam_a, &g->lam_b, &g->lam_c, &g->lam_v};
    for (double **p : b)
        if (!*p) CK3(cudaMalloc((void **)p, 8 * N * d));
    if (!g->lamq) CK3(cudaMalloc((void **)&g->lamq, 11 * P * d));
    if (!g->ck) g->ck = new (std::nothrow) std::vector<double *>;
    if (!g->ck_dt) g->ck_dt = new (std::nothrow) std::vector<double>;
    if (!g->ck || !g->ck_dt) return fail3(g, ESMM_ERR_ARG, "out of host memory");
    return ESMM_OK;
}

// lam = (d rhs/d cons)^T mu at (cons, J, x, xdot), device arrays
int rhs_vjp_core3(esmm3 *g, const double *cons, const double *J, const double *x, const double *xdot,
                  const double *mu, double *lam)
{
    size_t N = (size_t)g->g.N, P = (size_t)g->g.P, d = sizeof(double);
    node3(g, cons, J, x, xdot, nullptr, nullptr);
    fluxes3(g);   // the Powell term's div B~
    CK3(cudaMemsetAsync(g->lamq, 0, 11 * P * d, g->st));
    CK3(cudaMemsetAsync(lam, 0, 8 * N * d, g->st));
    Phys ph = phys3(g);
    for (int dir = 0; dir < 3; ++dir) {
        {
            Prof3 pr_(g, ESMM_KIND_PAIRS);
            launch3_pairs_vjp(g->g, ph, g->q, mu, g->lamq, dir, g->st);
        }
        if (g->w > 0) {
            Prof3 pr_(g, ESMM_KIND_IFACE);
            launch3_iface_vjp(g->g, ph, g->q, mu, g->lamq, dir, g->st);
        }
    }
    {
        Prof3 pr_(g, ESMM_KIND_NODE);
        launch3_node_vjp(g->g, g->gamma, g->q, g->lamq, g->iflux, mu, J, lam, g->st);
    }
    CK3(cudaGetLastError());
    return ESMM_OK;
}

int set_dt3(esmm3 *g, double dt)
{
    g->pin[0] = dt;
    CK3(cudaMemcpyAsync(g->dt_dev, g->pin, sizeof(double), cudaMemcpyHostToDevice, g->st));
    CK3(cudaStreamSynchronize(g->st));
    return ESMM_OK;
}

// one step with a given mesh velocity (device, [3][N]) and dt
int step_given3(esmm3 *g, const double *xd, double dt, int mem)
{
    int rc;
    if ((rc = set_dt3(g, dt))) return rc;
    if ((rc = copy3(g, g->xdot, xd, 3 * (size_t)g->g.N, mem, true))) return rc;
    g->xdot_zero = 0;
    node3(g, g->cons, g->J, g->x, g->xdot, g->zg[0], g->zg[1]);
    return stages3(g);
}

}  // namespace

// ---- the esmm3_* entry points (esmm_3d.h) ------------------------------------------
int esmm3_create(esmm3 **out, const int n[3], const double lo[3], const double hi[3], const int bc[3], void *stream)
{
    *out = nullptr;
    for (int k = 0; k < 3; ++k)
        if (n[k] < 4 || n[k] > 4096 || (bc[k] != ESMM_PERIODIC && bc[k] != ESMM_OUTFLOW && bc[k] != ESMM_INFLOW) ||
            !(hi[k] > lo[k]))
            return ESMM_ERR_ARG;
    esmm3 *g = new (std::nothrow) esmm3;
    if (!g) return ESMM_ERR_ARG;
    memset((void *)g, 0, sizeof *g);
    for (int k = 0; k < 3; ++k) {
        g->g.n[k] = n[k];
        g->g.pd[k] = n[k] + 2 * GH;
        g->g.bc[k] = bc[k];
        if (bc[k] == ESMM_INFLOW) g->needs_inflow = 1;
        g->g.per[k] = hi[k] - lo[k];
        g->lo[k] = lo[k];
        g->hi[k] = hi[k];
    }
    g->g.N = (long long)n[0] * n[1] * n[2];
    g->g.P = (long long)g->g.pd[0] * g->g.pd[1] * g->g.pd[2];
    g->st = (cudaStream_t)stream;
    g->gamma = 4.0 / 3.0;
    g->p = 2;
    g->w = 5;
    g->prm.cfl = 0.3;
    g->prm.weno_eps = 1e-6;
    g->prm.monitor = ESMM_MONITOR_LNRHO;
    g->prm.alpha = 800.0;
    g->prm.alpha_lap = 0.0;
    g->prm.sweep = ESMM_SWEEP_AUTO;   // 2D RHD only; kept for esmm_get_params
    g->prm.n_filter = 4;
    g->prm.mu = 10;
    g->prm.move_mesh = 1;
    g->prm.precision = ESMM_FP64;
    size_t N = (size_t)g->g.N, P = (size_t)g->g.P, d = sizeof(double);
    size_t nb = N / BS3 + 2;
    struct { double **p; size_t n; } al[] = {
        {&g->cons, 8 * N}, {&g->J, N}, {&g->x, 3 * N}, {&g->xdot, 3 * N}, {&g->c1, 8 * N}, {&g->J1, N},
        {&g->x1, 3 * N}, {&g->c2, 8 * N}, {&g->J2, N}, {&g->x2, 3 * N}, {&g->q, (size_t)NQ3 * P},
        {&g->zg[0], N}, {&g->zg[1], N}, {&g->zg[2], N}, {&g->iflux, (size_t)3 * NF3 * P}, {&g->out_dc, 8 * N},
        {&g->out_dJ, N}, {&g->in_cons, 8 * N}, {&g->in_J, N}, {&g->in_x, 3 * N}, {&g->in_xdot, 3 * N},
        {&g->grad, N}, {&g->om, N}, {&g->om2, N}, {&g->X, 3 * N}, {&g->Xn, 3 * N}, {&g->dt_dev, 1},
        {&g->t_dev, 1}, {&g->partials, 3 * nb}, {&g->tot, 3}, {&g->xe, (size_t)NXE * ext_count3(g->g)},
        {&g->inflow_dev, 8}, {&g->cflb, 9 * N}, {&g->npart, 6 * nb}};
    bool ok = true;
    for (auto &a : al) ok = ok && cudaMalloc((void **)a.p, a.n * d) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&g->red, NR3 * sizeof(unsigned long long)) == cudaSuccess &&
         cudaMalloc((void **)&g->ds, sizeof(DtSolve)) == cudaSuccess &&
         cudaMalloc((void **)&g->status, 2 * sizeof(int)) == cudaSuccess &&
         cudaMallocHost((void **)&g->pin, 16 * sizeof(double)) == cudaSuccess;
    for (int k = 0; ok && k < 3; ++k) ok = cudaMemsetAsync(g->zg[k], 0xff, N * d, g->st) == cudaSuccess;
    ok = ok && cudaMemsetAsync(g->status, 0, 2 * sizeof(int), g->st) == cudaSuccess &&
         cudaMemsetAsync(g->t_dev, 0, d, g->st) == cudaSuccess && cudaStreamSynchronize(g->st) == cudaSuccess;
    if (!ok) {
        free3(g);
        delete g;
        return ESMM_ERR_CUDA;
    }
    *out = g;
    return ESMM_OK;
}

void esmm3_destroy(esmm3 *g)
{
    if (!g) return;
    cudaStreamSynchronize(g->st);
    prof_clear3(g);
    delete[] g->ev;
    free3(g);
    delete g;
}

int esmm3_set_stream(esmm3 *g, void *stream)
{
    CK3(cudaStreamSynchronize(g->st));
    g->st = (cudaStream_t)stream;
    return ESMM_OK;
}

int esmm3_set_eos(esmm3 *g, double gamma) { g->gamma = gamma; return ESMM_OK; }
int esmm3_set_order(esmm3 *g, int p, int w) { g->p = p; g->w = w; return ESMM_OK; }
int esmm3_set_params(esmm3 *g, const esmm_params *prm)
{
    if (prm->precision != ESMM_FP64) return fail3(g, ESMM_ERR_ARG, "3D grids compute in FP64 only");
    g->prm = *prm;
    return ESMM_OK;
}
int esmm3_get_params(const esmm3 *g, esmm_params *prm) { *prm = g->prm; return ESMM_OK; }

int esmm3_state_set(esmm3 *g, const double *prim, const double *x, int mem)
{
    size_t N = (size_t)g->g.N;
    int rc;
    if (x) {
        if ((rc = copy3(g, g->x, x, 3 * N, mem, true))) return rc;
    } else {
        std::vector<double> hx(3 * N);
        int den[3];
        for (int k = 0; k < 3; ++k) den[k] = g->g.bc[k] == ESMM_PERIODIC ? g->g.n[k] : g->g.n[k] - 1;
        for (int k = 0; k < g->g.n[2]; ++k)
            for (int j = 0; j < g->g.n[1]; ++j)
                for (int i = 0; i < g->g.n[0]; ++i) {
                    size_t id = ((size_t)k * g->g.n[1] + j) * g->g.n[0] + i;
                    int ijk[3] = {i, j, k};
                    for (int c = 0; c < 3; ++c)
                        hx[c * N + id] = g->lo[c] + (g->hi[c] - g->lo[c]) * ijk[c] / den[c];
                }
        CK3(cudaMemcpyAsync(g->x, hx.data(), 3 * N * sizeof(double), cudaMemcpyHostToDevice, g->st));
        CK3(cudaStreamSynchronize(g->st));
    }
    if ((rc = copy3(g, g->out_dc, prim, 8 * N, mem, true))) return rc;
    CK3(cudaMemsetAsync(g->status, 0, 2 * sizeof(int), g->st));
    Prof3 pr_(g, ESMM_KIND_OTHER);
    unsigned nb = nb3(g->g.N);
    if (g->p == 1) k3_init<1><<<nb, BS3, 0, g->st>>>(g->g, g->gamma, g->out_dc, g->x, g->cons, g->J, g->status);
    else if (g->p == 2) k3_init<2><<<nb, BS3, 0, g->st>>>(g->g, g->gamma, g->out_dc, g->x, g->cons, g->J, g->status);
    else k3_init<3><<<nb, BS3, 0, g->st>>>(g->g, g->gamma, g->out_dc, g->x, g->cons, g->J, g->status);
    CK3(cudaGetLastError());
    CK3(cudaMemsetAsync(g->xdot, 0, 3 * N * sizeof(double), g->st));
    for (int k = 0; k < 3; ++k) CK3(cudaMemsetAsync(g->zg[k], 0xff, N * sizeof(double), g->st));
    CK3(cudaMemsetAsync(g->t_dev, 0, sizeof(double), g->st));
    int h[2];
    CK3(cudaMemcpyAsync(h, g->status, sizeof h, cudaMemcpyDeviceToHost, g->st));
    CK3(cudaStreamSynchronize(g->st));
    g->xdot_zero = 1;
    if (h[1] > 0) {
        CK3(cudaMemsetAsync(g->status, 0, 2 * sizeof(int), g->st));
        g->has_state = 0;
        return fail3(g, ESMM_ERR_ARG, "non-admissible initial state or tangled mesh");
    }
    g->has_state = 1;
    return ESMM_OK;
}

int esmm3_state_set_cons(esmm3 *g, const double *cons, const double *J, const double *x, double t, int mem)
{
    size_t N = (size_t)g->g.N;
    int rc;
    if ((rc = copy3(g, g->cons, cons, 8 * N, mem, true)) || (rc = copy3(g, g->J, J, N, mem, true)) ||
        (rc = copy3(g, g->x, x, 3 * N, mem, true)))
        return rc;
    g->pin[0] = t;
    CK3(cudaMemcpyAsync(g->t_dev, g->pin, sizeof(double), cudaMemcpyHostToDevice, g->st));
    CK3(cudaMemsetAsync(g->xdot, 0, 3 * N * sizeof(double), g->st));
    for (int k = 0; k < 3; ++k) CK3(cudaMemsetAsync(g->zg[k], 0xff, N * sizeof(double), g->st));
    CK3(cudaStreamSynchronize(g->st));
    g->xdot_zero = 1;
    g->has_state = 1;
    return ESMM_OK;
}

int esmm3_state_get(esmm3 *g, int what, double *out, int mem)
{
    if (!g->has_state) return fail3(g, ESMM_ERR_STATE, "no state");
    size_t N = (size_t)g->g.N;
    int rc = ESMM_OK;
    switch (what) {
    case ESMM_GET_PRIM:
        g->launches++;
        g->nl[ESMM_KIND_OTHER]++;
        k3_prim_out<<<nb3(g->g.N), BS3, 0, g->st>>>(g->g, g->gamma, g->cons, g->J, g->out_dc, g->status);
        CK3(cudaGetLastError());
        rc = copy3(g, out, g->out_dc, 8 * N, mem, false);
        break;
    case ESMM_GET_CONS: rc = copy3(g, out, g->cons, 8 * N, mem, false); break;
    case ESMM_GET_J: rc = copy3(g, out, g->J, N, mem, false); break;
    case ESMM_GET_X: rc = copy3(g, out, g->x, 3 * N, mem, false); break;
    case ESMM_GET_XDOT: rc = copy3(g, out, g->xdot, 3 * N, mem, false); break;
    default: return fail3(g, ESMM_ERR_ARG, "unknown field");
    }
    if (rc) return rc;
    CK3(cudaStreamSynchronize(g->st));
    return what == ESMM_GET_PRIM ? check3(g) : ESMM_OK;
}

int esmm3_get_time(esmm3 *g, double *t)
{
    CK3(cudaMemcpyAsync(g->pin, g->t_dev, sizeof(double), cudaMemcpyDeviceToHost, g->st));
    CK3(cudaStreamSynchronize(g->st));
    *t = g->pin[0];
    return ESMM_OK;
}

// every call that runs a node pass: an inflow end needs its state
static int inflow_ok3(esmm3 *g)
{
    return g->needs_inflow && !g->has_inflow ? fail3(g, ESMM_ERR_STATE, "an inflow end without an inflow state")
                                             : ESMM_OK;
}

int esmm3_set_inflow(esmm3 *g, const double *prim)
{
    CK3(cudaMemcpyAsync(g->inflow_dev, prim, 8 * sizeof(double), cudaMemcpyHostToDevice, g->st));
    CK3(cudaStreamSynchronize(g->st));
    g->has_inflow = 1;
    return ESMM_OK;
}

int esmm3_rhs(esmm3 *g, const double *cons, const double *J, const double *x, const double *xdot, double *dcons,
              double *dJ, int mem)
{
    size_t N = (size_t)g->g.N;
    int rc;
    if ((rc = inflow_ok3(g))) return rc;
    if (mem == ESMM_MEM_HOST) {
        if ((rc = copy3(g, g->in_cons, cons, 8 * N, mem, true)) || (rc = copy3(g, g->in_J, J, N, mem, true)) ||
            (rc = copy3(g, g->in_x, x, 3 * N, mem, true)))
            return rc;
        if (xdot && (rc = copy3(g, g->in_xdot, xdot, 3 * N, mem, true))) return rc;
        cons = g->in_cons;
        J = g->in_J;
        x = g->in_x;
        xdot = xdot ? g->in_xdot : nullptr;
    }
    node3(g, cons, J, x, xdot, nullptr, nullptr);
    fluxes3(g);
    double *dc = mem == ESMM_MEM_HOST ? g->out_dc : dcons;
    double *dj = mem == ESMM_MEM_HOST ? g->out_dJ : dJ;
    update3(g, dc, dj, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, 0.0, nullptr, nullptr, nullptr);
    CK3(cudaGetLastError());
    if (mem == ESMM_MEM_HOST) {
        if ((rc = copy3(g, dcons, g->out_dc, 8 * N, mem, false)) || (rc = copy3(g, dJ, g->out_dJ, N, mem, false)))
            return rc;
        CK3(cudaStreamSynchronize(g->st));
        return check3(g);
    }
    return ESMM_OK;
}

int esmm3_cfl_dt(esmm3 *g, double *dt)
{
    if (!g->has_state) return fail3(g, ESMM_ERR_STATE, "no state");
    if (int rc = inflow_ok3(g)) return rc;
    node3(g, g->cons, g->J, g->x, nullptr, nullptr, nullptr);
    g->launches += 3;
    g->nl[ESMM_KIND_OTHER] += 3;
    k3_red_init<<<1, 32, 0, g->st>>>(g->red);
    k3_cfl<<<nb3(g->g.N), BS3, 0, g->st>>>(g->g, g->gamma, g->q, g->J, g->red, nullptr);
    k3_dt<<<1, 32, 0, g->st>>>(g->prm.cfl, 0.0, g->red, g->ds, g->dt_dev);
    CK3(cudaMemcpyAsync(g->pin, g->dt_dev, sizeof(double), cudaMemcpyDeviceToHost, g->st));
    CK3(cudaStreamSynchronize(g->st));
    *dt = g->pin[0];
    return check3(g);
}

int esmm3_mesh_redistribute(esmm3 *g, double dt, double *xdot, double *dtau, double *dt_used, int mem)
{
    if (!g->has_state) return fail3(g, ESMM_ERR_STATE, "no state");
    if (int rc = inflow_ok3(g)) return rc;
    node3(g, g->cons, g->J, g->x, nullptr, nullptr, nullptr);
    int rc = mesh_and_dt3(g, dt);
    if (rc) return rc;
    if (xdot && (rc = copy3(g, xdot, g->xdot, 3 * (size_t)g->g.N, mem, false))) return rc;
    CK3(cudaMemcpyAsync(g->pin, g->red + 1, sizeof(double), cudaMemcpyDeviceToHost, g->st));
    CK3(cudaMemcpyAsync(g->pin + 1, g->dt_dev, sizeof(double), cudaMemcpyDeviceToHost, g->st));
    CK3(cudaStreamSynchronize(g->st));
    if (dtau) *dtau = g->prm.move_mesh ? g->pin[0] : 0.0;
    if (dt_used) *dt_used = g->pin[1];
    return check3(g);
}

static int rk_step_async3(esmm3 *g, double dt)
{
    node3(g, g->cons, g->J, g->x, nullptr, g->zg[0], g->zg[1]);
    int rc = mesh_and_dt3(g, dt);
    if (rc) return rc;
    {
        Prof3 pr_(g, ESMM_KIND_OTHER);
        k3_tmetric<<<nb3(g->g.P), BS3, 0, g->st>>>(g->g, g->xdot, g->q);
    }
    return stages3(g);
}

int esmm3_rk_step(esmm3 *g, double dt, double *dt_used)
{
    if (!g->has_state) return fail3(g, ESMM_ERR_STATE, "no state");
    if (int rc = inflow_ok3(g)) return rc;
    int rc = rk_step_async3(g, dt);
    if (rc) return rc;
    if (dt_used) {
        CK3(cudaMemcpyAsync(g->pin, g->dt_dev, sizeof(double), cudaMemcpyDeviceToHost, g->st));
        CK3(cudaStreamSynchronize(g->st));
        *dt_used = g->pin[0];
        return check3(g);
    }
    return ESMM_OK;
}

int esmm3_rk_step_given(esmm3 *g, const double *xdot, double dt, int mem)
{
    if (!g->has_state) return fail3(g, ESMM_ERR_STATE, "no state");
    if (int rc = inflow_ok3(g)) return rc;
    int rc = step_given3(g, xdot, dt, mem);
    if (rc) return rc;
    CK3(cudaStreamSynchronize(g->st));
    return check3(g);
}

int esmm3_advance(esmm3 *g, int nsteps, double dt)
{
    if (!g->has_state) return fail3(g, ESMM_ERR_STATE, "no state");
    if (int rc = inflow_ok3(g)) return rc;
    for (int s = 0; s < nsteps; ++s) {
        int rc = rk_step_async3(g, dt);
        if (rc) return rc;
    }
    return ESMM_OK;
}

int esmm3_totals(esmm3 *g, double out[3])
{
    if (!g->has_state) return fail3(g, ESMM_ERR_STATE, "no state");
    if (int rc = inflow_ok3(g)) return rc;
    node3(g, g->cons, g->J, g->x, nullptr, nullptr, nullptr);
    unsigned nb = nb3(g->g.N);
    g->launches += 2;
    g->nl[ESMM_KIND_OTHER] += 2;
    k3_totals<<<nb, BS3, 0, g->st>>>(g->g, g->gamma, g->q, g->cons, g->J, g->partials);
    k3_totals_final<<<1, 32, 0, g->st>>>((int)nb, g->partials, g->tot);
    CK3(cudaMemcpyAsync(g->pin, g->tot, 3 * sizeof(double), cudaMemcpyDeviceToHost, g->st));
    CK3(cudaStreamSynchronize(g->st));
    for (int k = 0; k < 3; ++k) out[k] = g->pin[k];
    return check3(g);
}

int esmm3_last_error(esmm3 *g, int *n_c2p_fail, char *msg, int len)
{
    int h[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(h, g->status, sizeof h, cudaMemcpyDeviceToHost, g->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
    if (e == cudaSuccess) cudaMemsetAsync(g->status, 0, sizeof(int), g->st);
    if (n_c2p_fail) *n_c2p_fail = h[0];
    if (msg && len > 0) {
        strncpy(msg, g->msg, (size_t)len - 1);
        msg[len - 1] = 0;
    }
    return e == cudaSuccess ? ESMM_OK : ESMM_ERR_CUDA;
}

long long esmm3_launches(const esmm3 *g) { return g->launches; }

int esmm3_profile(esmm3 *g, int mask)
{
    CK3(cudaStreamSynchronize(g->st));
    if (!g->ev) g->ev = new (std::nothrow) std::vector<std::pair<cudaEvent_t, cudaEvent_t>>[ESMM_NKINDS];
    if (!g->ev) return fail3(g, ESMM_ERR_ARG, "out of host memory");
    prof_clear3(g);
    for (int k = 0; k < ESMM_NKINDS; ++k) g->nl[k] = 0;
    g->prof_mask = mask;
    return ESMM_OK;
}

int esmm3_profile_read(esmm3 *g, double ms[ESMM_NKINDS], long long launches[ESMM_NKINDS],
                       long long timed[ESMM_NKINDS])
{
    CK3(cudaStreamSynchronize(g->st));
    for (int k = 0; k < ESMM_NKINDS; ++k) {
        double acc = 0.0;
        if (g->ev)
            for (auto &pr : g->ev[k]) {
                float t = 0.0f;
                CK3(cudaEventElapsedTime(&t, pr.first, pr.second));
                acc += t;
            }
        if (ms) ms[k] = acc;
        if (launches) launches[k] = g->nl[k];
        if (timed) timed[k] = g->ev ? (long long)g->ev[k].size() : 0;
    }
    return ESMM_OK;
}

// ---- adjoint entry points --------------------------------------------------------
int esmm3_rhs_vjp(esmm3 *g, const double *cons, const double *J, const double *x, const double *xdot,
                  const double *mu, double *lam, int mem)
{
    int rc;
    if ((rc = adj_alloc3(g))) return rc;
    size_t N = (size_t)g->g.N;
    if (mem == ESMM_MEM_HOST) {
        if ((rc = copy3(g, g->in_cons, cons, 8 * N, mem, true)) || (rc = copy3(g, g->in_J, J, N, mem, true)) ||
            (rc = copy3(g, g->in_x, x, 3 * N, mem, true)) || (rc = copy3(g, g->lam_a, mu, 8 * N, mem, true)))
            return rc;
        if (xdot && (rc = copy3(g, g->in_xdot, xdot, 3 * N, mem, true))) return rc;
        cons = g->in_cons;
        J = g->in_J;
        x = g->in_x;
        xdot = xdot ? g->in_xdot : nullptr;
        mu = g->lam_a;
    }
    double *out = mem == ESMM_MEM_HOST ? g->lam_v : lam;
    if ((rc = rhs_vjp_core3(g, cons, J, x, xdot, mu, out))) return rc;
    if (mem == ESMM_MEM_HOST) {
        if ((rc = copy3(g, lam, g->lam_v, 8 * N, mem, false))) return rc;
        CK3(cudaStreamSynchronize(g->st));
        return check3(g);
    }
    return ESMM_OK;
}

int esmm3_adjoint_record(esmm3 *g, int nsteps, double dt)
{
    if (!g->has_state) return fail3(g, ESMM_ERR_STATE, "no state");
    int rc;
    if ((rc = adj_alloc3(g))) return rc;
    size_t N = (size_t)g->g.N, d = sizeof(double);
    g->ck_dt->clear();
    g->ck_n = 0;
    for (int n = 0; n < nsteps; ++n) {
        if ((int)g->ck->size() <= n) {
            double *b = nullptr;
            CK3(cudaMalloc((void **)&b, 15 * N * d));   // cons, J, x, xdot
            g->ck->push_back(b);
        }
        double *b = (*g->ck)[n];
        CK3(cudaMemcpyAsync(b, g->cons, 8 * N * d, cudaMemcpyDeviceToDevice, g->st));
        CK3(cudaMemcpyAsync(b + 8 * N, g->J, N * d, cudaMemcpyDeviceToDevice, g->st));
        CK3(cudaMemcpyAsync(b + 9 * N, g->x, 3 * N * d, cudaMemcpyDeviceToDevice, g->st));
        if ((rc = rk_step_async3(g, dt))) return rc;
        CK3(cudaMemcpyAsync(b + 12 * N, g->xdot, 3 * N * d, cudaMemcpyDeviceToDevice, g->st));
        CK3(cudaMemcpyAsync(g->pin, g->dt_dev, d, cudaMemcpyDeviceToHost, g->st));
        CK3(cudaStreamSynchronize(g->st));
        g->ck_dt->push_back(g->pin[0]);
        g->ck_n = n + 1;
    }
    return check3(g);
}

int esmm3_adjoint_steps(esmm3 *g, int *nsteps, double *dt)
{
    *nsteps = g->ck_n;
    if (dt)
        for (int n = 0; n < g->ck_n; ++n) dt[n] = (*g->ck_dt)[n];
    return ESMM_OK;
}

int esmm3_adjoint_checkpoint(esmm3 *g, int step, int what, double *out, int mem)
{
    if (step < 0 || step >= g->ck_n) return ESMM_ERR_ARG;
    size_t N = (size_t)g->g.N;
    const double *b = (*g->ck)[step];
    int rc;
    switch (what) {
    case ESMM_GET_CONS: rc = copy3(g, out, b, 8 * N, mem, false); break;
    case ESMM_GET_J: rc = copy3(g, out, b + 8 * N, N, mem, false); break;
    case ESMM_GET_X: rc = copy3(g, out, b + 9 * N, 3 * N, mem, false); break;
    case ESMM_GET_XDOT: rc = copy3(g, out, b + 12 * N, 3 * N, mem, false); break;
    default: return fail3(g, ESMM_ERR_ARG, "unknown field");
    }
    if (rc) return rc;
    CK3(cudaStreamSynchronize(g->st));
    return ESMM_OK;
}

int esmm3_adjoint_replay(esmm3 *g, int nsteps)
{
    if (nsteps < 0 || nsteps > g->ck_n) return ESMM_ERR_ARG;
    if (!g->has_state) return fail3(g, ESMM_ERR_STATE, "no state");
    size_t N = (size_t)g->g.N;
    for (int n = 0; n < nsteps; ++n) {
        int rc = step_given3(g, (*g->ck)[n] + 12 * N, (*g->ck_dt)[n], ESMM_MEM_DEVICE);
        if (rc) return rc;
    }
    CK3(cudaStreamSynchronize(g->st));
    return check3(g);
}

// the three SSP-RK3 stages in reverse, per recorded step (as in 2D)
int esmm3_adjoint_vjp(esmm3 *g, const double *lam_final, double *lam_cons0, double *lam_prim0, int mem)
{
    if (g->ck_n < 1) return fail3(g, ESMM_ERR_STATE, "no recorded steps");
    int rc;
    if ((rc = adj_alloc3(g))) return rc;
    size_t N = (size_t)g->g.N;
    const long long n8 = 8 * (long long)N;
    double *la = g->lam_a, *lb = g->lam_b, *lc = g->lam_c, *v = g->lam_v;
    if ((rc = copy3(g, la, lam_final, 8 * N, mem, true))) return rc;
    for (int n = g->ck_n - 1; n >= 0; --n) {
        double *b = (*g->ck)[n];
        double *c0 = b, *J0 = b + 8 * N, *x0 = b + 9 * N, *xd = b + 12 * N;
        const double dt = (*g->ck_dt)[n];
        if ((rc = set_dt3(g, dt))) return rc;
        CK3(cudaMemcpyAsync(g->xdot, xd, 3 * N * sizeof(double), cudaMemcpyDeviceToDevice, g->st));
        g->xdot_zero = 0;
        // recompute the stage states (c1, J1, x1), (c2, J2, x2)
        node3(g, c0, J0, x0, xd, nullptr, nullptr);
        fluxes3(g);
        update3(g, nullptr, nullptr, c0, J0, x0, c0, J0, x0, 0.0, 1.0, g->c1, g->J1, g->x1);
        node3(g, g->c1, g->J1, g->x1, xd, nullptr, nullptr);
        fluxes3(g);
        update3(g, nullptr, nullptr, c0, J0, x0, g->c1, g->J1, g->x1, 0.75, 0.25, g->c2, g->J2, g->x2);
        // stage 3: c3 = 1/3 c0 + 2/3 (c2 + dt L(c2))
        if ((rc = rhs_vjp_core3(g, g->c2, g->J2, g->x2, xd, la, v))) return rc;
        launch3_lincomb(n8, 2.0 / 3.0, la, 2.0 / 3.0 * dt, v, lb, g->st);    // lambda_c2
        launch3_lincomb(n8, 1.0 / 3.0, la, 0.0, nullptr, lc, g->st);         // lambda_c0
        // stage 2: c2 = 3/4 c0 + 1/4 (c1 + dt L(c1))
        if ((rc = rhs_vjp_core3(g, g->c1, g->J1, g->x1, xd, lb, v))) return rc;
        launch3_lincomb(n8, 0.25, lb, 0.25 * dt, v, la, g->st);              // lambda_c1
        launch3_lincomb(n8, 1.0, lc, 0.75, lb, lc, g->st);
        // stage 1: c1 = c0 + dt L(c0)
        if ((rc = rhs_vjp_core3(g, c0, J0, x0, xd, la, v))) return rc;
        launch3_lincomb(n8, 1.0, lc, 1.0, la, lc, g->st);
        launch3_lincomb(n8, 1.0, lc, dt, v, la, g->st);                      // lambda of c^n
        g->launches += 6;
    }
    CK3(cudaGetLastError());
    if (lam_cons0 && (rc = copy3(g, lam_cons0, la, 8 * N, mem, false))) return rc;
    if (lam_prim0) {
        double *b0 = (*g->ck)[0];
        launch3_prim_grad(g->g, g->gamma, b0, b0 + 8 * N, la, v, g->status, g->st);
        if ((rc = copy3(g, lam_prim0, v, 8 * N, mem, false))) return rc;
    }
    CK3(cudaStreamSynchronize(g->st));
    return check3(g);
}
