// esmm_mhd.cu -- RMHD kernels (esmm_mhd.cuh) and their host launchers
// (declared in esmm_launch.h).
#include "esmm_launch.h"
#include "esmm_mhd.cuh"
#include "esmm_reduce.cuh"

namespace esmm {

__global__ void k_prim_out_mhd(ProbArg pa, double gam, const double *__restrict__ cons,
                               const double *__restrict__ J, double *__restrict__ prim, int *status)
{
    ProbDesc D;
    long long lb;
    locate(pa, D, lb);
    const Geom &g = D.g;
    long long id = lb * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    double iJ = 1.0 / J[id];
    double U[8], w[8], Z;
#pragma unroll
    for (int a = 0; a < 8; ++a) U[a] = cons[a * g.N + id] * iJ;
    if (cons2prim_mhd(gam, U, -1.0, w, Z)) atomicAdd(status, 1);
#pragma unroll
    for (int a = 0; a < 8; ++a) prim[a * g.N + id] = w[a];
}


// Spectral radius of the 8-wave system per node and direction (eq. cfl),
// with the speeds from the eigen-system in the working precision R (FP32 in
// the mixed form: the step carries ~1e-6 relative rounding, harmless for a
// stability bound).
// With cflb (the moving-mesh step) also the speed bounds L_k lambda_min/J and
// L_k lambda_max/J of every node into its rows 2 + k and 4 + k.
template <typename R>
__global__ void k_cfl_mhd(ProbArg pa, double gam, const double *__restrict__ q, const double *__restrict__ J,
                          unsigned long long *red, double *__restrict__ cflb)
{
    ProbDesc D;
    long long lb;
    int b = locate(pa, D, lb);
    const Geom &g = D.g;
    long long id = lb * blockDim.x + threadIdx.x;
    double r[2] = {0.0, 0.0};
    if (id < g.N) {
        int i = (int)(id % g.nx), j = (int)(id / g.nx);
        long long c = pidx(g, i, j);
        double iW = 1.0 / q[Q_W * g.P + c];
        double w[8] = {q[Q_RHO * g.P + c], q[Q_UX * g.P + c] * iW, q[Q_UY * g.P + c] * iW,
                       q[QM_UZ * g.P + c] * iW, q[Q_P * g.P + c], q[QM_B1 * g.P + c], q[QM_B2 * g.P + c],
                       q[QM_B3 * g.P + c]};
        double iJ = 1.0 / J[id];
        for (int k = 0; k < 2; ++k) {
            double mx = q[(Q_M00 + 2 * k) * g.P + c], my = q[(Q_M01 + 2 * k) * g.P + c];
            double Lk = sqrt(mx * mx + my * my);
            double nx = mx / Lk, ny = my / Lk;
            R wr[8] = {(R)w[0], (R)(nx * w[1] + ny * w[2]), (R)(-ny * w[1] + nx * w[2]), (R)w[3],
                       (R)w[4], (R)(nx * w[5] + ny * w[6]), (R)(-ny * w[5] + nx * w[6]), (R)w[7]};
            R lam[8], Rm[8][8];
            eigen_mhd<R>(gam, wr, lam, Rm, false);
            double a = 0.0, lo = (double)lam[0], hi = (double)lam[0];
            for (int m = 0; m < 8; ++m) {
                a = fmax(a, fabs((double)lam[m]));
                lo = fmin(lo, (double)lam[m]);
                hi = fmax(hi, (double)lam[m]);
            }
            r[k] = owned_row(g, j) ? Lk * a * iJ : 0.0;
            if (cflb) {
                cflb[6 * D.on + (2 + k) * g.N + id] = Lk * lo * iJ;
                cflb[6 * D.on + (4 + k) * g.N + id] = Lk * hi * iJ;
            }
        }
    }
    for (int k = 0; k < 2; ++k) {
        double m = block_reduce<0>(r[k]);
        if (threadIdx.x == 0) atomic_max_nonneg(red + (long long)NRED * b + 2 + k, m);
    }
}

void launch_node_mhd(const LaunchDom &L, int p, double gam, const double *cons, const double *J, const double *x,
                     const double *xdot, const double *zg_in, double *zg_out, double *q, int *status,
                     const double *inflow, int f32_logs, cudaStream_t st)
{
    if (p == 1)
        k_node_mhd<1><<<L.nblk, L.bs, 0, st>>>(L.pa, gam, cons, J, x, xdot, zg_in, zg_out, q, status, inflow,
                                               f32_logs);
    else if (p == 2)
        k_node_mhd<2><<<L.nblk, L.bs, 0, st>>>(L.pa, gam, cons, J, x, xdot, zg_in, zg_out, q, status, inflow,
                                               f32_logs);
    else
        k_node_mhd<3><<<L.nblk, L.bs, 0, st>>>(L.pa, gam, cons, J, x, xdot, zg_in, zg_out, q, status, inflow,
                                               f32_logs);
}

void launch_iface_mhd(const LaunchDom &L, const Phys &ph, const double *q, void *iflux, int dir, cudaStream_t st)
{
    launch_iface_mhd_t<double>(L, ph, q, iflux, dir, st);
}

void launch_update_mhd(const LaunchDom &L, const double *q, const void *fl, double *dcons, double *dJ,
                       const double *cn, const double *Jn, const double *xn, const double *cs, const double *Js,
                       const double *xs, const double *xdot, double A, double B, const double *dt_dev, double *co,
                       double *Jo, double *xo, cudaStream_t st)
{
    launch_update_mhd_t<double>(L, q, fl, dcons, dJ, cn, Jn, xn, cs, Js, xs, xdot, A, B, dt_dev, co, Jo, xo, st);
}

void launch_cfl_mhd(const LaunchDom &L, double gam, const double *q, const double *J, unsigned long long *red,
                    bool f32, double *cflb, cudaStream_t st)
{
    if (f32) k_cfl_mhd<float><<<L.nblk, L.bs, 0, st>>>(L.pa, gam, q, J, red, cflb);
    else k_cfl_mhd<double><<<L.nblk, L.bs, 0, st>>>(L.pa, gam, q, J, red, cflb);
}

void launch_init_mhd(const LaunchDom &L, int p, double gam, const double *prim, const double *x, double *cons,
                     double *J, int *status, cudaStream_t st)
{
    if (p == 1) k_init_state_mhd<1><<<L.nblk, L.bs, 0, st>>>(L.pa, gam, prim, x, cons, J, status);
    else if (p == 2) k_init_state_mhd<2><<<L.nblk, L.bs, 0, st>>>(L.pa, gam, prim, x, cons, J, status);
    else k_init_state_mhd<3><<<L.nblk, L.bs, 0, st>>>(L.pa, gam, prim, x, cons, J, status);
}

void launch_prim_out_mhd(const LaunchDom &L, double gam, const double *cons, const double *J, double *prim,
                         int *status, cudaStream_t st)
{
    k_prim_out_mhd<<<L.nblk, L.bs, 0, st>>>(L.pa, gam, cons, J, prim, status);
}

}  // namespace esmm
