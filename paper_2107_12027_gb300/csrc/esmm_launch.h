// esmm_launch.h -- host-side launchers of the kernels that live outside
// esmm_api.cu: the RHD flux kernels (one translation unit per working
// precision: esmm_flux_f64.cu, esmm_flux_f32.cu, and the fused sweep in
// esmm_sweep_f64.cu, esmm_sweep_f32.cu), the adjoint
// (esmm_adjoint.cu) and the RMHD kernels (esmm_mhd.cu).
#pragma once

#include <cuda_runtime.h>

#include "esmm_device.cuh"

namespace esmm {

// Launch domain of one kernel: the problem addressing and the grid shape.
// The RHD flux kernels also take a tile shape (tx threads along x_1 by
// bs / tx along x_2; 0: one flat run of sites along the sweep) and the
// number of tiles, over which a grid of nblk <= ntiles blocks strides
// (nblk < ntiles: a persistent grid).  ntiles < 0 means nblk.
struct LaunchDom {
    ProbArg pa;
    unsigned nblk;
    int bs;
    int tx = 0;
    long long ntiles = -1;
};

// resident blocks per SM of the RHD flux kernels at block size bs (the
// persistent grid of a tiled launch): kind 0 pairs, 1 interfaces
int flux_occupancy_f64(int kind, int p, int w, int bs);
int flux_occupancy_f32(int kind, int p, int w, int bs);

// The fused sweep kernel of one 2D RHD direction (esmm_sweep_f64.cu,
// esmm_sweep_f32.cu): pair and interface fluxes in one launch, bs / 32
// lines per block, one segment of 33 - p interfaces per line and tile.
void launch_sweep_f64(const LaunchDom &L, const Phys &ph, const double *q, const float *q32, void *iflux, int dir,
                      cudaStream_t st);
void launch_sweep_f32(const LaunchDom &L, const Phys &ph, const double *q, const float *q32, void *iflux, int dir,
                      cudaStream_t st);
int sweep_occupancy_f64(int p, int w, int bs);
int sweep_occupancy_f32(int p, int w, int bs);
// tiles of one problem in the fused sweep of direction dir with nw lines per block
inline long long sweep_tiles(const Geom &g, int dir, int p, int nw)
{
    const long long nd = dir == 0 ? g.nx : g.ny, no = dir == 0 ? g.ny : g.nx;
    const long long ta = 33 - p;
    return ((no + nw - 1) / nw) * ((nd + 1 + ta - 1) / ta);
}

struct Phys;

// Pair fluxes of direction dir; pairs holds PMAX * 4 * 2 arrays of P elements
// of the working precision (double or float).  q32: the FP32 copies of the
// node arrays ([NQ32][P]), read by the float kernels (unused by the FP64 ones).
void launch_pairs_f64(const LaunchDom &L, const Phys &ph, const double *q, const float *q32, void *pairs, int dir,
                      cudaStream_t st);
void launch_pairs_f32(const LaunchDom &L, const Phys &ph, const double *q, const float *q32, void *pairs, int dir,
                      cudaStream_t st);
// Interface fluxes (4 components + metric flux) of direction dir.
void launch_iface_f64(const LaunchDom &L, const Phys &ph, const double *q, const float *q32, const void *pairs,
                      void *iflux, int dir, cudaStream_t st);
void launch_iface_f32(const LaunchDom &L, const Phys &ph, const double *q, const float *q32, const void *pairs,
                      void *iflux, int dir, cudaStream_t st);

// Adjoint (esmm_adjoint.cu): local Jacobian-vector products of the pair and
// interface fluxes against the node adjoint mu ([4][N]) of d(cons)/dt, written
// per (pair | interface, node, quantity); the node kernel gathers them and
// adds (d rhs/d cons)^T mu into lam ([4][N], accumulated).
void launch_pairs_vjp(const LaunchDom &L, const Phys &ph, const double *q, const double *mu, double *Gp, int dir,
                      cudaStream_t st);
void launch_iface_vjp(const LaunchDom &L, const Phys &ph, const double *q, const double *mu, double *G, int dir,
                      cudaStream_t st);
void launch_node_vjp(const LaunchDom &L, double gam, int p, int w, const double *q, const double *G,
                     const double *Gp, const double *J, double *lam, cudaStream_t st);
void launch_lincomb(long long n, double a, const double *x, double b, const double *y, double *out, cudaStream_t st);
void launch_prim_grad(const LaunchDom &L, double gam, const double *cons, const double *J, const double *lam,
                      double *out, cudaStream_t st);
// RMHD (esmm_mhd.cu), single problems: node pass (zg: warm starts of
// Z = rho h W^2), interface fluxes (10 values per direction: F[8], the metric
// flux, the magnetic flux B~), update with the Powell source, CFL radius,
// state set-up and read-out, all FP64; the _f32 pair (esmm_mhd_f32.cu) keeps
// the interface fluxes in FP32 for the mixed form.  The node arrays hold 18
// fields per padded node.
constexpr int NQ_MHD = 18;
constexpr int NF_MHD = 10;
void launch_node_mhd(const LaunchDom &L, int p, double gam, const double *cons, const double *J, const double *x,
                     const double *xdot, const double *zg_in, double *zg_out, double *q, int *status,
                     const double *inflow, int f32_logs, cudaStream_t st);
void launch_iface_mhd(const LaunchDom &L, const Phys &ph, const double *q, void *iflux, int dir, cudaStream_t st);
void launch_update_mhd(const LaunchDom &L, const double *q, const void *fl, double *dcons, double *dJ,
                       const double *cn, const double *Jn, const double *xn, const double *cs, const double *Js,
                       const double *xs, const double *xdot, double A, double B, const double *dt_dev, double *co,
                       double *Jo, double *xo, cudaStream_t st);
void launch_iface_mhd_f32(const LaunchDom &L, const Phys &ph, const double *q, void *iflux, int dir,
                          cudaStream_t st);
void launch_update_mhd_f32(const LaunchDom &L, const double *q, const void *fl, double *dcons, double *dJ,
                           const double *cn, const double *Jn, const double *xn, const double *cs, const double *Js,
                           const double *xs, const double *xdot, double A, double B, const double *dt_dev,
                           double *co, double *Jo, double *xo, cudaStream_t st);
void launch_cfl_mhd(const LaunchDom &L, double gam, const double *q, const double *J, unsigned long long *red,
                    bool f32, double *cflb, cudaStream_t st);
void launch_init_mhd(const LaunchDom &L, int p, double gam, const double *prim, const double *x, double *cons,
                     double *J, int *status, cudaStream_t st);
void launch_prim_out_mhd(const LaunchDom &L, double gam, const double *cons, const double *J, double *prim,
                         int *status, cudaStream_t st);

// RMHD adjoint (esmm_mhd_adjoint.cu): node-quantity adjoints lamq[11][P]
// accumulated by the pair and interface passes, then the node pass.
void launch_pairs_vjp_mhd(const LaunchDom &L, const Phys &ph, const double *q, const double *mu, double *lamq,
                          int dir, cudaStream_t st);
void launch_iface_vjp_mhd(const LaunchDom &L, const Phys &ph, const double *q, const double *mu, double *lamq,
                          int dir, cudaStream_t st);
void launch_node_vjp_mhd(const LaunchDom &L, double gam, const double *q, const double *lamq, const double *iflux,
                         const double *mu, const double *J, double *lam, cudaStream_t st);
void launch_prim_grad_mhd(const LaunchDom &L, double gam, const double *cons, const double *J, const double *lam,
                          double *out, int *status, cudaStream_t st);
constexpr long long ADJ_LAMQ_PER_NODE = 11;
// esmm_mhd_eigen (host arrays): 0, or 1 on a CUDA failure
int mhd_eigen_host(double gam, int n, const double *w, const double *dw, double *lam, double *R, double *dlam,
                   double *dR);

// sizes of the adjoint's contribution buffers, in doubles per padded node
constexpr long long ADJ_G_PER_NODE = 2 * 6 * 7;
constexpr long long ADJ_GP_PER_NODE = 2 * PMAX * 2 * 7;

}  // namespace esmm
