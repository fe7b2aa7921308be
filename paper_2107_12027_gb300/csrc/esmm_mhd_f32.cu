// esmm_mhd_f32.cu -- the RMHD interface and update kernels instantiated for
// the FP32 bulk form (FP64 recovery, near-equal log means and state).
#include "esmm_launch.h"
#include "esmm_mhd.cuh"

namespace esmm {

void launch_iface_mhd_f32(const LaunchDom &L, const Phys &ph, const double *q, void *iflux, int dir,
                          cudaStream_t st)
{
    launch_iface_mhd_t<float>(L, ph, q, iflux, dir, st);
}

void launch_update_mhd_f32(const LaunchDom &L, const double *q, const void *fl, double *dcons, double *dJ,
                           const double *cn, const double *Jn, const double *xn, const double *cs, const double *Js,
                           const double *xs, const double *xdot, double A, double B, const double *dt_dev,
                           double *co, double *Jo, double *xo, cudaStream_t st)
{
    launch_update_mhd_t<float>(L, q, fl, dcons, dJ, cn, Jn, xn, cs, Js, xs, xdot, A, B, dt_dev, co, Jo, xo, st);
}

}  // namespace esmm
