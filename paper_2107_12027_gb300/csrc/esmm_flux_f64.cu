// esmm_flux_f64.cu -- flux kernels instantiated for the double working precision.
#include "esmm_flux.cuh"

namespace esmm {

void launch_pairs_f64(const LaunchDom &L, const Phys &ph, const double *q, const float *q32, void *pairs, int dir,
                      cudaStream_t st)
{
    launch_pairs_t<double>(L, ph, q, q32, pairs, dir, st);
}

void launch_iface_f64(const LaunchDom &L, const Phys &ph, const double *q, const float *q32, const void *pairs,
                      void *iflux, int dir, cudaStream_t st)
{
    launch_iface_t<double>(L, ph, q, q32, pairs, iflux, dir, st);
}

int flux_occupancy_f64(int kind, int p, int w, int bs) { return flux_occupancy_t<double>(kind, p, w, bs); }

}  // namespace esmm
