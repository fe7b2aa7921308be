// esmm_sweep_f64.cu -- the fused sweep kernel instantiated for the double working precision.
#include "esmm_sweep.cuh"

namespace esmm {

void launch_sweep_f64(const LaunchDom &L, const Phys &ph, const double *q, const float *q32, void *iflux, int dir,
                      cudaStream_t st)
{
    launch_sweep_t<double>(L, ph, q, q32, iflux, dir, st);
}

int sweep_occupancy_f64(int p, int w, int bs) { return sweep_occupancy_t<double>(p, w, bs); }

}  // namespace esmm
