// esmm_launch.h -- host-side launchers of the flux kernels, one translation
// unit per working precision (esmm_flux_f64.cu, esmm_flux_f32.cu).
#pragma once

#include <cuda_runtime.h>

#include "esmm_device.cuh"

namespace esmm {

// Launch domain of one kernel: the problem addressing and the grid shape.
struct LaunchDom {
    ProbArg pa;
    unsigned nblk;
    int bs;
};

struct Phys;

// Pair fluxes of direction dir; pairs holds PMAX * 4 * 2 arrays of P elements
// of the working precision (double or float).
void launch_pairs_f64(const LaunchDom &L, const Phys &ph, const double *q, void *pairs, int dir, cudaStream_t st);
void launch_pairs_f32(const LaunchDom &L, const Phys &ph, const double *q, void *pairs, int dir, cudaStream_t st);
// Interface fluxes (4 components + metric flux) of direction dir.
void launch_iface_f64(const LaunchDom &L, const Phys &ph, const double *q, const void *pairs, void *iflux, int dir,
                      cudaStream_t st);
void launch_iface_f32(const LaunchDom &L, const Phys &ph, const double *q, const void *pairs, void *iflux, int dir,
                      cudaStream_t st);

}  // namespace esmm
