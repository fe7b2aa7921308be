// esmm_3d_iface.cu -- instantiations of the 3D interface-flux kernel (its
// own translation unit: the kernel, with the RMHD eigen-system inlined, is the
// slowest to compile).
#include "esmm_3d.cuh"

namespace esmm {
namespace d3 {

template <int P>
static void iface3_p(const Geom3 &g, const Phys &ph, int w, const double *q, double *iflux, int dir, unsigned nb,
                     cudaStream_t st)
{
    switch (w) {
    case 0: k3_iface<P, 0><<<nb, 128, 0, st>>>(g, ph, q, iflux, dir); break;
    case 3: k3_iface<P, 3><<<nb, 128, 0, st>>>(g, ph, q, iflux, dir); break;
    default: k3_iface<P, 5><<<nb, 128, 0, st>>>(g, ph, q, iflux, dir); break;
    }
}

void launch3_iface(const Geom3 &g, const Phys &ph, int p, int w, const double *q, double *iflux, int dir,
                   unsigned nb, cudaStream_t st)
{
    if (p == 1) iface3_p<1>(g, ph, w, q, iflux, dir, nb, st);
    else if (p == 2) iface3_p<2>(g, ph, w, q, iflux, dir, nb, st);
    else iface3_p<3>(g, ph, w, q, iflux, dir, nb, st);
}

}  // namespace d3
}  // namespace esmm
