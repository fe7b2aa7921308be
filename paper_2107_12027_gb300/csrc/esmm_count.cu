// esmm_count.cu -- algorithmic operation counts of the 2D RHD flux arithmetic
// (a measurement addition; the paper has no counterpart).
//
// The flux templates of esmm_flux.cuh / esmm_device.cuh are evaluated on a
// counting number type by one thread, for one node pair (ec_pair) and for
// the dissipation of one interface (es_dissipation): every add, subtract,
// multiply, divide, reciprocal, square root and reciprocal square root
// counts as one operation; negation, comparison, absolute value and max as
// none.  These are the operations the method asks for as this library
// writes it; the profiler's executed-instruction counts also include the
// instruction sequences that implement each divide and root.
#include <cuda_runtime.h>

#include "esmm.h"
#include "esmm_flux.cuh"

namespace esmm {

__device__ unsigned long long g_nops;

struct cnt {
    double v;
    __device__ cnt() {}
    __device__ cnt(double a) : v(a) {}
};
__device__ __forceinline__ cnt op1(double r)
{
    ++g_nops;
    return cnt(r);
}
__device__ __forceinline__ cnt operator+(cnt a, cnt b) { return op1(a.v + b.v); }
__device__ __forceinline__ cnt operator-(cnt a, cnt b) { return op1(a.v - b.v); }
__device__ __forceinline__ cnt operator*(cnt a, cnt b) { return op1(a.v * b.v); }
__device__ __forceinline__ cnt operator/(cnt a, cnt b) { return op1(a.v / b.v); }
__device__ __forceinline__ cnt operator-(cnt a) { return cnt(-a.v); }
__device__ __forceinline__ cnt operator+(cnt a, double b) { return op1(a.v + b); }
__device__ __forceinline__ cnt operator+(double a, cnt b) { return op1(a + b.v); }
__device__ __forceinline__ cnt operator-(cnt a, double b) { return op1(a.v - b); }
__device__ __forceinline__ cnt operator-(double a, cnt b) { return op1(a - b.v); }
__device__ __forceinline__ cnt operator*(cnt a, double b) { return op1(a.v * b); }
__device__ __forceinline__ cnt operator*(double a, cnt b) { return op1(a * b.v); }
__device__ __forceinline__ cnt operator/(cnt a, double b) { return op1(a.v / b); }
__device__ __forceinline__ cnt operator/(double a, cnt b) { return op1(a / b.v); }
__device__ __forceinline__ cnt &operator+=(cnt &a, cnt b) { a = a + b; return a; }
__device__ __forceinline__ cnt &operator-=(cnt &a, cnt b) { a = a - b; return a; }
__device__ __forceinline__ cnt &operator*=(cnt &a, cnt b) { a = a * b; return a; }
__device__ __forceinline__ double val(cnt x) { return x.v; }
__device__ __forceinline__ cnt vmax(cnt a, cnt b) { return a.v >= b.v ? a : b; }
__device__ __forceinline__ int sgn_d(cnt a) { return (a.v > 0.0) - (a.v < 0.0); }
__device__ __forceinline__ bool le(cnt a, cnt b) { return a.v <= b.v; }
template <> struct LogT<cnt> { using type = cnt; };
template <> __device__ __forceinline__ cnt rcp<cnt>(cnt x) { return op1(1.0 / x.v); }
template <> __device__ __forceinline__ cnt rsq<cnt>(cnt x) { return op1(rsqrt(x.v)); }
template <> __device__ __forceinline__ cnt sq_rt<cnt>(cnt x) { return op1(sqrt(x.v)); }
template <> __device__ __forceinline__ cnt fab<cnt>(cnt x) { return cnt(fabs(x.v)); }

namespace {

// a generic node (no equal neighbours): rho, v_x, v_y, p and the parameter
// variables of the flux arguments
__device__ void node_state(double rho, double vx, double vy, double p, cnt st[6], NodeV<cnt> &nv)
{
    const double W = 1.0 / sqrt(1.0 - vx * vx - vy * vy), beta = rho / p;
    st[0] = cnt(beta);
    st[1] = cnt(W * vx);
    st[2] = cnt(W * vy);
    st[3] = cnt(W);
    st[4] = cnt(log(rho));
    st[5] = cnt(log(beta));
    nv.rho = cnt(rho);
    nv.beta = cnt(beta);
    nv.lnr = st[4];
    nv.lnb = st[5];
    nv.r = cnt(rho);
    nv.b = cnt(beta);
    nv.ux = st[1];
    nv.uy = st[2];
    nv.W = st[3];
}

__global__ void k_count_rhd(double gamma, int w, unsigned long long *out)
{
    if (threadIdx.x || blockIdx.x) return;
    Phys ph;
    ph.gamma = gamma;
    ph.gm1i = 1.0 / (gamma - 1.0);
    ph.eps = 1e-6;
    ph.ln_thr = 1e-4;
    ph.sign_tol = 1e-10;
    cnt st[6][6];
    NodeV<cnt> nv[6];
    const double rho[6] = {0.5, 0.62, 0.71, 0.66, 0.58, 0.47}, p[6] = {0.3, 0.36, 0.45, 0.41, 0.33, 0.29};
    const double vx[6] = {0.2, 0.15, 0.1, 0.05, 0.12, 0.18}, vy[6] = {-0.1, 0.0, 0.3, 0.25, 0.1, -0.05};
    for (int k = 0; k < 6; ++k) node_state(rho[k], vx[k], vy[k], p[k], st[k], nv[k]);
    cnt f[4];
    g_nops = 0;
    ec_pair<cnt>(nv[2], nv[3], cnt(0.05), cnt(1.1), cnt(0.1), cnt(ph.gm1i), ph.ln_thr, f);
    out[0] = g_nops;
    cnt diss[4];
    g_nops = 0;
    if (w == 5) {
        ArrStencil<cnt, 6> s{st};
        es_dissipation<cnt, cnt, 5>(cnt(1.1), cnt(0.1), cnt(0.05), nv[2].rho, nv[3].rho, nv[2].lnr, nv[3].lnr,
                                    nv[2].r, nv[3].r, s, ph, diss);
    } else {
        ArrStencil<cnt, 4> s{st + 1};
        es_dissipation<cnt, cnt, 3>(cnt(1.1), cnt(0.1), cnt(0.05), nv[2].rho, nv[3].rho, nv[2].lnr, nv[3].lnr,
                                    nv[2].r, nv[3].r, s, ph, diss);
    }
    out[1] = g_nops;
}

}  // namespace
}  // namespace esmm

// ops[0]: one two-point EC flux; ops[1]: the ES dissipation of one interface
// (w = 3 or 5); ops[2]: the interface kernel's combination of the pair
// fluxes (eq. ECFlux_O2p and the metric flux: per component p(p-1)/2 adds
// inside the n-sums, p multiplies by alpha_{p,n} and p - 1 adds, over 4 flux
// and 1 metric components, then 4 subtractions of the dissipation).
extern "C" int esmm_flux_ops(double gamma, int p, int w, double ops[3])
{
    using namespace esmm;
    if (!ops || !(gamma > 1.0 && gamma <= 2.0) || p < 1 || p > 3 || (w != 3 && w != 5)) return ESMM_ERR_ARG;
    if (cudaPeekAtLastError() != cudaSuccess) return ESMM_ERR_CUDA;
    unsigned long long *d = nullptr, h[2] = {0, 0};
    if (cudaMalloc((void **)&d, sizeof h) != cudaSuccess) return ESMM_ERR_CUDA;
    k_count_rhd<<<1, 32>>>(gamma, w, d);
    cudaError_t e = cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return ESMM_ERR_CUDA;
    ops[0] = (double)h[0];
    ops[1] = (double)h[1];
    ops[2] = 5.0 * (p * (p - 1) / 2 + 2 * p - 1) + 4.0;
    return ESMM_OK;
}
