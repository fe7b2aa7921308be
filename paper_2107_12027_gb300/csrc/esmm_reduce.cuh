// esmm_reduce.cuh -- block reductions and bit-pattern atomics shared by the
// CFL, mesh and totals kernels of both systems.
#pragma once

#include "esmm_device.cuh"

namespace esmm {

// ---------------------------------------------------------------------------
// block reductions (warp shuffles, then one value per warp in shared memory)
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

// OP: 0 max, 1 min, 2 sum; the result is valid in thread 0.  Every thread of
// the block must call it.
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
    __syncthreads();
    return v;
}

// Non-negative doubles order like their bit patterns, so the max/min of such
// values over many blocks is an integer atomic on the bits.
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *a, double v)
{
    atomicMax(a, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ void atomic_min_nonneg(unsigned long long *a, double v)
{
    atomicMin(a, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ double bits_to_double(unsigned long long b) { return __longlong_as_double((long long)b); }

// per-problem reduction slots: [0] max |grad sigma|, [1] Delta tau (min),
// [2], [3] max spectral radius per direction, [4], [5] max mesh Courant
// number per direction of the full displacement x^[mu] - x^n, [6] max
// |lap sigma| (monitor with a Laplacian term), [7] unused
constexpr int NRED = 8;

}  // namespace esmm
