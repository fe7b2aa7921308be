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

// Max and min of non-negative values on their bit patterns (which order like
// the values), on the integer pipes rather than the FP64 one.  A NaN is
// ignored (as fmax/fmin would), a negative value counts as 0.
__device__ __forceinline__ unsigned long long ord_bits(double v, bool for_min)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    if ((b & 0x7fffffffffffffffull) > 0x7ff0000000000000ull) return for_min ? 0x7ff0000000000000ull : 0ull;
    return (b >> 63) ? 0ull : b;
}
__device__ __forceinline__ unsigned long long warp_max_bits(unsigned long long v)
{
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}
__device__ __forceinline__ unsigned long long warp_min_bits(unsigned long long v)
{
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w < v ? w : v;
    }
    return v;
}

// OP: 0 max, 1 min (of non-negative values, min capped at 1e300), 2 sum; the
// result is valid in thread 0.  Every thread of the block must call it.
template <int OP>
__device__ double block_reduce(double v)
{
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int nw = (blockDim.x + 31) >> 5;
    if (OP == 2) {
        __shared__ double sh[32];
        v = warp_sum(v);
        if (lane == 0) sh[wid] = v;
        __syncthreads();
        if (wid == 0) {
            v = lane < nw ? sh[lane] : 0.0;
            v = warp_sum(v);
        }
        __syncthreads();
        return v;
    }
    __shared__ unsigned long long shb[32];
    const unsigned long long init = OP == 0 ? 0ull : (unsigned long long)__double_as_longlong(1.0e300);
    unsigned long long b = ord_bits(v, OP == 1);
    if (OP == 1 && b > init) b = init;
    b = OP == 0 ? warp_max_bits(b) : warp_min_bits(b);
    if (lane == 0) shb[wid] = b;
    __syncthreads();
    if (wid == 0) {
        b = lane < nw ? shb[lane] : init;
        b = OP == 0 ? warp_max_bits(b) : warp_min_bits(b);
    }
    __syncthreads();
    return __longlong_as_double((long long)b);
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
