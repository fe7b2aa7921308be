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
// the values), on the integer pipes rather than the FP64 one.  A negative
// value counts as 0.  A NaN counts as +infinity in a max, so that a node
// whose recovery failed (NaN speeds) cannot drop out of the CFL spectral
// radius: the step becomes 0 instead of one sized by the healthy nodes.  In
// a min a NaN is ignored.
__device__ __forceinline__ unsigned long long ord_bits(double v, bool for_min)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    if ((b & 0x7fffffffffffffffull) > 0x7ff0000000000000ull) return 0x7ff0000000000000ull;
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

// ---------------------------------------------------------------------------
// eq. cfl with the mesh velocity in the spectral radius, solved for dt.
//
// With the step's displacement d = x^[mu] - x^n, a_{k,i} = d_i.(J xi_k,x)_i / J_i
// and the speed bounds bmin, bmax = L_k lambda_min / J, L_k lambda_max / J of
// every node, eq. cfl reads g(dt) = CFL with
//   g(t) = sum_k max_i max(t bmax_{k,i} - tau a_{k,i}, tau a_{k,i} - t bmin_{k,i}),
// the left side dt sum_k max_i rho_{k,i} with rho_{k,i} = max_m |(J xi_k)_t +
// L_k lambda_m| / J_i and (J xi_k)_t = -tau d.(J xi_k,x)/dt.  g is convex and
// piecewise linear; Newton's method from the right end (CFL + C_m)/S steps to
// the root of the line active at each iterate (the smaller slope on a tie),
// which a convex g lies above, so the iterates fall monotonically onto the
// root's piece.  The solve stops once g <= CFL or the Newton step is below
// 2^-50 t (the root up to rounding); after DT_NEWTON evaluations without
// that, or with a slope <= 0, the safe lower bound (CFL - C_m)/S is used.  k_dt sets the state up; every Newton launch
// evaluates g at the current iterate over all nodes of a problem, and the
// last of the problem's blocks to finish reduces their partial results
// (in any order: the (value, slope) maximum below does not depend on it)
// and advances the iterate.
constexpr int DT_NEWTON = 6;
constexpr int DT_NPT = 1;   // nodes per thread of a Newton evaluation (8 measured slower: 26 vs 15 us)

struct DtSolve {
    double t, t_safe;    // current iterate, the fallback
    int iter, done;      // evaluations so far; 1 when dt_dev holds the step
    unsigned count;      // blocks of the current launch that have finished
    int pad_;
};

// The (value, slope) maximum -- the larger value, on equal values the
// smaller slope -- reduced on order-preserving 64-bit integer keys: the
// values are >= 0, so their bit patterns order like them (a NaN maps to 0
// and never wins), and the slopes' bits are mapped so that unsigned order is
// their order.  On this GPU FP64 compares run on the FP64 pipe, at a small
// fraction of the integer pipes' rate.  A total order, so reductions in any
// order agree.  No site: (0, ~0).  (The values max(t bmax - ta, ta - t bmin)
// are never negative: the two lines sum to t (bmax - bmin) >= 0.)
__device__ __forceinline__ unsigned long long vkey(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return ((b & 0x7fffffffffffffffull) > 0x7ff0000000000000ull || (b >> 63)) ? 0ull : b;   // NaN, -0
}
__device__ __forceinline__ unsigned long long skey(double s)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(s);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double skey_inv(unsigned long long k)
{
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}
__device__ __forceinline__ void vs_take(unsigned long long &v, unsigned long long &s, unsigned long long v2,
                                        unsigned long long s2)
{
    if (v2 > v || (v2 == v && s2 < s)) {
        v = v2;
        s = s2;
    }
}

// the line of one node at t that attains its max(t bmax - ta, ta - t bmin),
// as the keys of (value, slope); the smaller slope where the two lines tie
__device__ __forceinline__ void cfl_line(double t, double ta, double bmin, double bmax, unsigned long long &v,
                                         unsigned long long &s)
{
    const double up = t * bmax - ta, dn = ta - t * bmin;
    const unsigned long long ku = skey(up), kd = skey(dn), kmax = skey(bmax), kmin = skey(-bmin);
    v = vkey(ku > kd ? up : dn);
    s = ku > kd ? kmax : (kd > ku ? kmin : (kmax < kmin ? kmax : kmin));
}

// block-wide (value, slope) maximum of NDIR key pairs; valid in thread 0
template <int NDIR>
__device__ void block_vs_max(unsigned long long (&v)[NDIR], unsigned long long (&s)[NDIR])
{
    __shared__ unsigned long long shv[32][NDIR], shs[32][NDIR];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NDIR; ++k)
        for (int o = 16; o > 0; o >>= 1)
            vs_take(v[k], s[k], __shfl_xor_sync(0xffffffffu, v[k], o), __shfl_xor_sync(0xffffffffu, s[k], o));
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NDIR; ++k) {
            shv[wid][k] = v[k];
            shs[wid][k] = s[k];
        }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NDIR; ++k) {
            v[k] = lane < nw ? shv[lane][k] : 0ull;
            s[k] = lane < nw ? shs[lane][k] : ~0ull;
            for (int o = 16; o > 0; o >>= 1)
                vs_take(v[k], s[k], __shfl_xor_sync(0xffffffffu, v[k], o), __shfl_xor_sync(0xffffffffu, s[k], o));
        }
    }
    __syncthreads();
}

// One Newton update from g(t) and the active slope: the solve ends at
// g <= CFL or at a step below 2^-50 t (the root up to rounding), falls back
// to the safe bound without a positive slope or after DT_NEWTON evaluations,
// and otherwise steps to the root of the active line.
__host__ __device__ inline void dt_newton_update(DtSolve *S, double g, double slope, double cfl, double *dt_out)
{
    const double step = (g - cfl) / slope;
    if (g <= cfl || (slope > 0.0 && step <= 0x1p-50 * S->t)) {
        *dt_out = S->t;
        S->done = 1;
    } else if (!(slope > 0.0) || S->iter + 1 >= DT_NEWTON) {
        *dt_out = S->t_safe;
        S->done = 1;
    } else {
        S->t -= step;
        S->iter += 1;
    }
}

// The block's part of one Newton evaluation: (v, s) are this thread's values
// (-1, 0 where it has no node).  gblock is the block's index in the launch,
// [first, first + nb) the blocks of its problem, part [blocks][NDIR][2] the
// partial results.  The last block of the problem to finish advances S and
// writes the step to *dt_out when the solve ends.  Every thread of the block
// must call it.
//   With vs_out (a slab of a decomposed grid) the last block writes the
// problem's (value, slope) per direction to vs_out[2k], vs_out[2k + 1] for
// the host to combine over the slabs, and leaves S as it is.
template <int NDIR>
__device__ void dt_newton_block(DtSolve *S, unsigned long long (&v)[NDIR], unsigned long long (&s)[NDIR],
                                long long gblock, long long first, long long nb, unsigned long long *part, double cfl,
                                double *dt_out, double *vs_out = nullptr)
{
    __shared__ int last;
    block_vs_max<NDIR>(v, s);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NDIR; ++k) {
            part[(gblock * NDIR + k) * 2] = v[k];
            part[(gblock * NDIR + k) * 2 + 1] = s[k];
        }
        __threadfence();
        last = atomicAdd(&S->count, 1u) == (unsigned)(nb - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
#pragma unroll
    for (int k = 0; k < NDIR; ++k) {
        v[k] = 0ull;
        s[k] = ~0ull;
    }
    for (long long q = threadIdx.x; q < nb; q += blockDim.x)
#pragma unroll
        for (int k = 0; k < NDIR; ++k)
            vs_take(v[k], s[k], __ldcg(part + ((first + q) * NDIR + k) * 2),
                    __ldcg(part + ((first + q) * NDIR + k) * 2 + 1));
    block_vs_max<NDIR>(v, s);
    if (threadIdx.x == 0 && vs_out) {
        S->count = 0u;
#pragma unroll
        for (int k = 0; k < NDIR; ++k) {
            vs_out[2 * k] = __longlong_as_double((long long)v[k]);
            vs_out[2 * k + 1] = skey_inv(s[k]);
        }
        return;
    }
    if (threadIdx.x == 0) {
        double g = 0.0, slope = 0.0;
#pragma unroll
        for (int k = 0; k < NDIR; ++k) {
            g += __longlong_as_double((long long)v[k]);
            slope += skey_inv(s[k]);
        }
        S->count = 0u;
        dt_newton_update(S, g, slope, cfl, dt_out);
    }
}

// Set-up of the solve for one problem (one thread): the displacement's
// Courant number C_m = tau sum_k A_k (A_k = max_i |a_{k,i}|), Delta tau scaled
// so that C_m = CFL/2 where C_m >= CFL (no step satisfies eq. cfl there; *tau
// is updated), S = sum_k S_k the static radius.  A given dt > 0, or C_m = 0,
// ends the solve at once.
__device__ __forceinline__ void dt_setup(DtSolve *S, double cfl, double dt_fixed, double C1, double Ssum,
                                         double *tau, double *dt_out)
{
    double C = *tau * C1;
    if (C >= cfl) {
        *tau = *tau * (0.5 * cfl / C);
        C = 0.5 * cfl;
    }
    S->count = 0u;
    S->iter = 0;
    S->done = 1;
    if (dt_fixed > 0.0) {
        *dt_out = dt_fixed;
    } else if (!(C > 0.0)) {
        *dt_out = cfl / Ssum;
    } else {
        S->t = (cfl + C) / Ssum;
        S->t_safe = (cfl - C) / Ssum;
        S->done = 0;
    }
}

// per-problem reduction slots: [0] max |grad sigma|, [1] Delta tau (min),
// [2], [3] max spectral radius per direction, [4], [5] max mesh Courant
// number per direction of the full displacement x^[mu] - x^n, [6] max
// |lap sigma| (monitor with a Laplacian term), [7] unused
constexpr int NRED = 8;

}  // namespace esmm
