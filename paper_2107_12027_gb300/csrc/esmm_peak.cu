// esmm_peak.cu -- FMA throughput of the FP64 and FP32 pipes, the denominator
// of the roofline fraction of the arithmetic-bound kernels (the paper has no
// counterpart; it is a measurement addition).
//
// Every thread runs UNR independent FMA chains x <- x*m + c for iters
// rounds; the grid holds 8 blocks of 256 threads per SM, enough warps to
// hide the pipes' latency.  flops = 2 per FMA.
#include <cuda_runtime.h>

#include "esmm.h"

namespace {

constexpr int UNR = 8;
constexpr int BS_PEAK = 256;

template <typename T>
__global__ void k_fma_peak(long long iters, T m, T c, T *out)
{
    T x[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) x[u] = (T)(threadIdx.x + u) * (T)1e-3;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            if constexpr (sizeof(T) == 4) x[u] = fmaf(x[u], m, c);
            else x[u] = fma(x[u], m, c);
        }
    }
    T s = (T)0;
#pragma unroll
    for (int u = 0; u < UNR; ++u) s += x[u];
    if (s == (T)-1.0) out[blockIdx.x] = s;   // never true (x stays positive); keeps the chains live
}

template <typename T>
int run(double seconds, double *flops_per_s, double *ms_out)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return ESMM_ERR_CUDA;
    const unsigned blocks = (unsigned)sms * 8u;
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    T *out = nullptr;
    int rc = ESMM_ERR_CUDA;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&a) != cudaSuccess ||
        cudaEventCreate(&b) != cudaSuccess || cudaMalloc((void **)&out, blocks * sizeof(T)) != cudaSuccess)
        goto done;
    {
        const T m = (T)0.9999999, c = (T)1e-7;
        long long iters = 1024;
        float ms = 0.0f;
        // grow the launch until it takes ~1/8 of the requested time, then time
        // enough launches to fill it (each launch a few tens of ms at most)
        for (int k = 0; k < 40; ++k) {
            k_fma_peak<T><<<blocks, BS_PEAK, 0, st>>>(iters, m, c, out);
            cudaEventRecord(a, st);
            k_fma_peak<T><<<blocks, BS_PEAK, 0, st>>>(iters, m, c, out);
            cudaEventRecord(b, st);
            if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) goto done;
            if (ms > 1e3 * seconds / 8.0 || ms > 50.0) break;
            iters *= 2;
        }
        int reps = (int)(1e3 * seconds / (ms > 0.0f ? ms : 1.0f));
        reps = reps < 1 ? 1 : (reps > 1000 ? 1000 : reps);
        cudaEventRecord(a, st);
        for (int r = 0; r < reps; ++r) k_fma_peak<T><<<blocks, BS_PEAK, 0, st>>>(iters, m, c, out);
        cudaEventRecord(b, st);
        if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) goto done;
        const double fl = 2.0 * UNR * (double)iters * (double)blocks * BS_PEAK * reps;
        if (flops_per_s) *flops_per_s = fl / (1e-3 * ms);
        if (ms_out) *ms_out = ms / reps;
        rc = cudaGetLastError() == cudaSuccess ? ESMM_OK : ESMM_ERR_CUDA;
    }
done:
    if (out) cudaFree(out);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (st) cudaStreamDestroy(st);
    return rc;
}

}  // namespace

extern "C" int esmm_fma_peak(int precision, double seconds, double *flops_per_s, double *ms_per_launch)
{
    if (!(seconds > 0.0) || seconds > 60.0 || !flops_per_s) return ESMM_ERR_ARG;
    if (precision == ESMM_FP64) return run<double>(seconds, flops_per_s, ms_per_launch);
    if (precision == ESMM_MIXED) return run<float>(seconds, flops_per_s, ms_per_launch);
    return ESMM_ERR_ARG;
}
