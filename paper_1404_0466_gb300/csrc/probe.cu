// Fused multiply-add throughput of this GPU's FP32 and FP64 pipes, for the
// roofline denominators of the ALU-bound kernels (pichol_probe_fma).  Every
// thread runs eight independent FMA chains, so the pipes, not latency, bound
// the rate; the chains' sums land in a device word so that no work is dropped.
#include "internal.cuh"

namespace pichol {

static __device__ double g_probe_sink;

template <typename T>
__global__ void __launch_bounds__(256) k_probe_fma(int64_t iters, T a, T b)
{
    T x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = (T)(threadIdx.x + j) * (T)1e-3;
    for (int64_t i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
    T s = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == (T)12345.678) g_probe_sink = (double)s;   // never true for these inputs; keeps the chains live
}

}  // namespace pichol

using namespace pichol;

extern "C" pichol_status pichol_probe_fma(int32_t fp64, int64_t iters, double* tflops)
{
    if (!tflops || (fp64 != 0 && fp64 != 1) || iters < 1 || iters > ((int64_t)1 << 24)) return PICHOL_ERR_INVALID_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PICHOL_ERR_CUDA;
    const int blocks = nsm * 8;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return PICHOL_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return PICHOL_ERR_CUDA;
    }
    cudaError_t e = cudaSuccess;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first run warms the clocks up
        cudaEventRecord(e0, 0);
        if (fp64) k_probe_fma<double><<<blocks, 256>>>(iters, 0.999999, 1e-7);
        else k_probe_fma<float><<<blocks, 256>>>(iters, 0.999999f, 1e-7f);
        cudaEventRecord(e1, 0);
        e = cudaEventSynchronize(e1);
    }
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || !(ms > 0.0f)) return PICHOL_ERR_CUDA;
    const double fmas = (double)blocks * 256.0 * 8.0 * (double)iters;
    *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
    return PICHOL_OK;
}
