// Fused multiply-add throughput of this GPU's FP32 and FP64 pipes, for the
// roofline denominators of the ALU-bound kernels (pichol_probe_fma).  Every
// thread runs eight independent FMA chains, so the pipes, not latency, bound
// the rate; the chains' sums land in a device word so that no work is dropped.
// And the issue rate of tcgen05.mma kind::tf32 (M = 128, K = 8) for a given N
// (pichol_probe_mma): one CTA per SM issues MMAs back to back on operands in
// shared memory, so the tensor pipe alone bounds the rate.
#include "internal.cuh"
#include "tcgen05.cuh"

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

// One thread issues `iters` MMAs 128 x N x 8 into two alternating accumulators
// (columns 0 and 256 of a 512-column allocation), the operands being zeroed
// 16 KB (A, 128 rows) and 32 KB (B, up to 256 rows) tiles in the 128-byte
// swizzle layout; K offsets rotate over the four 32-byte steps of a row.  The
// completion wait is bounded; *status = 1 once every MMA has completed.
template <int N>
__global__ void __launch_bounds__(128, 1) k_probe_mma(int64_t iters, int* status)
{
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
    __shared__ uint32_t tslot;
    __shared__ __align__(8) uint64_t bar;
    for (int i = threadIdx.x; i < 49152 / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(sm)[i] = 0u;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (threadIdx.x < 32) tc5::alloc(&tslot, 512);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // the zeroed operands, for the tensor pipe
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    const uint32_t tmem = tslot;
    if (threadIdx.x == 0) {
        const uint64_t da = tc5::sw128_desc(smem_u32(sm)), db = tc5::sw128_desc(smem_u32(sm + 16384));
        constexpr uint32_t id = tc5::idesc_tf32(128, N);
        for (int64_t i = 0; i < iters; ++i)
            tc5::mma_tf32(tmem + ((i & 1) ? 256u : 0u), da + 2 * (i & 3), db + 2 * (i & 3), id, i > 1 ? 1u : 0u);
        tc5::commit(&bar);
        if (mbar_wait(&bar, 0) && blockIdx.x == 0) *status = 1;
    }
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    if (threadIdx.x < 32) tc5::dealloc(tmem, 512);
}

}  // namespace pichol

using namespace pichol;

extern "C" pichol_status pichol_probe_mma(int32_t n_cols, int64_t iters, double* tflops)
{
    if (!tflops || (n_cols != 64 && n_cols != 128 && n_cols != 256) || iters < 1 || iters > ((int64_t)1 << 22))
        return PICHOL_ERR_INVALID_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PICHOL_ERR_CUDA;
    // 120 KB of shared memory per CTA keeps one CTA (and one tensor-memory
    // allocation) per SM
    constexpr int SMEM = 120 * 1024;
    auto kern = n_cols == 64 ? k_probe_mma<64> : (n_cols == 128 ? k_probe_mma<128> : k_probe_mma<256>);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM) != cudaSuccess)
        return PICHOL_ERR_CUDA;
    int* dstat = nullptr;
    if (cudaMalloc(&dstat, sizeof(int)) != cudaSuccess) return PICHOL_ERR_CUDA;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) {
        cudaFree(dstat);
        return PICHOL_ERR_CUDA;
    }
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaFree(dstat);
        return PICHOL_ERR_CUDA;
    }
    cudaError_t e = cudaMemset(dstat, 0, sizeof(int));
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first run warms the clocks up
        cudaEventRecord(e0, 0);
        kern<<<nsm, 128, SMEM>>>(iters, dstat);
        cudaEventRecord(e1, 0);
        e = cudaEventSynchronize(e1);
    }
    float ms = 0.0f;
    int done = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaMemcpy(&done, dstat, sizeof(int), cudaMemcpyDeviceToHost);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(dstat);
    if (e != cudaSuccess || !(ms > 0.0f)) return PICHOL_ERR_CUDA;
    if (!done) return PICHOL_ERR_TIMEOUT;
    const double macs = (double)nsm * (double)iters * 128.0 * (double)n_cols * 8.0;
    *tflops = 2.0 * macs / (ms * 1e-3) / 1e12;
    return PICHOL_OK;
}

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
