// Polynomial fit of Algorithm 1 (steps 2-6): Theta_f = P T_f, P = V^+ ((r+1) x g,
// computed in double by k_setup), T_f = the g sampled factors of fold f.
// T_f is never assembled: each CTA reads one tile of all g factors and writes
// the (r+1) coefficient planes of that tile, adjacent in memory.
// Double-precision mode accumulates in double; mixed mode in float with P
// rounded to float (P is well conditioned for the Chebyshev-log basis).
#include "internal.cuh"

namespace pichol {

template <typename T>
__global__ void __launch_bounds__(256)
k_fit(const T* __restrict__ F, const double* __restrict__ pinv, int g, int p, int64_t ntiles,
      T* __restrict__ Theta)
{
    __shared__ T P[MAX_P * MAX_G];
    const int tile = blockIdx.x, f = blockIdx.y;
    for (int e = threadIdx.x; e < p * g; e += 256) P[e] = (T)pinv[e];
    __syncthreads();
    T* out = Theta + ((int64_t)f * ntiles + tile) * p * TILE_ELEMS;
    for (int e = threadIdx.x; e < TILE_ELEMS; e += 256) {
        T l[MAX_G];
        for (int s = 0; s < g; ++s) l[s] = F[(((int64_t)f * g + s) * ntiles + tile) * TILE_ELEMS + e];
        for (int m = 0; m < p; ++m) {
            T acc = P[m * g] * l[0];
            for (int s = 1; s < g; ++s) acc = fma(P[m * g + s], l[s], acc);
            out[(int64_t)m * TILE_ELEMS + e] = acc;
        }
    }
}

cudaError_t launch_fit(pichol_ctx* ctx, cudaStream_t s)
{
    const pichol_config& c = ctx->cfg;
    dim3 grid((unsigned)ctx->ntiles, c.k);
    StageScope sc_(ctx, ST_FIT, s);
    if (c.mode == PICHOL_MODE_FP64)
        k_fit<double><<<grid, 256, 0, s>>>((const double*)ctx->F, ctx->pinv, c.g, ctx->p, ctx->ntiles,
                                           (double*)ctx->Theta);
    else
        k_fit<float><<<grid, 256, 0, s>>>((const float*)ctx->F, ctx->pinv, c.g, ctx->p, ctx->ntiles,
                                          (float*)ctx->Theta);
    ctx->launches++;
    return cudaGetLastError();
}

}  // namespace pichol
