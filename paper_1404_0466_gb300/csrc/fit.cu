// Polynomial fit of Algorithm 1: Theta_f = P T_f, P = V^+ ((r+1) x g,
// computed in double by k_setup), T_f = the g sampled factors of fold f.
// T_f is never assembled: each CTA reads one tile of all g factors and writes
// the (r+1) coefficient planes of that tile, adjacent in memory.
// Double-precision mode accumulates in double; mixed mode in float with P
// rounded to float (P is well conditioned for the Chebyshev-log basis).
// With the warm start (warm_samples = g'), the folds f > 0 are corrected from
// fold 0's coefficients by their g' factors (k_fit_warm).
#include "internal.cuh"

#include <cstring>

namespace pichol {

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int N = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int N = 2; };

// Each thread carries 16 bytes of a tile at a time (4 fp32 or 2 fp64 entries):
// the g factor values in, the p coefficients out.
template <typename T, int G>
__global__ void __launch_bounds__(256)
k_fit(const T* __restrict__ F, const double* __restrict__ pinv, int p, int64_t ntiles, T* __restrict__ Theta)
{
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::N;
    __shared__ T P[MAX_P * MAX_G];
    const int tile = blockIdx.x, f = blockIdx.y;
    for (int e = threadIdx.x; e < p * G; e += 256) P[e] = (T)pinv[e];
    __syncthreads();
    T* out = Theta + ((int64_t)f * ntiles + tile) * p * TILE_ELEMS;
    const T* in = F + ((int64_t)f * G * ntiles + tile) * TILE_ELEMS;
    const int64_t sstride = ntiles * TILE_ELEMS;      // between the g factors of fold f
    for (int v = threadIdx.x; v < TILE_ELEMS / VN; v += 256) {
        T l[G][VN];
#pragma unroll
        for (int s = 0; s < G; ++s) {
            const V x = reinterpret_cast<const V*>(in + s * sstride)[v];
            memcpy(l[s], &x, sizeof(V));
        }
        for (int m = 0; m < p; ++m) {
            T acc[VN];
#pragma unroll
            for (int u = 0; u < VN; ++u) acc[u] = P[m * G] * l[0][u];
#pragma unroll
            for (int s = 1; s < G; ++s)
#pragma unroll
                for (int u = 0; u < VN; ++u) acc[u] = fma(P[m * G + s], l[s][u], acc[u]);
            V y;
            memcpy(&y, acc, sizeof(V));
            reinterpret_cast<V*>(out + (int64_t)m * TILE_ELEMS)[v] = y;
        }
    }
}

// Warm start of fold f = blockIdx.y + 1 from fold 0's coefficients: with the
// GW warm factors l_s of the tile, the residuals e_s = l_s - sum_m Vw[s][m]
// Theta_0m, then Theta_fm = Theta_0m + sum_s Pw[m][s] e_s for m < pw and
// Theta_0m for the rest.  16 bytes of the tile per thread at a time.
template <typename T, int GW>
__global__ void __launch_bounds__(256)
k_fit_warm(const T* __restrict__ F, const double* __restrict__ pinv_w, const double* __restrict__ vw, int p,
           int pw, int g, int64_t ntiles, T* __restrict__ Theta)
{
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::N;
    __shared__ T Pw[MAX_P * MAX_G];
    __shared__ T Vw[MAX_G * MAX_P];
    const int tile = blockIdx.x, f = blockIdx.y + 1;
    for (int e = threadIdx.x; e < pw * GW; e += 256) Pw[e] = (T)pinv_w[e];
    for (int e = threadIdx.x; e < GW * p; e += 256) Vw[e] = (T)vw[e];
    __syncthreads();
    const T* base = Theta + (int64_t)tile * p * TILE_ELEMS;                   // fold 0
    T* out = Theta + ((int64_t)f * ntiles + tile) * p * TILE_ELEMS;
    const T* in = F + ((int64_t)f * g * ntiles + tile) * TILE_ELEMS;          // slots f g + s
    const int64_t sstride = ntiles * TILE_ELEMS;
    for (int v = threadIdx.x; v < TILE_ELEMS / VN; v += 256) {
        // loops over m run to MAX_P with a guard so that th stays in registers
        T th[MAX_P][VN], res[GW][VN];
#pragma unroll
        for (int m = 0; m < MAX_P; ++m)
            if (m < p) {
                const V x = reinterpret_cast<const V*>(base + (int64_t)m * TILE_ELEMS)[v];
                memcpy(th[m], &x, sizeof(V));
            }
#pragma unroll
        for (int s = 0; s < GW; ++s) {
            const V x = reinterpret_cast<const V*>(in + s * sstride)[v];
            memcpy(res[s], &x, sizeof(V));
#pragma unroll
            for (int m = 0; m < MAX_P; ++m)
                if (m < p)
#pragma unroll
                    for (int u = 0; u < VN; ++u) res[s][u] = fma(-Vw[s * p + m], th[m][u], res[s][u]);
        }
#pragma unroll
        for (int m = 0; m < MAX_P; ++m)
            if (m < p) {
                T acc[VN];
#pragma unroll
                for (int u = 0; u < VN; ++u) acc[u] = th[m][u];
                if (m < pw) {
#pragma unroll
                    for (int s = 0; s < GW; ++s)
#pragma unroll
                        for (int u = 0; u < VN; ++u) acc[u] = fma(Pw[m * GW + s], res[s][u], acc[u]);
                }
                V y;
                memcpy(&y, acc, sizeof(V));
                reinterpret_cast<V*>(out + (int64_t)m * TILE_ELEMS)[v] = y;
            }
    }
}

template <typename T>
static cudaError_t fit_warm_dispatch(int gw, dim3 grid, const T* F, const double* pinv_w, const double* vw, int p,
                                     int pw, int g, int64_t ntiles, T* Theta, cudaStream_t s)
{
    switch (gw) {
#define PICHOL_FIT_WARM_CASE(G) \
    case G: k_fit_warm<T, G><<<grid, 256, 0, s>>>(F, pinv_w, vw, p, pw, g, ntiles, Theta); break;
        PICHOL_FIT_WARM_CASE(2) PICHOL_FIT_WARM_CASE(3) PICHOL_FIT_WARM_CASE(4) PICHOL_FIT_WARM_CASE(5)
        PICHOL_FIT_WARM_CASE(6) PICHOL_FIT_WARM_CASE(7) PICHOL_FIT_WARM_CASE(8)
#undef PICHOL_FIT_WARM_CASE
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
static cudaError_t fit_dispatch(int g, dim3 grid, const T* F, const double* pinv, int p, int64_t ntiles, T* Theta,
                                cudaStream_t s)
{
    switch (g) {
#define PICHOL_FIT_CASE(G) \
    case G: k_fit<T, G><<<grid, 256, 0, s>>>(F, pinv, p, ntiles, Theta); break;
        PICHOL_FIT_CASE(1) PICHOL_FIT_CASE(2) PICHOL_FIT_CASE(3) PICHOL_FIT_CASE(4) PICHOL_FIT_CASE(5)
        PICHOL_FIT_CASE(6) PICHOL_FIT_CASE(7) PICHOL_FIT_CASE(8) PICHOL_FIT_CASE(9) PICHOL_FIT_CASE(10)
        PICHOL_FIT_CASE(11) PICHOL_FIT_CASE(12) PICHOL_FIT_CASE(13) PICHOL_FIT_CASE(14) PICHOL_FIT_CASE(15)
        PICHOL_FIT_CASE(16) PICHOL_FIT_CASE(17) PICHOL_FIT_CASE(18) PICHOL_FIT_CASE(19) PICHOL_FIT_CASE(20)
        PICHOL_FIT_CASE(21) PICHOL_FIT_CASE(22) PICHOL_FIT_CASE(23) PICHOL_FIT_CASE(24) PICHOL_FIT_CASE(25)
        PICHOL_FIT_CASE(26) PICHOL_FIT_CASE(27) PICHOL_FIT_CASE(28) PICHOL_FIT_CASE(29) PICHOL_FIT_CASE(30)
        PICHOL_FIT_CASE(31) PICHOL_FIT_CASE(32)
#undef PICHOL_FIT_CASE
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_fit(pichol_ctx* ctx, cudaStream_t s)
{
    const pichol_config& c = ctx->cfg;
    const int gw = c.warm_samples;
    // with the warm start only fold 0 is fitted from all g samples; the other
    // folds follow from it
    dim3 grid((unsigned)ctx->ntiles, gw ? 1 : c.k);
    cudaError_t e;
    {
        StageScope sc_(ctx, ST_FIT, s);
        if (c.mode == PICHOL_MODE_FP64)
            e = fit_dispatch<double>(c.g, grid, (const double*)ctx->F, ctx->pinv, ctx->p, ctx->ntiles,
                                     (double*)ctx->Theta, s);
        else
            e = fit_dispatch<float>(c.g, grid, (const float*)ctx->F, ctx->pinv, ctx->p, ctx->ntiles,
                                    (float*)ctx->Theta, s);
    }
    ctx->launches++;
    if (e == cudaSuccess && !gw && ctx->Th) e = launch_theta_split(ctx, s);
    if (e != cudaSuccess || !gw) return e;
    const int pw = gw < ctx->p ? gw : ctx->p;
    dim3 wgrid((unsigned)ctx->ntiles, c.k - 1);
    {
        StageScope sc_(ctx, ST_FIT, s);
        if (c.mode == PICHOL_MODE_FP64)
            e = fit_warm_dispatch<double>(gw, wgrid, (const double*)ctx->F, ctx->pinv_w, ctx->vw, ctx->p, pw, c.g,
                                          ctx->ntiles, (double*)ctx->Theta, s);
        else
            e = fit_warm_dispatch<float>(gw, wgrid, (const float*)ctx->F, ctx->pinv_w, ctx->vw, ctx->p, pw, c.g,
                                         ctx->ntiles, (float*)ctx->Theta, s);
    }
    ctx->launches++;
    if (e == cudaSuccess && ctx->Th) e = launch_theta_split(ctx, s);
    return e;
}

}  // namespace pichol
