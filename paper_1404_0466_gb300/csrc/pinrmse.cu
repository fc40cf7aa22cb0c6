// PINRMSE (the paper's supplementary comparator): Algorithm 1 with the g x D
// target matrix T replaced by the g x 1 vector t_f of exact hold-out errors at
// the sampled lambdas.  The sampled factors of pichol_factor_samples are
// solved and scored exactly (the kernels of the exact path, the g samples as
// one batch), then one small kernel fits theta_f = V^+ t_f per fold and
// evaluates E_f(lambda_t) = phi(lambda_t) . theta_f on the whole grid.
#include "internal.cuh"

#include <cfloat>

namespace pichol {

// One CTA: (1) t_f[s] = (yy_f + sum of the tile partials of sample s) / (n_f c),
// +inf where the exact factor's diagonal is unusable; (2) theta_f = P t_f;
// (3) E[f][t] = phi_t . theta_f, +inf for a fold with a non-finite sample;
// (4) the first argmin of the mean over folds.
__global__ void __launch_bounds__(256)
k_pinrmse(const double* __restrict__ Epart, const int* __restrict__ flags, const float* __restrict__ dmax,
          const float* __restrict__ dmin, const double* __restrict__ yy, const int64_t* __restrict__ nf_c,
          const double* __restrict__ pinv, const double* __restrict__ phi, int k, int g, int p, int q, int nt,
          double* __restrict__ E_out, double* __restrict__ Eint, int32_t* __restrict__ t_star, DevStatus* st)
{
    __shared__ double ts[MAX_K * MAX_G];
    __shared__ double th[MAX_K * MAX_P];
    __shared__ int badf[MAX_K];
    __shared__ double best_v[256];
    __shared__ int best_t[256];
    __shared__ int nbad;
    const int tid = threadIdx.x;
    const double thr_rel = 1e3 * DBL_EPSILON;
    if (tid < k) badf[tid] = 0;
    if (tid == 0) nbad = 0;
    __syncthreads();
    for (int e = tid; e < k * g; e += 256) {
        const int f = e / g, s = e % g;
        const int64_t o = ((int64_t)f * q + s) * nt;
        double sum = yy[f];
        int bad = 0;
        float mx = 0.0f, mn = FLT_MAX;
        for (int i = 0; i < nt; ++i) {
            sum += Epart[o + i];
            bad |= flags[o + i];
            mx = fmaxf(mx, dmax[o + i]);
            mn = fminf(mn, dmin[o + i]);
        }
        if ((double)mn <= thr_rel * (double)mx) bad = 1;
        const double v = bad ? INFINITY : sum / (double)nf_c[f];
        ts[e] = v;
        if (!isfinite(v)) {
            badf[f] = 1;
            atomicAdd(&nbad, 1);
        }
    }
    __syncthreads();
    for (int e = tid; e < k * p; e += 256) {
        const int f = e / p, m = e % p;
        double v = 0.0;
        for (int s = 0; s < g; ++s) v = fma(pinv[m * g + s], ts[f * g + s], v);
        th[e] = v;
    }
    __syncthreads();
    double bv = INFINITY;
    int bt = -1;
    for (int t = tid; t < q; t += 256) {
        double sum = 0.0;
        for (int f = 0; f < k; ++f) {
            double e = INFINITY;
            if (!badf[f]) {
                e = 0.0;
                for (int m = 0; m < p; ++m) e = fma(phi[t * p + m], th[f * p + m], e);
            }
            E_out[(int64_t)f * q + t] = e;
            Eint[(int64_t)f * q + t] = e;
            sum += e;
        }
        const double eb = sum / (double)k;
        if (isfinite(eb) && eb < bv) {   // t increases per thread: the first minimum is kept
            bv = eb;
            bt = t;
        }
    }
    best_v[tid] = bv;
    best_t[tid] = bt;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (tid < w) {
            const double v2 = best_v[tid + w];
            const int t2 = best_t[tid + w];
            if (t2 >= 0 && (best_t[tid] < 0 || v2 < best_v[tid] || (v2 == best_v[tid] && t2 < best_t[tid]))) {
                best_v[tid] = v2;
                best_t[tid] = t2;
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        *t_star = best_t[0];
        st->unusable = nbad;
    }
}

cudaError_t launch_pinrmse(pichol_ctx* ctx, double* E_out, int32_t* t_star, cudaStream_t s)
{
    const pichol_config& cf = ctx->cfg;
    // the g sampled factors are slots f g + i of the factor buffer: solve and
    // score them as one exact batch of g "lambdas" t = 0 .. g-1
    const int64_t keep = ctx->exact_batch;
    ctx->exact_batch = cf.g;
    cudaError_t e = launch_eval(ctx, 1, 0, cf.g, s);
    ctx->exact_batch = keep;
    if (e != cudaSuccess) return e;
    {
        StageScope sc_(ctx, ST_SELECT, s);
        k_pinrmse<<<1, 256, 0, s>>>(ctx->Epart, ctx->flags, ctx->dmax, ctx->dmin, ctx->yy, ctx->nfc, ctx->pinv,
                                    ctx->phi, cf.k, cf.g, ctx->p, cf.q, ctx->nt, E_out, ctx->E, t_star,
                                    ctx->status);
    }
    ctx->launches++;
    return cudaGetLastError();
}

}  // namespace pichol
