// Multi-level narrowing of the lambda range (MChol, Sec. 6.2), run entirely
// on the device so that the whole search enqueues without a host round trip.
//
// Each level evaluates the exact hold-out error at the three lambdas
// tau 10^(c-s), tau 10^c, tau 10^(c+s) with the exact-Cholesky path of the
// library (the factorisation, solve and scoring kernels of the `Chol`
// comparator), then one small kernel takes the first argmin of the mean over
// folds, sets c <- log10(lambda_opt / tau) and halves s.  The number of
// levels depends on s and s_min only, so the host knows it in advance.  After
// the last level the grid, the samples and V^+ are set up again on the final
// window [10^(c-s), 10^(c+s)], so piCholesky then searches that window.
//
// State lives in the workspace (ctx->mlam): [0..2] the level's lambdas (the
// shifts the exact factorisation reads), [4] c, [5] s, [6..7] the window.
#include "internal.cuh"

#include <cfloat>

namespace pichol {

__global__ void k_mchol_init(double* __restrict__ m, double c, double s)
{
    m[4] = c;
    m[5] = s;
}

// lambda_i = tau 10^(c + (i - 1) s), i = 0, 1, 2
__global__ void k_mchol_lams(const double* __restrict__ scal, double* __restrict__ m)
{
    const int i = threadIdx.x;
    if (i < 3) m[i] = scal[0] * pow(10.0, m[4] + (double)(i - 1) * m[5]);
}

// One warp per candidate lambda (blockDim 96).  For every fold the warp sums
// the per-tile hold-out partials and the diagonal checks of that (fold,
// lambda), E_f = (yy_f + sum) / (n_f c) or +inf where the factor's diagonal
// is unusable; then the mean over folds, the first argmin over finite means,
// the update of (c, s) and the trace row
//   [lambda_0, lambda_1, lambda_2, Ebar_0, Ebar_1, Ebar_2, c, s] (after the update).
__global__ void __launch_bounds__(96)
k_mchol_step(const double* __restrict__ Epart, const int* __restrict__ flags, const float* __restrict__ dmax,
             const float* __restrict__ dmin, const double* __restrict__ yy, const int64_t* __restrict__ nf_c,
             const double* __restrict__ scal, int k, int q, int nt, double* __restrict__ m,
             double* __restrict__ trace_row)
{
    __shared__ double Ebar[3];
    const int t = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double thr_rel = 1e3 * DBL_EPSILON;
    double sum = 0.0;
    for (int f = 0; f < k; ++f) {
        const int64_t o = ((int64_t)f * q + t) * nt;
        double s = 0.0;
        int bad = 0;
        float mx = 0.0f, mn = FLT_MAX;
        for (int i = lane; i < nt; i += 32) {
            s += Epart[o + i];
            bad |= flags[o + i];
            mx = fmaxf(mx, dmax[o + i]);
            mn = fminf(mn, dmin[o + i]);
        }
        for (int w = 16; w > 0; w >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, w);
            bad |= __shfl_xor_sync(0xffffffffu, bad, w);
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, w));
            mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, w));
        }
        if ((double)mn <= thr_rel * (double)mx) bad = 1;
        sum += bad ? INFINITY : (yy[f] + s) / (double)nf_c[f];
    }
    if (lane == 0) Ebar[t] = sum / (double)k;
    __syncthreads();
    if (threadIdx.x == 0) {
        int best = -1;
        double bv = INFINITY;
        for (int i = 0; i < 3; ++i)
            if (isfinite(Ebar[i]) && Ebar[i] < bv) {
                bv = Ebar[i];
                best = i;
            }
        double c = m[4];
        const double s = 0.5 * m[5];
        if (best >= 0) c = log10(m[best] / scal[0]);
        m[4] = c;
        m[5] = s;
        m[6] = pow(10.0, c - s);
        m[7] = pow(10.0, c + s);
        if (trace_row) {
            for (int i = 0; i < 3; ++i) {
                trace_row[i] = m[i];
                trace_row[3 + i] = Ebar[i];
            }
            trace_row[6] = c;
            trace_row[7] = s;
        }
    }
}

int mchol_levels(double s, double s_min)
{
    int n = 0;
    do {
        ++n;
        s *= 0.5;
    } while (s > s_min && n <= 64);
    return n;
}

cudaError_t launch_mchol(pichol_ctx* ctx, double c, double s, int levels, double* trace_out, cudaStream_t st)
{
    const pichol_config& cf = ctx->cfg;
    // the three lambdas of a level are factored in batches of up to three
    // problems per fold; the factor buffer holds nfac / k slots per fold
    const int64_t keep_batch = ctx->exact_batch;
    double* keep_lam = ctx->lam;
    const int per = (int)((ctx->nfac / cf.k) < 3 ? (ctx->nfac / cf.k) : 3);
    ctx->exact_batch = per;
    ctx->lam = ctx->mlam;   // the exact factorisation reads its shifts from here
    cudaError_t e = cudaSuccess;
    k_mchol_init<<<1, 1, 0, st>>>(ctx->mlam, c, s);
    ctx->launches++;
    e = cudaGetLastError();
    for (int lv = 0; lv < levels && e == cudaSuccess; ++lv) {
        {
            StageScope sc_(ctx, ST_SETUP, st);
            k_mchol_lams<<<1, 32, 0, st>>>(ctx->scal, ctx->mlam);
        }
        ctx->launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        for (int t0 = 0; t0 < 3 && e == cudaSuccess; t0 += per) {
            const int cnt = (3 - t0) < per ? (3 - t0) : per;
            e = launch_factor(ctx, cnt, 1, t0, st);
            if (e == cudaSuccess) e = launch_eval(ctx, 1, t0, cnt, st);
        }
        if (e != cudaSuccess) break;
        {
            StageScope sc_(ctx, ST_SELECT, st);
            k_mchol_step<<<1, 96, 0, st>>>(ctx->Epart, ctx->flags, ctx->dmax, ctx->dmin, ctx->yy, ctx->nfc,
                                           ctx->scal, cf.k, cf.q, ctx->nt, ctx->mlam,
                                           trace_out ? trace_out + (int64_t)lv * 8 : nullptr);
        }
        ctx->launches++;
        e = cudaGetLastError();
    }
    ctx->lam = keep_lam;
    ctx->exact_batch = keep_batch;
    if (e == cudaSuccess) e = launch_setup(ctx, ctx->mlam + 6, st);
    return e;
}

}  // namespace pichol
