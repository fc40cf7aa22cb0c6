// C ABI of libpichol: argument checking, workspace planning and the order of
// kernel launches.  Every call below only enqueues work on the caller's
// stream; see include/pichol.h for the contract of each entry point.
#include "internal.cuh"

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

using namespace pichol;

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Lay the workspace sections out from `base` (nullptr: only count bytes).
size_t plan(pichol_ctx* ctx, char* base)
{
    const pichol_config& c = ctx->cfg;
    const int64_t k = c.k, q = c.q, g = c.g, p = ctx->p, dp = ctx->dp, nt = ctx->nt;
    const int64_t eb = ctx->eb, cc = c.c, ntl = ctx->ntiles;
    size_t off = 0;
    ctx->nguard = 0;
    auto take = [&](size_t bytes) -> void* {
        void* ptr = base ? (void*)(base + off) : nullptr;
        off += align256(bytes);
        if (GUARD_BYTES && ctx->nguard < MAX_GUARDS) {
            ctx->guard_off[ctx->nguard++] = off;
            off += GUARD_BYTES;
        }
        return ptr;
    };
    ctx->status = (DevStatus*)take(sizeof(DevStatus));
    ctx->scal = (double*)take(8 * sizeof(double));
    ctx->lam = (double*)take(q * sizeof(double));
    ctx->lam_grid = (double*)take(q * sizeof(double));
    ctx->mlam = (double*)take(8 * sizeof(double));
    ctx->lam_s = (double*)take(g * sizeof(double));
    ctx->pinv = (double*)take(p * g * sizeof(double));
    ctx->lam_w = (double*)take(g * sizeof(double));
    ctx->pinv_w = (double*)take(p * g * sizeof(double));
    ctx->vw = (double*)take(g * p * sizeof(double));
    ctx->phi = (double*)take(q * p * sizeof(double));
    ctx->dphi = (double*)take(q * p * sizeof(double));
    ctx->nfc = (int64_t*)take(k * sizeof(int64_t));
    ctx->yy = (double*)take(k * sizeof(double));
    ctx->G = take((size_t)(k * dp * dp * eb));
    ctx->Bv = take((size_t)(k * dp * cc * eb));
    ctx->Btr = take((size_t)(k * dp * cc * eb));
    ctx->xpart = (double*)take(xty_part_bytes((int)k, dp, cc));
    ctx->Hf = take((size_t)(k * ntl * TILE_ELEMS * eb));
    ctx->F = take((size_t)(ctx->nfac * ntl * TILE_ELEMS * eb));
    const bool mixed = c.mode == PICHOL_MODE_MIXED;
    ctx->Ph = mixed ? (float*)take((size_t)(2 * ctx->nfac * nt * TILE_ELEMS * sizeof(float))) : nullptr;
    ctx->Pl = mixed ? (float*)take((size_t)(2 * ctx->nfac * nt * TILE_ELEMS * sizeof(float))) : nullptr;
    ctx->Theta = take((size_t)(k * ntl * p * TILE_ELEMS * eb));
    ctx->Dinv = take((size_t)(k * q * nt * TILE_ELEMS * eb));
    ctx->W = take((size_t)(k * q * dp * cc * eb));
    const bool refine = c.mode == PICHOL_MODE_MIXED && c.refine_steps > 0;
    const bool rexact = refine && c.refine_target == PICHOL_REFINE_EXACT;
    ctx->U = (refine && !rexact) ? take((size_t)(2 * k * q * dp * cc * sizeof(float))) : nullptr;
    const bool rtc = c.mode == PICHOL_MODE_MIXED;   // Theta split for the tensor-core solve and residual
    const size_t tplanes = (size_t)(k * ntl * p + 1) * TILE_ELEMS * sizeof(float);
    ctx->Th = rtc ? (float*)take(tplanes) : nullptr;
    ctx->Tl = rtc ? (float*)take(tplanes) : nullptr;
    ctx->TTh = rtc ? (float*)take(tplanes) : nullptr;
    ctx->TTl = rtc ? (float*)take(tplanes) : nullptr;
    ctx->Sh = rtc ? (float*)take((size_t)(k * q * cc * dp * sizeof(float))) : nullptr;
    ctx->Sl = rtc ? (float*)take((size_t)(k * q * cc * dp * sizeof(float))) : nullptr;
    ctx->Rres = refine ? take((size_t)(k * q * dp * cc * eb)) : nullptr;
    if (c.mode == PICHOL_MODE_MIXED) {
        const int64_t qc = q * cc;
        ctx->Xh = (float*)take((size_t)(dp * ctx->kpad_cap * 4));
        ctx->Xl = (float*)take((size_t)(dp * ctx->kpad_cap * 4));
        ctx->Yh = (float*)take((size_t)(cc * ctx->kpad_cap * 4));
        ctx->Yl = (float*)take((size_t)(cc * ctx->kpad_cap * 4));
        ctx->Gh = (float*)take((size_t)(k * dp * dp * 4));
        ctx->Gl = (float*)take((size_t)(k * dp * dp * 4));
        ctx->Wth = (float*)take((size_t)(k * qc * dp * 4));
        ctx->Wtl = (float*)take((size_t)(k * qc * dp * 4));
        ctx->U2 = rexact ? (float*)take((size_t)(k * dp * ctx->ldu * 4)) : nullptr;
        ctx->Xrh = (float*)take((size_t)(c.n * dp * 4));
        ctx->Xrl = (float*)take((size_t)(c.n * dp * 4));
        ctx->Ycp = (float*)take((size_t)(c.n * cc * 4));
        ctx->Escore = (double*)take((size_t)(k * ctx->mt_cap * ctx->ldu * 8));
        ctx->Gah = rexact ? (float*)take((size_t)(dp * dp * 4)) : nullptr;
        ctx->Gal = rexact ? (float*)take((size_t)(dp * dp * 4)) : nullptr;
        ctx->U3 = rexact ? (float*)take((size_t)(k * dp * ctx->ldu * 4)) : nullptr;
    }
    ctx->gW = take((size_t)(3 * k * dp * cc * eb));
    ctx->gDinv = take((size_t)(k * nt * TILE_ELEMS * eb));
    ctx->gP = (double*)take((size_t)(GRAD_CHUNKS * 4 * k * dp * cc * sizeof(double)));
    ctx->gL = take((size_t)(2 * k * ntl * TILE_ELEMS * eb));
    ctx->gphi = (double*)take((size_t)(2 * MAX_P + 1) * sizeof(double));
    ctx->gflags = (int*)take((size_t)(k * nt * sizeof(int)));
    ctx->gdmax = (float*)take((size_t)(k * nt * sizeof(float)));
    ctx->gdmin = (float*)take((size_t)(k * nt * sizeof(float)));
    ctx->Epart = (double*)take((size_t)(k * q * nt * sizeof(double)));
    ctx->E = (double*)take((size_t)(k * q * sizeof(double)));
    ctx->flags = (int*)take((size_t)(k * q * nt * sizeof(int)));
    // wavefront solve: two tickets (in a 256-byte head), then per pass the exchanged
    // solved blocks of up to WAVE_SYS_CAP systems (mixed mode only)
    ctx->wave_sys = c.mode == PICHOL_MODE_MIXED ? (k * q < WAVE_SYS_CAP ? k * q : WAVE_SYS_CAP) : 0;
    ctx->wave = ctx->wave_sys ? (int*)take((size_t)(WAVE_HEAD_INTS * 4 + 2 * ctx->wave_sys * dp * cc * 4)) : nullptr;
    ctx->dmax = (float*)take((size_t)(k * q * nt * sizeof(float)));
    ctx->dmin = (float*)take((size_t)(k * q * nt * sizeof(float)));
    return off;
}

pichol_status cuda_status(cudaError_t e) { return e == cudaSuccess ? PICHOL_OK : PICHOL_ERR_CUDA; }

struct GuardList {
    int n;
    int64_t off[MAX_GUARDS];
};

// One CTA per guard band: the first byte that is not GUARD_FILL latches the error.
__global__ void k_check_guards(const unsigned char* ws, GuardList gl, DevStatus* st)
{
    const unsigned char* band = ws + gl.off[blockIdx.x];
    for (int i = threadIdx.x; i < (int)GUARD_BYTES; i += blockDim.x)
        if (band[i] != GUARD_FILL) latch_error(st, PICHOL_ERR_WORKSPACE, -1, (int)blockIdx.x, i);
}

bool ready(const pichol_ctx* ctx) { return ctx && ctx->ws; }

// Caller lambdas: every value finite and positive.
bool lambdas_ok(const double* v, int n)
{
    for (int i = 0; i < n; ++i)
        if (!(v[i] > 0.0) || !std::isfinite(v[i])) return false;
    return true;
}

// Caller fold offsets: offs[0] = 0, offs[k] = n, strictly increasing.
bool offsets_ok(const int64_t* o, int k, int64_t n)
{
    if (o[0] != 0 || o[k] != n) return false;
    for (int f = 0; f < k; ++f)
        if (!(o[f + 1] > o[f])) return false;
    return true;
}

}  // namespace

namespace pichol {
cudaError_t launch_check_guards(pichol_ctx* ctx, cudaStream_t s)
{
    GuardList gl;
    gl.n = ctx->nguard;
    for (int i = 0; i < ctx->nguard; ++i) gl.off[i] = (int64_t)ctx->guard_off[i];
    k_check_guards<<<ctx->nguard, 256, 0, s>>>((const unsigned char*)ctx->ws, gl, ctx->status);
    return cudaGetLastError();
}
}  // namespace pichol

extern "C" {

void pichol_config_default(pichol_config* cfg)
{
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->lam_lo = 1e-3;
    cfg->lam_hi = 1e1;
    cfg->scale_by_trace = 1;
    cfg->basis = PICHOL_BASIS_MONO;
    cfg->mode = PICHOL_MODE_FP64;
    cfg->refine_steps = 0;
    cfg->gram_passes = 3;
    cfg->exact_batch = 0;
}

pichol_status pichol_create(const pichol_config* cfg, pichol_ctx** out)
{
    if (out) *out = nullptr;
    if (!cfg || !out) return PICHOL_ERR_INVALID_ARG;
    const pichol_config& c = *cfg;
    if (c.k < 2 || c.k > MAX_K) return PICHOL_ERR_INVALID_ARG;
    if (c.n < c.k || c.d < 1 || c.d > 16384 || c.c < 1 || c.c > 32) return PICHOL_ERR_INVALID_ARG;
    if (c.q < 1 || c.q > 4096) return PICHOL_ERR_INVALID_ARG;
    if (c.r < 0 || c.r > 5) return PICHOL_ERR_INVALID_ARG;
    if (c.g <= c.r || c.g > c.q || c.g > MAX_G) return PICHOL_ERR_INVALID_ARG;
    if (!(c.lam_lo > 0.0) || !(c.lam_hi >= c.lam_lo) || !std::isfinite(c.lam_hi)) return PICHOL_ERR_INVALID_ARG;
    if (c.scale_by_trace != 0 && c.scale_by_trace != 1) return PICHOL_ERR_INVALID_ARG;
    if (c.basis != PICHOL_BASIS_MONO && c.basis != PICHOL_BASIS_CHEB_LOG) return PICHOL_ERR_INVALID_ARG;
    if (c.mode != PICHOL_MODE_FP64 && c.mode != PICHOL_MODE_MIXED) return PICHOL_ERR_INVALID_ARG;
    if (c.refine_steps < 0 || c.refine_steps > 4) return PICHOL_ERR_INVALID_ARG;
    if (c.gram_passes != 1 && c.gram_passes != 3) return PICHOL_ERR_INVALID_ARG;
    if (c.exact_batch < 0 || c.exact_batch > c.q) return PICHOL_ERR_INVALID_ARG;
    if (c.refine_target != PICHOL_REFINE_INTERPOLATED && c.refine_target != PICHOL_REFINE_EXACT)
        return PICHOL_ERR_INVALID_ARG;
    for (int i = 0; i < 3; ++i)
        if (c.reserved[i] != 0) return PICHOL_ERR_INVALID_ARG;
    if (c.refine_residual != PICHOL_RESIDUAL_TENSOR && c.refine_residual != PICHOL_RESIDUAL_DOUBLE_FLOAT)
        return PICHOL_ERR_INVALID_ARG;
    if (c.warm_samples != 0 && (c.warm_samples < 2 || c.warm_samples > c.g || c.warm_samples > 8))
        return PICHOL_ERR_INVALID_ARG;
    if (c.refine_target == PICHOL_REFINE_EXACT && c.mode != PICHOL_MODE_MIXED) return PICHOL_ERR_UNSUPPORTED;
    // the interpolate-on-load solve keeps p coefficient planes and the
    // right-hand-side blocks of two lambdas in shared memory (227 KB per CTA)
    if (solve_smem_bytes(c.mode == PICHOL_MODE_FP64 ? 8 : 4, c.r + 1, c.c) > 227 * 1024)
        return PICHOL_ERR_UNSUPPORTED;
    pichol_ctx* ctx = new (std::nothrow) pichol_ctx();
    if (!ctx) return PICHOL_ERR_INVALID_ARG;
    ctx->cfg = c;
    ctx->nt = (int)((c.d + TB - 1) / TB);
    ctx->dp = (int64_t)ctx->nt * TB;
    ctx->ntiles = num_tiles(ctx->nt);
    ctx->p = c.r + 1;
    ctx->eb = c.mode == PICHOL_MODE_FP64 ? 8 : 4;
    for (int f = 0; f <= c.k; ++f) ctx->offs[f] = (int64_t)f * c.n / c.k;
    ctx->exact_batch = c.exact_batch > 0 ? c.exact_batch : c.q;
    ctx->nfac = (int64_t)c.k * (ctx->exact_batch > c.g ? ctx->exact_batch : c.g);
    ctx->kpad = tc_kpad(ctx);
    ctx->kpad_cap = (c.n + 31 * (int64_t)c.k) / 32 * 32;
    ctx->ldu = ((int64_t)c.q * c.c + 3) / 4 * 4;
    // the largest fold any split can make has n - (k - 1) rows
    ctx->mt_cap = (int)((c.n - (c.k - 1) + 127) / 128);
    ctx->need_bytes = plan(ctx, nullptr);
    ctx->tune.update_strip = 4;
    ctx->tune.diag_threads = 512;
    ctx->tune.diag_exclusive = 1;
    ctx->tune.update_engine = 1;   // CUDA cores: see pichol_tuning
    ctx->tune.solve_engine = 2;    // automatic: see pichol_tuning
    *out = ctx;
    return PICHOL_OK;
}

pichol_status pichol_workspace_size(const pichol_ctx* ctx, size_t* bytes)
{
    if (!ctx || !bytes) return PICHOL_ERR_INVALID_ARG;
    *bytes = ctx->need_bytes;
    return PICHOL_OK;
}

pichol_status pichol_set_workspace(pichol_ctx* ctx, void* workspace, size_t bytes)
{
    if (!ctx || !workspace) return PICHOL_ERR_INVALID_ARG;
    if (bytes < ctx->need_bytes || ((uintptr_t)workspace & 255u)) return PICHOL_ERR_WORKSPACE;
    // the host resources come first; the context takes the workspace only once
    // they exist and its status word reads "no error", so a failure leaves it
    // without a workspace (and without half-made resources)
    if (!ctx->aux) {
        int dev = 0, least = 0, greatest = 0;
        cudaStream_t aux = nullptr;
        cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
        bool ok = cudaGetDevice(&dev) == cudaSuccess &&
                  cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
                  cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess &&
                  cudaStreamCreateWithPriority(&aux, cudaStreamNonBlocking, greatest) == cudaSuccess;
        for (int i = 0; i < 4 && ok; ++i) ok = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            for (cudaEvent_t e : ev)
                if (e) cudaEventDestroy(e);
            if (aux) cudaStreamDestroy(aux);
            return PICHOL_ERR_CUDA;
        }
        ctx->aux = aux;
        ctx->ev_fork = ev[0];
        ctx->ev_panel = ev[1];
        ctx->ev_upd = ev[2];
        ctx->ev_join = ev[3];
    }
    ctx->ws = (char*)workspace;
    ctx->ws_bytes = bytes;
    plan(ctx, ctx->ws);
    ctx->have_hessian = ctx->have_factors = ctx->have_fit = false;
    // debug build: fill the guard bands
    for (int i = 0; i < ctx->nguard; ++i)
        if (cudaMemset(ctx->ws + ctx->guard_off[i], GUARD_FILL, GUARD_BYTES) != cudaSuccess) {
            ctx->ws = nullptr;
            ctx->ws_bytes = 0;
            return PICHOL_ERR_CUDA;
        }
    // the status word must read "no error" before any kernel runs
    if (cudaMemset(ctx->status, 0, sizeof(DevStatus)) != cudaSuccess) {
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
        return PICHOL_ERR_CUDA;
    }
    return PICHOL_OK;
}

pichol_status pichol_hessian(pichol_ctx* ctx, const void* X, const void* Y, const int64_t* fold_offsets,
                             void* stream)
{
    CallRange range_(__func__);
    if (!ctx || !X || !Y) return PICHOL_ERR_INVALID_ARG;
    const pichol_config& c = ctx->cfg;
    if (fold_offsets && !offsets_ok(fold_offsets, c.k, c.n)) return PICHOL_ERR_INVALID_ARG;
    if (!ready(ctx)) return PICHOL_ERR_WORKSPACE;
    for (int f = 0; f <= c.k; ++f) ctx->offs[f] = fold_offsets ? fold_offsets[f] : (int64_t)f * c.n / c.k;
    ctx->kpad = tc_kpad(ctx);   // <= kpad_cap for every split
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(ctx->status, 0, sizeof(DevStatus), s);
    pichol_status st = cuda_status(e == cudaSuccess ? launch_gram(ctx, X, Y, s) : e);
    ctx->have_hessian = st == PICHOL_OK;
    ctx->have_factors = ctx->have_fit = false;
    return st;
}

pichol_status pichol_factor_samples(pichol_ctx* ctx, const double* lam_s, void* stream)
{
    CallRange range_(__func__);
    if (!ctx) return PICHOL_ERR_INVALID_ARG;
    if (lam_s && !lambdas_ok(lam_s, ctx->cfg.g)) return PICHOL_ERR_INVALID_ARG;
    if (!ready(ctx)) return PICHOL_ERR_WORKSPACE;
    if (!ctx->have_hessian) return PICHOL_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_set_samples(ctx, lam_s, s);
    if (e == cudaSuccess) e = launch_factor(ctx, ctx->cfg.g, 0, 0, s);
    pichol_status st = cuda_status(e);
    ctx->have_factors = st == PICHOL_OK;
    ctx->have_fit = false;
    return st;
}

pichol_status pichol_fit(pichol_ctx* ctx, void* theta_out, void* stream)
{
    CallRange range_(__func__);
    if (!ctx) return PICHOL_ERR_INVALID_ARG;
    if (!ready(ctx)) return PICHOL_ERR_WORKSPACE;
    if (!ctx->have_factors) return PICHOL_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_fit(ctx, s);
    if (e == cudaSuccess && theta_out)
        e = cudaMemcpyAsync(theta_out, ctx->Theta,
                            (size_t)ctx->cfg.k * ctx->ntiles * ctx->p * TILE_ELEMS * ctx->eb,
                            cudaMemcpyDeviceToDevice, s);
    pichol_status st = cuda_status(e);
    ctx->have_fit = st == PICHOL_OK;
    return st;
}

pichol_status pichol_eval_holdout(pichol_ctx* ctx, const double* lam_t, double* E_out, int32_t* t_star,
                                  void* W_out, void* stream)
{
    CallRange range_(__func__);
    if (!ctx || !E_out || !t_star) return PICHOL_ERR_INVALID_ARG;
    if (lam_t && !lambdas_ok(lam_t, ctx->cfg.q)) return PICHOL_ERR_INVALID_ARG;
    if (!ready(ctx)) return PICHOL_ERR_WORKSPACE;
    if (!ctx->have_fit) return PICHOL_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_set_evals(ctx, lam_t, s);
    if (e == cudaSuccess) e = launch_eval(ctx, 0, 0, ctx->cfg.q, s);
    if (e == cudaSuccess) e = launch_finish(ctx, E_out, t_star, s);
    if (e == cudaSuccess && W_out) e = launch_copy_w(ctx, W_out, s);
    return cuda_status(e);
}

pichol_status pichol_eval_holdout_exact(pichol_ctx* ctx, const double* lam_t, double* E_out, int32_t* t_star,
                                        void* W_out, void* stream)
{
    CallRange range_(__func__);
    if (!ctx || !E_out || !t_star) return PICHOL_ERR_INVALID_ARG;
    if (lam_t && !lambdas_ok(lam_t, ctx->cfg.q)) return PICHOL_ERR_INVALID_ARG;
    if (!ready(ctx)) return PICHOL_ERR_WORKSPACE;
    if (!ctx->have_hessian) return PICHOL_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    const int q = ctx->cfg.q, b = (int)ctx->exact_batch;
    cudaError_t e = launch_set_evals(ctx, lam_t, s);
    for (int t0 = 0; t0 < q && e == cudaSuccess; t0 += b) {
        const int cnt = (q - t0) < b ? (q - t0) : b;
        e = launch_factor(ctx, cnt, 1, t0, s);
        if (e == cudaSuccess) e = launch_eval(ctx, 1, t0, cnt, s);
    }
    ctx->have_factors = false;   // the sampled factors were overwritten
    if (e == cudaSuccess) e = launch_finish(ctx, E_out, t_star, s);
    if (e == cudaSuccess && W_out) e = launch_copy_w(ctx, W_out, s);
    return cuda_status(e);
}

pichol_status pichol_eval_pinrmse(pichol_ctx* ctx, double* E_out, int32_t* t_star, void* stream)
{
    CallRange range_(__func__);
    if (!ctx || !E_out || !t_star) return PICHOL_ERR_INVALID_ARG;
    if (!ready(ctx)) return PICHOL_ERR_WORKSPACE;
    if (ctx->cfg.warm_samples) return PICHOL_ERR_UNSUPPORTED;
    if (!ctx->have_factors) return PICHOL_ERR_STATE;
    return cuda_status(launch_pinrmse(ctx, E_out, t_star, (cudaStream_t)stream));
}

pichol_status pichol_mchol_levels(double s, double s_min, int32_t* levels)
{
    if (!levels || !(s > 0.0) || !(s <= 300.0) || !(s_min > 0.0) || !(s_min <= 300.0)) return PICHOL_ERR_INVALID_ARG;
    const int n = mchol_levels(s, s_min);
    if (n > 64) return PICHOL_ERR_INVALID_ARG;
    *levels = n;
    return PICHOL_OK;
}

pichol_status pichol_mchol(pichol_ctx* ctx, double c, double s, double s_min, double* trace_out, void* stream)
{
    CallRange range_(__func__);
    int32_t levels = 0;
    if (!ctx || !(c >= -300.0 && c <= 300.0)) return PICHOL_ERR_INVALID_ARG;
    pichol_status st = pichol_mchol_levels(s, s_min, &levels);
    if (st != PICHOL_OK) return st;
    if (!ready(ctx)) return PICHOL_ERR_WORKSPACE;
    if (!ctx->have_hessian) return PICHOL_ERR_STATE;
    if (ctx->cfg.q < 3) return PICHOL_ERR_UNSUPPORTED;
    st = cuda_status(launch_mchol(ctx, c, s, levels, trace_out, (cudaStream_t)stream));
    ctx->have_factors = ctx->have_fit = false;   // the factor buffer was reused; the grid moved
    return st;
}

pichol_status pichol_holdout_grad(pichol_ctx* ctx, double log_lam, double* E_out, double* dE_out, void* stream)
{
    CallRange range_(__func__);
    if (!ctx || !E_out || !dE_out || !(log_lam == log_lam) || log_lam > 700.0 || log_lam < -700.0)
        return PICHOL_ERR_INVALID_ARG;
    if (!ready(ctx)) return PICHOL_ERR_WORKSPACE;
    if (!ctx->have_fit) return PICHOL_ERR_STATE;
    return cuda_status(launch_grad(ctx, log_lam, E_out, dE_out, (cudaStream_t)stream));
}

pichol_status pichol_get_lambdas(pichol_ctx* ctx, double* lam_out, void* stream)
{
    if (!ctx || !lam_out) return PICHOL_ERR_INVALID_ARG;
    if (!ready(ctx)) return PICHOL_ERR_WORKSPACE;
    if (!ctx->have_hessian) return PICHOL_ERR_STATE;
    return cuda_status(cudaMemcpyAsync(lam_out, ctx->lam, sizeof(double) * ctx->cfg.q, cudaMemcpyDeviceToDevice,
                                       (cudaStream_t)stream));
}

pichol_status pichol_export_factor(pichol_ctx* ctx, int32_t f, int32_t s, double* L_out, void* stream)
{
    if (!ctx || !L_out || f < 0 || f >= ctx->cfg.k || s < 0 || s >= ctx->cfg.g) return PICHOL_ERR_INVALID_ARG;
    if (f > 0 && ctx->cfg.warm_samples && s >= ctx->cfg.warm_samples) return PICHOL_ERR_INVALID_ARG;
    if (!ready(ctx)) return PICHOL_ERR_WORKSPACE;
    if (!ctx->have_factors) return PICHOL_ERR_STATE;
    const int64_t slot = (int64_t)f * ctx->cfg.g + s;
    const char* src = (const char*)ctx->F + slot * ctx->ntiles * TILE_ELEMS * ctx->eb;
    return cuda_status(launch_export_tiles(ctx, src, 0, TILE_ELEMS, L_out, (cudaStream_t)stream));
}

pichol_status pichol_export_theta(pichol_ctx* ctx, int32_t f, double* theta_out, void* stream)
{
    if (!ctx || !theta_out || f < 0 || f >= ctx->cfg.k) return PICHOL_ERR_INVALID_ARG;
    if (!ready(ctx)) return PICHOL_ERR_WORKSPACE;
    if (!ctx->have_fit) return PICHOL_ERR_STATE;
    const int64_t d = ctx->cfg.d;
    const char* base = (const char*)ctx->Theta + (int64_t)f * ctx->ntiles * ctx->p * TILE_ELEMS * ctx->eb;
    for (int m = 0; m < ctx->p; ++m) {
        cudaError_t e = launch_export_tiles(ctx, base, (int64_t)m * TILE_ELEMS, (int64_t)ctx->p * TILE_ELEMS,
                                            theta_out + (int64_t)m * d * d, (cudaStream_t)stream);
        if (e != cudaSuccess) return PICHOL_ERR_CUDA;
    }
    return PICHOL_OK;
}

pichol_status pichol_export_hessian(pichol_ctx* ctx, int32_t f, double* H_out, double* B_out, void* stream)
{
    if (!ctx || !H_out || !B_out || f < 0 || f >= ctx->cfg.k) return PICHOL_ERR_INVALID_ARG;
    if (!ready(ctx)) return PICHOL_ERR_WORKSPACE;
    if (!ctx->have_hessian) return PICHOL_ERR_STATE;
    return cuda_status(launch_export_hessian(ctx, f, H_out, B_out, (cudaStream_t)stream));
}

pichol_status pichol_get_info(pichol_ctx* ctx, pichol_info* info, void* stream)
{
    if (!ctx || !info) return PICHOL_ERR_INVALID_ARG;
    if (!ready(ctx)) return PICHOL_ERR_WORKSPACE;
    DevStatus h;
    cudaStream_t s = (cudaStream_t)stream;
    if (ctx->nguard > 0 && launch_check_guards(ctx, s) != cudaSuccess) return PICHOL_ERR_CUDA;
    cudaError_t e = cudaMemcpyAsync(&h, ctx->status, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return PICHOL_ERR_CUDA;
    info->code = (pichol_status)h.code;
    info->fold = h.code ? h.fold : -1;
    info->index = h.code ? h.index : -1;
    info->pivot = h.code ? h.pivot : -1;
    info->unusable = h.unusable;
    return PICHOL_OK;
}

pichol_status pichol_clear_status(pichol_ctx* ctx, void* stream)
{
    if (!ctx) return PICHOL_ERR_INVALID_ARG;
    if (!ready(ctx)) return PICHOL_ERR_WORKSPACE;
    return cuda_status(cudaMemsetAsync(ctx->status, 0, sizeof(DevStatus), (cudaStream_t)stream));
}

pichol_status pichol_check_rsqrt(int64_t n, uint64_t seed, double* max_rel_err, void* stream)
{
    if (n < 1 || n > ((int64_t)1 << 32) || !max_rel_err) return PICHOL_ERR_INVALID_ARG;
    return cuda_status(launch_check_rsqrt(n, seed, max_rel_err, (cudaStream_t)stream));
}

int64_t pichol_launch_count(const pichol_ctx* ctx) { return ctx ? ctx->launches : 0; }

static void free_timing(pichol_ctx* ctx)
{
    if (ctx->ev) {
        for (int i = 0; i < 2 * ctx->ev_cap; ++i) cudaEventDestroy(ctx->ev[i]);
        std::free(ctx->ev);
        std::free(ctx->ev_stage);
    }
    ctx->ev = nullptr;
    ctx->ev_stage = nullptr;
    ctx->ev_cap = ctx->ev_used = 0;
    ctx->timing = 0;
}

pichol_status pichol_set_timing(pichol_ctx* ctx, int32_t max_launches)
{
    if (!ctx || max_launches < 0 || max_launches > (1 << 20)) return PICHOL_ERR_INVALID_ARG;
    free_timing(ctx);
    if (max_launches == 0) return PICHOL_OK;
    ctx->ev = (cudaEvent_t*)std::calloc((size_t)2 * max_launches, sizeof(cudaEvent_t));
    ctx->ev_stage = (int*)std::calloc((size_t)max_launches, sizeof(int));
    if (!ctx->ev || !ctx->ev_stage) { free_timing(ctx); return PICHOL_ERR_INVALID_ARG; }
    for (int i = 0; i < 2 * max_launches; ++i) {
        if (cudaEventCreate(&ctx->ev[i]) != cudaSuccess) {
            ctx->ev_cap = i / 2;
            free_timing(ctx);
            return PICHOL_ERR_CUDA;
        }
        ctx->ev_cap = (i + 1) / 2;
    }
    ctx->ev_cap = max_launches;
    ctx->ev_used = 0;
    ctx->timing = 1;
    return PICHOL_OK;
}

pichol_status pichol_stage_times(pichol_ctx* ctx, double* ms, int64_t* launches, int32_t n_stages, void* stream)
{
    if (!ctx || !ms || !launches || n_stages < 1) return PICHOL_ERR_INVALID_ARG;
    for (int i = 0; i < n_stages; ++i) { ms[i] = 0.0; launches[i] = 0; }
    if (!ctx->timing) return PICHOL_ERR_STATE;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return PICHOL_ERR_CUDA;
    for (int k = 0; k < ctx->ev_used; ++k) {
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, ctx->ev[2 * k], ctx->ev[2 * k + 1]) != cudaSuccess) return PICHOL_ERR_CUDA;
        const int st = ctx->ev_stage[k];
        if (st < n_stages) { ms[st] += t; launches[st] += 1; }
    }
    const int overflow = ctx->ev_used >= ctx->ev_cap;
    ctx->ev_used = 0;
    return overflow ? PICHOL_ERR_WORKSPACE : PICHOL_OK;
}

pichol_status pichol_check_timeout(pichol_ctx* ctx, int64_t cycles, void* stream)
{
    if (!ctx || cycles < 1 || cycles > ((int64_t)1 << 34)) return PICHOL_ERR_INVALID_ARG;
    if (!ready(ctx)) return PICHOL_ERR_WORKSPACE;
    return cuda_status(launch_wait_check(ctx, (long long)cycles, (cudaStream_t)stream));
}

pichol_status pichol_check_wave_timeout(pichol_ctx* ctx, int64_t cycles, void* stream)
{
    if (!ctx || cycles < 1 || cycles > ((int64_t)1 << 34)) return PICHOL_ERR_INVALID_ARG;
    if (!ready(ctx)) return PICHOL_ERR_WORKSPACE;
    const cudaError_t e = launch_wave_check(ctx, (long long)cycles, (cudaStream_t)stream);
    if (e == cudaErrorNotSupported) return PICHOL_ERR_UNSUPPORTED;
    return cuda_status(e);
}

pichol_status pichol_get_tuning(const pichol_ctx* ctx, pichol_tuning* t)
{
    if (!ctx || !t) return PICHOL_ERR_INVALID_ARG;
    *t = ctx->tune;
    return PICHOL_OK;
}

pichol_status pichol_set_tuning(pichol_ctx* ctx, const pichol_tuning* t)
{
    if (!ctx || !t) return PICHOL_ERR_INVALID_ARG;
    if (t->update_strip < 1 || t->update_strip > 8) return PICHOL_ERR_INVALID_ARG;
    if (t->diag_threads != 256 && t->diag_threads != 512) return PICHOL_ERR_INVALID_ARG;
    if (t->diag_exclusive != 0 && t->diag_exclusive != 1) return PICHOL_ERR_INVALID_ARG;
    if (t->eval_overlap != 0 && t->eval_overlap != 1) return PICHOL_ERR_INVALID_ARG;
    if (t->update_engine != 0 && t->update_engine != 1) return PICHOL_ERR_INVALID_ARG;
    if (t->solve_engine < 0 || t->solve_engine > 2) return PICHOL_ERR_INVALID_ARG;
    for (int i = 0; i < 2; ++i)
        if (t->reserved[i] != 0) return PICHOL_ERR_INVALID_ARG;
    ctx->tune = *t;
    return PICHOL_OK;
}

pichol_status pichol_get_state(const pichol_ctx* ctx, int32_t* state)
{
    if (!ctx || !state) return PICHOL_ERR_INVALID_ARG;
    *state = (ctx->have_hessian ? PICHOL_STATE_HESSIAN : 0) | (ctx->have_factors ? PICHOL_STATE_FACTORS : 0) |
             (ctx->have_fit ? PICHOL_STATE_FIT : 0);
    return PICHOL_OK;
}

pichol_status pichol_resume(pichol_ctx* ctx, int32_t state)
{
    constexpr int32_t all = PICHOL_STATE_HESSIAN | PICHOL_STATE_FACTORS | PICHOL_STATE_FIT;
    if (!ctx || (state & ~all)) return PICHOL_ERR_INVALID_ARG;
    if ((state & (PICHOL_STATE_FACTORS | PICHOL_STATE_FIT)) && !(state & PICHOL_STATE_HESSIAN))
        return PICHOL_ERR_INVALID_ARG;
    if (!ready(ctx)) return PICHOL_ERR_WORKSPACE;
    ctx->have_hessian = (state & PICHOL_STATE_HESSIAN) != 0;
    ctx->have_factors = (state & PICHOL_STATE_FACTORS) != 0;
    ctx->have_fit = (state & PICHOL_STATE_FIT) != 0;
    return PICHOL_OK;
}

void pichol_destroy(pichol_ctx* ctx)
{
    if (!ctx) return;
    free_timing(ctx);
    if (ctx->aux) cudaStreamDestroy(ctx->aux);
    for (cudaEvent_t e : {ctx->ev_fork, ctx->ev_panel, ctx->ev_upd, ctx->ev_join})
        if (e) cudaEventDestroy(e);
    delete ctx;
}

int32_t pichol_version(void) { return 100 * PICHOL_VERSION_MAJOR + PICHOL_VERSION_MINOR; }

pichol_status pichol_debug_guards(const pichol_ctx* ctx, int64_t* offsets, int32_t capacity, int32_t* count)
{
    if (!ctx || !count || capacity < 0 || (capacity > 0 && !offsets)) return PICHOL_ERR_INVALID_ARG;
    *count = ctx->nguard;
    for (int i = 0; i < ctx->nguard && i < capacity; ++i) offsets[i] = (int64_t)ctx->guard_off[i];
    return PICHOL_OK;
}

int32_t pichol_debug_build(void) { return GUARD_BYTES > 0 ? 1 : 0; }

const char* pichol_status_string(pichol_status s)
{
    switch (s) {
    case PICHOL_OK: return "ok";
    case PICHOL_ERR_INVALID_ARG: return "invalid argument";
    case PICHOL_ERR_NOT_SPD: return "matrix not positive definite";
    case PICHOL_ERR_CUDA: return "CUDA runtime error";
    case PICHOL_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    case PICHOL_ERR_TIMEOUT: return "bounded device wait gave up";
    case PICHOL_ERR_UNSUPPORTED: return "unsupported";
    case PICHOL_ERR_STATE: return "calls out of order";
    }
    return "unknown status";
}

}  // extern "C"
