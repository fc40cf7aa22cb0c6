// Evaluation of the interpolated factor and the hold-out solves (Sec. 3.3,
// last paragraph: L(lambda_t) = sum_m phi_m(lambda_t) Theta_m; Sec. 3.2: two
// triangular solves; Sec. 3.1: hold-out error and the argmin over lambda).
//
//   k_diag_inv : for every (fold, lambda, tile row i) the diagonal tile
//                L~_ii(lambda) is built from Theta and inverted; its diagonal is
//                checked (an entry <= 0, or <= 1e3 eps max|diag|, makes the
//                pair unusable and it is scored +inf).
//   k_solve    : forward (L~ Z = B) and back (L~^T W = Z) block substitution
//                for a group of LG lambdas of one fold per CTA.  Each
//                off-diagonal tile's coefficient planes are copied into shared
//                memory once (fp32: TMA boxes with 128-byte swizzle, one thread
//                issuing; fp64: cp.async, XOR-swizzled) and evaluated there for
//                all LG lambdas, so L~(lambda) never exists in global memory.
//   (the refinement residual r = B - L~ (L~^T W) is in resid.cu)
//   k_score    : E partials <W_I, (G_f W)_I> - 2 <Bv_I, W_I> per tile row.
//   k_select   : E_f(t), mean over folds, first argmin.
#include "internal.cuh"
#include "solve_common.cuh"
#include "tma.cuh"

#include <algorithm>
#include <cfloat>
#include <cstring>

namespace pichol {



// ---------------------------------------------------------------------------
// Diagonal tiles: build, check, invert.
// ---------------------------------------------------------------------------
struct DiagArgs {
    const void* src;     // Theta (interp) or factor buffer (exact)
    void* dinv;          // [f][t][i][64x64]
    const double* phi;   // [t][p]
    int* flags;          // [f][t][i]
    float* dmax;
    float* dmin;
    int p, nt, q, t0, per;
    int64_t ntiles, d;
};

constexpr int DIAG_INV_THREADS = 256;
constexpr int DIAG_INV_LD = TB + 2;   // row stride of the staged tiles: even, so entry pairs are aligned

template <typename T, bool EXACT>
__global__ void __launch_bounds__(DIAG_INV_THREADS)
k_diag_inv(DiagArgs a)
{
    constexpr int NT = DIAG_INV_THREADS;
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::N;
    constexpr int NV = TILE_ELEMS / VN / NT;       // 16-byte vectors per thread and plane
    constexpr int GP = 16 / NV;                     // planes whose loads are in flight together
    constexpr int LD = DIAG_INV_LD;
    using V2 = typename VecN<T, 2>::type;
    extern __shared__ __align__(16) unsigned char dsm[];
    T (*Ls)[LD] = reinterpret_cast<T (*)[LD]>(dsm);
    T (*Xs)[LD] = reinterpret_cast<T (*)[LD]>(dsm + sizeof(T) * TB * LD);
    __shared__ float rmax[TB], rmin[TB];
    __shared__ int rbad[TB];
    __shared__ T rinv[TB];
    __shared__ __align__(16) T Ts[TB * TB / 4];     // T = B A^-1 of the lower-left blocks being doubled
    const int i = blockIdx.x, t = a.t0 + blockIdx.y, f = blockIdx.z, tid = threadIdx.x;
    const int64_t ti = tile_index(i, i);
    const int np = EXACT ? 1 : a.p;
    const T* base;
    if constexpr (EXACT) {
        const int pr = f * a.per + (t - a.t0);
        base = (const T*)a.src + ((int64_t)pr * a.ntiles + ti) * TILE_ELEMS;
    } else {
        base = (const T*)a.src + ((int64_t)f * a.ntiles + ti) * a.p * TILE_ELEMS;
    }
    // L~_ii = Theta_0 + sum_{m >= 1} phi_m Theta_m (phi_0 = 1 for both bases; FMAs in m,
    // the solve's order), every thread NV vectors of each plane, the loads of GP
    // planes issued before their first use
    const V* bv = reinterpret_cast<const V*>(base);
    V acc[NV];
#pragma unroll
    for (int u = 0; u < NV; ++u) acc[u] = bv[tid + NT * u];
    if constexpr (!EXACT) {
        for (int m0 = 1; m0 < np; m0 += GP) {
            V tv[GP][NV];
#pragma unroll
            for (int h = 0; h < GP; ++h)
                if (m0 + h < np)
#pragma unroll
                    for (int u = 0; u < NV; ++u) tv[h][u] = bv[(int64_t)(m0 + h) * (TILE_ELEMS / VN) + tid + NT * u];
#pragma unroll
            for (int h = 0; h < GP; ++h)
                if (m0 + h < np) {
                    const T w = (T)a.phi[(int64_t)t * a.p + m0 + h];
#pragma unroll
                    for (int u = 0; u < NV; ++u) {
                        T* x = reinterpret_cast<T*>(&acc[u]);
                        const T* y = reinterpret_cast<const T*>(&tv[h][u]);
#pragma unroll
                        for (int j = 0; j < VN; ++j) x[j] = fma(w, y[j], x[j]);
                    }
                }
        }
    }
#pragma unroll
    for (int u = 0; u < NV; ++u) {
        const T* x = reinterpret_cast<const T*>(&acc[u]);
        const int e = VN * (tid + NT * u), r = e / TB, c0 = e % TB;
#pragma unroll
        for (int j = 0; j < VN; ++j) {
            Ls[r][c0 + j] = (c0 + j <= r) ? x[j] : T(0);
            Xs[r][c0 + j] = T(0);
        }
    }
    __syncthreads();
    if (tid < TB) {
        const T dv = Ls[tid][tid];
        const bool valid = (int64_t)i * TB + tid < a.d;
        rmax[tid] = valid ? (float)fabs((double)dv) : 0.0f;
        rmin[tid] = valid ? (float)fabs((double)dv) : FLT_MAX;
        rbad[tid] = (valid && !(dv > T(0))) ? 1 : 0;
        rinv[tid] = T(1) / dv;
    }
    __syncthreads();
    // Blocked inverse.  The eight 8 x 8 diagonal blocks are inverted by forward
    // substitution on unit vectors (thread (b, c): column c of block b):
    //   X[r][c] = -(sum_{c <= q < r} L[r][q] X[q][c]) / L[r][r].
    // Then the inverted blocks are doubled three times (h = 8, 16, 32): for
    //   L = [A 0; B C],  L^-1 = [A^-1 0; -C^-1 (B A^-1) C^-1],
    // first T = B A^-1, then the lower-left block -C^-1 T, every two adjacent
    // entries of a row by one thread (one load of B or C^-1 serves both; each
    // entry's sum keeps its order).
    if (tid < TB) {
        const int b0 = (tid >> 3) * 8, c = b0 + (tid & 7);
        Xs[c][c] = rinv[c];
        for (int r = c + 1; r < b0 + 8; ++r) {
            T s = T(0);
            for (int qq = c; qq < r; ++qq) s = fma(Ls[r][qq], Xs[qq][c], s);
            Xs[r][c] = -s * rinv[r];
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int h = 8; h < TB; h *= 2) {
        const int hh = h * h, ne = (TB / (2 * h)) * hh;     // entries of all lower-left blocks: 32 h
        for (int e = 2 * tid; e < ne; e += 2 * NT) {
            const int b0 = (e / hh) * 2 * h, r = (e % hh) / h, c = e % h;   // c even
            // (A^-1 is lower triangular: its entry (c, c + 1) is zero, so both sums start at k = c)
            T s0 = T(0), s1 = T(0);
            for (int k = c; k < h; ++k) {
                const T bv = Ls[b0 + h + r][b0 + k];
                const V2 x = *reinterpret_cast<const V2*>(&Xs[b0 + k][b0 + c]);
                s0 = fma(bv, x.x, s0);
                s1 = fma(bv, x.y, s1);
            }
            V2 o2;
            o2.x = s0;
            o2.y = s1;
            *reinterpret_cast<V2*>(&Ts[e]) = o2;
        }
        __syncthreads();
        for (int e = 2 * tid; e < ne; e += 2 * NT) {
            const int b0 = (e / hh) * 2 * h, r = (e % hh) / h, c = e % h;
            const T* tcol = Ts + (e / hh) * hh + c;
            T s0 = T(0), s1 = T(0);
            for (int k = 0; k <= r; ++k) {
                const T cv = Xs[b0 + h + r][b0 + h + k];
                const V2 t2 = *reinterpret_cast<const V2*>(tcol + k * h);
                s0 = fma(cv, t2.x, s0);
                s1 = fma(cv, t2.y, s1);
            }
            Xs[b0 + h + r][b0 + c] = -s0;
            Xs[b0 + h + r][b0 + c + 1] = -s1;
        }
        __syncthreads();
    }
    T* out = (T*)a.dinv + (((int64_t)f * a.q + t) * a.nt + i) * TILE_ELEMS;
    for (int e = tid; e < TILE_ELEMS; e += NT) out[e] = Xs[e / TB][e % TB];
    if (tid == 0) {
        float mx = 0.0f, mn = FLT_MAX;
        int bad = 0;
        for (int r = 0; r < TB; ++r) { mx = fmaxf(mx, rmax[r]); mn = fminf(mn, rmin[r]); bad |= rbad[r]; }
        const int64_t o = ((int64_t)f * a.q + t) * a.nt + i;
        a.flags[o] = bad;
        a.dmax[o] = mx;
        a.dmin[o] = mn;
    }
}

// y += x over the systems t0 .. t0 + tcount - 1 of every fold ([f][t][dp][c]
// blocks of `len` values).
template <typename T>
__global__ void k_axpy(T* __restrict__ y, const T* __restrict__ x, int k, int q, int t0, int tcount, int64_t len)
{
    const int64_t per = (int64_t)tcount * len, n = (int64_t)k * per;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int f = (int)(e / per);
        const int64_t g = ((int64_t)f * q + t0) * len + e % per;
        y[g] += x[g];
    }
}

// ---------------------------------------------------------------------------
// Hold-out score partials: for tile row I and LG lambdas of fold f,
//   part = sum_{rows in I} sum_o W[row][o] ((G_f W)[row][o] - 2 Bv_f[row][o])
// with G_f = X_f^T X_f (the fold's own Gram block, dense).  Products in the
// working type per 64-column tile, everything above that in double.
// ---------------------------------------------------------------------------
struct ScoreArgs {
    const void* G;       // [j][dp][dp]
    const void* Bv;      // [j][dp][c]
    const void* W;       // [f][t][dp][c]
    double* Epart;       // [f][t][I]
    int nt, q, t0, tcount;
    int64_t dp, c;
};

template <typename T, int LG, int CB>
__global__ void __launch_bounds__(256)
k_score(ScoreArgs a)
{
    constexpr int VN = Vec16<T>::N;
    constexpr int CBP = (CB + VN - 1) / VN * VN;
    constexpr int PB = TILE_ELEMS * (int)sizeof(T);
    using V = typename Vec16<T>::type;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* plane = smem;
    T* Zs = reinterpret_cast<T*>(smem + PB);                 // [LG][64][CBP]
    double* Ud = reinterpret_cast<double*>(Zs + LG * TB * CBP); // [LG][64][CBP]
    __shared__ double red[256];
    const int I = blockIdx.x, f = blockIdx.z, tid = threadIdx.x;
    const int r = tid & 63, kq = tid >> 6;
    const int64_t c = a.c, dp = a.dp;
    int tl[LG];
    bool live[LG];
#pragma unroll
    for (int l = 0; l < LG; ++l) {
        const int li = blockIdx.y * LG + l;
        live[l] = li < a.tcount;
        tl[l] = a.t0 + (live[l] ? li : a.tcount - 1);
    }
    const T* G = (const T*)a.G + (int64_t)f * dp * dp;
    const T* Wt = (const T*)a.W;
    for (int e = tid; e < LG * TB * CBP; e += 256) Zs[e] = T(0);
    double tot[LG][CBP];
#pragma unroll
    for (int l = 0; l < LG; ++l)
#pragma unroll
        for (int o = 0; o < CBP; ++o) tot[l][o] = 0.0;
#pragma unroll 1
    for (int J = 0; J < a.nt; ++J) {
        __syncthreads();
        stage_planes<T>(plane, G + (int64_t)I * TB * dp + (int64_t)J * TB, 1, dp, 0);
        cp_async_commit();
        for (int e = tid; e < LG * TB * c; e += 256) {
            const int l = e / (TB * (int)c), rem = e % (TB * (int)c);
            const int kk = rem / (int)c, o = rem % (int)c;
            Zs[(l * TB + kk) * CBP + o] = Wt[((int64_t)f * a.q + tl[l]) * dp * c + (int64_t)J * TB * c + rem];
        }
        cp_async_wait<0>();
        __syncthreads();
        T acc[LG][CBP];
#pragma unroll
        for (int l = 0; l < LG; ++l)
#pragma unroll
            for (int o = 0; o < CBP; ++o) acc[l][o] = T(0);
#pragma unroll 1
        for (int ch = 0; ch < 16 / VN; ++ch) {
            const int kc = (kq * 16) / VN + ch;
            V x = *reinterpret_cast<const V*>(plane + r * TB * (int)sizeof(T) + ((kc ^ (r & 7)) << 4));
            T gv[VN];
            memcpy(gv, &x, 16);
#pragma unroll
            for (int e = 0; e < VN; ++e) {
                const int kk = kc * VN + e;
#pragma unroll
                for (int l = 0; l < LG; ++l) {
                    const T* zrow = Zs + (l * TB + kk) * CBP;
#pragma unroll
                    for (int o = 0; o < CBP; ++o) acc[l][o] = fma(gv[e], zrow[o], acc[l][o]);
                }
            }
        }
#pragma unroll
        for (int l = 0; l < LG; ++l)
#pragma unroll
            for (int o = 0; o < CBP; ++o) tot[l][o] += (double)acc[l][o];
    }
    __syncthreads();
#pragma unroll 1
    for (int qq = 3; qq >= 0; --qq) {
        if (kq == qq) {
#pragma unroll
            for (int l = 0; l < LG; ++l)
#pragma unroll
                for (int o = 0; o < CBP; ++o) {
                    double* dst = Ud + (l * TB + r) * CBP + o;
                    *dst = (qq == 3) ? tot[l][o] : *dst + tot[l][o];
                }
        }
        __syncthreads();
    }
    // per-lambda dot products over this tile row
    const T* Bv = (const T*)a.Bv + (int64_t)f * dp * c;
#pragma unroll 1
    for (int l = 0; l < LG; ++l) {
        double s = 0.0;
        if (tid < TB) {
            const int64_t row = (int64_t)I * TB + tid;
            const T* wr = Wt + ((int64_t)f * a.q + tl[l]) * dp * c + row * c;
            for (int o = 0; o < c; ++o) {
                const double wv = (double)wr[o];
                s += wv * (Ud[(l * TB + tid) * CBP + o] - 2.0 * (double)Bv[row * c + o]);
            }
        }
        red[tid] = s;
        __syncthreads();
        for (int wdt = 128; wdt > 0; wdt >>= 1) {
            if (tid < wdt) red[tid] += red[tid + wdt];
            __syncthreads();
        }
        if (tid == 0 && live[l]) a.Epart[((int64_t)f * a.q + tl[l]) * a.nt + I] = red[0];
        __syncthreads();
    }
}

// E_f(t) = (yy_f + sum_I part) / (n_f c), +inf if unusable; Ebar; first argmin.
__global__ void __launch_bounds__(256)
k_select(const double* __restrict__ Epart, const int* __restrict__ flags, const float* __restrict__ dmax,
         const float* __restrict__ dmin, const double* __restrict__ yy, const int64_t* __restrict__ nf_c,
         int k, int q, int nt, double* __restrict__ E_out, double* __restrict__ Eint, int32_t* __restrict__ t_star,
         DevStatus* st)
{
    __shared__ double Ebar[4096];
    __shared__ int nbad[256];
    int bad_count = 0;
    const double thr_rel = 1e3 * DBL_EPSILON;
    for (int t = threadIdx.x; t < q; t += 256) {
        double sum = 0.0;
        for (int f = 0; f < k; ++f) {
            const int64_t o = ((int64_t)f * q + t) * nt;
            int bad = 0;
            float mx = 0.0f, mn = FLT_MAX;
            double s = yy[f];
            for (int i = 0; i < nt; ++i) {
                bad |= flags[o + i];
                mx = fmaxf(mx, dmax[o + i]);
                mn = fminf(mn, dmin[o + i]);
                s += Epart[o + i];
            }
            if ((double)mn <= thr_rel * (double)mx) bad = 1;
            const double e = bad ? INFINITY : s / (double)nf_c[f];
            bad_count += bad;
            E_out[(int64_t)f * q + t] = e;
            Eint[(int64_t)f * q + t] = e;
            sum += e;
        }
        Ebar[t] = sum / (double)k;
    }
    nbad[threadIdx.x] = bad_count;
    __syncthreads();
    if (threadIdx.x == 0) {
        int best = -1;
        double bv = INFINITY;
        int nb = 0;
        for (int t = 0; t < q; ++t) {
            if (isfinite(Ebar[t]) && Ebar[t] < bv) { bv = Ebar[t]; best = t; }
        }
        for (int u = 0; u < 256; ++u) nb += nbad[u];
        *t_star = best;
        st->unusable = nb;
    }
}

// ---------------------------------------------------------------------------
// host-side launch plumbing
// ---------------------------------------------------------------------------

// Dynamic shared memory the solve kernel needs for a mode (element bytes eb),
// p coefficient planes and c outputs; mirrors SolveCfg.
size_t solve_smem_bytes(int eb, int p, int64_t c)
{
    const int LG = 2, cb = pick_cb(c), vn = 16 / eb;
    const int zvn = cb % vn == 0 ? vn : (cb % 2 == 0 ? 2 : 1);
    const int cbp = (cb + zvn - 1) / zvn * zvn;
    const size_t zs = (size_t)2 * LG * (TB / 2) * cbp * eb, rb = (size_t)4 * LG * TB * cbp * eb;
    const size_t dinv = (size_t)LG * TB * TB * eb, hpb = (size_t)(TB / 2) * TB * eb;
    size_t most = 0;
    for (int nps : {p, LG}) {          // interpolated (p planes) and exact (LG planes)
        const size_t stage = (size_t)nps * hpb;
        if (eb == 4) {
            const size_t loop = 2 * stage;
            const size_t ring = loop > dinv + rb ? loop : dinv + rb;
            most = std::max(most, ring + zs + 1024);
        } else {
            const size_t ring = 2 * stage > dinv ? 2 * stage : dinv;
            most = std::max(most, ring + zs + rb);
        }
    }
    return most;
}

// The map the fp32 solve and residual stage coefficient (or factor) planes
// through: the buffer viewed as [rows][64] fp32, 32 x 32 boxes.
cudaError_t plane_map(CUtensorMap* m, const void* buf, int64_t planes)
{
    const int64_t rows = planes * TB;
    if (rows > INT32_MAX) return cudaErrorInvalidValue;   // TMA coordinates are 32-bit
    return make_map_f32(m, (const float*)buf, TB, (uint64_t)rows, TB, 32, 32) ? cudaSuccess : cudaErrorInvalidValue;
}

// Two lambdas per CTA share each staged coefficient tile.  When every
// system can have an SM of its own (a single lambda, as in the gradient, or a
// few, as in an MChol level) the systems take one-lambda CTAs with a deeper
// copy ring instead: there each CTA's serial chain sets the time, and a
// two-lambda CTA would double it.  A system's arithmetic does not depend on LG.
template <typename T, bool EXACT>
static cudaError_t solve_dispatch(pichol_ctx* ctx, const SolveArgs& sa, cudaStream_t s)
{
    if (sa.tcount == 1 || (int64_t)ctx->cfg.k * sa.tcount <= ctx->nsm) {
        if constexpr (std::is_same<T, float>::value) {
            if (ctx->tune.solve_engine != 1) {           // the wavefront unless the CUDA-core chain is asked for
                const cudaError_t e = launch_solve_wave(ctx, sa, EXACT, s);
                if (e != cudaErrorNotSupported) return e;
            }
        }
        return launch_solve_single(ctx, sa, EXACT, s);
    }
    constexpr int LG = 2;
    switch (pick_cb(ctx->cfg.c)) {
    case 4: return solve_np<T, LG, 4, EXACT>(ctx, sa, s);
    case 10: return solve_np<T, LG, 10, EXACT>(ctx, sa, s);
    case 12: return solve_np<T, LG, 12, EXACT>(ctx, sa, s);
    default: return solve_np<T, LG, 32, EXACT>(ctx, sa, s);
    }
}

template <typename T, int LG, int CB>
static cudaError_t run_score(pichol_ctx* ctx, const ScoreArgs& sc, cudaStream_t s)
{
    constexpr int VN = Vec16<T>::N;
    constexpr int CBP = (CB + VN - 1) / VN * VN;
    const int smem = TILE_ELEMS * (int)sizeof(T) + LG * TB * CBP * (int)sizeof(T) + LG * TB * CBP * 8;
    static std::atomic<unsigned long long> set{0};
    {
        const cudaError_t e = smem_limit_once(k_score<T, LG, CB>, smem, set);
        if (e != cudaSuccess) return e;
    }
    dim3 grid(ctx->nt, (unsigned)((sc.tcount + LG - 1) / LG), ctx->cfg.k);
    {
        StageScope sc_(ctx, ST_SCORE, s);
        k_score<T, LG, CB><<<grid, 256, smem, s>>>(sc);
    }
    ctx->launches++;
    return cudaGetLastError();
}

template <typename T>
static cudaError_t score_dispatch(pichol_ctx* ctx, const ScoreArgs& sc, cudaStream_t s)
{
    switch (pick_cb(ctx->cfg.c)) {
    case 4: return run_score<T, 2, 4>(ctx, sc, s);
    case 10:
    case 12: return run_score<T, 2, 12>(ctx, sc, s);
    default: return run_score<T, 1, 32>(ctx, sc, s);
    }
}

template <typename T, bool EXACT>
static cudaError_t eval_impl(pichol_ctx* ctx, int t0, int tcount, cudaStream_t s)
{
    const pichol_config& cf = ctx->cfg;
    DiagArgs da;
    da.src = EXACT ? ctx->F : ctx->Theta;
    da.dinv = ctx->Dinv;
    da.phi = ctx->phi;
    da.flags = ctx->flags;
    da.dmax = ctx->dmax;
    da.dmin = ctx->dmin;
    da.p = ctx->p;
    da.nt = ctx->nt;
    da.q = cf.q;
    da.t0 = t0;
    da.per = (int)ctx->exact_batch;
    da.ntiles = ctx->ntiles;
    da.d = cf.d;
    const int dsm = 2 * (int)sizeof(T) * TB * DIAG_INV_LD;
    static std::atomic<unsigned long long> set{0};
    {
        const cudaError_t ea = smem_limit_once(k_diag_inv<T, EXACT>, dsm, set);
        if (ea != cudaSuccess) return ea;
    }
    {
        StageScope sc_(ctx, ST_DIAG_INV, s);
        k_diag_inv<T, EXACT><<<dim3(ctx->nt, tcount, cf.k), DIAG_INV_THREADS, dsm, s>>>(da);
    }
    ctx->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;

    // the interpolated (or exact) solves of systems [t0h, t0h + tch) and their
    // refinement steps, on stream `st`
    auto solve_refine = [&](int t0h, int tch, cudaStream_t st, cudaEvent_t solved) -> cudaError_t {
        SolveArgs sa;
        sa.src = da.src;
        sa.dinv = ctx->Dinv;
        sa.rhs = ctx->Btr;
        sa.zbuf = ctx->W;
        sa.out = ctx->W;
        sa.phi = ctx->phi;
        sa.p = ctx->p;
        sa.nt = ctx->nt;
        sa.q = cf.q;
        sa.t0 = t0h;
        sa.tcount = tch;
        sa.per = (int)ctx->exact_batch;
        sa.rhs_per_system = 0;
        sa.ntiles = ctx->ntiles;
        sa.dp = ctx->dp;
        sa.c = cf.c;
        sa.st = ctx->status;
        // mixed mode, interpolated systems: all lambdas per fold on the tensor cores when tuned so
        // automatic: the tensor cores when a fold's planes stream from HBM for every lambda pair
        const bool big = (double)ctx->ntiles * ctx->p * TILE_ELEMS * sizeof(float) > 64.0 * 1024 * 1024;
        const int eng = ctx->tune.solve_engine == 2 ? (big ? 0 : 1) : ctx->tune.solve_engine;
        const bool tcs = std::is_same<T, float>::value && !EXACT && eng == 0 && ctx->Sh;
        cudaError_t er = tcs ? launch_solve_tc(ctx, t0h, tch, ctx->Btr, 0, ctx->W, st)
                             : solve_dispatch<T, EXACT>(ctx, sa, st);
        if (er == cudaSuccess && solved) er = cudaEventRecord(solved, st);
        if (er != cudaSuccess) return er;
        if constexpr (std::is_same<T, float>::value && !EXACT) {
            for (int it = 0; it < cf.refine_steps; ++it) {
                // the residual of the system this step refines (see refine_target)
                if (cf.refine_target == PICHOL_REFINE_EXACT) {
                    if ((er = launch_resid_exact(ctx, t0h, tch, st)) != cudaSuccess) return er;
                } else if (cf.refine_residual == PICHOL_RESIDUAL_TENSOR) {
                    if ((er = launch_resid_tc(ctx, t0h, tch, st)) != cudaSuccess) return er;
                } else {
                    ResidArgs ra;
                    ra.theta = (const float*)ctx->Theta;
                    ra.W = (const float*)ctx->W;
                    ra.uhi = (const float*)ctx->U;
                    ra.ulo = (const float*)ctx->U + (int64_t)cf.k * cf.q * ctx->dp * cf.c;
                    ra.ohi = (float*)ctx->U;
                    ra.olo = (float*)ctx->U + (int64_t)cf.k * cf.q * ctx->dp * cf.c;
                    ra.B = (const float*)ctx->Btr;
                    ra.R = (float*)ctx->Rres;
                    ra.phi = ctx->phi;
                    ra.p = ctx->p;
                    ra.nt = ctx->nt;
                    ra.q = cf.q;
                    ra.t0 = t0h;
                    ra.tcount = tch;
                    ra.ntiles = ctx->ntiles;
                    ra.dp = ctx->dp;
                    ra.c = cf.c;
                    ra.st = ctx->status;
                    if ((er = launch_resid_pass(ctx, ra, 0, st)) != cudaSuccess) return er;
                    if ((er = launch_resid_pass(ctx, ra, 1, st)) != cudaSuccess) return er;
                }
                SolveArgs sc = sa;
                sc.rhs = ctx->Rres;
                sc.rhs_per_system = 1;
                sc.zbuf = ctx->Rres;
                sc.out = ctx->Rres;
                er = tcs ? launch_solve_tc(ctx, t0h, tch, ctx->Rres, 1, ctx->Rres, st) : solve_dispatch<T, EXACT>(ctx, sc, st);
                if (er != cudaSuccess) return er;
                {
                    StageScope sc_(ctx, ST_RESID, st);
                    k_axpy<float><<<1024, 256, 0, st>>>((float*)ctx->W, (const float*)ctx->Rres, cf.k, cf.q, t0h,
                                                        tch, ctx->dp * cf.c);
                }
                ctx->launches++;
            }
        }
        return cudaGetLastError();
    };

    // With refinement and the overlap tuning, the systems are split in two
    // halves: the second half starts on the internal high-priority stream when
    // the first half's solve ends, so its solve runs beside the first half's
    // residual passes (the solve alone leaves most issue slots idle).  Each
    // system's arithmetic is unchanged.
    const bool overlap = std::is_same<T, float>::value && !EXACT && cf.refine_steps > 0 && ctx->tune.eval_overlap &&
                         ctx->aux && tcount >= 4;
    if (overlap) {
        const int tA = (tcount / 2) & ~1, tB = tcount - tA;
        if ((e = solve_refine(t0, tA, s, ctx->ev_panel)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(ctx->aux, ctx->ev_panel, 0)) != cudaSuccess) return e;
        if ((e = solve_refine(t0 + tA, tB, ctx->aux, nullptr)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(ctx->ev_join, ctx->aux)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s, ctx->ev_join, 0)) != cudaSuccess) return e;
    } else {
        if ((e = solve_refine(t0, tcount, s, nullptr)) != cudaSuccess) return e;
    }

    if constexpr (std::is_same<T, float>::value) {
        // mixed mode: G_f W for all lambdas on tensor cores, then the dot products
        return launch_score_tc(ctx, t0, tcount, s);
    }
    ScoreArgs sc;
    sc.G = ctx->G;
    sc.Bv = ctx->Bv;
    sc.W = ctx->W;
    sc.Epart = ctx->Epart;
    sc.nt = ctx->nt;
    sc.q = cf.q;
    sc.t0 = t0;
    sc.tcount = tcount;
    sc.dp = ctx->dp;
    sc.c = cf.c;
    return score_dispatch<T>(ctx, sc, s);
}

// One interpolated system per fold at the lambda whose basis values are
// phi_row[0..p): optional diagonal inverses (into dinv_out, with the gradient's
// own diagonal checks), then the solve of (L~ L~^T) out = rhs.
template <typename T>
static cudaError_t diag_solve_one_impl(pichol_ctx* ctx, const double* phi_row, const void* rhs, int rhs_per_system,
                                       void* out, void* dinv_out, cudaStream_t s)
{
    const pichol_config& cf = ctx->cfg;
    if (dinv_out) {
        DiagArgs da;
        da.src = ctx->Theta;
        da.dinv = dinv_out;
        da.phi = phi_row;
        da.flags = ctx->gflags;
        da.dmax = ctx->gdmax;
        da.dmin = ctx->gdmin;
        da.p = ctx->p;
        da.nt = ctx->nt;
        da.q = 1;
        da.t0 = 0;
        da.per = 1;
        da.ntiles = ctx->ntiles;
        da.d = cf.d;
        const int dsm = 2 * (int)sizeof(T) * TB * DIAG_INV_LD;
        static std::atomic<unsigned long long> set{0};
        const cudaError_t ea = smem_limit_once(k_diag_inv<T, false>, dsm, set);
        if (ea != cudaSuccess) return ea;
        {
            StageScope sc_(ctx, ST_DIAG_INV, s);
            k_diag_inv<T, false><<<dim3(ctx->nt, 1, cf.k), DIAG_INV_THREADS, dsm, s>>>(da);
        }
        ctx->launches++;
    }
    SolveArgs sa;
    sa.src = ctx->Theta;
    sa.dinv = ctx->gDinv;
    sa.rhs = rhs;
    sa.zbuf = out;
    sa.out = out;
    sa.phi = phi_row;
    sa.p = ctx->p;
    sa.nt = ctx->nt;
    sa.q = 1;
    sa.t0 = 0;
    sa.tcount = 1;
    sa.per = 1;
    sa.rhs_per_system = rhs_per_system;
    sa.ntiles = ctx->ntiles;
    sa.dp = ctx->dp;
    sa.c = cf.c;
    sa.st = ctx->status;
    return solve_dispatch<T, false>(ctx, sa, s);
}

cudaError_t launch_diag_solve_one(pichol_ctx* ctx, const double* phi_row, const void* rhs, int rhs_per_system,
                                  void* out, void* dinv, cudaStream_t s)
{
    if (ctx->cfg.mode == PICHOL_MODE_FP64)
        return diag_solve_one_impl<double>(ctx, phi_row, rhs, rhs_per_system, out, dinv, s);
    return diag_solve_one_impl<float>(ctx, phi_row, rhs, rhs_per_system, out, dinv, s);
}

cudaError_t launch_eval(pichol_ctx* ctx, int exact, int t0, int tcount, cudaStream_t s)
{
    if (ctx->cfg.mode == PICHOL_MODE_FP64)
        return exact ? eval_impl<double, true>(ctx, t0, tcount, s) : eval_impl<double, false>(ctx, t0, tcount, s);
    return exact ? eval_impl<float, true>(ctx, t0, tcount, s) : eval_impl<float, false>(ctx, t0, tcount, s);
}

cudaError_t launch_finish(pichol_ctx* ctx, double* E_out, int32_t* t_star, cudaStream_t s)
{
    const pichol_config& cf = ctx->cfg;
    {
        StageScope sc_(ctx, ST_SELECT, s);
        k_select<<<1, 256, 0, s>>>(ctx->Epart, ctx->flags, ctx->dmax, ctx->dmin, ctx->yy, ctx->nfc, cf.k, cf.q, ctx->nt,
                                   E_out, ctx->E, t_star, ctx->status);
    }
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t launch_copy_w(pichol_ctx* ctx, void* W_out, cudaStream_t s)
{
    const pichol_config& cf = ctx->cfg;
    const size_t eb = (size_t)ctx->eb;
    return cudaMemcpy2DAsync(W_out, (size_t)cf.d * cf.c * eb, ctx->W, (size_t)ctx->dp * cf.c * eb,
                             (size_t)cf.d * cf.c * eb, (size_t)cf.k * cf.q, cudaMemcpyDeviceToDevice, s);
}

}  // namespace pichol
