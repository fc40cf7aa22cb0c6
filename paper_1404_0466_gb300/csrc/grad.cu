// Hold-out error and its derivative in log(lambda) through the interpolated
// factor (the differentiable use of Algorithm 1's polynomials):
//
//   A(lambda) = L~ L~^T,  L~ = sum_m phi_m(lambda) Theta_m,
//   L~' = dL~/dlambda = sum_m phi_m'(lambda) Theta_m,
//   W = A^{-1} B_f,  V = G_f W - Bv_f,  U = A^{-1} V,
//   E_f = (yy_f + <W, V> - <W, Bv_f>) / (n_f c)              (= ||Y_f - X_f W||^2 / (n_f c))
//   dE_f/dlambda = -(2 / (n_f c)) (<L~'^T U, L~^T W> + <L~^T U, L~'^T W>)
//   dE_f/dlog(lambda) = lambda dE_f/dlambda.
//
// The derivative follows from dW = -A^{-1} (L~' L~^T + L~ L~'^T) W and the
// symmetry of A.  The two solves reuse k_diag_inv / k_solve with a one-entry
// basis table holding phi(lambda); the triangular products build tiles of
// L~ or L~' from Theta in shared memory like the solve.
#include "internal.cuh"

#include <cfloat>
#include <type_traits>

namespace pichol {

cudaError_t launch_diag_solve_one(pichol_ctx* ctx, const double* phi_row, const void* rhs, int rhs_per_system,
                                  void* out, void* dinv, cudaStream_t s);

// phi(lambda) and phi'(lambda) at lambda = exp(log_lam): gphi[0..p) and gphi[p..2p)
__global__ void k_grad_setup(int basis, int p, int g, double log_lam, const double* __restrict__ lam_s,
                             double* __restrict__ gphi, double* __restrict__ glam)
{
    if (threadIdx.x != 0) return;
    double smin = lam_s[0], smax = lam_s[0];
    for (int i = 1; i < g; ++i) { smin = fmin(smin, lam_s[i]); smax = fmax(smax, lam_s[i]); }
    const double lam = exp(log_lam);
    *glam = lam;
    const double a = log(smin), b = log(smax);
    if (basis == PICHOL_BASIS_MONO) {
        const double x = lam / smax;
        double xm = 1.0;
        gphi[p] = 0.0;
        for (int m = 0; m < p; ++m) {
            gphi[m] = xm;
            if (m + 1 < p) gphi[p + m + 1] = (m + 1) * xm / smax;
            xm *= x;
        }
    } else {
        const double u = (b > a) ? 2.0 * (log(lam) - a) / (b - a) - 1.0 : 0.0;
        const double du = (b > a) ? 2.0 / ((b - a) * lam) : 0.0;
        double t0 = 1.0, t1 = u, d0 = 0.0, d1 = 1.0;
        gphi[0] = 1.0;
        gphi[p] = 0.0;
        if (p > 1) { gphi[1] = u; gphi[p + 1] = du; }
        for (int m = 2; m < p; ++m) {
            const double t2 = 2.0 * u * t1 - t0, d2 = 2.0 * t1 + 2.0 * u * d1 - d0;
            gphi[m] = t2;
            gphi[p + m] = d2 * du;
            t0 = t1; t1 = t2; d0 = d1; d1 = d2;
        }
    }
}

// V = G_f W - Bv_f for every fold (dense G_f, dp x dp).  Block (tile row I,
// fold f) walks the columns of its 64 rows in blocks of 32: the G block and the
// matching 32 x c block of W are staged in shared memory (coalesced rows),
// thread (row r, column group cq) multiplies them in the working type, and the
// per-block sums are added in double.
template <typename T>
__global__ void __launch_bounds__(256)
k_grad_gv(const T* __restrict__ G, const T* __restrict__ W, const T* __restrict__ Bv, int64_t dp, int64_t c,
          T* __restrict__ V)
{
    constexpr int KB = 32;
    __shared__ T Gs[TB][KB + 1];
    __shared__ T Ws[KB][32];
    const int I = blockIdx.x, f = blockIdx.y, tid = threadIdx.x, r = tid & 63, cq = tid >> 6;
    const int64_t row = (int64_t)I * TB + r;
    const T* Gf = G + (int64_t)f * dp * dp + (int64_t)I * TB * dp;
    const T* Wf = W + (int64_t)f * dp * c;
    double acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = 0.0;
    const int nb = (int)(dp / KB);
    for (int J = 0; J < nb; ++J) {
        __syncthreads();
        for (int e = tid; e < TB * KB; e += 256) Gs[e / KB][e % KB] = Gf[(int64_t)(e / KB) * dp + J * KB + e % KB];
        for (int e = tid; e < KB * 32; e += 256) {
            const int kk = e / 32, o = e % 32;
            Ws[kk][o] = (o < c) ? Wf[((int64_t)J * KB + kk) * c + o] : T(0);
        }
        __syncthreads();
        T t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) t[u] = T(0);
#pragma unroll 4
        for (int kk = 0; kk < KB; ++kk) {
            const T g = Gs[r][kk];
#pragma unroll
            for (int u = 0; u < 8; ++u) t[u] = fma(g, Ws[kk][cq * 8 + u], t[u]);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] += (double)t[u];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int o = cq * 8 + u;
        if (o < c) {
            const int64_t g = (int64_t)f * dp * c + row * c + o;
            V[g] = (T)(acc[u] - (double)Bv[g]);
        }
    }
}

// L~ = sum_m phi_m Theta_m and L~' = sum_m phi_m' Theta_m of every fold, tile by
// tile, into ML[0] and ML[1] ([which][f][tile][64 x 64]), in the working type
// with the weights rounded to it, as the solves evaluate L~.
template <typename T>
__global__ void __launch_bounds__(256)
k_grad_eval(const T* __restrict__ Theta, int p, int64_t ntiles, int k, const double* __restrict__ gphi,
            T* __restrict__ ML)
{
    const int64_t tile = blockIdx.x;
    const int f = blockIdx.y;
    T w[2][MAX_P];
#pragma unroll
    for (int m = 0; m < MAX_P; ++m) {
        w[0][m] = m < p ? (T)gphi[m] : T(0);
        w[1][m] = m < p ? (T)gphi[p + m] : T(0);
    }
    const T* th = Theta + ((int64_t)f * ntiles + tile) * p * TILE_ELEMS;
    T* o0 = ML + ((int64_t)f * ntiles + tile) * TILE_ELEMS;
    T* o1 = ML + (((int64_t)k + f) * ntiles + tile) * TILE_ELEMS;
    for (int e = threadIdx.x; e < TILE_ELEMS; e += 256) {
        T v0 = w[0][0] * th[e], v1 = w[1][0] * th[e];
#pragma unroll
        for (int m = 1; m < MAX_P; ++m)
            if (m < p) {
                const T x = th[(int64_t)m * TILE_ELEMS + e];
                v0 = fma(w[0][m], x, v0);
                v1 = fma(w[1][m], x, v1);
            }
        o0[e] = v0;
        o1[e] = v1;
    }
}

// out_i = sum_{j >= i} M_ji^T x_j for the four products (M, x) in {L~, L~'} x
// {W, U} (blockIdx.z = 2 which_m + which_x), M's tiles read from ML.  Tile row
// i's range of j is split into nch chunks of at most clen tiles (blockIdx.x =
// i nch + chunk), so every CTA walks a few tiles; each chunk's partial sums go
// to its own slot (k_grad_sum adds the slots in order).  Each tile's product
// is summed in the working type and the tiles are added in double.
template <typename T, int CB>
__global__ void __launch_bounds__(256)
k_grad_tmv(const T* __restrict__ ML, int64_t ntiles, int nt, int nch, int clen, int64_t dp, int64_t c,
           const T* __restrict__ Wv, const T* __restrict__ Uv, double* __restrict__ out)
{
    extern __shared__ __align__(16) unsigned char gsm[];
    double (*red)[CB + 1] = reinterpret_cast<double (*)[CB + 1]>(gsm);                          // 64 x (CB+1)
    T (*Ms)[TB + 1] = reinterpret_cast<T (*)[TB + 1]>(gsm + sizeof(double) * TB * (CB + 1));   // 64 x 65
    T (*xs)[CB] = reinterpret_cast<T (*)[CB]>(gsm + sizeof(double) * TB * (CB + 1) + sizeof(T) * TB * (TB + 1));
    const int i = blockIdx.x / nch, chunk = blockIdx.x % nch, f = blockIdx.y, combo = blockIdx.z;
    const int j0 = i + chunk * clen, j1 = (j0 + clen < nt) ? j0 + clen : nt;   // empty when j0 >= nt
    const int which_m = combo >> 1, which_x = combo & 1;
    const int col = threadIdx.x & 63, kq = threadIdx.x >> 6;
    const T* x = (which_x ? Uv : Wv) + (int64_t)f * dp * c;
    const T* M = ML + ((int64_t)which_m * gridDim.y + f) * ntiles * TILE_ELEMS;
    double acc[CB];
#pragma unroll
    for (int o = 0; o < CB; ++o) acc[o] = 0.0;
    for (int j = j0; j < j1; ++j) {
        const T* mt = M + tile_index(j, i) * TILE_ELEMS;
        __syncthreads();
        for (int e = threadIdx.x; e < TILE_ELEMS; e += 256) Ms[e / TB][e % TB] = mt[e];
        for (int e = threadIdx.x; e < TB * CB; e += 256) {
            const int kk = e / CB, o = e % CB;
            xs[kk][o] = (o < c) ? x[((int64_t)j * TB + kk) * c + o] : T(0);
        }
        __syncthreads();
        if constexpr (std::is_same<T, double>::value) {
#pragma unroll 4
            for (int kk = kq * 16; kk < kq * 16 + 16; ++kk) {
                const double mv = Ms[kk][col];
#pragma unroll
                for (int o = 0; o < CB; ++o) acc[o] = fma(mv, xs[kk][o], acc[o]);
            }
        } else {
            T t[CB];
#pragma unroll
            for (int o = 0; o < CB; ++o) t[o] = T(0);
#pragma unroll 4
            for (int kk = kq * 16; kk < kq * 16 + 16; ++kk) {
                const T mv = Ms[kk][col];
#pragma unroll
                for (int o = 0; o < CB; ++o) t[o] = fma(mv, xs[kk][o], t[o]);
            }
#pragma unroll
            for (int o = 0; o < CB; ++o) acc[o] += (double)t[o];
        }
    }
    __syncthreads();
    for (int qq = 3; qq >= 0; --qq) {
        if (kq == qq) {
#pragma unroll
            for (int o = 0; o < CB; ++o) red[col][o] = (qq == 3) ? acc[o] : red[col][o] + acc[o];
        }
        __syncthreads();
    }
    if (kq == 0) {
        double* dst = out + (((int64_t)chunk * 4 + combo) * gridDim.y + f) * dp * c + ((int64_t)i * TB + col) * c;
        for (int o = 0; o < c; ++o) dst[o] = red[col][o];
    }
}

// slot 0 of P += slots 1 .. nch-1, in slot order (n values per slot)
__global__ void k_grad_sum(double* __restrict__ P, int nch, int64_t n)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double v = P[e];
        for (int ch = 1; ch < nch; ++ch) v += P[(int64_t)ch * n + e];
        P[e] = v;
    }
}

// E_f and dE_f/dlog(lambda) from W, V, Bv and the four products.
template <typename T>
__global__ void __launch_bounds__(256)
k_grad_final(const T* __restrict__ W, const T* __restrict__ V, const T* __restrict__ Bv, const double* __restrict__ P,
             const double* __restrict__ yy, const int64_t* __restrict__ nfc, const double* __restrict__ glam, int k,
             int64_t dp, int64_t c, double* __restrict__ E_out, double* __restrict__ dE_out)
{
    __shared__ double red[2][256];
    const int f = blockIdx.x;
    const int64_t len = dp * c, base = (int64_t)f * len;
    // products (slot 0 after k_grad_sum): combo 0 = L~^T W (P1), 1 = L~^T U (Q1),
    // 2 = L~'^T W (P2), 3 = L~'^T U (Q2)
    const double* P1 = P + ((int64_t)0 * k + f) * len;
    const double* Q1 = P + ((int64_t)1 * k + f) * len;
    const double* P2 = P + ((int64_t)2 * k + f) * len;
    const double* Q2 = P + ((int64_t)3 * k + f) * len;
    double se = 0.0, sd = 0.0;
    for (int64_t e = threadIdx.x; e < len; e += 256) {
        const double wv = (double)W[base + e];
        se += wv * ((double)V[base + e] - (double)Bv[base + e]);
        sd += Q2[e] * P1[e] + Q1[e] * P2[e];
    }
    red[0][threadIdx.x] = se;
    red[1][threadIdx.x] = sd;
    __syncthreads();
    for (int wdt = 128; wdt > 0; wdt >>= 1) {
        if (threadIdx.x < wdt) {
            red[0][threadIdx.x] += red[0][threadIdx.x + wdt];
            red[1][threadIdx.x] += red[1][threadIdx.x + wdt];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double nc = (double)nfc[f];
        E_out[f] = (yy[f] + red[0][0]) / nc;
        dE_out[f] = *glam * (-2.0 / nc) * red[1][0];
    }
}

template <typename T, int CB>
static cudaError_t launch_tmv(dim3 grid, const T* ML, pichol_ctx* ctx, int nch, int clen, const T* gW, const T* gU,
                              cudaStream_t s)
{
    const int smem = (int)(sizeof(double) * TB * (CB + 1) + sizeof(T) * TB * (TB + 1) + sizeof(T) * TB * CB);
    static std::atomic<unsigned long long> set{0};
    const cudaError_t e = smem_limit_once(k_grad_tmv<T, CB>, smem, set);
    if (e != cudaSuccess) return e;
    k_grad_tmv<T, CB><<<grid, 256, smem, s>>>(ML, ctx->ntiles, ctx->nt, nch, clen, ctx->dp, ctx->cfg.c, gW, gU,
                                              ctx->gP);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t grad_impl(pichol_ctx* ctx, double log_lam, double* E_out, double* dE_out, cudaStream_t s)
{
    const pichol_config& cf = ctx->cfg;
    const int64_t dp = ctx->dp, c = cf.c;
    T* gW = (T*)ctx->gW;
    T* gU = gW + (int64_t)cf.k * dp * c;
    T* gV = gU + (int64_t)cf.k * dp * c;
    {
        StageScope sc_(ctx, ST_MISC, s);
        k_grad_setup<<<1, 32, 0, s>>>(cf.basis, ctx->p, cf.g, log_lam, ctx->lam_s, ctx->gphi, ctx->gphi + 2 * MAX_P);
    }
    ctx->launches++;
    cudaError_t e = launch_diag_solve_one(ctx, ctx->gphi, ctx->Btr, 0, gW, ctx->gDinv, s);
    if (e != cudaSuccess) return e;
    {
        StageScope sc_(ctx, ST_SCORE, s);
        k_grad_gv<T><<<dim3(ctx->nt, cf.k), 256, 0, s>>>((const T*)ctx->G, gW, (const T*)ctx->Bv, dp, c, gV);
    }
    ctx->launches++;
    e = launch_diag_solve_one(ctx, ctx->gphi, gV, 1, gU, nullptr, s);   // same lambda: reuse the inverses
    if (e != cudaSuccess) return e;
    // tile row i's tiles j = i .. nt-1 in at most GRAD_CHUNKS chunks of clen tiles
    const int nch = ctx->nt < GRAD_CHUNKS ? ctx->nt : GRAD_CHUNKS;
    const int clen = (ctx->nt + nch - 1) / nch;
    T* ML = (T*)ctx->gL;
    {
        StageScope sc_(ctx, ST_RESID, s);
        k_grad_eval<T><<<dim3((unsigned)ctx->ntiles, cf.k), 256, 0, s>>>((const T*)ctx->Theta, ctx->p, ctx->ntiles,
                                                                        cf.k, ctx->gphi, ML);
    }
    {
        StageScope sc_(ctx, ST_RESID, s);
        const dim3 grid(ctx->nt * nch, cf.k, 4);
        if (c <= 4)
            e = launch_tmv<T, 4>(grid, ML, ctx, nch, clen, gW, gU, s);
        else if (c <= 12)
            e = launch_tmv<T, 12>(grid, ML, ctx, nch, clen, gW, gU, s);
        else
            e = launch_tmv<T, 32>(grid, ML, ctx, nch, clen, gW, gU, s);
        if (e != cudaSuccess) return e;
    }
    {
        StageScope sc_(ctx, ST_RESID, s);
        k_grad_sum<<<1024, 256, 0, s>>>(ctx->gP, nch, (int64_t)4 * cf.k * dp * c);
    }
    {
        StageScope sc_(ctx, ST_SELECT, s);
        k_grad_final<T><<<cf.k, 256, 0, s>>>(gW, gV, (const T*)ctx->Bv, ctx->gP, ctx->yy, ctx->nfc,
                                             ctx->gphi + 2 * MAX_P, cf.k, dp, c, E_out, dE_out);
    }
    ctx->launches += 4;
    return cudaGetLastError();
}

cudaError_t launch_grad(pichol_ctx* ctx, double log_lam, double* E_out, double* dE_out, cudaStream_t s)
{
    if (ctx->cfg.mode == PICHOL_MODE_FP64) return grad_impl<double>(ctx, log_lam, E_out, dE_out, s);
    return grad_impl<float>(ctx, log_lam, E_out, dE_out, s);
}

}  // namespace pichol
