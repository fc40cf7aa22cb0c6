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

// out_i = sum_{j >= i} M_ji^T x_j with M = sum_m w_m Theta_m (w = phi or phi'),
// for the four products (M, x) in {L~, L~'} x {W, U} (blockIdx.z = 2 which_m + which_x).
// M's tiles are evaluated in the working type with w rounded to it, as the
// solves evaluate L~; each tile's product is summed in the working type and
// the tiles are added in double.
template <typename T>
__global__ void __launch_bounds__(256)
k_grad_tmv(const T* __restrict__ Theta, int p, int64_t ntiles, int nt, int64_t dp, int64_t c,
           const double* __restrict__ gphi, const T* __restrict__ Wv, const T* __restrict__ Uv,
           double* __restrict__ out)
{
    extern __shared__ __align__(16) unsigned char gsm[];
    T (*Ms)[TB + 1] = reinterpret_cast<T (*)[TB + 1]>(gsm);                                   // 64 x 65
    T (*xs)[33] = reinterpret_cast<T (*)[33]>(gsm + sizeof(T) * TB * (TB + 1));             // 64 x 33
    double (*red)[33] = reinterpret_cast<double (*)[33]>(gsm + sizeof(T) * TB * (TB + 1 + 33)); // 64 x 33
    const int i = blockIdx.x, f = blockIdx.y, combo = blockIdx.z;
    const int which_m = combo >> 1, which_x = combo & 1;
    const int col = threadIdx.x & 63, kq = threadIdx.x >> 6;
    const T* x = (which_x ? Uv : Wv) + (int64_t)f * dp * c;
    T w[MAX_P];
    for (int m = 0; m < p; ++m) w[m] = (T)gphi[which_m * p + m];
    double acc[32];
#pragma unroll
    for (int o = 0; o < 32; ++o) acc[o] = 0.0;
    for (int j = i; j < nt; ++j) {
        const T* th = Theta + ((int64_t)f * ntiles + tile_index(j, i)) * p * TILE_ELEMS;
        __syncthreads();
        for (int e = threadIdx.x; e < TILE_ELEMS; e += 256) {
            T v = w[0] * th[e];
            for (int m = 1; m < p; ++m) v = fma(w[m], th[(int64_t)m * TILE_ELEMS + e], v);
            Ms[e / TB][e % TB] = v;
        }
        for (int e = threadIdx.x; e < TB * 32; e += 256) {
            const int kk = e / 32, o = e % 32;
            xs[kk][o] = (o < c) ? x[((int64_t)j * TB + kk) * c + o] : T(0);
        }
        __syncthreads();
        T t[32];
#pragma unroll
        for (int o = 0; o < 32; ++o) t[o] = T(0);
        for (int kk = kq * 16; kk < kq * 16 + 16; ++kk) {
            const T mv = Ms[kk][col];
#pragma unroll
            for (int o = 0; o < 32; ++o)
                if (o < c) t[o] = fma(mv, xs[kk][o], t[o]);
        }
#pragma unroll
        for (int o = 0; o < 32; ++o)
            if (o < c) acc[o] += (double)t[o];
    }
    __syncthreads();
    for (int qq = 3; qq >= 0; --qq) {
        if (kq == qq) {
#pragma unroll
            for (int o = 0; o < 32; ++o) red[col][o] = (qq == 3) ? acc[o] : red[col][o] + acc[o];
        }
        __syncthreads();
    }
    if (kq == 0) {
        double* dst = out + ((int64_t)combo * gridDim.y + f) * dp * c + ((int64_t)i * TB + col) * c;
        for (int o = 0; o < c; ++o) dst[o] = red[col][o];
    }
}

// E_f and dE_f/dlog(lambda) from W, V, Bv and the four products.
template <typename T>
__global__ void __launch_bounds__(256)
k_grad_final(const T* __restrict__ W, const T* __restrict__ V, const T* __restrict__ Bv, const double* __restrict__ P,
             const double* __restrict__ yy, const int64_t* __restrict__ nfc, const double* __restrict__ glam,
             int k, int64_t dp, int64_t c, double* __restrict__ E_out, double* __restrict__ dE_out)
{
    __shared__ double red[2][256];
    const int f = blockIdx.x;
    const int64_t len = dp * c, base = (int64_t)f * len;
    // products: combo 0 = L~^T W (P1), 1 = L~^T U (Q1), 2 = L~'^T W (P2), 3 = L~'^T U (Q2)
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
    const int tmv_smem = (int)(sizeof(T) * TB * (TB + 1 + 33) + sizeof(double) * TB * 33);
    static bool attr_done = false;
    if (!attr_done) {
        e = cudaFuncSetAttribute(k_grad_tmv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, tmv_smem);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    {
        StageScope sc_(ctx, ST_RESID, s);
        k_grad_tmv<T><<<dim3(ctx->nt, cf.k, 4), 256, tmv_smem, s>>>((const T*)ctx->Theta, ctx->p, ctx->ntiles,
                                                                     ctx->nt, dp, c, ctx->gphi, gW, gU, ctx->gP);
    }
    {
        StageScope sc_(ctx, ST_SELECT, s);
        k_grad_final<T><<<cf.k, 256, 0, s>>>(gW, gV, (const T*)ctx->Bv, ctx->gP, ctx->yy, ctx->nfc,
                                             ctx->gphi + 2 * MAX_P, cf.k, dp, c, E_out, dE_out);
    }
    ctx->launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_grad(pichol_ctx* ctx, double log_lam, double* E_out, double* dE_out, cudaStream_t s)
{
    if (ctx->cfg.mode == PICHOL_MODE_FP64) return grad_impl<double>(ctx, log_lam, E_out, dE_out, s);
    return grad_impl<float>(ctx, log_lam, E_out, dE_out, s);
}

}  // namespace pichol
