// Normal-equation blocks (Sec. 3.1, Eq. 2: H = X^T X, g = X^T y) per fold,
// the lambda grid, and the Vandermonde pseudo-inverse of Algorithm 1.
//
//   G_j  = X_j^T X_j   (dense dp x dp, fold j's rows)       k_gram_simt
//   Bv_j = X_j^T Y_j   (dp x c)                             k_xty + k_bsum
//   yy_j = ||Y_j||_F^2                                      k_yy
//   tau, lambda grid, sampled lambdas, V, P = V^+, phi      k_setup
//   B_f  = sum_{j != f} Bv_j                                k_bsum
//   H_f  = sum_{j != f} G_j, lower tiles                    k_hf_tiles
#include "internal.cuh"

#include <cuda.h>
#include <cmath>
#include <cstring>
#include <mutex>

namespace pichol {

struct FoldOffs { int64_t o[MAX_K + 1]; };

// ---------------------------------------------------------------------------
// G_j = X_j^T X_j, one 64 x 64 output tile per CTA (lower tiles; the upper
// tile is written by mirroring).  Rows are consumed 32 at a time; each chunk
// sum is accumulated in the working type and folded into a compensated
// (Kahan) total so that long folds do not lose accuracy.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_gram_simt(const T* __restrict__ X, int64_t d, int64_t dp, FoldOffs fo, T* __restrict__ G)
{
    int I, J;
    tile_coords(blockIdx.x, I, J);
    const int j = blockIdx.y;
    const int64_t r0 = fo.o[j], r1 = fo.o[j + 1];
    __shared__ T As[32][TB];
    __shared__ T Bs[32][TB];
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    T tot[4][4], cmp[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) { tot[a][b] = T(0); cmp[a][b] = T(0); }

    for (int64_t rb = r0; rb < r1; rb += 32) {
        for (int qq = tid; qq < 32 * TB; qq += 256) {
            int rr = qq / TB, cc = qq % TB;
            int64_t row = rb + rr;
            int64_t ci = (int64_t)I * TB + cc, cj = (int64_t)J * TB + cc;
            As[rr][cc] = (row < r1 && ci < d) ? X[row * d + ci] : T(0);
            Bs[rr][cc] = (row < r1 && cj < d) ? X[row * d + cj] : T(0);
        }
        __syncthreads();
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {   // Kahan: tot += acc
                T y = acc[a][b] - cmp[a][b];
                T t = tot[a][b] + y;
                cmp[a][b] = (t - tot[a][b]) - y;
                tot[a][b] = t;
            }
        __syncthreads();
    }
    T* Gj = G + (int64_t)j * dp * dp;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            int64_t row = (int64_t)I * TB + ty + 16 * a;
            int64_t col = (int64_t)J * TB + tx + 16 * b;
            Gj[row * dp + col] = tot[a][b];
            if (I != J) Gj[col * dp + row] = tot[a][b];
        }
}

// ---------------------------------------------------------------------------
// Bv_j = X_j^T Y_j in two deterministic passes.  k_xty: CTA (tile, fold j,
// row split rs) sums rows [r0 + rs*chunk, ...) of fold j; thread (feature fi,
// output phase oc) accumulates outputs o = oc + 4u over 32-row chunks in the
// working type, chunk totals in double, into part[j][rs][dp][c].
// k_bsum: Bv_j = sum_rs part (increasing rs), B_f = sum_{j != f} Bv_j.
// ---------------------------------------------------------------------------
constexpr int XTY_SPLITS = 16;

template <typename T>
__global__ void __launch_bounds__(256)
k_xty(const T* __restrict__ X, const T* __restrict__ Y, int64_t d, int64_t dp, int64_t c,
      FoldOffs fo, double* __restrict__ part)
{
    const int tile = blockIdx.x, j = blockIdx.y, rs = blockIdx.z;
    const int fi = threadIdx.x & 63, oc = threadIdx.x >> 6;
    const int64_t col = (int64_t)tile * TB + fi;
    const int64_t nj = fo.o[j + 1] - fo.o[j];
    const int64_t chunk = ((nj + XTY_SPLITS - 1) / XTY_SPLITS + 31) / 32 * 32;
    const int64_t r0 = fo.o[j] + rs * chunk;
    const int64_t r1 = (r0 + chunk < fo.o[j + 1]) ? r0 + chunk : fo.o[j + 1];
    double tot[16];
    T acc[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) tot[u] = 0.0;
    for (int64_t rb = r0; rb < r1; rb += 32) {
#pragma unroll
        for (int u = 0; u < 16; ++u) acc[u] = T(0);
        const int64_t re = rb + 32 < r1 ? rb + 32 : r1;
        // 32 rows, fully unrolled so the loads of X are independent of each other
#pragma unroll
        for (int rr = 0; rr < 32; ++rr) {
            const int64_t row = rb + rr;
            if (row < re) {
                const T x = col < d ? X[row * d + col] : T(0);
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int64_t o = oc + 4 * u;
                    if (o < c) acc[u] = fma(x, Y[row * c + o], acc[u]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) tot[u] += (double)acc[u];
    }
    double* P = part + ((int64_t)j * XTY_SPLITS + rs) * dp * c;
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const int64_t o = oc + 4 * u;
        if (o < c) P[col * c + o] = tot[u];
    }
}

template <typename T>
__global__ void k_bsum(const double* __restrict__ part, int k, int64_t len, T* __restrict__ Bv,
                       T* __restrict__ Btr)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len;
         e += (int64_t)gridDim.x * blockDim.x) {
        double bv[MAX_K];
        double all = 0.0;
        for (int j = 0; j < k; ++j) {
            double s = 0.0;
            for (int rs = 0; rs < XTY_SPLITS; ++rs) s += part[((int64_t)j * XTY_SPLITS + rs) * len + e];
            bv[j] = s;
            Bv[(int64_t)j * len + e] = (T)s;
        }
        for (int f = 0; f < k; ++f) {
            all = 0.0;
            for (int j = 0; j < k; ++j)
                if (j != f) all += bv[j];
            Btr[(int64_t)f * len + e] = (T)all;
        }
    }
}

// yy_j = ||Y_j||_F^2 in double, fixed reduction order.
template <typename T>
__global__ void __launch_bounds__(256)
k_yy(const T* __restrict__ Y, int64_t c, FoldOffs fo, double* __restrict__ yy, int64_t* __restrict__ nfc)
{
    const int j = blockIdx.x;
    if (threadIdx.x == 0) nfc[j] = (fo.o[j + 1] - fo.o[j]) * c;
    const int64_t a = fo.o[j] * c, b = fo.o[j + 1] * c;
    double s = 0.0;
    for (int64_t e = a + threadIdx.x; e < b; e += 256) {
        double v = (double)Y[e];
        s += v * v;
    }
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) yy[j] = red[0];
}

// B_f = sum_{j != f} Bv_j (summed in double in increasing j) when Bv is already formed.
template <typename T>
__global__ void k_btrain_from_bv(const T* __restrict__ Bv, int k, int64_t len, T* __restrict__ Btr)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len;
         e += (int64_t)gridDim.x * blockDim.x) {
        for (int f = 0; f < k; ++f) {
            double all = 0.0;
            for (int j = 0; j < k; ++j)
                if (j != f) all += (double)Bv[(int64_t)j * len + e];
            Btr[(int64_t)f * len + e] = (T)all;
        }
    }
}

// ---------------------------------------------------------------------------
// Set-up in double precision (one CTA):
//   tau = tr(sum_j G_j) / d (if scale_by_trace, else 1)
//   lambda_t = tau lo (hi/lo)^(t/(q-1))                 (Sec. 6.3 grid)
//   idx_s = round(s (q-1)/(g-1)), lambda_s = lambda_{idx_s}
//   V[s][m] = phi_m(lambda_s); V = Q R by modified Gram-Schmidt with one
//   re-orthogonalisation pass; P = R^{-1} Q^T = V^+ (Algorithm 1's observation matrix and least squares)
//   phi[t][m] = phi_m(lambda_t), dphi[t][m] = d phi_m / d lambda at lambda_t
//   warm start (gw > 0): lam_w[i] = lambda at round(i (q-1)/(gw-1)),
//   vw[i][m] = phi_m(lam_w[i]), pinv_w = (first min(gw, p) columns of vw)^+
// ---------------------------------------------------------------------------
__device__ inline void basis_eval(int basis, int p, double lam, double a, double b, double smax,
                                  double* phi, double* dphi)
{
    if (basis == PICHOL_BASIS_MONO) {
        // phi_m = x^m, d phi_m / d lambda = m x^(m-1) / smax, x = lambda / smax
        double x = lam / smax, xm = 1.0;
        dphi[0] = 0.0;
        for (int m = 0; m < p; ++m) {
            phi[m] = xm;
            if (m + 1 < p) dphi[m + 1] = (m + 1) * xm / smax;
            xm *= x;
        }
    } else {
        double u = (b > a) ? 2.0 * (log(lam) - a) / (b - a) - 1.0 : 0.0;
        double du = (b > a) ? 2.0 / ((b - a) * lam) : 0.0;
        double t0 = 1.0, t1 = u, d0 = 0.0, d1 = 1.0;
        phi[0] = 1.0; dphi[0] = 0.0;
        if (p > 1) { phi[1] = u; dphi[1] = du; }
        for (int m = 2; m < p; ++m) {
            double t2 = 2.0 * u * t1 - t0;
            double d2 = 2.0 * t1 + 2.0 * u * d1 - d0;
            phi[m] = t2; dphi[m] = d2 * du;
            t0 = t1; t1 = t2; d0 = d1; d1 = d2;
        }
    }
}

// Pseudo-inverse P = V^+ (cols x rows, row-major P[m * rows + i]) of the first
// `cols` columns of V (rows x cols, full column rank) by modified Gram-Schmidt
// with one re-orthogonalisation pass, V = Q R, then P = R^{-1} Q^T by back
// substitution.  False if a column is dependent on the previous ones.
__device__ inline bool pinv_mgs(const double (*V)[MAX_P], int rows, int cols, double* P)
{
    double Q[MAX_G][MAX_P], R[MAX_P][MAX_P];
    for (int m = 0; m < cols; ++m)
        for (int l = 0; l < cols; ++l) R[m][l] = 0.0;
    bool ok = true;
    for (int m = 0; m < cols; ++m) {
        double v[MAX_G];
        for (int i = 0; i < rows; ++i) v[i] = V[i][m];
        for (int pass = 0; pass < 2; ++pass)
            for (int l = 0; l < m; ++l) {
                double dot = 0.0;
                for (int i = 0; i < rows; ++i) dot += Q[i][l] * v[i];
                R[l][m] += dot;
                for (int i = 0; i < rows; ++i) v[i] -= dot * Q[i][l];
            }
        double nrm = 0.0;
        for (int i = 0; i < rows; ++i) nrm += v[i] * v[i];
        nrm = sqrt(nrm);
        if (!(nrm > 0.0)) { ok = false; nrm = 1.0; }
        R[m][m] = nrm;
        for (int i = 0; i < rows; ++i) Q[i][m] = v[i] / nrm;
    }
    for (int i = 0; i < rows; ++i)
        for (int m = cols - 1; m >= 0; --m) {
            double v = Q[i][m];
            for (int l = m + 1; l < cols; ++l) v -= R[m][l] * P[l * rows + i];
            P[m * rows + i] = v / R[m][m];
        }
    return ok;
}

// Basis normalisation, V and P = V^+ from the sampled lambdas lam_s (one
// thread): scal[1..3] = (ln min lam_s, ln max lam_s, max lam_s); with a warm
// start (gw > 0) also the warm-start lambdas (grid indices of lam_grid), V'
// and V'^+.  A rank-deficient V latches PICHOL_ERR_INVALID_ARG.
__device__ void samples_basis(int basis, int g, int p, int q, const double* lam_s, const double* lam_grid,
                              double* scal, double* pinv, int gw, double* lam_w, double* pinv_w, double* vw,
                              DevStatus* st)
{
    double smin = lam_s[0], smax = lam_s[0];
    for (int i = 1; i < g; ++i) { smin = fmin(smin, lam_s[i]); smax = fmax(smax, lam_s[i]); }
    const double a = log(smin), b = log(smax);
    double V[MAX_G][MAX_P], dummy[MAX_P];
    for (int i = 0; i < g; ++i) basis_eval(basis, p, lam_s[i], a, b, smax, V[i], dummy);
    if (!pinv_mgs(V, g, p, pinv)) latch_error(st, PICHOL_ERR_INVALID_ARG, -1, -1, -1);
    if (gw > 0) {
        // warm start: gw samples at round(i (q-1)/(gw-1)), the same basis
        // (normalised by the g samples), the first pw functions fitted
        const int pw = gw < p ? gw : p;
        double Vw[MAX_G][MAX_P];
        for (int i = 0; i < gw; ++i) {
            const int idx = (2 * i * (q - 1) + (gw - 1)) / (2 * (gw - 1));
            lam_w[i] = lam_grid[idx];
            basis_eval(basis, p, lam_w[i], a, b, smax, Vw[i], dummy);
            for (int m = 0; m < p; ++m) vw[i * p + m] = Vw[i][m];
        }
        if (!pinv_mgs(Vw, gw, pw, pinv_w)) latch_error(st, PICHOL_ERR_INVALID_ARG, -1, -1, -1);
    }
    scal[1] = a;
    scal[2] = b;
    scal[3] = smax;
}

__global__ void __launch_bounds__(256)
k_setup(const void* G, int mode_fp64, int64_t d, int64_t dp, int k, int g, int p, int q,
        double lo, double hi, const double* __restrict__ window, int scale_by_trace, int basis,
        double* scal, double* lam_grid, double* lam, double* lam_s, double* pinv, double* phi, double* dphi,
        int gw, double* lam_w, double* pinv_w, double* vw, DevStatus* st)
{
    if (window) {
        lo = window[0];
        hi = window[1];
    }
    __shared__ double red[256];
    double s = 0.0;
    for (int64_t e = threadIdx.x; e < (int64_t)k * d; e += 256) {
        const int j = (int)(e / d);
        const int64_t i = e % d;
        const int64_t off = (int64_t)j * dp * dp + i * dp + i;
        s += mode_fp64 ? ((const double*)G)[off] : (double)((const float*)G)[off];
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double tau = scale_by_trace ? red[0] / (double)d : 1.0;
    for (int t = threadIdx.x; t < q; t += 256) {
        const double v = (q == 1) ? tau * lo : tau * lo * pow(hi / lo, (double)t / (double)(q - 1));
        lam_grid[t] = v;
        lam[t] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!(tau > 0.0) || isinf(tau) || !(lo > 0.0) || !(hi >= lo) || isinf(hi))
            latch_error(st, PICHOL_ERR_INVALID_ARG, -1, -1, -1);
        scal[0] = tau;
        for (int i = 0; i < g; ++i) {
            const int idx = (g == 1) ? 0 : (2 * i * (q - 1) + (g - 1)) / (2 * (g - 1));
            lam_s[i] = lam_grid[idx];
        }
        samples_basis(basis, g, p, q, lam_s, lam_grid, scal, pinv, gw, lam_w, pinv_w, vw, st);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < q; t += 256)
        basis_eval(basis, p, lam[t], scal[1], scal[2], scal[3], phi + t * p, dphi + t * p);
}

// The sampled lambdas of pichol_factor_samples: the caller's values (given)
// or the default grid samples, then samples_basis and the basis values of
// the current evaluation lambdas under the new normalisation.
__global__ void __launch_bounds__(256)
k_set_samples(LamValues vals, int given, int basis, int g, int p, int q, double* scal,
              const double* __restrict__ lam_grid, const double* __restrict__ lam, double* lam_s, double* pinv,
              double* phi, double* dphi, int gw, double* lam_w, double* pinv_w, double* vw, DevStatus* st)
{
    if (threadIdx.x == 0) {
        for (int i = 0; i < g; ++i) {
            const int idx = (g == 1) ? 0 : (2 * i * (q - 1) + (g - 1)) / (2 * (g - 1));
            lam_s[i] = given ? vals.v[i] : lam_grid[idx];
        }
        samples_basis(basis, g, p, q, lam_s, lam_grid, scal, pinv, gw, lam_w, pinv_w, vw, st);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < q; t += 256)
        basis_eval(basis, p, lam[t], scal[1], scal[2], scal[3], phi + t * p, dphi + t * p);
}

// Evaluation lambdas [t0, t0 + count): the caller's values (given) or the
// grid, and their basis values under the samples' normalisation.
__global__ void __launch_bounds__(256)
k_set_evals(LamValues vals, int given, int t0, int count, int basis, int p, const double* __restrict__ scal,
            const double* __restrict__ lam_grid, double* lam, double* phi, double* dphi)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int t = t0 + i;
    const double v = given ? vals.v[i] : lam_grid[t];
    lam[t] = v;
    basis_eval(basis, p, v, scal[1], scal[2], scal[3], phi + (int64_t)t * p, dphi + (int64_t)t * p);
}

cudaError_t launch_set_samples(pichol_ctx* ctx, const double* lam_s_host, cudaStream_t s)
{
    const pichol_config& c = ctx->cfg;
    LamValues v;
    memset(&v, 0, sizeof(v));
    if (lam_s_host)
        for (int i = 0; i < c.g; ++i) v.v[i] = lam_s_host[i];
    {
        StageScope sc_(ctx, ST_SETUP, s);
        k_set_samples<<<1, 256, 0, s>>>(v, lam_s_host != nullptr, c.basis, c.g, ctx->p, c.q, ctx->scal,
                                        ctx->lam_grid, ctx->lam, ctx->lam_s, ctx->pinv, ctx->phi, ctx->dphi,
                                        c.warm_samples, ctx->lam_w, ctx->pinv_w, ctx->vw, ctx->status);
    }
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t launch_set_evals(pichol_ctx* ctx, const double* lam_t_host, cudaStream_t s)
{
    const pichol_config& c = ctx->cfg;
    for (int t0 = 0; t0 < c.q; t0 += LAM_CHUNK) {
        const int cnt = (c.q - t0) < LAM_CHUNK ? (c.q - t0) : LAM_CHUNK;
        LamValues v;
        memset(&v, 0, sizeof(v));
        if (lam_t_host)
            for (int i = 0; i < cnt; ++i) v.v[i] = lam_t_host[t0 + i];
        {
            StageScope sc_(ctx, ST_SETUP, s);
            k_set_evals<<<(cnt + 255) / 256, 256, 0, s>>>(v, lam_t_host != nullptr, t0, cnt, c.basis, ctx->p,
                                                         ctx->scal, ctx->lam_grid, ctx->lam, ctx->phi, ctx->dphi);
        }
        ctx->launches++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// H_f = sum_{j != f} G_j on the lower tiles, tile-major, summed in increasing j
// (the padding stays zero; the factorisation input adds the shift and the
// identity on the padding).  FP64 mode sums in double.  In fp32 the sum is
// compensated on the FP32 pipes (TwoSum per term, the rounding errors added at
// the end), which keeps it within an ulp of the correctly rounded sum; a double
// accumulation would occupy GB300's FP64 unit (one warp instruction per 64
// cycles) for most of the kernel.
template <typename T>
__global__ void __launch_bounds__(256)
k_hf_tiles(const T* __restrict__ G, int k, int64_t dp, int64_t ntiles, T* __restrict__ Hf)
{
    int I, J;
    tile_coords(blockIdx.x, I, J);
    const int f = blockIdx.y;
    T* dst = Hf + ((int64_t)f * ntiles + blockIdx.x) * TILE_ELEMS;
    if constexpr (std::is_same<T, float>::value) {
        // thread: four 16-byte groups (rows r, r + 16, r + 32, r + 48; columns 4 cc .. 4 cc + 3)
        const int cc = threadIdx.x & 15, r0 = threadIdx.x >> 4;
        float s[16], comp[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) { s[u] = 0.0f; comp[u] = 0.0f; }
        bool first = true;
        for (int j0 = 0; j0 < k; j0 += 2) {
            float4 x[2][4];                       // two blocks' loads in flight
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = j0 + h;
                if (j < k && j != f) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int64_t row = (int64_t)I * TB + r0 + 16 * u, col = (int64_t)J * TB + 4 * cc;
                        x[h][u] = *reinterpret_cast<const float4*>(G + (int64_t)j * dp * dp + row * dp + col);
                    }
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = j0 + h;
                if (j < k && j != f) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float* xv = reinterpret_cast<const float*>(&x[h][u]);
#pragma unroll
                        for (int w = 0; w < 4; ++w) {
                            const int q = 4 * u + w;
                            if (first) {
                                s[q] = xv[w];
                            } else {          // TwoSum: s + x = t + err exactly
                                const float t = s[q] + xv[w];
                                const float bp = t - s[q];
                                comp[q] += (s[q] - (t - bp)) + (xv[w] - bp);
                                s[q] = t;
                            }
                        }
                    }
                    first = false;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float4 o;
            o.x = s[4 * u] + comp[4 * u];
            o.y = s[4 * u + 1] + comp[4 * u + 1];
            o.z = s[4 * u + 2] + comp[4 * u + 2];
            o.w = s[4 * u + 3] + comp[4 * u + 3];
            *reinterpret_cast<float4*>(dst + (r0 + 16 * u) * TB + 4 * cc) = o;
        }
        return;
    }
    for (int e = threadIdx.x; e < TILE_ELEMS; e += 256) {
        const int r = e / TB, c = e % TB;
        const int64_t row = (int64_t)I * TB + r, col = (int64_t)J * TB + c;
        double v = 0.0;
        for (int j = 0; j < k; ++j)
            if (j != f) v += (double)G[(int64_t)j * dp * dp + row * dp + col];
        dst[e] = (T)v;
    }
}

template <typename T>
static cudaError_t gram_impl(pichol_ctx* ctx, const T* X, const T* Y, cudaStream_t s)
{
    const pichol_config& c = ctx->cfg;
    FoldOffs fo;
    for (int j = 0; j <= c.k; ++j) fo.o[j] = ctx->offs[j];
    T* G = (T*)ctx->G;
    cudaError_t e = cudaMemsetAsync(G, 0, sizeof(T) * (size_t)c.k * ctx->dp * ctx->dp, s);
    if (e != cudaSuccess) return e;
    if constexpr (std::is_same<T, float>::value) {
        // mixed mode: G_j and Bv_j = X_j^T Y_j on tensor cores (split TF32 when gram_passes = 3)
        ctx->Yin = Y;
        e = launch_gram_tc(ctx, X, s);
        if (e == cudaSuccess && ctx->Gah) e = launch_gall_split(ctx, s);
        if (e != cudaSuccess) return e;
    } else {
        {
            StageScope sc_(ctx, ST_GRAM, s);
            k_gram_simt<T><<<dim3((unsigned)ctx->ntiles, c.k), 256, 0, s>>>(X, c.d, ctx->dp, fo, G);
        }
        StageScope sc_(ctx, ST_XTY, s);
        k_xty<T><<<dim3(ctx->nt, c.k, XTY_SPLITS), 256, 0, s>>>(X, Y, c.d, ctx->dp, c.c, fo, ctx->xpart);
    }
    {
        StageScope sc_(ctx, ST_MISC, s);
        k_yy<T><<<c.k, 256, 0, s>>>(Y, c.c, fo, ctx->yy, ctx->nfc);
    }
    if ((e = launch_setup(ctx, nullptr, s)) != cudaSuccess) return e;
    const int64_t len = ctx->dp * c.c;
    if constexpr (std::is_same<T, float>::value) {
        StageScope sc_(ctx, ST_XTY, s);
        k_btrain_from_bv<T><<<(unsigned)((len + 255) / 256), 256, 0, s>>>((const T*)ctx->Bv, c.k, len, (T*)ctx->Btr);
    } else {
        StageScope sc_(ctx, ST_XTY, s);
        k_bsum<T><<<(unsigned)((len + 255) / 256), 256, 0, s>>>(ctx->xpart, c.k, len, (T*)ctx->Bv, (T*)ctx->Btr);
    }
    {
        StageScope sc_(ctx, ST_MISC, s);
        k_hf_tiles<T><<<dim3((unsigned)ctx->ntiles, c.k), 256, 0, s>>>(G, c.k, ctx->dp, ctx->ntiles, (T*)ctx->Hf);
    }
    ctx->launches += 6;
    return cudaGetLastError();
}

cudaError_t launch_setup(pichol_ctx* ctx, const double* window, cudaStream_t s)
{
    const pichol_config& c = ctx->cfg;
    {
        StageScope sc_(ctx, ST_SETUP, s);
        k_setup<<<1, 256, 0, s>>>(ctx->G, c.mode == PICHOL_MODE_FP64, c.d, ctx->dp, c.k, c.g, ctx->p, c.q,
                                  c.lam_lo, c.lam_hi, window, c.scale_by_trace, c.basis, ctx->scal, ctx->lam_grid,
                                  ctx->lam, ctx->lam_s, ctx->pinv, ctx->phi, ctx->dphi, c.warm_samples, ctx->lam_w,
                                  ctx->pinv_w, ctx->vw, ctx->status);
    }
    ctx->launches++;
    return cudaGetLastError();
}

size_t xty_part_bytes(int k, int64_t dp, int64_t c) { return sizeof(double) * (size_t)k * XTY_SPLITS * dp * c; }

// ---------------------------------------------------------------------------
// Fold right-hand sides without allocating (pichol_fold_rhs_noalloc).
//
// Some callers cannot allocate device memory at all: a plug-in inside a
// framework that owns every byte of the GPU through its own pool, a real-time
// path that cannot pay for cudaMalloc's implicit device-wide synchronisation,
// or code that is handed only its input and output buffers.  For them the
// partial sums of X_j^T Y_j live in a fixed array in the library's own device
// memory instead of a workspace: NOALLOC_PART_DOUBLES doubles (8 MiB) per GPU,
// held by every GPU that loads the library until the process exits.
// ---------------------------------------------------------------------------
constexpr size_t NOALLOC_PART_DOUBLES = (size_t)1 << 20;
static __device__ __align__(256) double g_noalloc_part[NOALLOC_PART_DOUBLES];

static std::mutex g_noalloc_mu;
// Device address of g_noalloc_part per device, and the driver context it was
// looked up in: the address belongs to that context's copy of the module, so
// after a device reset (or under another context on the same device) it is
// looked up again.
static double* g_noalloc_ptr[256];
static CUcontext g_noalloc_ctx[256];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
static CtxGetCurrentFn ctx_get_current_fn()
{
    static CtxGetCurrentFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (CtxGetCurrentFn)p;
    }
    return fn;
}

// Bv_j (k x d x c) and B_f (k x d x c), unpadded, from the partial sums.
template <typename T>
__global__ void k_bsum_unpadded(const double* __restrict__ part, int k, int64_t dp, int64_t d, int64_t c,
                                T* __restrict__ Bv, T* __restrict__ B)
{
    const int64_t len = d * c, plen = dp * c;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len;
         e += (int64_t)gridDim.x * blockDim.x) {
        double bv[MAX_K];
        for (int j = 0; j < k; ++j) {
            double s = 0.0;
            for (int rs = 0; rs < XTY_SPLITS; ++rs) s += part[((int64_t)j * XTY_SPLITS + rs) * plen + e];
            bv[j] = s;
            Bv[(int64_t)j * len + e] = (T)s;
        }
        for (int f = 0; f < k; ++f) {
            double all = 0.0;
            for (int j = 0; j < k; ++j)
                if (j != f) all += bv[j];
            B[(int64_t)f * len + e] = (T)all;
        }
    }
}

template <typename T>
static cudaError_t fold_rhs_noalloc(const T* X, const T* Y, int64_t n, int64_t d, int64_t c, int k, T* Bv,
                                    T* B, double* part, cudaStream_t s)
{
    FoldOffs fo;
    for (int j = 0; j <= k; ++j) fo.o[j] = (int64_t)j * n / k;
    const int nt = (int)((d + TB - 1) / TB);
    const int64_t dp = (int64_t)nt * TB;
    k_xty<T><<<dim3(nt, k, XTY_SPLITS), 256, 0, s>>>(X, Y, d, dp, c, fo, part);
    const int64_t len = d * c;
    const unsigned blocks = (unsigned)((len + 255) / 256 < 4096 ? (len + 255) / 256 : 4096);
    k_bsum_unpadded<T><<<blocks, 256, 0, s>>>(part, k, dp, d, c, Bv, B);
    return cudaGetLastError();
}

cudaError_t launch_gram(pichol_ctx* ctx, const void* X, const void* Y, cudaStream_t s)
{
    if (ctx->cfg.mode == PICHOL_MODE_FP64)
        return gram_impl<double>(ctx, (const double*)X, (const double*)Y, s);
    return gram_impl<float>(ctx, (const float*)X, (const float*)Y, s);
}

}  // namespace pichol

extern "C" PICHOL_API pichol_status pichol_fold_rhs_noalloc(int32_t mode, const void* X, const void* Y, int64_t n,
                                                           int64_t d, int64_t c, int32_t k, void* Bv_out,
                                                           void* B_out, void* stream)
{
    using namespace pichol;
    if (mode != PICHOL_MODE_FP64 && mode != PICHOL_MODE_MIXED) return PICHOL_ERR_INVALID_ARG;
    if (!X || !Y || !Bv_out || !B_out) return PICHOL_ERR_INVALID_ARG;
    if (k < 2 || k > MAX_K || n < k || d < 1 || c < 1 || c > 64) return PICHOL_ERR_INVALID_ARG;
    const int64_t dp = (d + TB - 1) / TB * TB;
    // the partial sums need k * 16 * dp * c doubles of the fixed array
    if ((double)k * XTY_SPLITS * (double)dp * (double)c > (double)NOALLOC_PART_DOUBLES) return PICHOL_ERR_WORKSPACE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return PICHOL_ERR_CUDA;
    double* part = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        CUcontext cur = nullptr;
        CtxGetCurrentFn cfn = ctx_get_current_fn();
        if (!cfn || cfn(&cur) != CUDA_SUCCESS) cur = nullptr;
        if (!g_noalloc_ptr[dev] || g_noalloc_ctx[dev] != cur) {
            void* addr = nullptr;
            if (cudaGetSymbolAddress(&addr, g_noalloc_part) != cudaSuccess || !addr) return PICHOL_ERR_CUDA;
            g_noalloc_ptr[dev] = (double*)addr;
            g_noalloc_ctx[dev] = cur;
        }
        part = g_noalloc_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = (mode == PICHOL_MODE_FP64)
        ? fold_rhs_noalloc<double>((const double*)X, (const double*)Y, n, d, c, k, (double*)Bv_out,
                                   (double*)B_out, part, s)
        : fold_rhs_noalloc<float>((const float*)X, (const float*)Y, n, d, c, k, (float*)Bv_out, (float*)B_out,
                                  part, s);
    return e == cudaSuccess ? PICHOL_OK : PICHOL_ERR_CUDA;
}
