// Blocked right-looking Cholesky factorisation of many shifted Hessians at once
// (Sec. 3.2; Algorithm 1, step 1).  For each factorisation problem pr (a fold
// f and a shift lambda), A = H_f + lambda I with H_f = sum_{j != f} G_j is
// written tile-major, then for every tile column J:
//   k_chol_diag   : L_JJ = chol(A_JJ), in double precision
//   k_chol_panel  : L_IJ = A_IJ L_JJ^{-T} by substitution, row by row (I > J)
//   k_chol_update : A_IK -= L_IJ L_KJ^T               (J < K <= I)
// All problems advance one tile column per launch.  A non-positive pivot
// latches PICHOL_ERR_NOT_SPD with (fold, sample, row) and the factorisation
// continues with a unit pivot so no NaN spreads.
#include "internal.cuh"

namespace pichol {

struct ProbMap {
    int per;        // problem slots per fold
    int count;      // live slots per fold (slots >= count are skipped)
    int exact;      // 0: shifts are the sampled lambdas; 1: grid lambdas t0 + i
    int t0;
};

__device__ inline bool prob_dead(const ProbMap& pm, int pr) { return pr % pm.per >= pm.count; }

__device__ inline double prob_lambda(const ProbMap& pm, int pr, const double* lam, const double* lam_s) {
    int i = pr % pm.per;
    return pm.exact ? lam[pm.t0 + i] : lam_s[i];
}

// A = H_f + lambda I on the lower tiles (H_f tile-major from the Gram step);
// identity on the padding.
template <typename T>
__global__ void __launch_bounds__(256)
k_chol_init(const T* __restrict__ Hf, int64_t d, int64_t ntiles, ProbMap pm,
            const double* __restrict__ lam, const double* __restrict__ lam_s, T* __restrict__ F)
{
    int I, J;
    tile_coords(blockIdx.x, I, J);
    const int pr = blockIdx.y;
    if (prob_dead(pm, pr)) return;
    const int f = pr / pm.per;
    const double shift = prob_lambda(pm, pr, lam, lam_s);
    const T* src = Hf + ((int64_t)f * ntiles + blockIdx.x) * TILE_ELEMS;
    T* dst = F + ((int64_t)pr * ntiles + blockIdx.x) * TILE_ELEMS;
    for (int e = threadIdx.x; e < TILE_ELEMS; e += 256) {
        const int r = e / TB, c = e % TB;
        const int64_t row = (int64_t)I * TB + r, col = (int64_t)J * TB + c;
        T v;
        if (I == J && c > r) v = T(0);
        else if (row >= d || col >= d) v = (row == col) ? T(1) : T(0);
        else v = (row == col) ? (T)((double)src[e] + shift) : src[e];
        dst[e] = v;
    }
}

// One CTA per problem: factor the 64 x 64 diagonal tile in double precision,
// right-looking inside the tile (pivot, scale the column by 1/L_jj, rank-1
// update of the trailing triangle).
template <typename T>
__global__ void __launch_bounds__(256)
k_chol_diag(T* __restrict__ F, int64_t ntiles, int J, int64_t d, ProbMap pm, DevStatus* st)
{
    __shared__ double A[TB][TB + 1];
    __shared__ double piv_inv;
    const int pr = blockIdx.x, tid = threadIdx.x;
    if (prob_dead(pm, pr)) return;
    T* tile = F + ((int64_t)pr * ntiles + tile_index(J, J)) * TILE_ELEMS;
    for (int e = tid; e < TILE_ELEMS; e += 256) {
        const int r = e / TB, c = e % TB;
        A[r][c] = (c <= r) ? (double)tile[e] : 0.0;
    }
    for (int j = 0; j < TB; ++j) {
        __syncthreads();
        if (tid == 0) {
            double piv = A[j][j];
            if (!(piv > 0.0)) {
                if ((int64_t)J * TB + j < d)
                    latch_error(st, PICHOL_ERR_NOT_SPD, pr / pm.per,
                                pm.exact ? pm.t0 + pr % pm.per : pr % pm.per, (long long)J * TB + j);
                piv = 1.0;
            }
            const double ljj = sqrt(piv);
            A[j][j] = ljj;
            piv_inv = 1.0 / ljj;
        }
        __syncthreads();
        const double inv = piv_inv;
        for (int i = j + 1 + tid; i < TB; i += 256) A[i][j] *= inv;
        __syncthreads();
        // rank-1 update of the trailing triangle: thread (row i = tid & 63,
        // phase ph = tid >> 6) updates columns c = j+1+ph, j+5+ph, ... <= i
        const int i = tid & 63, ph = tid >> 6;
        if (i > j) {
            const double aij = A[i][j];
            for (int c = j + 1 + ph; c <= i; c += 4) A[i][c] -= aij * A[c][j];
        }
    }
    __syncthreads();
    for (int e = tid; e < TILE_ELEMS; e += 256) {
        const int r = e / TB, c = e % TB;
        tile[e] = (c <= r) ? (T)A[r][c] : T(0);
    }
}

// Load a 64 x 64 row-major tile transposed into shared memory: S[k][r] = src[r][k].
template <typename T, typename S>
__device__ inline void load_tile_transposed(const S* __restrict__ src, T (*dst)[TB + 1])
{
    for (int e = threadIdx.x; e < TILE_ELEMS; e += blockDim.x) {
        int r = e / TB, k = e % TB;
        dst[k][r] = (T)src[e];
    }
}

// acc[a][b] += sum_k As[k][ty + 16a] * Bs[k][tx + 16b]   (C = A B^T for row-major A, B)
template <typename T>
__device__ inline void mm_nt(T (*As)[TB + 1], T (*Bs)[TB + 1], T acc[4][4])
{
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll 4
    for (int k = 0; k < TB; ++k) {
        T av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = As[k][ty + 16 * a];
#pragma unroll
        for (int b = 0; b < 4; ++b) bv[b] = Bs[k][tx + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
}

// L_IJ = A_IJ L_JJ^{-T}: every row x of L_IJ solves L_JJ x^T = a^T by forward
// substitution, x_c = (a_c - sum_{k<c} L_JJ[c][k] x_k) / L_JJ[c][c].  One
// thread per row, 256 / 64 = 4 tiles per CTA, the row in registers.
template <typename T>
__global__ void __launch_bounds__(256)
k_chol_panel(T* __restrict__ F, int64_t ntiles, int J, int m, ProbMap pm)
{
    if (prob_dead(pm, blockIdx.y)) return;
    __shared__ T Ls[TB][TB + 1];
    __shared__ T inv[TB];
    const int pr = blockIdx.y, tid = threadIdx.x;
    T* base = F + (int64_t)pr * ntiles * TILE_ELEMS;
    const T* ljj = base + tile_index(J, J) * TILE_ELEMS;
    for (int e = tid; e < TILE_ELEMS; e += 256) Ls[e / TB][e % TB] = ljj[e];
    __syncthreads();
    if (tid < TB) inv[tid] = T(1) / Ls[tid][tid];
    __syncthreads();
    const int it = blockIdx.x * 4 + (tid >> 6);
    if (it >= m) return;
    const int r = tid & 63;
    T* row = base + tile_index(J + 1 + it, J) * TILE_ELEMS + r * TB;
    T x[TB];
#pragma unroll
    for (int c = 0; c < TB; ++c) x[c] = row[c];
#pragma unroll
    for (int c = 0; c < TB; ++c) {
        T sacc = x[c];
#pragma unroll
        for (int k2 = 0; k2 < c; ++k2) sacc = fma(-Ls[c][k2], x[k2], sacc);
        x[c] = sacc * inv[c];
    }
#pragma unroll
    for (int c = 0; c < TB; ++c) row[c] = x[c];
}

// A_IK -= L_IJ L_KJ^T for the trailing lower tiles J < K <= I.
template <typename T>
__global__ void __launch_bounds__(256)
k_chol_update(T* __restrict__ F, int64_t ntiles, int J, ProbMap pm)
{
    if (prob_dead(pm, blockIdx.y)) return;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T (*As)[TB + 1] = reinterpret_cast<T (*)[TB + 1]>(sm_raw);
    T (*Bs)[TB + 1] = reinterpret_cast<T (*)[TB + 1]>(sm_raw + sizeof(T) * TB * (TB + 1));
    int ii, kk;
    tile_coords(blockIdx.x, ii, kk);
    const int I = J + 1 + ii, K = J + 1 + kk, pr = blockIdx.y;
    T* base = F + (int64_t)pr * ntiles * TILE_ELEMS;
    load_tile_transposed<T, T>(base + tile_index(I, J) * TILE_ELEMS, As);
    load_tile_transposed<T, T>(base + tile_index(K, J) * TILE_ELEMS, Bs);
    __syncthreads();
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    mm_nt<T>(As, Bs, acc);
    T* out = base + tile_index(I, K) * TILE_ELEMS;
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            int e = (ty + 16 * a) * TB + tx + 16 * b;
            out[e] = out[e] - acc[a][b];
        }
}

template <typename T>
static cudaError_t factor_impl(pichol_ctx* ctx, int count, int exact, int t0, cudaStream_t s)
{
    const pichol_config& c = ctx->cfg;
    ProbMap pm;
    pm.exact = exact;
    pm.t0 = t0;
    pm.per = exact ? (int)ctx->exact_batch : c.g;
    pm.count = count;
    const int nprob = c.k * pm.per;
    T* F = (T*)ctx->F;
    const size_t sm_mm = 2 * sizeof(T) * TB * (TB + 1);
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(k_chol_update<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_mm);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    {
        StageScope sc_(ctx, ST_CHOL_INIT, s);
        k_chol_init<T><<<dim3((unsigned)ctx->ntiles, nprob), 256, 0, s>>>(
            (const T*)ctx->Hf, c.d, ctx->ntiles, pm, ctx->lam, ctx->lam_s, F);
    }
    ctx->launches++;
    for (int J = 0; J < ctx->nt; ++J) {
        {
            StageScope sc_(ctx, ST_CHOL_DIAG, s);
            k_chol_diag<T><<<nprob, 256, 0, s>>>(F, ctx->ntiles, J, c.d, pm, ctx->status);
        }
        ctx->launches++;
        const int m = ctx->nt - 1 - J;
        if (m > 0) {
            {
                StageScope sc_(ctx, ST_CHOL_PANEL, s);
                k_chol_panel<T><<<dim3((m + 3) / 4, nprob), 256, 0, s>>>(F, ctx->ntiles, J, m, pm);
            }
            {
                StageScope sc_(ctx, ST_CHOL_UPDATE, s);
                k_chol_update<T><<<dim3(m * (m + 1) / 2, nprob), 256, sm_mm, s>>>(F, ctx->ntiles, J, pm);
            }
            ctx->launches += 2;
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_factor(pichol_ctx* ctx, int count, int exact, int t0, cudaStream_t s)
{
    if (ctx->cfg.mode == PICHOL_MODE_FP64) return factor_impl<double>(ctx, count, exact, t0, s);
    return factor_impl<float>(ctx, count, exact, t0, s);
}

// ---------------------------------------------------------------------------
// Inspection: tile-major planes -> dense row-major double (lower triangle).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_export_tiles(const T* __restrict__ src, int64_t tile_stride, int64_t d, double* __restrict__ out)
{
    int I, J;
    tile_coords(blockIdx.x, I, J);
    const T* t = src + (int64_t)blockIdx.x * tile_stride;
    for (int e = threadIdx.x; e < TILE_ELEMS; e += 256) {
        int r = e / TB, c = e % TB;
        int64_t row = (int64_t)I * TB + r, col = (int64_t)J * TB + c;
        if (row < d && col < d && col <= row) out[row * d + col] = (double)t[e];
    }
}

cudaError_t launch_export_tiles(pichol_ctx* ctx, const void* tiles, int64_t plane_offset_elems,
                                int64_t tile_stride_elems, double* out, cudaStream_t s)
{
    const int64_t d = ctx->cfg.d;
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * (size_t)(d * d), s);
    if (e != cudaSuccess) return e;
    if (ctx->cfg.mode == PICHOL_MODE_FP64)
        k_export_tiles<double><<<(unsigned)ctx->ntiles, 256, 0, s>>>(
            (const double*)tiles + plane_offset_elems, tile_stride_elems, d, out);
    else
        k_export_tiles<float><<<(unsigned)ctx->ntiles, 256, 0, s>>>(
            (const float*)tiles + plane_offset_elems, tile_stride_elems, d, out);
    ctx->launches++;
    return cudaGetLastError();
}

// H_f = sum_{j != f} G_j (dense) and B_f, as doubles.
template <typename T>
__global__ void k_export_hessian(const T* __restrict__ G, const T* __restrict__ Btr, int k, int f,
                                 int64_t d, int64_t dp, int64_t c, double* __restrict__ H,
                                 double* __restrict__ B)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < d * d;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t row = e / d, col = e % d;
        double v = 0.0;
        for (int j = 0; j < k; ++j)
            if (j != f) v += (double)G[(int64_t)j * dp * dp + row * dp + col];
        H[e] = v;
    }
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < d * c;
         e += (int64_t)gridDim.x * blockDim.x)
        B[e] = (double)Btr[(int64_t)f * dp * c + e];
}

cudaError_t launch_export_hessian(pichol_ctx* ctx, int f, double* H, double* B, cudaStream_t s)
{
    const pichol_config& c = ctx->cfg;
    if (c.mode == PICHOL_MODE_FP64)
        k_export_hessian<double><<<256, 256, 0, s>>>((const double*)ctx->G, (const double*)ctx->Btr, c.k, f,
                                                     c.d, ctx->dp, c.c, H, B);
    else
        k_export_hessian<float><<<256, 256, 0, s>>>((const float*)ctx->G, (const float*)ctx->Btr, c.k, f,
                                                    c.d, ctx->dp, c.c, H, B);
    ctx->launches++;
    return cudaGetLastError();
}

}  // namespace pichol
