// Blocked right-looking Cholesky factorisation of many shifted Hessians at once
// (Sec. 3.2; the exact factors of Algorithm 1).  For each factorisation problem pr (a fold
// f and a shift lambda), A = H_f + lambda I with H_f = sum_{j != f} G_j is
// written tile-major, then for every tile column J:
//   k_chol_diag   : L_JJ = chol(A_JJ), in double precision
//   k_chol_panel  : L_IJ = A_IJ L_JJ^{-T} by substitution, row by row (I > J)
//   k_chol_update : A_IK -= L_IJ L_KJ^T               (J < K <= I)
// All problems advance one tile column per launch.  A non-positive pivot
// latches PICHOL_ERR_NOT_SPD with (fold, sample, row) and the factorisation
// continues with a unit pivot so no NaN spreads.
#include "internal.cuh"
#include "tcgen05.cuh"

#include <cstring>
#include <type_traits>

namespace pichol {

struct ProbMap {
    int per;        // problem slots per fold
    int count;      // live slots per fold (slots >= count are skipped)
    int exact;      // 0: shifts are the sampled lambdas; 1: grid lambdas t0 + i
    int t0;
    int warm;       // > 0: folds f > 0 have this many live slots, shifted by the warm-start lambdas
};

__device__ inline bool prob_dead(const ProbMap& pm, int pr)
{
    const int live = (pm.warm > 0 && pr >= pm.per) ? pm.warm : pm.count;
    return pr % pm.per >= live;
}

__device__ inline double prob_lambda(const ProbMap& pm, int pr, const double* lam, const double* lam_s,
                                     const double* lam_w)
{
    const int i = pr % pm.per;
    if (pm.exact) return lam[pm.t0 + i];
    return (pm.warm > 0 && pr >= pm.per) ? lam_w[i] : lam_s[i];
}

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int N = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int N = 2; };

// A = H_f + lambda I on the lower tiles (H_f tile-major from the Gram step);
// identity on the padding.
template <typename T>
__global__ void __launch_bounds__(256)
k_chol_init(const T* __restrict__ Hf, int64_t d, int64_t ntiles, ProbMap pm,
            const double* __restrict__ lam, const double* __restrict__ lam_s, const double* __restrict__ lam_w,
            T* __restrict__ F)
{
    int I, J;
    tile_coords(blockIdx.x, I, J);
    const int pr = blockIdx.y;
    if (prob_dead(pm, pr)) return;
    const int f = pr / pm.per;
    const double shift = prob_lambda(pm, pr, lam, lam_s, lam_w);
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::N, NV = TILE_ELEMS / VN / 256;   // 16-byte vectors per thread
    const V* src = reinterpret_cast<const V*>(Hf + ((int64_t)f * ntiles + blockIdx.x) * TILE_ELEMS);
    V* dst = reinterpret_cast<V*>(F + ((int64_t)pr * ntiles + blockIdx.x) * TILE_ELEMS);
    V in[NV];
#pragma unroll
    for (int u = 0; u < NV; ++u) in[u] = src[threadIdx.x + 256 * u];   // all loads in flight
#pragma unroll
    for (int u = 0; u < NV; ++u) {
        const int e0 = VN * (threadIdx.x + 256 * u), r = e0 / TB;
        T* x = reinterpret_cast<T*>(&in[u]);
#pragma unroll
        for (int j = 0; j < VN; ++j) {
            const int c = e0 % TB + j;
            const int64_t row = (int64_t)I * TB + r, col = (int64_t)J * TB + c;
            if (I == J && c > r) x[j] = T(0);
            else if (row >= d || col >= d) x[j] = (row == col) ? T(1) : T(0);
            else if (row == col) x[j] = (T)((double)x[j] + shift);
        }
        dst[threadIdx.x + 256 * u] = in[u];
    }
}

// 1/sqrt(p) in double precision with few FP64 instructions.  GB300 issues one
// FP64 warp instruction per 64 cycles on each SM sub-partition, so the pivot
// chain of the diagonal tiles is counted in FP64 instructions:
//  * seed: the float with p's exponent and top 20 mantissa bits (integer
//    arithmetic on the high word), rsqrtf of it (relative error below 2^-20
//    in all), widened back to double exactly by integer arithmetic;
//  * one third-order step from the binomial series of (1 - r)^(-1/2):
//    y1 = y + y r (1/2 + 3r/8), r = 1 - p y^2, which cubes the seed's error
//    (5/16 e^3 < 2^-62) and leaves the rounding of five FP64 operations.
// Outside [2^-99, 2^100) (and for NaN or p <= 0) the library quotient is used.
__device__ __forceinline__ bool rsqrt_seed_range(int hi) { return hi >= (924 << 20) && hi < (1123 << 20); }

__device__ __forceinline__ double rsqrt_cubic(double p)
{
    const int hi = __double2hiint(p);
    if (!rsqrt_seed_range(hi)) return 1.0 / sqrt(p);
    const float pf = __int_as_float((hi - 0x38000000) << 3);       // exponent 1023 -> 127
    const int fb = __float_as_int(rsqrtf(pf));
    const double y = __hiloint2double((fb >> 3) + 0x38000000, fb << 29);
    const double r = fma(-p * y, y, 1.0);
    return fma(y * r, fma(r, 0.375, 0.5), y);
}

// Largest relative difference between rsqrt_cubic and the library's 1 / sqrt
// over n values p = 2^u, u uniform in [-110, 110) from a splitmix64 stream
// (covers the seeded range and both fallbacks); one value per thread and
// grid-stride step, the maximum reduced with an atomic on the bit pattern
// (non-negative doubles order like their bits).
__global__ void k_check_rsqrt(int64_t n, uint64_t seed, unsigned long long* out)
{
    double mx = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const double u = (double)(z >> 11) * 0x1.0p-53;
        const double p = exp2(-110.0 + 220.0 * u);
        const double ref = 1.0 / sqrt(p);
        mx = fmax(mx, fabs(rsqrt_cubic(p) - ref) / ref);
    }
    atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

cudaError_t launch_check_rsqrt(int64_t n, uint64_t seed, double* max_rel, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(max_rel, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
    k_check_rsqrt<<<152, 256, 0, s>>>(n, seed, (unsigned long long*)max_rel);
    return cudaGetLastError();
}

// One CTA of DNT threads per problem: the 64 x 64 diagonal tile in double
// precision, right-looking with a look-ahead of one column.  In phase t:
//  * warp 0 finishes column t (pivot L_tt = sqrt(a_tt), column scaled by
//    1 / L_tt) and brings column t+1 up to date (the updates by columns t-1
//    and t), so pivot t+1 is ready at the next phase;
//  * the bulk warps apply column t-1 to the trailing columns >= t+2.
// One barrier per phase; every element receives its updates in column order,
// as in the plain right-looking loop.  Warp 0's sub-partition takes no bulk
// work (warps 4, 8, ... stay idle), so its FP64 unit serves the pivot chain
// alone.  The lower triangle is listed column by column in `tab`, so each
// trailing set is a suffix of the list that the bulk threads share evenly.
template <typename T, int DNT, int ILP>
__global__ void __launch_bounds__(DNT)
k_chol_diag(T* __restrict__ F, int64_t ntiles, int J, int64_t d, ProbMap pm, DevStatus* st)
{
    constexpr int NTRI = TB * (TB + 1) / 2;
    constexpr int NW = DNT / 32;
    constexpr int NB = NW - (NW + 3) / 4;       // bulk warps: those off sub-partition 0
    __shared__ double A[TB][TB + 1];
    __shared__ unsigned short tab[NTRI];
    const int pr = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (prob_dead(pm, pr)) return;
    T* tile = F + ((int64_t)pr * ntiles + tile_index(J, J)) * TILE_ELEMS;
    for (int e = tid; e < TILE_ELEMS; e += DNT) {
        const int r = e / TB, c = e % TB;
        A[r][c] = (c <= r) ? (double)tile[e] : 0.0;
        // column c starts at c TB - c (c - 1) / 2 in the list
        if (c <= r) tab[c * TB - c * (c - 1) / 2 + (r - c)] = (unsigned short)((r << 8) | c);
    }
    const int brank = (warp % 4 != 0) ? warp - warp / 4 - 1 : -1;
    __syncthreads();
    for (int t = 0; t < TB; ++t) {
        if (warp == 0) {
            double piv = A[t][t];
            if (!(piv > 0.0)) {
                if (lane == 0 && (int64_t)J * TB + t < d)
                    latch_error(st, PICHOL_ERR_NOT_SPD, pr / pm.per, pm.exact ? pm.t0 + pr % pm.per : pr % pm.per,
                                (long long)J * TB + t);
                piv = 1.0;
            }
            const double y = rsqrt_cubic(piv);       // every lane: no broadcast needed
            __syncwarp();
            if (lane == 0) A[t][t] = piv * y;
            for (int i = t + 1 + lane; i < TB; i += 32) A[i][t] *= y;
            __syncwarp();
            if (t + 1 < TB) {
                const double a1 = (t > 0) ? A[t + 1][t - 1] : 0.0;
                const double a2 = A[t + 1][t];
                for (int i = t + 1 + lane; i < TB; i += 32) {
                    double v = A[i][t + 1];
                    if (t > 0) v = fma(-A[i][t - 1], a1, v);
                    v = fma(-A[i][t], a2, v);
                    A[i][t + 1] = v;
                }
            }
        } else if (brank >= 0 && t >= 1) {
            const int j = t - 1;
            const int e0 = (t + 2) * TB - (t + 2) * (t + 1) / 2;   // column t+2 onwards
            for (int eb = e0 + brank * 32 + lane; eb < NTRI; eb += NB * 32 * ILP) {
                double a[ILP], b[ILP], c[ILP];
                int ii[ILP], cc[ILP];
#pragma unroll
                for (int u = 0; u < ILP; ++u) {
                    const int e = eb + u * NB * 32;
                    ii[u] = -1;
                    cc[u] = 0;
                    if (e < NTRI) {
                        const int ic = tab[e];
                        ii[u] = ic >> 8;
                        cc[u] = ic & 255;
                        a[u] = A[ii[u]][j];
                        b[u] = A[cc[u]][j];
                        c[u] = A[ii[u]][cc[u]];
                    }
                }
#pragma unroll
                for (int u = 0; u < ILP; ++u)
                    if (ii[u] >= 0) A[ii[u]][cc[u]] = fma(-a[u], b[u], c[u]);
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < TILE_ELEMS; e += DNT) {
        const int r = e / TB, c = e % TB;
        tile[e] = (c <= r) ? (T)A[r][c] : T(0);
    }
}


// Copy a row-major 64 x 64 tile into shared memory rows of LD elements (16-byte moves).
template <typename T, int LD, int NT>
__device__ __forceinline__ void stage_tile(T* __restrict__ dst, const T* __restrict__ src)
{
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::N, CPR = TB / VN;
    for (int q = threadIdx.x; q < TB * CPR; q += NT) {
        const int r = q / CPR, ch = q % CPR;
        *reinterpret_cast<V*>(dst + r * LD + ch * VN) = *reinterpret_cast<const V*>(src + r * TB + ch * VN);
    }
}

// L_IJ = A_IJ L_JJ^{-T}: every row x of L_IJ solves L_JJ x^T = a^T by forward
// substitution, x_c = (a_c - sum_{k<c} L_JJ[c][k] x_k) / L_JJ[c][c].  One
// thread per row (the row in registers), 256 / 64 = 4 tiles per CTA; the rows
// of L_JJ are read from shared memory 16 bytes at a time (the same address for
// the whole warp), and each sum runs as VN interleaved partial sums (one per
// element of the 16-byte chunk), added in a fixed order.
// With ph (fp32 only), each solved row is also written split into TF32 hi
// (ph) and remainder (pl) at panel-buffer row prow0 + (pr nt + I) 64 + r, the
// operands of the tensor-core trailing update.
template <typename T>
__global__ void __launch_bounds__(256)
k_chol_panel(T* __restrict__ F, int64_t ntiles, int J, int m, ProbMap pm, float* __restrict__ ph,
             float* __restrict__ pl, int64_t prow0, int nt)
{
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::N, LD = TB + VN;
    if (prob_dead(pm, blockIdx.y)) return;
    __shared__ __align__(16) T Ls[TB * LD];
    __shared__ T inv[TB];
    const int pr = blockIdx.y, tid = threadIdx.x;
    T* base = F + (int64_t)pr * ntiles * TILE_ELEMS;
    stage_tile<T, LD, 256>(Ls, base + tile_index(J, J) * TILE_ELEMS);
    __syncthreads();
    if (tid < TB) inv[tid] = T(1) / Ls[tid * LD + tid];
    __syncthreads();
    const int it = blockIdx.x * 4 + (tid >> 6);
    if (it >= m) return;
    const int r = tid & 63;
    T* row = base + tile_index(J + 1 + it, J) * TILE_ELEMS + r * TB;
    T x[TB];
#pragma unroll
    for (int ch = 0; ch < TB / VN; ++ch) {
        V v = reinterpret_cast<const V*>(row)[ch];
        memcpy(&x[ch * VN], &v, sizeof(V));
    }
#pragma unroll
    for (int c = 0; c < TB; ++c) {
        T sp[VN];
#pragma unroll
        for (int e = 0; e < VN; ++e) sp[e] = T(0);
#pragma unroll
        for (int k0 = 0; k0 < c; k0 += VN) {
            V lv = *reinterpret_cast<const V*>(Ls + c * LD + k0);
            T l[VN];
            memcpy(l, &lv, sizeof(V));
#pragma unroll
            for (int e = 0; e < VN; ++e)
                if (k0 + e < c) sp[e] = fma(l[e], x[k0 + e], sp[e]);
        }
        T sum = sp[0];
#pragma unroll
        for (int e = 1; e < VN; ++e) sum += sp[e];
        x[c] = (x[c] - sum) * inv[c];
    }
#pragma unroll
    for (int ch = 0; ch < TB / VN; ++ch) {
        V v;
        memcpy(&v, &x[ch * VN], sizeof(V));
        reinterpret_cast<V*>(row)[ch] = v;
    }
    if constexpr (std::is_same<T, float>::value) {
        if (ph) {
            const int64_t o = (prow0 + ((int64_t)pr * nt + J + 1 + it) * TB + r) * TB;
#pragma unroll
            for (int ch = 0; ch < TB / 4; ++ch) {
                float4 h, l;
                h.x = tc5::tf32_round(x[4 * ch]);
                h.y = tc5::tf32_round(x[4 * ch + 1]);
                h.z = tc5::tf32_round(x[4 * ch + 2]);
                h.w = tc5::tf32_round(x[4 * ch + 3]);
                l.x = x[4 * ch] - h.x;
                l.y = x[4 * ch + 1] - h.y;
                l.z = x[4 * ch + 2] - h.z;
                l.w = x[4 * ch + 3] - h.w;
                reinterpret_cast<float4*>(ph + o)[ch] = h;
                reinterpret_cast<float4*>(pl + o)[ch] = l;
            }
        }
    }
}

// Copy a row-major 64 x 64 tile into shared memory rows of LD elements with
// 16-byte cp.async copies (committed by the caller).
template <typename T, int LD, int NT>
__device__ __forceinline__ void stage_tile_async(T* __restrict__ dst, const T* __restrict__ src)
{
    constexpr int VN = Vec16<T>::N, CPR = TB / VN;
    for (int q = threadIdx.x; q < TB * CPR; q += NT) {
        const int r = q / CPR, ch = q % CPR;
        cp_async16(dst + r * LD + ch * VN, src + r * TB + ch * VN);
    }
}

// A_IK -= L_IJ L_KJ^T for trailing lower tiles.  One CTA takes a strip of up
// to `chunk` output tiles of one tile column: K = first + blockIdx.y, rows
// I = K + blockIdx.x * chunk, ... (I < nt); blockIdx.z is the problem.  L_KJ
// is staged once, the L_IJ tiles are double-buffered (cp.async), and the
// output tile's current values are loaded into registers before its product,
// so the global latency of each step hides behind the previous step's
// arithmetic.  NT threads per CTA; thread (ty, tx) = (t / 8, t % 8) owns rows
// ty + (NT/8) a and columns tx + 8 b.  Operand rows are padded to LD elements
// so that the 16-byte row reads of a warp hit distinct banks.
template <typename T, int NT>
__global__ void __launch_bounds__(NT)
k_chol_update(T* __restrict__ F, int64_t ntiles, int nt, int J, int first, int chunk, ProbMap pm)
{
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::N, LD = TB + VN;
    constexpr int TY = NT / 8, RA = TB / TY, RC = 8;
    const int pr = blockIdx.z;
    if (prob_dead(pm, pr)) return;
    const int K = first + (int)blockIdx.y;
    const int I0 = K + (int)blockIdx.x * chunk;
    if (I0 >= nt) return;
    const int n = (I0 + chunk < nt ? I0 + chunk : nt) - I0;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T* Bs = reinterpret_cast<T*>(sm_raw);
    T* As = Bs + TB * LD;                          // two buffers
    T* base = F + (int64_t)pr * ntiles * TILE_ELEMS;
    stage_tile_async<T, LD, NT>(Bs, base + tile_index(K, J) * TILE_ELEMS);
    stage_tile_async<T, LD, NT>(As, base + tile_index(I0, J) * TILE_ELEMS);
    cp_async_commit();
    const int ty = threadIdx.x >> 3, tx = threadIdx.x & 7;
#pragma unroll 1
    for (int u = 0; u < n; ++u) {
        const int I = I0 + u;
        const T* Au = As + (u & 1) * TB * LD;
        if (u + 1 < n)
            stage_tile_async<T, LD, NT>(As + ((u + 1) & 1) * TB * LD, base + tile_index(I + 1, J) * TILE_ELEMS);
        cp_async_commit();
        T* out = base + tile_index(I, K) * TILE_ELEMS;
        T cv[RA][RC];
#pragma unroll
        for (int a = 0; a < RA; ++a)
#pragma unroll
            for (int b = 0; b < RC; ++b) cv[a][b] = out[(ty + TY * a) * TB + tx + 8 * b];
        cp_async_wait<1>();                        // L_KJ and L_IJ have landed
        __syncthreads();
        T acc[RA][RC];
        if constexpr (std::is_same<T, float>::value) {
            // fp32: packed FMAs over pairs of k (even and odd k in the two halves of a
            // register pair, added at the end): half the FMA issue slots
            unsigned long long acc2[RA][RC];
#pragma unroll
            for (int a = 0; a < RA; ++a)
#pragma unroll
                for (int b = 0; b < RC; ++b) acc2[a][b] = 0ull;
#pragma unroll 2
            for (int k0 = 0; k0 < TB; k0 += 4) {
                ulonglong2 av[RA], bv[RC];
#pragma unroll
                for (int a = 0; a < RA; ++a) av[a] = *reinterpret_cast<const ulonglong2*>(Au + (ty + TY * a) * LD + k0);
#pragma unroll
                for (int b = 0; b < RC; ++b) bv[b] = *reinterpret_cast<const ulonglong2*>(Bs + (tx + 8 * b) * LD + k0);
#pragma unroll
                for (int a = 0; a < RA; ++a)
#pragma unroll
                    for (int b = 0; b < RC; ++b) {
                        acc2[a][b] = f32x2_fma(av[a].x, bv[b].x, acc2[a][b]);
                        acc2[a][b] = f32x2_fma(av[a].y, bv[b].y, acc2[a][b]);
                    }
            }
#pragma unroll
            for (int a = 0; a < RA; ++a)
#pragma unroll
                for (int b = 0; b < RC; ++b) {
                    const float2 h = f32x2_unpack(acc2[a][b]);
                    acc[a][b] = h.x + h.y;
                }
        } else {
#pragma unroll
            for (int a = 0; a < RA; ++a)
#pragma unroll
                for (int b = 0; b < RC; ++b) acc[a][b] = T(0);
#pragma unroll 2
            for (int k0 = 0; k0 < TB; k0 += VN) {
                T av[RA][VN], bv[RC][VN];
#pragma unroll
                for (int a = 0; a < RA; ++a) {
                    V v = *reinterpret_cast<const V*>(Au + (ty + TY * a) * LD + k0);
                    memcpy(av[a], &v, sizeof(V));
                }
#pragma unroll
                for (int b = 0; b < RC; ++b) {
                    V v = *reinterpret_cast<const V*>(Bs + (tx + 8 * b) * LD + k0);
                    memcpy(bv[b], &v, sizeof(V));
                }
#pragma unroll
                for (int e = 0; e < VN; ++e)
#pragma unroll
                    for (int a = 0; a < RA; ++a)
#pragma unroll
                        for (int b = 0; b < RC; ++b) acc[a][b] = fma(av[a][e], bv[b][e], acc[a][b]);
            }
        }
#pragma unroll
        for (int a = 0; a < RA; ++a)
#pragma unroll
            for (int b = 0; b < RC; ++b) out[(ty + TY * a) * TB + tx + 8 * b] = cv[a][b] - acc[a][b];
        __syncthreads();                           // this buffer is refilled two steps on
    }
}

template <typename T> struct UpdateThreads { static constexpr int value = 128; };
template <> struct UpdateThreads<double> { static constexpr int value = 256; };

template <typename T>
static cudaError_t factor_impl(pichol_ctx* ctx, int count, int exact, int t0, cudaStream_t s)
{
    const pichol_config& c = ctx->cfg;
    ProbMap pm;
    pm.exact = exact;
    pm.t0 = t0;
    pm.per = exact ? (int)ctx->exact_batch : c.g;
    pm.count = count;
    pm.warm = exact ? 0 : c.warm_samples;
    const int nprob = c.k * pm.per;
    T* F = (T*)ctx->F;
    constexpr int UNT = UpdateThreads<T>::value;
    const int UCH = ctx->tune.update_strip;     // output tiles per CTA in the bulk updates
    // The diagonal tiles are the critical path.  When the k g problems fit on
    // half the SMs (and the tuning allows), each diagonal CTA asks for enough
    // shared memory that no trailing-update CTA can share its SM.
    constexpr int DIAG_RESERVE = 160 * 1024;
    const size_t sm_mm = 3 * sizeof(T) * TB * (TB + Vec16<T>::N);
    static std::atomic<unsigned long long> set_upd{0}, set_d512{0}, set_d256{0};
    {
        cudaError_t e = smem_limit_once(k_chol_update<T, UNT>, (int)sm_mm, set_upd);
        if (e == cudaSuccess) e = smem_limit_once(k_chol_diag<T, 512, 2>, DIAG_RESERVE, set_d512);
        if (e == cudaSuccess) e = smem_limit_once(k_chol_diag<T, 256, 1>, DIAG_RESERVE, set_d256);
        if (e != cudaSuccess) return e;
    }
    {
        StageScope sc_(ctx, ST_CHOL_INIT, s);
        k_chol_init<T><<<dim3((unsigned)ctx->ntiles, nprob), 256, 0, s>>>(
            (const T*)ctx->Hf, c.d, ctx->ntiles, pm, ctx->lam, ctx->lam_s, ctx->lam_w, F);
    }
    ctx->launches++;
    // Look-ahead: the critical path (diagonal tile J, panel J, then the tiles
    // of column J+1) runs on the context's high-priority stream sh, so its
    // CTAs are dispatched ahead of the bulk of the trailing update (tiles
    // K >= J+2), which runs on the caller's stream s meanwhile.  The column
    // update J+1 waits for the bulk update J (both write column J+2).  sh forks
    // from s after the factor input is written and joins back at the end, so
    // the call stays capturable.
    cudaStream_t sh = ctx->aux ? ctx->aux : s;
    const bool split = sh != s;
    const size_t diag_smem = (ctx->tune.diag_exclusive && 2 * nprob <= ctx->nsm) ? DIAG_RESERVE : 0;
    cudaError_t e;
    if (split) {
        if ((e = cudaEventRecord(ctx->ev_fork, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(sh, ctx->ev_fork, 0)) != cudaSuccess) return e;
    }
    bool pending = false;   // a bulk update on s that sh has not yet waited for
    // mixed mode: the bulk updates run on the tensor cores from the panel
    // tiles split by k_chol_panel into panel buffer J & 1
    const bool tcu = std::is_same<T, float>::value && ctx->Ph != nullptr && ctx->tune.update_engine == 0;
    // output tiles per tensor-core CTA (pairs of 128 rows): at most two pairs;
    // CTAs of four pairs measured hundreds of times slower (not understood;
    // those shapes are not used)
    const int UCH_TC = UCH >= 2 ? 4 : 2;
    for (int J = 0; J < ctx->nt; ++J) {
        const int64_t prow0 = (int64_t)(J & 1) * ctx->nfac * ctx->nt * TB;
        {
            StageScope sc_(ctx, ST_CHOL_DIAG, sh);
            if (ctx->tune.diag_threads == 256)
                k_chol_diag<T, 256, 1><<<nprob, 256, diag_smem, sh>>>(F, ctx->ntiles, J, c.d, pm, ctx->status);
            else
                k_chol_diag<T, 512, 2><<<nprob, 512, diag_smem, sh>>>(F, ctx->ntiles, J, c.d, pm, ctx->status);
        }
        ctx->launches++;
        const int m = ctx->nt - 1 - J;
        if (m == 0) break;
        {
            StageScope sc_(ctx, ST_CHOL_PANEL, sh);
            k_chol_panel<T><<<dim3((m + 3) / 4, nprob), 256, 0, sh>>>(F, ctx->ntiles, J, m, pm, tcu ? ctx->Ph : nullptr,
                                                                       ctx->Pl, prow0, ctx->nt);
        }
        ctx->launches++;
        if (split && m > 1) {
            if ((e = cudaEventRecord(ctx->ev_panel, sh)) != cudaSuccess) return e;
            if (pending && (e = cudaStreamWaitEvent(sh, ctx->ev_upd, 0)) != cudaSuccess) return e;
            {
                StageScope sc_(ctx, ST_CHOL_UPDATE, sh);
                k_chol_update<T, UNT><<<dim3(m, 1, nprob), UNT, sm_mm, sh>>>(F, ctx->ntiles, ctx->nt, J, J + 1, 1,
                                                                           pm);
            }
            if ((e = cudaStreamWaitEvent(s, ctx->ev_panel, 0)) != cudaSuccess) return e;
            {
                StageScope sc_(ctx, ST_CHOL_UPDATE, s);
                if (tcu)
                    e = launch_update_tc(ctx, pm.per, pm.count, pm.warm, nprob, J, J + 2, m - 1, UCH_TC, s);
                else
                    k_chol_update<T, UNT><<<dim3((m - 1 + UCH - 1) / UCH, m - 1, nprob), UNT, sm_mm, s>>>(
                        F, ctx->ntiles, ctx->nt, J, J + 2, UCH, pm);
            }
            if (e != cudaSuccess) return e;
            if ((e = cudaEventRecord(ctx->ev_upd, s)) != cudaSuccess) return e;
            pending = true;
            ctx->launches += 2;
        } else {
            if (pending && (e = cudaStreamWaitEvent(sh, ctx->ev_upd, 0)) != cudaSuccess) return e;
            pending = false;
            {
                StageScope sc_(ctx, ST_CHOL_UPDATE, sh);
                if (tcu)
                    e = launch_update_tc(ctx, pm.per, pm.count, pm.warm, nprob, J, J + 1, m, UCH_TC, sh);
                else
                    k_chol_update<T, UNT><<<dim3((m + UCH - 1) / UCH, m, nprob), UNT, sm_mm, sh>>>(
                        F, ctx->ntiles, ctx->nt, J, J + 1, UCH, pm);
            }
            if (e != cudaSuccess) return e;
            ctx->launches++;
        }
    }
    if (split) {
        // s already follows every bulk update it ran; it now waits for sh
        if ((e = cudaEventRecord(ctx->ev_join, sh)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s, ctx->ev_join, 0)) != cudaSuccess) return e;
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
