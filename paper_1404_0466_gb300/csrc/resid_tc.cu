// Refinement residual on the tensor cores (mixed mode, interpolated target):
//   r_{f,t} = B_f - L~(lambda_t) (L~(lambda_t)^T W_{f,t}),
//   L~(lambda) = sum_m phi_m(lambda) Theta_{f,m}          (Algorithm 1's polynomials, Sec. 3.3)
// for every fold f and lambda t of a call at once.  Theta does not depend on
// lambda, so each triangular product is a sum over the coefficient planes of
// one contraction shared by all q lambdas (N = q c columns):
//   pass 0:  U = L~^T W:  U_i = sum_m phi_m(t) sum_{j >= i} Theta_{m,ji}^T W_j
//   pass 1:  R = B - L~ U: R_i = B_i - sum_m phi_m(t) sum_{j <= i} Theta_{m,ij} U_j
// Each CTA keeps one fp32 tensor-memory accumulator per plane m, so the
// basis values phi_m(lambda_t), which scale whole columns, are applied when
// the accumulators are drained: v = sum_m phi_m(t(col)) acc_m.  Operands are
// split TF32 (x = hi + lo; hi*hi + hi*lo + lo*hi) and every 32 rows of K the
// accumulators are drained into compensated (Kahan) fp32 totals: a residual
// is a small difference of large terms, and the tensor memory's fp32 sums of
// long K would carry an error of many roundings of those terms.
//
// Layouts: Theta split into hi/lo and, for pass 0, transposed tile by tile
// (k_theta_split): [f][tile][m][64 x 64] plus one zero plane at the end,
// read through a 2D TMA map [rows][64] with 64 x 32 boxes.  W^T and U^T are
// [f][q c][dp] hi/lo (K-major).  One CTA: 128 rows (tile rows 2 mt, 2 mt + 1)
// x BN columns; warp 0 issues TMA, warp 1 the MMAs, warps 2..9 drain.  Every
// mbarrier wait is bounded; a wait that runs out latches PICHOL_ERR_TIMEOUT,
// the CTA stops issuing work, waits (bounded) for its copies, frees its
// tensor memory and returns.
#include "internal.cuh"
#include "tcgen05.cuh"
#include "tma.cuh"

#include <cstring>

namespace pichol {

namespace rtc {

constexpr int BM = 128, BK = 32;
constexpr int NA = 4;                          // A ring stages (one coefficient plane, hi + lo)
constexpr int NB = 3;                          // B ring stages (one k-block of W^T / U^T, hi + lo)
constexpr int A_BYTES = 2 * BM * BK * 4;       // 32 KB
constexpr int CHUNK = 1;                       // k-blocks (32 rows of K) per drain
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 32 * (2 + EPI_WARPS);
constexpr int TMEM_COLS = 512;

template <int BN> struct Cfg {
    static constexpr int B_BYTES = 2 * BN * BK * 4;
    static constexpr int PHI_BYTES = MAX_P * BN * 4;
    static constexpr int SMEM = NA * A_BYTES + NB * B_BYTES + 1024 /* alignment */ + 256 /* barriers */ + PHI_BYTES;
};

}  // namespace rtc

// Theta_{f,m} tile (I, J) split into TF32 hi and remainder lo, as stored and
// transposed within the tile: th/tl[.][e] and tth/ttl[.][(b, a)] for element
// (a, b).  One CTA per (tile, fold), all p planes.
__global__ void __launch_bounds__(256)
k_theta_split(const float* __restrict__ theta, int p, int64_t ntiles, float* __restrict__ th,
              float* __restrict__ tl, float* __restrict__ tth, float* __restrict__ ttl)
{
    __shared__ float hs[TB][TB + 1], ls[TB][TB + 1];
    const int64_t base = ((int64_t)blockIdx.y * ntiles + blockIdx.x) * p * TILE_ELEMS;
    for (int m = 0; m < p; ++m) {
        const int64_t o = base + (int64_t)m * TILE_ELEMS;
        for (int e = threadIdx.x; e < TILE_ELEMS; e += 256) {
            const float v = theta[o + e];
            const float h = tc5::tf32_round(v);
            th[o + e] = h;
            tl[o + e] = v - h;
            hs[e / TB][e % TB] = h;
            ls[e / TB][e % TB] = v - h;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < TILE_ELEMS; e += 256) {
            const int a = e / TB, b = e % TB;     // output (a, b) = input (b, a)
            tth[o + e] = hs[b][a];
            ttl[o + e] = ls[b][a];
        }
        __syncthreads();
    }
}

struct ResidTcArgs {
    const double* phi;        // [t][p]
    const float* B;           // pass 1: [f][dp][c]
    float* R;                 // pass 1 output [f][t][dp][c]
    float* Uh;                // pass 0 output [f][q c][dp], hi
    float* Ul;                //                             lo
    int p, nt, q, t0, tcount;
    int64_t ntiles, dp, c, qc;
    int zero_row;             // first row of the zero plane in the Theta maps
    DevStatus* st;
};

// Row of the Theta map holding the 64 x 64 block that multiplies K tile column
// j for tile row i, plane m, in pass PASS; the zero plane where the triangle
// has no block (or i is past the last tile row).
template <int PASS>
__device__ __forceinline__ int a_row(const ResidTcArgs& a, int f, int i, int j, int m)
{
    int64_t tile;
    if (i >= a.nt) return a.zero_row;
    if (PASS == 1) {                    // Theta_{ij}, j <= i
        if (j > i) return a.zero_row;
        tile = tile_index(i, j);
    } else {                            // Theta_{ji}^T, j >= i
        if (j < i || j >= a.nt) return a.zero_row;
        tile = tile_index(j, i);
    }
    return (int)((((int64_t)f * a.ntiles + tile) * a.p + m) * TB);
}

template <int PASS, int BN>
__global__ void __launch_bounds__(320, 1)
k_resid_tc(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
           const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl, const ResidTcArgs a)
{
    using namespace rtc;
    using C = Cfg<BN>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* aring = smem;
    unsigned char* bring = smem + NA * A_BYTES;
    uint64_t* afull = (uint64_t*)(bring + NB * C::B_BYTES);
    uint64_t* aempty = afull + NA;
    uint64_t* bfull = aempty + NA;
    uint64_t* bempty = bfull + NB;
    uint64_t* tfull = bempty + NB;         // [2] accumulator set ready to drain
    uint64_t* tempty = tfull + 2;          // [2] accumulator set drained
    uint64_t* mdone = tempty + 2;          // every MMA of the issuer complete (its exit)
    uint32_t* tmem_slot = (uint32_t*)(mdone + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    volatile int* aconsumed = abort_flag + 1;
    volatile int* bconsumed = aconsumed + 1;
    float* phis = (float*)(smem + NA * A_BYTES + NB * C::B_BYTES + 256);   // [m][BN]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int f = blockIdx.y;
    const int64_t N = (int64_t)a.tcount * a.c;
    const int nN = (int)((N + BN - 1) / BN);
    const int nM = (a.nt + 1) / 2;
    const int nb = (int)blockIdx.x % nN;
    const int mi = (int)blockIdx.x / nN;
    // the CTAs with the longest K ranges first
    const int mt = PASS == 1 ? nM - 1 - mi : mi;
    const int i0 = 2 * mt, i1 = 2 * mt + 1;
    const int jlo = PASS == 1 ? 0 : i0;
    const int jhi = PASS == 1 ? (i1 < a.nt ? i1 : a.nt - 1) : a.nt - 1;
    const int nkb = 2 * (jhi - jlo + 1);
    const int nchunks = (nkb + CHUNK - 1) / CHUNK;
    const int p = a.p;
    const int brow = (int)((int64_t)f * a.qc + (int64_t)a.t0 * a.c + (int64_t)nb * BN);

    if (threadIdx.x == 0) {
        for (int s = 0; s < NA; ++s) { mbar_init(&afull[s], 1); mbar_init(&aempty[s], 1); }
        for (int s = 0; s < NB; ++s) { mbar_init(&bfull[s], 1); mbar_init(&bempty[s], 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], EPI_WARPS); }
        mbar_init(mdone, 1);
        *abort_flag = 0;
        *aconsumed = 0;
        *bconsumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    // basis values of the CTA's columns, phi_m(lambda_{t0 + (nb BN + col) / c})
    for (int e = threadIdx.x; e < p * BN; e += blockDim.x) {
        const int m = e / BN, col = e % BN;
        const int64_t n = (int64_t)nb * BN + col;
        phis[e] = n < N ? (float)a.phi[(int64_t)(a.t0 + n / a.c) * p + m] : 0.0f;
    }
    if (warp == 0) tc5::alloc(tmem_slot, TMEM_COLS);
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- producer: B (one k-block) then its p coefficient planes ----
            int aiss = 0, biss = 0;
            for (int kb = 0; kb < nkb && !*abort_flag; ++kb) {
                const int j = jlo + kb / 2, x = j * TB + (kb & 1) * BK;
                const int sb = kb % NB;
                if (!mbar_wait(&bempty[sb], ((kb / NB) & 1) ^ 1)) { *abort_flag = 1; break; }
                unsigned char* bs = bring + sb * C::B_BYTES;
                mbar_expect_tx(&bfull[sb], C::B_BYTES);
                tma_load_2d(bs, &mBh, &bfull[sb], x, brow);
                tma_load_2d(bs + C::B_BYTES / 2, &mBl, &bfull[sb], x, brow);
                ++biss;
                const int xa = (kb & 1) * BK;
                for (int m = 0; m < p; ++m) {
                    const int q = kb * p + m, sa = q % NA;
                    if (!mbar_wait(&aempty[sa], ((q / NA) & 1) ^ 1)) { *abort_flag = 1; break; }
                    unsigned char* as = aring + sa * A_BYTES;
                    mbar_expect_tx(&afull[sa], A_BYTES);
                    const int y0 = a_row<PASS>(a, f, i0, j, m), y1 = a_row<PASS>(a, f, i1, j, m);
                    tma_load_2d(as, &mAh, &afull[sa], xa, y0);
                    tma_load_2d(as + BM / 2 * 128, &mAh, &afull[sa], xa, y1);
                    tma_load_2d(as + BM * 128, &mAl, &afull[sa], xa, y0);
                    tma_load_2d(as + BM * 128 + BM / 2 * 128, &mAl, &afull[sa], xa, y1);
                    ++aiss;
                }
            }
            // wait (bounded) for copies that were issued but never consumed
            for (int q = *aconsumed; q < aiss; ++q) mbar_wait(&afull[q % NA], (q / NA) & 1);
            for (int kb = *bconsumed; kb < biss; ++kb) mbar_wait(&bfull[kb % NB], (kb / NB) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer: chunk ch accumulates plane m into set ch & 1, columns m BN ----
            constexpr uint32_t idesc = tc5::idesc_tf32(BM, BN);
            int kb = 0;
            for (int ch = 0; ch < nchunks && !*abort_flag; ++ch) {
                const int b = ch & 1, use = ch >> 1;
                if (!mbar_wait(&tempty[b], (use & 1) ^ 1)) { *abort_flag = 1; break; }
                tc5::fence_after();
                const int kend = (kb + CHUNK < nkb) ? kb + CHUNK : nkb;
                for (int kfirst = kb; kb < kend; ++kb) {
                    const int sb = kb % NB;
                    if (*abort_flag || !mbar_wait(&bfull[sb], (kb / NB) & 1)) { *abort_flag = 1; break; }
                    tc5::fence_after();
                    const uint32_t bh = smem_u32(bring + sb * C::B_BYTES), bl = bh + C::B_BYTES / 2;
                    for (int m = 0; m < p; ++m) {
                        const int q = kb * p + m, sa = q % NA;
                        if (*abort_flag || !mbar_wait(&afull[sa], (q / NA) & 1)) { *abort_flag = 1; break; }
                        tc5::fence_after();
                        const uint32_t ah = smem_u32(aring + sa * A_BYTES), al = ah + BM * 128;
                        const uint32_t acc = tmem + (uint32_t)((b * p + m) * BN);
                        tc5::mma_split3_k32(acc, ah, al, bh, bl, idesc, kb == kfirst);
                        tc5::commit(&aempty[sa]);
                        *aconsumed = q + 1;
                    }
                    tc5::commit(&bempty[sb]);
                    *bconsumed = kb + 1;
                }
                tc5::commit(&tfull[b]);   // set b holds the chunk's sums once its MMAs complete
            }
            // every MMA issued has completed before the tensor memory is freed
            tc5::commit(mdone);
            mbar_wait(mdone, 0);
        }
    } else {
        // ---- drain: v = sum_m phi_m(col) acc_m, compensated totals ----
        // warp w reads tensor-memory lanes 32 (w % 4) .. +31 (its tile rows);
        // the first four drain warps take columns [0, BN/2), the others [BN/2, BN)
        constexpr int HC = BN / 2;
        float tot[HC], cmp[HC];
        const int qtr = warp & 3, chalf = (warp - 2) >> 2;
#pragma unroll
        for (int u = 0; u < HC; ++u) { tot[u] = 0.0f; cmp[u] = 0.0f; }
        for (int ch = 0; ch < nchunks; ++ch) {
            const int b = ch & 1, use = ch >> 1;
            if (!mbar_wait(&tfull[b], use & 1)) { *abort_flag = 1; break; }
            tc5::fence_after();
#pragma unroll
            for (int cc = 0; cc < HC / 16; ++cc) {
                float v[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) v[u] = 0.0f;
                // the planes' loads in groups of G, one wait per group (G x 16 registers)
                constexpr int G = BN == 64 ? 2 : 4;
                for (int m0 = 0; m0 < p; m0 += G) {
                    uint32_t x[G][16];
#pragma unroll
                    for (int h = 0; h < G; ++h)
                        if (m0 + h < p)
                            tc5::ld16_issue(tmem + ((uint32_t)(qtr * 32) << 16) +
                                                (uint32_t)((b * p + m0 + h) * BN + chalf * HC + cc * 16),
                                            x[h]);
                    tc5::wait_ld();
#pragma unroll
                    for (int h = 0; h < G; ++h)
                        if (m0 + h < p) {
                            tc5::regs_ready(x[h]);
                            const float* ph = phis + (m0 + h) * BN + chalf * HC + cc * 16;
#pragma unroll
                            for (int u = 0; u < 16; ++u) v[u] = fmaf(ph[u], __uint_as_float(x[h][u]), v[u]);
                        }
                }
#pragma unroll
                for (int u = 0; u < 16; ++u) {   // Kahan: tot += v
                    const float y = v[u] - cmp[cc * 16 + u];
                    const float t = tot[cc * 16 + u] + y;
                    cmp[cc * 16 + u] = (t - tot[cc * 16 + u]) - y;
                    tot[cc * 16 + u] = t;
                }
            }
            tc5::fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(&tempty[b])) : "memory");
        }
        if (!*abort_flag) {
            const int64_t row = (int64_t)mt * BM + qtr * 32 + lane;    // row of dp
            const int64_t n0 = (int64_t)nb * BN + chalf * HC;
            if (row < a.dp) {
                if (PASS == 0) {
                    // U^T split for pass 1's B operand: [f][t0 c + n][row]
#pragma unroll
                    for (int u = 0; u < HC; ++u) {
                        const int64_t n = n0 + u;
                        if (n < N) {
                            const int64_t o = ((int64_t)f * a.qc + (int64_t)a.t0 * a.c + n) * a.dp + row;
                            const float h = tc5::tf32_round(tot[u]);
                            a.Uh[o] = h;
                            a.Ul[o] = tot[u] - h;
                        }
                    }
                } else {
                    // R[f][t][row][o] = B_f[row][o] - (L~ U)
#pragma unroll
                    for (int u = 0; u < HC; ++u) {
                        const int64_t n = n0 + u;
                        if (n < N) {
                            const int64_t t = a.t0 + n / a.c, oc = n % a.c;
                            const float bv = a.B[((int64_t)f * a.dp + row) * a.c + oc];
                            a.R[(((int64_t)f * a.q + t) * a.dp + row) * a.c + oc] = bv - tot[u];
                        }
                    }
                }
            }
        }
    }
    __syncwarp();
    tc5::fence_before();
    __syncthreads();
    if (*abort_flag && threadIdx.x == 0) latch_error(a.st, PICHOL_ERR_TIMEOUT, f, (int)blockIdx.x, -1);
    if (warp == 0) tc5::dealloc(tmem, TMEM_COLS);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
cudaError_t launch_theta_split(pichol_ctx* ctx, cudaStream_t s)
{
    const pichol_config& c = ctx->cfg;
    const size_t plane = (size_t)TILE_ELEMS * sizeof(float);
    const int64_t planes = (int64_t)c.k * ctx->ntiles * ctx->p;
    for (float* a : {ctx->Th, ctx->Tl, ctx->TTh, ctx->TTl}) {
        cudaError_t e = cudaMemsetAsync(a + planes * TILE_ELEMS, 0, plane, s);   // the zero plane
        if (e != cudaSuccess) return e;
    }
    {
        StageScope sc_(ctx, ST_FIT, s);
        k_theta_split<<<dim3((unsigned)ctx->ntiles, c.k), 256, 0, s>>>((const float*)ctx->Theta, ctx->p, ctx->ntiles,
                                                                       ctx->Th, ctx->Tl, ctx->TTh, ctx->TTl);
    }
    ctx->launches++;
    return cudaGetLastError();
}

template <int PASS, int BN>
static cudaError_t resid_pass(pichol_ctx* ctx, const CUtensorMap& ah, const CUtensorMap& al, const CUtensorMap& bh,
                              const CUtensorMap& bl, const ResidTcArgs& ra, cudaStream_t s)
{
    static std::atomic<unsigned long long> set{0};
    cudaError_t e = smem_limit_once(k_resid_tc<PASS, BN>, rtc::Cfg<BN>::SMEM, set);
    if (e != cudaSuccess) return e;
    const int64_t N = (int64_t)ra.tcount * ra.c;
    const unsigned nN = (unsigned)((N + BN - 1) / BN), nM = (unsigned)((ra.nt + 1) / 2);
    {
        StageScope sc_(ctx, ST_RESID, s);
        k_resid_tc<PASS, BN><<<dim3(nM * nN, ctx->cfg.k), rtc::THREADS, rtc::Cfg<BN>::SMEM, s>>>(ah, al, bh, bl, ra);
    }
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t launch_resid_tc(pichol_ctx* ctx, int t0, int tcount, cudaStream_t s)
{
    const pichol_config& c = ctx->cfg;
    const int64_t dp = ctx->dp, qc = (int64_t)c.q * c.c;
    const int p = ctx->p;
    if (p * 32 > 256) return cudaErrorInvalidValue;          // two accumulator sets of p x 32 columns
    cudaError_t e = launch_split_wt(ctx, t0, tcount, ST_RESID, s);
    if (e != cudaSuccess) return e;
    float* Uh = (float*)ctx->U;
    float* Ul = Uh + (int64_t)c.k * qc * dp;
    const int BN = p <= 4 ? 64 : 32;
    const uint64_t trows = (uint64_t)(c.k * ctx->ntiles * p + 1) * TB;
    CUtensorMap th, tl, tth, ttl, wh, wl, uh, ul;
    if (!make_map_f32(&th, ctx->Th, TB, trows, TB, rtc::BK, TB) || !make_map_f32(&tl, ctx->Tl, TB, trows, TB, rtc::BK, TB) ||
        !make_map_f32(&tth, ctx->TTh, TB, trows, TB, rtc::BK, TB) ||
        !make_map_f32(&ttl, ctx->TTl, TB, trows, TB, rtc::BK, TB) ||
        !make_map_f32(&wh, ctx->Wth, (uint64_t)dp, (uint64_t)(c.k * qc), (uint64_t)dp, rtc::BK, BN) ||
        !make_map_f32(&wl, ctx->Wtl, (uint64_t)dp, (uint64_t)(c.k * qc), (uint64_t)dp, rtc::BK, BN) ||
        !make_map_f32(&uh, Uh, (uint64_t)dp, (uint64_t)(c.k * qc), (uint64_t)dp, rtc::BK, BN) ||
        !make_map_f32(&ul, Ul, (uint64_t)dp, (uint64_t)(c.k * qc), (uint64_t)dp, rtc::BK, BN))
        return cudaErrorInvalidValue;
    ResidTcArgs ra;
    memset(&ra, 0, sizeof(ra));
    ra.phi = ctx->phi;
    ra.B = (const float*)ctx->Btr;
    ra.R = (float*)ctx->Rres;
    ra.Uh = Uh;
    ra.Ul = Ul;
    ra.p = p;
    ra.nt = ctx->nt;
    ra.q = c.q;
    ra.t0 = t0;
    ra.tcount = tcount;
    ra.ntiles = ctx->ntiles;
    ra.dp = dp;
    ra.c = c.c;
    ra.qc = qc;
    ra.zero_row = (int)((int64_t)c.k * ctx->ntiles * p * TB);
    ra.st = ctx->status;
    if (BN == 64) {
        if ((e = resid_pass<0, 64>(ctx, tth, ttl, wh, wl, ra, s)) != cudaSuccess) return e;
        return resid_pass<1, 64>(ctx, th, tl, uh, ul, ra, s);
    }
    if ((e = resid_pass<0, 32>(ctx, tth, ttl, wh, wl, ra, s)) != cudaSuccess) return e;
    return resid_pass<1, 32>(ctx, th, tl, uh, ul, ra, s);
}

}  // namespace pichol
