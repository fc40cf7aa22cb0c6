// Trailing update of the blocked Cholesky factorisation on the tensor cores
// (mixed mode; Sec. 3.2, the exact factors of Algorithm 1):
//   A_IK -= L_IJ L_KJ^T      for the tiles I >= K > J of every problem,
// after the panel J has been solved.  The panel kernel leaves each panel tile
// L_IJ split into TF32 hi and remainder lo in a scratch buffer (two buffers,
// by the parity of J, so that panel J+1 on the look-ahead stream never
// overwrites what the update of column J still reads).
//
// One CTA: problem pr, output tile column K, a strip of output tile rows
// I0 .. I0 + strip - 1 taken in pairs (M = 128 rows, N = 64 columns, K = 64).
// warp 0 loads L_KJ once and the L_IJ pairs through a two-stage ring (TMA,
// 64 x 32 boxes, 128-byte swizzle); warp 1 issues the split-TF32 MMAs
// (hi*hi + hi*lo + lo*hi) into one of two 64-column tensor-memory
// accumulators; warps 2..9 read the product back (tcgen05.ld) and subtract it
// from the output tiles in fp32.  Every mbarrier wait is bounded; a wait that
// runs out latches PICHOL_ERR_TIMEOUT, the CTA stops issuing work, waits
// (bounded) for its copies, frees its tensor memory and returns.
#include "internal.cuh"
#include "tcgen05.cuh"
#include "tma.cuh"

namespace pichol {

namespace ctc {

constexpr int BM = 128, BN = 64, BK = 32;
constexpr int HALF_BYTES = TB * BK * 4;          // one 64 x 32 box: 8 KB
constexpr int B_BYTES = 4 * HALF_BYTES;          // L_KJ: 2 K halves x (hi, lo)
constexpr int A_BYTES = 8 * HALF_BYTES;          // a pair: 2 K halves x (hi, lo) x 128 rows
constexpr int NSTG = 2;
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 32 * (2 + EPI_WARPS);
constexpr int TMEM_COLS = 128;                   // two 64-column accumulators
constexpr int SMEM = B_BYTES + NSTG * A_BYTES + 1024 /* alignment */ + 256 /* barriers */;

}  // namespace ctc

struct UpdTcArgs {
    float* F;               // factors, tile-major
    int64_t ntiles;
    int nt, J, first, chunk;
    int per, count, warm;   // problem map (see ProbMap in chol.cu)
    int64_t prow0;          // first row of this J's panel buffer in the scratch map
    int nfac;               // problem slots per panel buffer
    DevStatus* st;
};

__device__ __forceinline__ bool upd_dead(const UpdTcArgs& a, int pr)
{
    const int live = (a.warm > 0 && pr >= a.per) ? a.warm : a.count;
    return pr % a.per >= live;
}

// Shared-memory offset of K half h, part (0 hi, 1 lo) inside an operand: the
// halves are 64-row boxes of 128-byte rows; an A pair stacks the two tiles'
// boxes so each (h, part) is one 128-row K-major tile.
__device__ __forceinline__ uint32_t a_off(int h, int part, int tile2) { return ((h * 2 + part) * 2 + tile2) * ctc::HALF_BYTES; }
__device__ __forceinline__ uint32_t b_off(int h, int part) { return (h * 2 + part) * ctc::HALF_BYTES; }

__global__ void __launch_bounds__(320, 1)
k_chol_update_tc(const __grid_constant__ CUtensorMap mh, const __grid_constant__ CUtensorMap ml, const UpdTcArgs a)
{
    using namespace ctc;
    const int pr = blockIdx.z;
    if (upd_dead(a, pr)) return;
    const int K = a.first + (int)blockIdx.y;
    const int I0 = K + (int)blockIdx.x * a.chunk;
    if (I0 >= a.nt) return;
    const int nrow = (I0 + a.chunk < a.nt ? I0 + a.chunk : a.nt) - I0;   // output tiles of the strip
    const int npair = (nrow + 1) / 2;

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* bsm = smem;
    unsigned char* aring = smem + B_BYTES;
    uint64_t* bfull = (uint64_t*)(aring + NSTG * A_BYTES);
    uint64_t* afull = bfull + 1;
    uint64_t* aempty = afull + NSTG;
    uint64_t* tfull = aempty + NSTG;
    uint64_t* tempty = tfull + 2;
    uint64_t* mdone = tempty + 2;          // every MMA of the issuer complete (its exit)
    uint32_t* tmem_slot = (uint32_t*)(mdone + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    volatile int* consumed = abort_flag + 1;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t pbase = a.prow0 + (int64_t)pr * a.nt * TB;    // scratch row of panel tile 0 of this problem

    if (threadIdx.x == 0) {
        mbar_init(bfull, 1);
        for (int s = 0; s < NSTG; ++s) { mbar_init(&afull[s], 1); mbar_init(&aempty[s], 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], EPI_WARPS); }
        mbar_init(mdone, 1);
        *abort_flag = 0;
        *consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) tc5::alloc(tmem_slot, TMEM_COLS);
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- producer ----
            int issued = 0;
            mbar_expect_tx(bfull, B_BYTES);
            const int yk = (int)(pbase + (int64_t)K * TB);
            for (int h = 0; h < 2; ++h) {
                tma_load_2d(bsm + b_off(h, 0), &mh, bfull, h * BK, yk);
                tma_load_2d(bsm + b_off(h, 1), &ml, bfull, h * BK, yk);
            }
            for (int u = 0; u < npair; ++u) {
                const int s = u % NSTG;
                if (!mbar_wait(&aempty[s], ((u / NSTG) & 1) ^ 1)) { *abort_flag = 1; break; }
                if (*abort_flag) break;
                unsigned char* as = aring + s * A_BYTES;
                mbar_expect_tx(&afull[s], A_BYTES);
                const int I = I0 + 2 * u;
                const int I2 = (2 * u + 1 < nrow) ? I + 1 : I;      // a lone last tile repeats (not stored)
                const int y0 = (int)(pbase + (int64_t)I * TB), y1 = (int)(pbase + (int64_t)I2 * TB);
                for (int h = 0; h < 2; ++h) {
                    tma_load_2d(as + a_off(h, 0, 0), &mh, &afull[s], h * BK, y0);
                    tma_load_2d(as + a_off(h, 0, 1), &mh, &afull[s], h * BK, y1);
                    tma_load_2d(as + a_off(h, 1, 0), &ml, &afull[s], h * BK, y0);
                    tma_load_2d(as + a_off(h, 1, 1), &ml, &afull[s], h * BK, y1);
                }
                ++issued;
            }
            mbar_wait(bfull, 0);
            for (int u = *consumed; u < issued; ++u) mbar_wait(&afull[u % NSTG], (u / NSTG) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer: pair u into accumulator u & 1 ----
            constexpr uint32_t idesc = tc5::idesc_tf32(BM, BN);
            bool ok = mbar_wait(bfull, 0);
            if (!ok) *abort_flag = 1;
            tc5::fence_after();
            const uint32_t bbase = smem_u32(bsm);
            for (int u = 0; u < npair && ok && !*abort_flag; ++u) {
                const int s = u % NSTG, b = u & 1;
                if (!mbar_wait(&tempty[b], ((u >> 1) & 1) ^ 1) || !mbar_wait(&afull[s], (u / NSTG) & 1)) {
                    *abort_flag = 1;
                    break;
                }
                tc5::fence_after();
                const uint32_t abase = smem_u32(aring + s * A_BYTES);
                const uint32_t acc = tmem + (uint32_t)(b * BN);
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    tc5::mma_split3_k32(acc, abase + a_off(h, 0, 0), abase + a_off(h, 1, 0), bbase + b_off(h, 0),
                                        bbase + b_off(h, 1), idesc, h == 0);
                tc5::commit(&aempty[s]);
                tc5::commit(&tfull[b]);
                *consumed = u + 1;
            }
            // every MMA issued has completed before the tensor memory is freed
            tc5::commit(mdone);
            mbar_wait(mdone, 0);
        }
    } else {
        // ---- epilogue: out -= product; warp w reads lanes 32 (w % 4) .. +31 ----
        const int qtr = warp & 3, chalf = (warp - 2) >> 2;
        float* base = a.F + (int64_t)pr * a.ntiles * TILE_ELEMS;
        for (int u = 0; u < npair; ++u) {
            const int b = u & 1;
            if (!mbar_wait(&tfull[b], (u >> 1) & 1)) { *abort_flag = 1; break; }
            tc5::fence_after();
            float v[32];
            const uint32_t src = tmem + ((uint32_t)(qtr * 32) << 16) + (uint32_t)(b * BN + chalf * 32);
            tc5::ld16(src, *reinterpret_cast<float(*)[16]>(v));
            tc5::ld16(src + 16, *reinterpret_cast<float(*)[16]>(v + 16));
            tc5::fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(&tempty[b])) : "memory");
            const int tsel = qtr >> 1;                        // rows 0..63: tile I, 64..127: tile I + 1
            if (2 * u + tsel < nrow && !*abort_flag) {
                const int I = I0 + 2 * u + tsel;
                const int r = (qtr & 1) * 32 + lane;
                float4* o = reinterpret_cast<float4*>(base + tile_index(I, K) * TILE_ELEMS + r * TB + chalf * 32);
#pragma unroll
                for (int w = 0; w < 8; ++w) {
                    float4 x = o[w];
                    x.x -= v[4 * w];
                    x.y -= v[4 * w + 1];
                    x.z -= v[4 * w + 2];
                    x.w -= v[4 * w + 3];
                    o[w] = x;
                }
            }
        }
    }
    __syncwarp();
    tc5::fence_before();
    __syncthreads();
    if (*abort_flag && threadIdx.x == 0) latch_error(a.st, PICHOL_ERR_TIMEOUT, pr / a.per, K, -1);
    if (warp == 0) tc5::dealloc(tmem, TMEM_COLS);
}

}  // namespace pichol

namespace pichol {

// Bulk trailing update of tile column J on the tensor cores: output columns
// K = first .. first + ncols - 1, strips of `chunk` tiles from the diagonal
// down; the panel tiles of J must be in panel buffer J & 1.
cudaError_t launch_update_tc(pichol_ctx* ctx, int per, int count, int warm, int nprob, int J, int first, int ncols,
                             int chunk, cudaStream_t s)
{
    static std::atomic<unsigned long long> set{0};
    cudaError_t e = smem_limit_once(k_chol_update_tc, ctc::SMEM, set);
    if (e != cudaSuccess) return e;
    const uint64_t rows = (uint64_t)2 * ctx->nfac * ctx->nt * TB;
    CUtensorMap mh, ml;
    if (!make_map_f32(&mh, ctx->Ph, TB, rows, TB, ctc::BK, TB) || !make_map_f32(&ml, ctx->Pl, TB, rows, TB, ctc::BK, TB))
        return cudaErrorInvalidValue;
    UpdTcArgs a;
    a.F = (float*)ctx->F;
    a.ntiles = ctx->ntiles;
    a.nt = ctx->nt;
    a.J = J;
    a.first = first;
    a.chunk = chunk;
    a.per = per;
    a.count = count;
    a.warm = warm;
    a.prow0 = (int64_t)(J & 1) * ctx->nfac * ctx->nt * TB;
    a.nfac = (int)ctx->nfac;
    a.st = ctx->status;
    const int m = ctx->nt - first;                 // tiles in the longest output column
    k_chol_update_tc<<<dim3((unsigned)((m + chunk - 1) / chunk), (unsigned)ncols, (unsigned)nprob), ctc::THREADS,
                       ctc::SMEM, s>>>(mh, ml, a);
    return cudaGetLastError();
}

}  // namespace pichol
