// Tensor-core (tcgen05, TF32) contractions of the mixed-precision path:
//   Gram blocks     G_j = X_j^T X_j and X_j^T Y_j       (Sec. 3.1, Eq. 2)
//   hold-out scores E_f(t) = ||Y_f - X_f W_{f,t}||^2 for all q lambdas at once:
//                   X_f W_f (N = q c columns) with the squared residuals summed
//                   in the epilogue (Sec. 3.1's hold-out error, direct form)
//   exact-system refinement residual (refine_target exact; not in the paper):
//                   G_f W_f and G_all W_f, G_all = sum_j G_j, combined as
//                   R = B_f - lambda W - (G_all W - G_f W)
// and the bounded-wait check (pichol_check_timeout).
//
// C = sum_p A_p B_p^T with A (M x K) and B (N x K) both K-major fp32 in global
// memory.  With PASSES = 3 every operand is split as x = hi + lo, hi = x
// rounded to TF32 and lo = x - hi (exact in fp32), and the products
// hi*hi + hi*lo + lo*hi are accumulated in one fp32 accumulator: the dropped
// lo*lo term and the TF32 rounding of lo are ~2^-22 of |x y|, so the result is
// close to an fp32 product (the split-TF32 scheme of Ootomo & Yokota, 2022).
//
// One CTA computes one 128 x 128 tile of C:
//   warp 0 lane 0  TMA producer: 128 x 32 fp32 boxes (128-byte swizzle) of
//                  A_hi, A_lo, B_hi, B_lo per stage into a STAGES-deep ring
//   warp 1 lane 0  MMA issuer: tcgen05.mma kind::tf32, M = 128, N = 128,
//                  K = 8, into one of two 128-column tensor-memory
//                  accumulators, switching every CHUNK k-blocks
//   warps 2..9     drain each finished chunk (tcgen05.ld) into compensated
//                  (Kahan) fp32 totals in registers, then store C.  Summing
//                  128-row partial sums this way keeps the accumulation error
//                  of long K (the fold's rows) near one fp32 rounding.
// Every wait on an mbarrier is bounded (about two seconds of clock); a wait
// that runs out latches PICHOL_ERR_TIMEOUT, the CTA stops issuing work, waits
// (bounded) for its own copies and MMAs, frees its tensor memory and returns.
#include "internal.cuh"
#include "tcgen05.cuh"
#include "tma.cuh"

#include <algorithm>
#include <cstring>

namespace pichol {

namespace tc {

constexpr int BM = 128, BN = 128, BK = 32;     // BK fp32 = 128 bytes = one swizzle row
constexpr int STAGES = 3;
constexpr int TILE_BYTES = BM * BK * 4;        // 16 KB per operand tile
constexpr int STAGE_BYTES = 4 * TILE_BYTES;    // A_hi, A_lo, B_hi, B_lo
constexpr int RED_BYTES = 4 * BN * 4;           // score epilogue: one float per (row quarter, column)
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /* alignment */ + 256 /* barriers */ + RED_BYTES;
constexpr int TMEM_COLS = 256;                 // two 128-column accumulators
// k-blocks per accumulator drain: GemmArgs.chunk (1 = every 32 rows of K for
// the Gram blocks, whose fp32 tensor-memory sums of positive terms are the
// most exposed to the accumulation's rounding; 4 for the other products)
constexpr int EPI_WARPS = 8;                   // warps 2..9 drain and store
constexpr int THREADS = 32 * (2 + EPI_WARPS);

using tc5::sw128_desc;
using tc5::tf32_round;
__device__ __forceinline__ void tc_fence_before() { tc5::fence_before(); }
__device__ __forceinline__ void tc_fence_after() { tc5::fence_after(); }
__host__ __device__ constexpr uint32_t idesc_tf32_128x128() { return tc5::idesc_tf32(BM, BN); }
__device__ __forceinline__ void umma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    tc5::mma_tf32(tmem_d, a, b, idesc, acc);
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) { tc5::commit(bar); }
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) { tc5::ld16(taddr, v); }

}  // namespace tc

enum GemmMode { GEMM_GRAM = 0, GEMM_PLAIN = 1, GEMM_XTY = 2, GEMM_SCORE = 3 };

struct GemmArgs {
    int mode;
    int passes;
    int chunk;                // k-blocks of 32 rows of K per accumulator drain
    // GEMM_GRAM: lower tiles (I, J) of fold blockIdx.y; K range of fold f is
    // [k0[f], k0[f] + kn[f]) in the transposed, fold-padded X.
    int ntb;                  // 128-tiles per side
    int k0[MAX_K + 1];
    int kn[MAX_K];
    // GEMM_PLAIN: fold f uses A rows [f*a_rows_fold, ...) and B rows
    // [f*b_rows_fold + b_row_off, ...); output columns start at c_col_off
    int a_rows_fold, b_rows_fold, b_row_off, c_col_off;
    int K;
    // output
    float* C;                 // GRAM: G (k x dp x dp); PLAIN: C (k x M x ldc)
    float* Chi;               // GRAM: split of G for later contractions (may be null)
    float* Clo;
    int64_t ldc, M, N;        // valid rows / columns of one fold's C
    int64_t c_fold_stride;
    // GEMM_SCORE: A = X row-major split (fold f = rows [k0[f], k0[f] + kn[f])),
    // B = W^T of fold f (rows b_row_off + ..., N = lambdas x outputs), K = dp;
    // row i, column n of the tile gives the residual Y[k0[f] + i][(t0c + n) mod yc] - (X_f W)_in
    const float* Y;           // n x yc targets
    int64_t yc;
    int64_t t0c;              // column offset of the first lambda (t0 c)
    int mt_max;               // row tiles per fold in the grid
    double* epart;            // [f][mt_max][lde] per-column sums of squared residuals
    int64_t lde;
    DevStatus* st;
};

__global__ void __launch_bounds__(320, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
          const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl, const GemmArgs a)
{
    using namespace tc;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;      // [2] accumulator buffer ready to drain
    uint64_t* tempty = tfull + 2;          // [2] accumulator buffer drained
    uint64_t* mdone = tempty + 2;          // every MMA of the issuer complete (its exit)
    uint32_t* tmem_slot = (uint32_t*)(mdone + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    volatile int* consumed = abort_flag + 1;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int f = blockIdx.y;
    int tI, tJ, nk, kx0, arow, brow;
    if (a.mode == GEMM_GRAM) {
        tile_coords(blockIdx.x, tI, tJ);
        nk = (a.kn[f] + BK - 1) / BK;
        kx0 = a.k0[f];
        arow = tI * BM;
        brow = tJ * BN;
    } else if (a.mode == GEMM_XTY) {
        // X_f^T Y_f: A = X^T (feature tile blockIdx.x), B = Y^T (outputs), K = fold f's rows
        tI = blockIdx.x;
        tJ = 0;
        nk = (a.kn[f] + BK - 1) / BK;
        kx0 = a.k0[f];
        arow = tI * BM;
        brow = 0;
    } else if (a.mode == GEMM_SCORE) {
        tI = blockIdx.x % a.mt_max;
        tJ = blockIdx.x / a.mt_max;
        if ((int64_t)tI * BM >= a.kn[f]) return;   // past this fold's rows: the whole CTA leaves
        nk = (a.K + BK - 1) / BK;
        kx0 = 0;
        arow = a.k0[f] + tI * BM;
        brow = f * a.b_rows_fold + a.b_row_off + tJ * BN;
    } else {
        tI = blockIdx.x % ((int)((a.M + BM - 1) / BM));
        tJ = blockIdx.x / ((int)((a.M + BM - 1) / BM));
        nk = (a.K + BK - 1) / BK;
        kx0 = 0;
        arow = f * a.a_rows_fold + tI * BM;
        brow = f * a.b_rows_fold + a.b_row_off + tJ * BN;
    }
    const int CHUNK = a.chunk > 0 ? a.chunk : 4;
    const int nchunks = (nk + CHUNK - 1) / CHUNK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], EPI_WARPS);
        }
        mbar_init(mdone, 1);
        *abort_flag = 0;
        *consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t bytes_per_stage = (a.passes == 3 ? 4 : 2) * TILE_BYTES;

    if (warp == 0) {
        if (lane == 0) {
            // ---- producer ----
            int issued = 0;
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % STAGES;
                if (!mbar_wait(&empty[s], ((kb / STAGES) & 1) ^ 1)) { *abort_flag = 1; break; }
                if (*abort_flag) break;
                unsigned char* st = smem + s * STAGE_BYTES;
                mbar_expect_tx(&full[s], bytes_per_stage);
                const int x = kx0 + kb * BK;
                tma_load_2d(st, &mAh, &full[s], x, arow);
                tma_load_2d(st + 2 * TILE_BYTES, &mBh, &full[s], x, brow);
                if (a.passes == 3) {
                    tma_load_2d(st + TILE_BYTES, &mAl, &full[s], x, arow);
                    tma_load_2d(st + 3 * TILE_BYTES, &mBl, &full[s], x, brow);
                }
                ++issued;
            }
            // wait (bounded) for copies that were issued but never consumed
            for (int kb = *consumed; kb < issued; ++kb) mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer: chunk ch accumulates into buffer ch & 1 ----
            const uint32_t idesc = idesc_tf32_128x128();
            int kb = 0;
            for (int ch = 0; ch < nchunks && !*abort_flag; ++ch) {
                const int b = ch & 1, use = ch >> 1;
                if (!mbar_wait(&tempty[b], (use & 1) ^ 1)) { *abort_flag = 1; break; }
                tc_fence_after();
                const uint32_t acc = tmem + (uint32_t)(b * BN);
                const int kend = (kb + CHUNK < nk) ? kb + CHUNK : nk;
                for (int k0 = kb; kb < kend; ++kb) {
                    const int s = kb % STAGES;
                    if (*abort_flag || !mbar_wait(&full[s], (kb / STAGES) & 1)) { *abort_flag = 1; break; }
                    tc_fence_after();
                    const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
                    const uint32_t ah = base, al = base + TILE_BYTES, bh = base + 2 * TILE_BYTES,
                                   bl = base + 3 * TILE_BYTES;
                    if (a.passes == 3) {
                        tc5::mma_split3_k32(acc, ah, al, bh, bl, idesc, kb == k0);
                    } else {
#pragma unroll
                        for (int kk = 0; kk < BK / 8; ++kk) {
                            const uint32_t off = kk * 32;   // 8 tf32 = 32 bytes along K
                            umma_tf32(acc, sw128_desc(ah + off), sw128_desc(bh + off), idesc, ((kb - k0) | kk) != 0);
                        }
                    }
                    umma_commit(&empty[s]);
                    *consumed = kb + 1;
                }
                umma_commit(&tfull[b]);   // buffer b holds the chunk's sum once its MMAs complete
            }
            // every MMA issued has completed before the tensor memory is freed
            umma_commit(mdone);
            mbar_wait(mdone, 0);
        }
    } else {
        // ---- drain: add every chunk's partial sum into compensated fp32 totals ----
        // warp w may access TMEM lanes 32 (w % 4) .. +31: its tile rows; the
        // first four drain warps take columns 0..63, the next four 64..127
        float tot[64], cmp[64];
        const int qtr = warp & 3, chalf = (warp - 2) >> 2;
#pragma unroll
        for (int u = 0; u < 64; ++u) { tot[u] = 0.0f; cmp[u] = 0.0f; }
        for (int ch = 0; ch < nchunks; ++ch) {
            const int b = ch & 1, use = ch >> 1;
            if (!mbar_wait(&tfull[b], use & 1)) { *abort_flag = 1; break; }
            tc_fence_after();
            const uint32_t src = tmem + ((uint32_t)(qtr * 32) << 16) + (uint32_t)(b * BN + chalf * 64);
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                float v[16];
                tmem_ld16(src + (uint32_t)(cc * 16), v);
#pragma unroll
                for (int u = 0; u < 16; ++u) {   // Kahan: tot += v
                    const float y = v[u] - cmp[cc * 16 + u];
                    const float t = tot[cc * 16 + u] + y;
                    cmp[cc * 16 + u] = (t - tot[cc * 16 + u]) - y;
                    tot[cc * 16 + u] = t;
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(&tempty[b])) : "memory");
        }
        if (!*abort_flag) {
        const int row = qtr * 32 + lane;           // row inside the tile
        const int64_t grow = (int64_t)tI * BM + row;
        const int64_t gcol0 = (int64_t)tJ * BN + chalf * 64;
        float* Cf = a.C + (int64_t)f * a.c_fold_stride;
        if (a.mode == GEMM_GRAM) {
            if (grow < a.M) {
#pragma unroll
                for (int u = 0; u < 64; ++u) {
                    const int64_t gc = gcol0 + u;
                    if (gc < a.N) {
                        Cf[grow * a.ldc + gc] = tot[u];
                        if (a.Chi) {
                            const float hi = tc::tf32_round(tot[u]);
                            a.Chi[(int64_t)f * a.c_fold_stride + grow * a.ldc + gc] = hi;
                            a.Clo[(int64_t)f * a.c_fold_stride + grow * a.ldc + gc] = tot[u] - hi;
                        }
                    }
                }
            }
            if (tI != tJ && grow < a.N) {   // mirror into the upper tile
#pragma unroll
                for (int u = 0; u < 64; ++u) {
                    const int64_t gc = gcol0 + u;
                    if (gc < a.M) {
                        Cf[gc * a.ldc + grow] = tot[u];
                        if (a.Chi) {
                            const float hi = tc::tf32_round(tot[u]);
                            a.Chi[(int64_t)f * a.c_fold_stride + gc * a.ldc + grow] = hi;
                            a.Clo[(int64_t)f * a.c_fold_stride + gc * a.ldc + grow] = tot[u] - hi;
                        }
                    }
                }
            }
        } else if (a.mode != GEMM_SCORE && grow < a.M) {
#pragma unroll
            for (int u = 0; u < 64; ++u) {
                const int64_t gc = gcol0 + u;
                if (gc < a.N) Cf[grow * a.ldc + a.c_col_off + gc] = tot[u];
            }
        }
        }
        if (a.mode == GEMM_SCORE) {
            // Squared residuals (Y - X_f W)^2 of this thread's row for its 64
            // columns, then summed over the tile's 128 rows per column in a
            // fixed order: a reduce-scatter over the warp's 32 rows (five
            // halvings; lane l keeps the sums of columns col(l) and col(l) + 1,
            // col(l) = 32 l4 + 16 l3 + 8 l2 + 4 l1 + 2 l0 for the bits of l),
            // the four row quarters through shared memory, in double.
            const bool live = !*abort_flag;
            const int row = qtr * 32 + lane;
            const int64_t grow = (int64_t)tI * BM + row;
            const int64_t gcol0 = (int64_t)tJ * BN + chalf * 64;
            float v[64];
            const bool rv = live && grow < a.kn[f];
            const float* yrow = a.Y + (rv ? ((int64_t)a.k0[f] + grow) * a.yc : 0);
            int64_t o = (a.t0c + gcol0) % a.yc;
#pragma unroll
            for (int u = 0; u < 64; ++u) {
                float r = 0.0f;
                if (rv && gcol0 + u < a.N) r = yrow[o] - tot[u];
                v[u] = r * r;
                o = (o + 1 == a.yc) ? 0 : o + 1;
            }
#pragma unroll
            for (int h = 32, b = 16; h >= 2; h >>= 1, b >>= 1) {
                const bool up = (lane & b) != 0;
#pragma unroll
                for (int u = 0; u < h; ++u) {
                    const float keep = up ? v[u + h] : v[u];
                    const float send = up ? v[u] : v[u + h];
                    v[u] = keep + __shfl_xor_sync(0xffffffffu, send, b);
                }
            }
            float* red = (float*)(smem + STAGES * STAGE_BYTES + 256);
            const int col = ((lane >> 4) & 1) * 32 + ((lane >> 3) & 1) * 16 + ((lane >> 2) & 1) * 8 +
                            ((lane >> 1) & 1) * 4 + (lane & 1) * 2;
            red[qtr * BN + chalf * 64 + col] = v[0];
            red[qtr * BN + chalf * 64 + col + 1] = v[1];
            asm volatile("bar.sync 1, 256;\n" ::: "memory");   // the eight drain warps
            if (warp < 6) {
                const int cidx = threadIdx.x - 64;              // 0 .. 127
                const double s = (double)red[cidx] + (double)red[BN + cidx] + (double)red[2 * BN + cidx] +
                                 (double)red[3 * BN + cidx];
                const int64_t gc = (int64_t)tJ * BN + cidx;
                if (live && gc < a.N) a.epart[((int64_t)f * a.mt_max + tI) * a.lde + gc] = s;
            }
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (*abort_flag && threadIdx.x == 0) latch_error(a.st, PICHOL_ERR_TIMEOUT, f, (int)blockIdx.x, -1);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// ---------------------------------------------------------------------------
// Operand preparation
// ---------------------------------------------------------------------------

// XT_hi / XT_lo [dp][Kpad]: column kc of fold j (k0[j] <= kc < k0[j+1]) holds
// sample row o[j] + (kc - k0[j]) if that row is in fold j, else 0; rows >= d are 0.
// With Xrh / Xrl given, the same pass writes the row-major split [n][dp] of X
// (columns >= d zero) for the direct hold-out score: every sample row is read
// once, by the CTA whose 32 columns of XT hold it.
struct XtArgs {
    int64_t k0[MAX_K + 1];
    int64_t o[MAX_K + 1];
    int k;
};

__global__ void __launch_bounds__(256)
k_split_xt(const float* __restrict__ X, int64_t d, int64_t dp, int64_t kpad, XtArgs xa, float* __restrict__ Xh,
           float* __restrict__ Xl, float* __restrict__ Xrh, float* __restrict__ Xrl)
{
    __shared__ float t[32][33];
    const int64_t kc0 = (int64_t)blockIdx.x * 32, f0 = (int64_t)blockIdx.y * 32;
    int j = 0;
    while (j + 1 < xa.k && xa.k0[j + 1] <= kc0) ++j;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    for (int yy = ty; yy < 32; yy += 8) {
        const int64_t kc = kc0 + yy;
        const int64_t row = xa.o[j] + (kc - xa.k0[j]);
        const int64_t feat = f0 + tx;
        float v = 0.0f;
        if (row < xa.o[j + 1]) {
            if (feat < d) v = X[row * d + feat];
            if (Xrh) {
                const float hi = tc::tf32_round(v);
                Xrh[row * dp + feat] = hi;
                Xrl[row * dp + feat] = v - hi;
            }
        }
        t[yy][tx] = v;
    }
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
        const int64_t feat = f0 + yy, kc = kc0 + tx;
        if (feat < dp && kc < kpad) {
            const float v = t[tx][yy];
            const float hi = tc::tf32_round(v);
            Xh[feat * kpad + kc] = hi;
            Xl[feat * kpad + kc] = v - hi;
        }
    }
}

// YT_hi / YT_lo [c][Kpad]: the same fold-padded transpose for the targets Y.
__global__ void __launch_bounds__(256)
k_split_yt(const float* __restrict__ Y, int64_t c, int64_t kpad, XtArgs xa, float* __restrict__ Yh,
           float* __restrict__ Yl)
{
    __shared__ float t[32][33];
    const int64_t kc0 = (int64_t)blockIdx.x * 32, o0 = (int64_t)blockIdx.y * 32;
    int j = 0;
    while (j + 1 < xa.k && xa.k0[j + 1] <= kc0) ++j;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int yy = ty; yy < 32; yy += 8) {
        const int64_t kc = kc0 + yy;
        const int64_t row = xa.o[j] + (kc - xa.k0[j]);
        const int64_t o = o0 + tx;
        t[yy][tx] = (row < xa.o[j + 1] && o < c) ? Y[row * c + o] : 0.0f;
    }
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
        const int64_t o = o0 + yy, kc = kc0 + tx;
        if (o < c && kc < kpad) {
            const float v = t[tx][yy];
            const float hi = tc::tf32_round(v);
            Yh[o * kpad + kc] = hi;
            Yl[o * kpad + kc] = v - hi;
        }
    }
}

// Wt_hi / Wt_lo [f][t*c + o][dp] = split of W[f][t][k][o].
__global__ void __launch_bounds__(256)
k_split_wt(const float* __restrict__ W, int q, int t0, int64_t dp, int64_t c, float* __restrict__ Wh,
           float* __restrict__ Wl)
{
    const int t = t0 + blockIdx.y, f = blockIdx.z;
    const float* Wt = W + ((int64_t)f * q + t) * dp * c;
    float* oh = Wh + ((int64_t)f * q + t) * c * dp;
    float* ol = Wl + ((int64_t)f * q + t) * c * dp;
    for (int64_t kk = (int64_t)blockIdx.x * 256 + threadIdx.x; kk < dp; kk += (int64_t)gridDim.x * 256)
        for (int o = 0; o < c; ++o) {
            const float v = Wt[kk * c + o];
            const float hi = tc::tf32_round(v);
            oh[(int64_t)o * dp + kk] = hi;
            ol[(int64_t)o * dp + kk] = v - hi;
        }
}

cudaError_t launch_split_wt(pichol_ctx* ctx, int t0, int tcount, int stage, cudaStream_t s)
{
    const pichol_config& c = ctx->cfg;
    const int64_t dp = ctx->dp;
    {
        StageScope sc_(ctx, stage, s);
        k_split_wt<<<dim3((unsigned)((dp + 255) / 256), tcount, c.k), 256, 0, s>>>((const float*)ctx->W, c.q, t0, dp,
                                                                                  c.c, ctx->Wth, ctx->Wtl);
    }
    ctx->launches++;
    return cudaGetLastError();
}

// Score partials from U = G_f W (dp x ldu per fold, column t*c + o):
// Epart[f][t][I] = sum_{rows in 64-tile I} sum_o W (U - 2 Bv), in double.
__global__ void __launch_bounds__(64)
k_score_reduce(const float* __restrict__ U, int64_t ldu, const float* __restrict__ W, const float* __restrict__ Bv,
               int q, int t0, int nt, int64_t dp, int64_t c, double* __restrict__ Epart)
{
    __shared__ double red[64];
    const int I = blockIdx.x, t = t0 + blockIdx.y, f = blockIdx.z;
    const int64_t row = (int64_t)I * TB + threadIdx.x;
    const float* wr = W + (((int64_t)f * q + t) * dp + row) * c;
    const float* ur = U + ((int64_t)f * dp + row) * ldu + (int64_t)t * c;
    const float* br = Bv + ((int64_t)f * dp + row) * c;
    double s = 0.0;
    for (int o = 0; o < c; ++o) s += (double)wr[o] * ((double)ur[o] - 2.0 * (double)br[o]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 32; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) Epart[((int64_t)f * q + t) * nt + I] = red[0];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// 2D fp32 K-major map: `rows` rows of `cols` elements, leading dimension `ld`,
// boxes of 32 (K) x 128 (rows).
static bool make_map(CUtensorMap* m, const float* base, uint64_t cols, uint64_t rows, uint64_t ld)
{
    return make_map_f32(m, base, cols, rows, ld, tc::BK, tc::BM);
}

static cudaError_t gemm_attr()
{
    static std::atomic<unsigned long long> set{0};
    return smem_limit_once(k_tc_gemm, tc::SMEM_BYTES, set);
}


int64_t tc_kpad(const pichol_ctx* ctx)
{
    int64_t kp = 0;
    for (int j = 0; j < ctx->cfg.k; ++j) kp += (ctx->offs[j + 1] - ctx->offs[j] + 31) / 32 * 32;
    return kp;
}

cudaError_t launch_gram_tc(pichol_ctx* ctx, const float* X, cudaStream_t s)
{
    const pichol_config& c = ctx->cfg;
    const int64_t dp = ctx->dp, kpad = ctx->kpad;
    XtArgs xa;
    xa.k = c.k;
    xa.k0[0] = 0;
    for (int j = 0; j < c.k; ++j) {
        xa.o[j] = ctx->offs[j];
        xa.k0[j + 1] = xa.k0[j] + (ctx->offs[j + 1] - ctx->offs[j] + 31) / 32 * 32;
    }
    xa.o[c.k] = ctx->offs[c.k];
    {
        StageScope sc_(ctx, ST_GRAM, s);
        // X and Y are read only during this call: the row-major split of X for the
        // direct hold-out scores of the evaluation is written in the same pass
        k_split_xt<<<dim3((unsigned)(kpad / 32), (unsigned)((dp + 31) / 32)), 256, 0, s>>>(
            X, c.d, dp, kpad, xa, ctx->Xh, ctx->Xl, ctx->Xrh, ctx->Xrl);
    }
    ctx->launches++;
    CUtensorMap mh, ml;
    if (!make_map(&mh, ctx->Xh, (uint64_t)kpad, (uint64_t)dp, (uint64_t)kpad) ||
        !make_map(&ml, ctx->Xl, (uint64_t)kpad, (uint64_t)dp, (uint64_t)kpad))
        return cudaErrorInvalidValue;
    cudaError_t e = gemm_attr();
    if (e != cudaSuccess) return e;
    GemmArgs ga;
    memset(&ga, 0, sizeof(ga));
    ga.mode = GEMM_GRAM;
    ga.passes = c.gram_passes;
    ga.chunk = 1;
    ga.ntb = (int)((dp + tc::BM - 1) / tc::BM);
    for (int j = 0; j <= c.k; ++j) ga.k0[j] = (int)xa.k0[j];
    for (int j = 0; j < c.k; ++j) ga.kn[j] = (int)(ctx->offs[j + 1] - ctx->offs[j]);
    ga.C = (float*)ctx->G;
    ga.Chi = ctx->Gh;
    ga.Clo = ctx->Gl;
    ga.ldc = dp;
    ga.M = dp;
    ga.N = dp;
    ga.c_fold_stride = dp * dp;
    ga.st = ctx->status;
    const unsigned tiles = (unsigned)((int64_t)ga.ntb * (ga.ntb + 1) / 2);
    {
        StageScope sc_(ctx, ST_GRAM, s);
        k_tc_gemm<<<dim3(tiles, c.k), tc::THREADS, tc::SMEM_BYTES, s>>>(mh, ml, mh, ml, ga);
    }
    ctx->launches++;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // and a copy of Y
    if (ctx->Ycp &&
        (e = cudaMemcpyAsync(ctx->Ycp, ctx->Yin, sizeof(float) * (size_t)(c.n * c.c), cudaMemcpyDeviceToDevice, s)) !=
            cudaSuccess)
        return e;

    // Bv_j = X_j^T Y_j on the same operands: B = Y^T (c rows, zero-filled to 128)
    {
        StageScope sc_(ctx, ST_XTY, s);
        k_split_yt<<<dim3((unsigned)(kpad / 32), (unsigned)((c.c + 31) / 32)), 256, 0, s>>>(ctx->Yin, c.c, kpad, xa,
                                                                                          ctx->Yh, ctx->Yl);
    }
    ctx->launches++;
    CUtensorMap yh, yl;
    if (!make_map(&yh, ctx->Yh, (uint64_t)kpad, (uint64_t)c.c, (uint64_t)kpad) ||
        !make_map(&yl, ctx->Yl, (uint64_t)kpad, (uint64_t)c.c, (uint64_t)kpad))
        return cudaErrorInvalidValue;
    GemmArgs gy = ga;
    gy.mode = GEMM_XTY;
    gy.C = (float*)ctx->Bv;
    gy.Chi = nullptr;
    gy.Clo = nullptr;
    gy.ldc = c.c;
    gy.M = dp;
    gy.N = c.c;
    gy.c_col_off = 0;
    gy.c_fold_stride = dp * c.c;
    {
        StageScope sc_(ctx, ST_XTY, s);
        k_tc_gemm<<<dim3((unsigned)ga.ntb, c.k), tc::THREADS, tc::SMEM_BYTES, s>>>(mh, ml, yh, yl, gy);
    }
    ctx->launches++;
    return cudaGetLastError();
}

// The error path of every bounded copy wait, exercised on purpose: one
// mbarrier expecting one arrival that nothing makes, waited on with a limit of
// `limit` clocks; when the wait runs out the kernel latches PICHOL_ERR_TIMEOUT
// and returns, like a copy wait that gives up.
__global__ void k_wait_check(long long limit, DevStatus* st)
{
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    mbar_init_fence();
    if (!mbar_wait(&bar, 0, limit)) latch_error(st, PICHOL_ERR_TIMEOUT, -1, -1, -1);
}

cudaError_t launch_wait_check(pichol_ctx* ctx, long long limit, cudaStream_t s)
{
    k_wait_check<<<1, 32, 0, s>>>(limit, ctx->status);
    ctx->launches++;
    return cudaGetLastError();
}

// G_all = sum_j G_j (the fp32 blocks summed in double, in increasing j),
// rounded to fp32 and split into a TF32 part and an fp32 remainder for the
// products with W of the exact-system refinement.
__global__ void __launch_bounds__(256)
k_gall_split(const float* __restrict__ G, int k, int64_t n, float* __restrict__ hi, float* __restrict__ lo)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int j = 0; j < k; ++j) v += (double)G[(int64_t)j * n + e];
        const float vf = (float)v;
        const float h = tc::tf32_round(vf);
        hi[e] = h;
        lo[e] = vf - h;
    }
}

cudaError_t launch_gall_split(pichol_ctx* ctx, cudaStream_t s)
{
    const int64_t n = ctx->dp * ctx->dp;
    {
        StageScope sc_(ctx, ST_MISC, s);
        k_gall_split<<<1216, 256, 0, s>>>((const float*)ctx->G, ctx->cfg.k, n, ctx->Gah, ctx->Gal);
    }
    ctx->launches++;
    return cudaGetLastError();
}

// Residual of the exact shifted system for every (fold f, lambda t) of the batch:
//   R = B_f - lambda_t W - (G_all W - G_f W)     (H_f = G_all - G_f),
// combined in double from the two split-TF32 products.
__global__ void __launch_bounds__(256)
k_resid_exact(const float* __restrict__ U2, const float* __restrict__ U3, int64_t ldu, const float* __restrict__ W,
              const float* __restrict__ B, const double* __restrict__ lam, int q, int t0, int tcount, int64_t dp,
              int64_t c, float* __restrict__ R)
{
    const int f = blockIdx.z, t = t0 + blockIdx.y;
    const int64_t len = dp * c;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / c, o = e % c;
        const int64_t u = ((int64_t)f * dp + i) * ldu + (int64_t)t * c + o;
        const int64_t w = ((int64_t)f * q + t) * len + e;
        const double hw = (double)U3[u] - (double)U2[u];
        R[w] = (float)((double)B[(int64_t)f * len + e] - lam[t] * (double)W[w] - hw);
    }
}

cudaError_t launch_resid_exact(pichol_ctx* ctx, int t0, int tcount, cudaStream_t s)
{
    const pichol_config& c = ctx->cfg;
    const int64_t dp = ctx->dp, qc = (int64_t)c.q * c.c;
    {
        StageScope sc_(ctx, ST_RESID, s);
        k_split_wt<<<dim3((unsigned)((dp + 255) / 256), tcount, c.k), 256, 0, s>>>((const float*)ctx->W, c.q, t0, dp,
                                                                                  c.c, ctx->Wth, ctx->Wtl);
    }
    ctx->launches++;
    CUtensorMap fh, fl, ah, al, bh, bl;
    if (!make_map(&fh, ctx->Gh, (uint64_t)dp, (uint64_t)(c.k * dp), (uint64_t)dp) ||
        !make_map(&fl, ctx->Gl, (uint64_t)dp, (uint64_t)(c.k * dp), (uint64_t)dp) ||
        !make_map(&ah, ctx->Gah, (uint64_t)dp, (uint64_t)dp, (uint64_t)dp) ||
        !make_map(&al, ctx->Gal, (uint64_t)dp, (uint64_t)dp, (uint64_t)dp) ||
        !make_map(&bh, ctx->Wth, (uint64_t)dp, (uint64_t)(c.k * qc), (uint64_t)dp) ||
        !make_map(&bl, ctx->Wtl, (uint64_t)dp, (uint64_t)(c.k * qc), (uint64_t)dp))
        return cudaErrorInvalidValue;
    cudaError_t e = gemm_attr();
    if (e != cudaSuccess) return e;
    GemmArgs ga;
    memset(&ga, 0, sizeof(ga));
    ga.mode = GEMM_PLAIN;
    ga.passes = 3;
    ga.a_rows_fold = (int)dp;
    ga.b_rows_fold = (int)qc;
    ga.b_row_off = t0 * (int)c.c;
    ga.c_col_off = t0 * (int)c.c;
    ga.K = (int)dp;
    ga.C = ctx->U2;
    ga.ldc = ctx->ldu;
    ga.M = dp;
    ga.N = (int64_t)tcount * c.c;
    ga.c_fold_stride = dp * ctx->ldu;
    ga.st = ctx->status;
    const unsigned mt = (unsigned)((dp + tc::BM - 1) / tc::BM), nt = (unsigned)((ga.N + tc::BN - 1) / tc::BN);
    {
        StageScope sc_(ctx, ST_RESID, s);
        k_tc_gemm<<<dim3(mt * nt, c.k), tc::THREADS, tc::SMEM_BYTES, s>>>(fh, fl, bh, bl, ga);   // G_f W
    }
    GemmArgs gb = ga;
    gb.a_rows_fold = 0;                       // one A for every fold
    gb.C = ctx->U3;
    {
        StageScope sc_(ctx, ST_RESID, s);
        k_tc_gemm<<<dim3(mt * nt, c.k), tc::THREADS, tc::SMEM_BYTES, s>>>(ah, al, bh, bl, gb);   // G_all W
    }
    {
        StageScope sc_(ctx, ST_RESID, s);
        k_resid_exact<<<dim3((unsigned)((dp * c.c + 255) / 256), tcount, c.k), 256, 0, s>>>(
            ctx->U2, ctx->U3, ctx->ldu, (const float*)ctx->W, (const float*)ctx->Btr, ctx->lam, c.q, t0, tcount, dp,
            c.c, (float*)ctx->Rres);
    }
    ctx->launches += 3;
    return cudaGetLastError();
}

// E_f(t) sums from the per-(row tile, column) partials of the direct score:
// S = sum over the fold's row tiles (in order) and outputs o (in order) of
// epart[f][mt][(t - t0) c + o].  The consumers of Epart (selection, MChol,
// PINRMSE) form yy_f + sum of a (fold, lambda)'s nt slots, so slot 0 gets
// S - yy_f and the others zero; adding yy_f back in double changes S by a few
// units of yy_f's last place (yy_f / S is ~1e2 at most here, so ~1e-14).
__global__ void __launch_bounds__(256)
k_score_direct_sum(const double* __restrict__ ep, int mt_max, int64_t lde, const int64_t* __restrict__ nfc,
                   const double* __restrict__ yy, int64_t c, int q, int t0, int tcount, int nt,
                   double* __restrict__ Epart)
{
    const int f = blockIdx.y;
    const int tl = blockIdx.x * blockDim.x + threadIdx.x;
    if (tl >= tcount) return;
    const int64_t nf = nfc[f] / c;
    const int mts = (int)((nf + 127) / 128);
    double s = 0.0;
    for (int mt = 0; mt < mts && mt < mt_max; ++mt) {
        const double* row = ep + ((int64_t)f * mt_max + mt) * lde + (int64_t)tl * c;
        for (int64_t o = 0; o < c; ++o) s += row[o];
    }
    double* out = Epart + ((int64_t)f * q + t0 + tl) * nt;
    out[0] = s - yy[f];
    for (int i = 1; i < nt; ++i) out[i] = 0.0;
}

// Mixed-mode hold-out scores of systems [t0, t0 + tcount) in the direct form
// ||Y_f - X_f W||^2: W^T split into TF32 parts, then one split-TF32 product
// X_f W per fold over all those lambdas (N = tcount c) whose epilogue squares
// and sums the residuals, then the per-(fold, lambda) sums.  The expansion
// yy - 2 <Bv, W> + <W, G_f W> cancels about ||Y_f||^2 / E_f digits of its
// fp32 terms; the direct form does not.
cudaError_t launch_score_tc(pichol_ctx* ctx, int t0, int tcount, cudaStream_t s)
{
    const pichol_config& c = ctx->cfg;
    const int64_t dp = ctx->dp, qc = (int64_t)c.q * c.c;
    {
        StageScope sc_(ctx, ST_SCORE, s);
        k_split_wt<<<dim3((unsigned)((dp + 255) / 256), tcount, c.k), 256, 0, s>>>((const float*)ctx->W, c.q, t0, dp,
                                                                                  c.c, ctx->Wth, ctx->Wtl);
    }
    ctx->launches++;
    CUtensorMap ah, al, bh, bl;
    if (!make_map(&ah, ctx->Xrh, (uint64_t)dp, (uint64_t)c.n, (uint64_t)dp) ||
        !make_map(&al, ctx->Xrl, (uint64_t)dp, (uint64_t)c.n, (uint64_t)dp) ||
        !make_map(&bh, ctx->Wth, (uint64_t)dp, (uint64_t)(c.k * qc), (uint64_t)dp) ||
        !make_map(&bl, ctx->Wtl, (uint64_t)dp, (uint64_t)(c.k * qc), (uint64_t)dp))
        return cudaErrorInvalidValue;
    cudaError_t e = gemm_attr();
    if (e != cudaSuccess) return e;
    GemmArgs ga;
    memset(&ga, 0, sizeof(ga));
    ga.mode = GEMM_SCORE;
    ga.passes = 3;
    int64_t nf_max = 0;
    for (int j = 0; j < c.k; ++j) {
        ga.k0[j] = (int)ctx->offs[j];
        ga.kn[j] = (int)(ctx->offs[j + 1] - ctx->offs[j]);
        nf_max = std::max<int64_t>(nf_max, ga.kn[j]);
    }
    ga.b_rows_fold = (int)qc;
    ga.b_row_off = t0 * (int)c.c;
    ga.K = (int)dp;
    ga.N = (int64_t)tcount * c.c;
    ga.Y = ctx->Ycp;
    ga.yc = c.c;
    ga.t0c = (int64_t)t0 * c.c;
    ga.mt_max = (int)((nf_max + tc::BM - 1) / tc::BM);
    ga.epart = ctx->Escore;
    ga.lde = ctx->ldu;
    ga.st = ctx->status;
    if (ga.mt_max > ctx->mt_cap) return cudaErrorInvalidValue;
    const unsigned nn = (unsigned)((ga.N + tc::BN - 1) / tc::BN);
    {
        StageScope sc_(ctx, ST_SCORE, s);
        k_tc_gemm<<<dim3((unsigned)ga.mt_max * nn, c.k), tc::THREADS, tc::SMEM_BYTES, s>>>(ah, al, bh, bl, ga);
    }
    {
        StageScope sc_(ctx, ST_SCORE, s);
        k_score_direct_sum<<<dim3((unsigned)((tcount + 255) / 256), c.k), 256, 0, s>>>(
            ctx->Escore, ga.mt_max, ctx->ldu, ctx->nfc, ctx->yy, c.c, c.q, t0, tcount, ctx->nt, ctx->Epart);
    }
    ctx->launches += 2;
    return cudaGetLastError();
}

}  // namespace pichol
