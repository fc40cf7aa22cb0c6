// Definitions shared by the interpolate-on-load solve (solve.cu, and
// solve_single.cu for one lambda per CTA) and the refinement residual
// (resid.cu): vector types, the staging of half tiles (TMA and cp.async), the
// staged layouts, the solve kernel and its launch, and the residual's
// arguments.
#pragma once

#include <cuda.h>

#include <cstring>
#include <type_traits>

#include "internal.cuh"
#include "tma.cuh"

namespace pichol {

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int N = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int N = 2; };

// N consecutive values of T as one load (N = 4, 2 or 1 for float; 2 or 1 for double)
template <typename T, int N> struct VecN;
template <> struct VecN<float, 4> { using type = float4; };
template <> struct VecN<float, 2> { using type = float2; };
template <> struct VecN<float, 1> { using type = float; };
template <> struct VecN<double, 2> { using type = double2; };
template <> struct VecN<double, 1> { using type = double; };


// Byte offset of element (row, col) of a row half (rows [32 h, 32 h + 32), all
// 64 columns) of an fp32 plane staged by two TMA boxes of 32 x 32: the box of
// columns [32 b, 32 b + 32) at b * 4096, rows of 128 bytes whose 16-byte
// chunks are permuted by XOR with (row & 7) (the 128-byte swizzle).
__device__ __forceinline__ int rowhalf_off_f32(int row, int col)
{
    return (col >> 5) * 4096 + row * 128 + (((((col & 31) >> 2) ^ (row & 7))) << 4) + ((col & 3) << 2);
}

// TMA copy of half of the NPS fp32 planes of one tile into a stage (1024-byte
// aligned), the same layouts stage_half writes for cols = true, and the
// rowhalf_off_f32 layout for cols = false.  row0(pl) is the first row of plane
// pl in the map's [rows][64] view.  Issued by one thread; completes on `bar`.
template <int NPS, typename Row0>
__device__ __forceinline__ void tma_stage_half(unsigned char* sdst, const CUtensorMap* map, uint64_t* bar, int h,
                                               bool cols, Row0 row0)
{
    constexpr int HPB = (TB / 2) * TB * 4;
    mbar_expect_tx(bar, (uint32_t)(NPS * HPB));
#pragma unroll
    for (int pl = 0; pl < NPS; ++pl) {
        const int y = row0(pl);
        unsigned char* d = sdst + pl * HPB;
        if (cols) {
            tma_load_2d(d, map, bar, 32 * h, y);
            tma_load_2d(d + 4096, map, bar, 32 * h, y + 32);
        } else {
            tma_load_2d(d, map, bar, 0, y + 32 * h);
            tma_load_2d(d + 4096, map, bar, 32, y + 32 * h);
        }
    }
}

// ---------------------------------------------------------------------------
// Refinement residual r = B - L~ (L~^T W), double-float accumulation.
//   pass 0: u_i = sum_{j >= i} L~_ji^T W_j      -> (uhi, ulo)
//   pass 1: r_i = B_i - sum_{j <= i} L~_ij u_j  -> R (rounded to float)
// Products are split error-free (p = a*b, e = fma(a, b, -p)); sums use TwoSum.
// ---------------------------------------------------------------------------
struct ResidArgs {
    const float* theta;
    const float* W;      // pass 0 input
    const float* uhi;    // pass 1 input
    const float* ulo;
    float* ohi;          // pass 0 outputs
    float* olo;
    const float* B;      // pass 1: per-fold right-hand side [f][dp][c]
    float* R;            // pass 1 output [f][t][dp][c]
    const double* phi;
    int p, nt, q, t0, tcount;
    int64_t ntiles, dp, c;
    DevStatus* st;       // PICHOL_ERR_TIMEOUT if a bounded copy wait runs out
};

// Copy nplanes consecutive 64 x 64 planes (row stride `ld` elements inside a
// plane, `pstride` elements between planes) into swizzled shared planes.
template <typename T>
__device__ __forceinline__ void stage_planes(unsigned char* sdst, const T* gsrc, int nplanes, int64_t ld,
                                             int64_t pstride)
{
    constexpr int CPR = TB * (int)sizeof(T) / 16;   // 16-byte chunks per row
    constexpr int PB = TILE_ELEMS * (int)sizeof(T); // bytes per plane
    const int total = nplanes * TB * CPR;
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
        const int pl = q / (TB * CPR), rem = q % (TB * CPR);
        const int row = rem / CPR, ch = rem % CPR;
        const T* g = gsrc + pl * pstride + row * ld + ch * (16 / (int)sizeof(T));
        cp_async16(sdst + pl * PB + row * TB * (int)sizeof(T) + ((ch ^ (row & 7)) << 4), g);
    }
}

template <typename T>
__device__ __forceinline__ T sm_elem(const unsigned char* plane, int row, int col)
{
    return *reinterpret_cast<const T*>(plane + swz_off(row, col, sizeof(T)));
}

// ---------------------------------------------------------------------------
// Block forward/back substitution with interpolate-on-load tiles.
// ---------------------------------------------------------------------------
struct SolveArgs {
    const void* src;     // Theta [f][tile][p][64x64] or factors [pr][tile][64x64]
    const void* dinv;    // [f][t][i][64x64]
    const void* rhs;     // [f][dp][c] (per fold) or [f][t][dp][c] (per system)
    void* zbuf;          // forward result [f][t][dp][c] (may alias out)
    void* out;           // solution [f][t][dp][c]
    const double* phi;   // [t][p]
    int p, nt, q, t0, tcount, per, rhs_per_system;
    int64_t ntiles, dp, c;
    DevStatus* st;       // PICHOL_ERR_TIMEOUT if a bounded copy wait runs out
};

template <typename T, int LG, int CB, int NP, bool EXACT>
struct SolveCfg {
    static constexpr int VN = Vec16<T>::N;
    static constexpr int ESZ = (int)sizeof(T);
    // the staged solved blocks are read ZVN values at a time: 16 bytes when CB is a
    // multiple of the 16-byte vector, else pairs (CB = 10: no padded columns)
    static constexpr int ZVN = CB % VN == 0 ? VN : (CB % 2 == 0 ? 2 : 1);
    static constexpr int CBP = (CB + ZVN - 1) / ZVN * ZVN;
    static constexpr int NPS = EXACT ? LG : NP;            // coefficient planes per tile
    // rows per thread: two when the accumulators (2 x LG x CBP) fit in registers
    static constexpr int RB = (CBP * ESZ <= 48) ? 2 : 1;
    static constexpr int RPT = TB / RB;                   // row groups (threads per k slice)
    static constexpr int NKQ = 256 / RPT;                 // k slices per half tile: 8 or 4
    static constexpr int KW = (TB / 2) / NKQ;             // k per slice per half tile: 4 or 8
    static constexpr int HPB = (TB / 2) * TB * ESZ;       // bytes of a half plane (32 x 64)
    static constexpr int STAGE_BYTES = NPS * HPB;
    static constexpr int DINV_BYTES = LG * TB * TB * ESZ; // the diagonal inverses reuse the ring
    static constexpr int ZS_BYTES = 2 * LG * (TB / 2) * CBP * ESZ;     // staged solved half blocks
    static constexpr int R_BYTES = 4 * LG * TB * CBP * ESZ;            // 4 reduction slots
    static constexpr bool TMA = std::is_same<T, float>::value;          // fp32 planes arrive by TMA
    // Two stages (one half tile in flight while one is read); a third stage
    // measured slower on the mixed case.  In fp32 the reduction slots live in
    // the ring too, after the inverses (both are used only after the k loop).
    // One-lambda CTAs (a single system per fold, as in the gradient) are few and
    // wait on each copy, so they keep three half tiles in flight instead.
    static constexpr int NSTAGE = (TMA && LG == 1) ? 4 : 2;
    static constexpr int RING_LOOP = NSTAGE * STAGE_BYTES;
    static constexpr int RING_AFTER = DINV_BYTES + (TMA ? R_BYTES : 0);
    static constexpr int PLANE_BYTES = RING_LOOP > RING_AFTER ? RING_LOOP : RING_AFTER;
    static constexpr int R_OFFSET = TMA ? DINV_BYTES : PLANE_BYTES + ZS_BYTES;
    static constexpr int SMEM = PLANE_BYTES + ZS_BYTES + (TMA ? 1024 : R_BYTES);   // fp32: + alignment
    // (one-lambda fp32 CTAs: at most 4 x 6 half planes + staged blocks = 201 KB)
    static constexpr int ZPER = (LG * (TB / 2) * CB + 255) / 256;      // staged values per thread
};

// Copy half of the NPS coefficient planes of one tile into a swizzled stage.
//  forward (cols = true):  columns [32 h, 32 h + 32) of all 64 rows, 32-wide rows
//  backward (cols = false): rows [32 h, 32 h + 32) with all 64 columns
// In both layouts the 16-byte chunks of a row are permuted by XOR with (row & 7).
template <typename T>
__device__ __forceinline__ void stage_half(unsigned char* sdst, const T* gsrc, int nplanes, int h, bool cols)
{
    constexpr int ESZ = (int)sizeof(T);
    constexpr int HPB = (TB / 2) * TB * ESZ;
    if (cols) {
        constexpr int CPR = (TB / 2) * ESZ / 16;      // chunks per 32-wide row
        const int total = nplanes * TB * CPR;
        for (int q = threadIdx.x; q < total; q += 256) {
            const int pl = q / (TB * CPR), rem = q % (TB * CPR);
            const int row = rem / CPR, ch = rem % CPR;
            const T* g = gsrc + (int64_t)pl * TILE_ELEMS + row * TB + h * (TB / 2) + ch * (16 / ESZ);
            cp_async16(sdst + pl * HPB + row * (TB / 2) * ESZ + ((ch ^ (row & 7)) << 4), g);
        }
    } else {
        constexpr int CPR = TB * ESZ / 16;            // chunks per 64-wide row
        const int total = nplanes * (TB / 2) * CPR;
        for (int q = threadIdx.x; q < total; q += 256) {
            const int pl = q / ((TB / 2) * CPR), rem = q % ((TB / 2) * CPR);
            const int row = rem / CPR, ch = rem % CPR;
            const T* g = gsrc + (int64_t)pl * TILE_ELEMS + (h * (TB / 2) + row) * TB + ch * (16 / ESZ);
            cp_async16(sdst + pl * HPB + row * TB * ESZ + ((ch ^ (row & 7)) << 4), g);
        }
    }
}

// Thread layout of k_solve (256 threads, LG systems): with RB rows per thread,
// thread t owns rows {rp + RPT h} (rp = t mod RPT) of the current tile for all
// LG systems and, inside each half tile, the k slice [KW kq, KW kq + KW)
// (kq = t / RPT); the lanes of a warp share one k slice, so the staged
// solved-block values they read are the same (broadcast).  The NKQ k-slice
// partial sums are combined in a fixed order through four shared slots.
template <typename T, int LG, int CB, int NP, bool EXACT>
__global__ void __launch_bounds__(256, 2)
k_solve(SolveArgs a, const __grid_constant__ CUtensorMap tmap)
{
    using C = SolveCfg<T, LG, CB, NP, EXACT>;
    constexpr int VN = C::VN, CBP = C::CBP, NPS = C::NPS, ESZ = C::ESZ, ZVN = C::ZVN;
    using ZV = typename VecN<T, ZVN>::type;
    constexpr int RB = C::RB, RPT = C::RPT, KW = C::KW, HPB = C::HPB, ZPER = C::ZPER;
    constexpr int HT = TB / 2;
    constexpr bool TMA = C::TMA;
    using V = typename Vec16<T>::type;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw;
    if constexpr (TMA) smem += (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;   // 128-byte swizzle atoms
    __shared__ uint64_t tbar[C::NSTAGE];
    uint32_t phase = 0;                 // bit s: parity of the next completion of stage s
    unsigned char* planes = smem;
    constexpr int NSTAGE = C::NSTAGE;
    T* Zs = reinterpret_cast<T*>(smem + C::PLANE_BYTES);              // [2][LG][32][CBP]
    T* Rs = reinterpret_cast<T*>(smem + C::R_OFFSET);                 // [4][LG][64][CBP]

    const int f = blockIdx.y, tid = threadIdx.x;
    const int rp = tid % RPT, kq = tid / RPT;
    const int64_t c = a.c, dp = a.dp;
    int tl[LG];
    bool live[LG];
#pragma unroll
    for (int l = 0; l < LG; ++l) {
        const int li = blockIdx.x * LG + l;
        live[l] = li < a.tcount;
        tl[l] = a.t0 + (live[l] ? li : a.tcount - 1);
    }
    // basis weights; phi_0 = 1 for both bases, so the evaluation starts at Theta_0
    T w[LG][NP > 1 ? NP : 1];
    if constexpr (!EXACT) {
#pragma unroll
        for (int l = 0; l < LG; ++l)
#pragma unroll
            for (int m = 0; m < NP; ++m) w[l][m] = (T)a.phi[(int64_t)tl[l] * a.p + m];
    }
    const T* src = (const T*)a.src;
    const T* dinv = (const T*)a.dinv;
    const T* rhs = (const T*)a.rhs;
    T* zb = (T*)a.zbuf;
    T* out = (T*)a.out;
    for (int e = tid; e < 2 * LG * HT * CBP; e += 256) Zs[e] = T(0);
    // (every reduction slot is written before it is read, so Rs needs no clearing)
    if (TMA && tid == 0) {
        for (int st = 0; st < NSTAGE; ++st) mbar_init(&tbar[st], 1);
        mbar_init_fence();
    }
    __syncthreads();

    auto sys_base = [&](int l) -> int64_t { return ((int64_t)f * a.q + tl[l]) * dp * c; };
    // the staged values of this thread: system l, row kk of the half block, output o
    int64_t zg[ZPER];
    int zs_off[ZPER];
#pragma unroll
    for (int u = 0; u < ZPER; ++u) {
        const int e = tid + 256 * u;
        if (e < LG * HT * (int)c) {
            const int l = e / (HT * (int)c), rem = e % (HT * (int)c);
            zg[u] = sys_base(l) + rem;
            zs_off[u] = (l * HT + rem / (int)c) * CBP + rem % (int)c;
        } else {
            zg[u] = -1;
            zs_off[u] = 0;
        }
    }
    auto tile_src = [&](int I, int J, int l) -> const T* {
        const int64_t tix = tile_index(I, J);
        if constexpr (EXACT) {
            const int pr = f * a.per + (tl[l] - a.t0);
            return src + ((int64_t)pr * a.ntiles + tix) * TILE_ELEMS;
        } else {
            return src + ((int64_t)f * a.ntiles + tix) * a.p * TILE_ELEMS;
        }
    };
    auto issue = [&](int I, int J, int h, bool cols, int stage) {
        unsigned char* dst = planes + stage * C::STAGE_BYTES;
        if constexpr (TMA) {
            if (tid == 0) {
                const int64_t tix = tile_index(I, J);
                tma_stage_half<NPS>(dst, &tmap, &tbar[stage], h, cols, [&](int pl) -> int {
                    if constexpr (EXACT)
                        return (int)(((int64_t)(f * a.per + (tl[pl] - a.t0)) * a.ntiles + tix) * TB);
                    else
                        return (int)((((int64_t)f * a.ntiles + tix) * a.p + pl) * TB);
                });
            }
        } else {
            if constexpr (EXACT) {
#pragma unroll
                for (int l = 0; l < LG; ++l) stage_half<T>(dst + l * HPB, tile_src(I, J, l), 1, h, cols);
            } else {
                stage_half<T>(dst, tile_src(I, J, 0), NPS, h, cols);
            }
            cp_async_commit();
        }
    };
    // a bounded copy wait ran out at half tile `it`: latch, wait (bounded) for
    // this CTA's copies still in flight (half tiles it .. it + NSTAGE - 2), and
    // let every thread return
    auto give_up = [&](int it, int nit) {
        if (tid == 0) {
            latch_error(a.st, PICHOL_ERR_TIMEOUT, f, (int)blockIdx.x, -1);
            for (int u = it; u < it + NSTAGE - 1 && u < nit; ++u) {
                const int st = u % NSTAGE;
                mbar_wait(&tbar[st], (phase >> st) & 1u);
            }
        }
    };
    auto evalv = [&](const T* v, int l) -> T {
        if constexpr (EXACT) {
            return v[l];
        } else {
            T sacc = v[0];
#pragma unroll
            for (int m = 1; m < NP; ++m) sacc = fma(w[l][m], v[m], sacc);
            return sacc;
        }
    };

    // fp32: accumulators in column pairs, updated by packed FMAs (each column's sum
    // keeps its order, so the results are those of scalar FMAs)
    constexpr bool PAIRED = std::is_same<T, float>::value && ZVN >= 2;
    constexpr int NACC = PAIRED ? CBP / 2 : CBP;
    using AccT = typename std::conditional<PAIRED, unsigned long long, T>::type;
    AccT acc[RB][LG][NACC];
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
        const bool back = pass == 1;
        const T* zsrc = back ? out : zb;   // solved blocks read during the j loop
#pragma unroll 1
        for (int step = 0; step < a.nt; ++step) {
            const int i = back ? a.nt - 1 - step : step;
            const int nj = back ? a.nt - 1 - i : i;       // off-diagonal tiles in this row
            const int nit = 2 * nj;                       // half tiles
#pragma unroll
            for (int hh = 0; hh < RB; ++hh)
#pragma unroll
                for (int l = 0; l < LG; ++l)
#pragma unroll
                    for (int o = 0; o < NACC; ++o) acc[hh][l][o] = AccT(0);
            auto tj = [&](int it) { return back ? i + 1 + (it >> 1) : (it >> 1); };
            T zr[ZPER];
            auto load_z = [&](int it) {
                const int64_t blk = ((int64_t)tj(it) * TB + (it & 1) * HT) * c;
#pragma unroll
                for (int u = 0; u < ZPER; ++u) zr[u] = (zg[u] >= 0) ? zsrc[zg[u] + blk] : T(0);
            };
            auto store_z = [&](int buf) {
                T* zsb = Zs + buf * LG * HT * CBP;
#pragma unroll
                for (int u = 0; u < ZPER; ++u)
                    if (zg[u] >= 0) zsb[zs_off[u]] = zr[u];
            };
            if (nit > 0) {
                // TMA: NSTAGE - 1 half tiles in flight ahead of the one being read
                const int pre = TMA ? NSTAGE - 1 : 1;
                for (int u = 0; u < pre && u < nit; ++u)
                    issue(back ? tj(u) : i, back ? i : tj(u), u & 1, !back, u);
                load_z(0);
                store_z(0);
            }
#pragma unroll 1
            for (int it = 0; it < nit; ++it) {
                const int stage = TMA ? it % NSTAGE : it & 1;
                bool ok = true;
                if constexpr (TMA) {
                    // one barrier per half tile: the next stage is refilled after it, when
                    // every thread has finished reading that stage (previous half tile)
                    ok = mbar_wait(&tbar[stage], (phase >> stage) & 1u);
                    fence_proxy_async();
                } else {
                    if (it + 1 < nit) {
                        issue(back ? tj(it + 1) : i, back ? i : tj(it + 1), (it + 1) & 1, !back, (it + 1) & 1);
                        cp_async_wait<1>();
                    } else {
                        cp_async_wait<0>();
                    }
                }
                if (__syncthreads_or(!ok)) {
                    give_up(it, nit);
                    return;
                }
                if constexpr (TMA) {
                    phase ^= 1u << stage;
                    const int nx = it + NSTAGE - 1;
                    if (nx < nit) issue(back ? tj(nx) : i, back ? i : tj(nx), nx & 1, !back, nx % NSTAGE);
                }
                if (it + 1 < nit) load_z(it + 1);
                const unsigned char* pl = planes + stage * C::STAGE_BYTES;
                const T* zs = Zs + (it & 1) * LG * HT * CBP;      // the solved blocks are double-buffered
                if (!back) {
                    // row-owner: rows rp + RPT hh of tile (i, j), local k in [KW kq, KW kq + KW)
#pragma unroll
                    for (int ch = 0; ch < KW / VN; ++ch) {
                        const int kc = (kq * KW) / VN + ch;
                        T v[RB][NPS][VN];
#pragma unroll
                        for (int hh = 0; hh < RB; ++hh) {
                            const int r = rp + RPT * hh;
#pragma unroll
                            for (int m = 0; m < NPS; ++m) {
                                V x = *reinterpret_cast<const V*>(pl + m * HPB + r * HT * ESZ + ((kc ^ (r & 7)) << 4));
                                memcpy(v[hh][m], &x, 16);
                            }
                        }
#pragma unroll
                        for (int e = 0; e < VN; ++e) {
                            const int kk = kc * VN + e;
#pragma unroll
                            for (int l = 0; l < LG; ++l) {
                                T lv[RB];
#pragma unroll
                                for (int hh = 0; hh < RB; ++hh) {
                                    T ve[NPS];
#pragma unroll
                                    for (int m = 0; m < NPS; ++m) ve[m] = v[hh][m][e];
                                    lv[hh] = evalv(ve, l);
                                }
                                const T* zrow = zs + (l * HT + kk) * CBP;
                                if constexpr (PAIRED) {
                                    unsigned long long lb[RB];
#pragma unroll
                                    for (int hh = 0; hh < RB; ++hh) lb[hh] = f32x2_pack(lv[hh], lv[hh]);
#pragma unroll
                                    for (int o = 0; o < CBP; o += ZVN) {
                                        unsigned long long zp[ZVN >= 2 ? ZVN / 2 : 1];
                                        if constexpr (ZVN == 4) {
                                            const ulonglong2 z2 = *reinterpret_cast<const ulonglong2*>(zrow + o);
                                            zp[0] = z2.x;
                                            zp[ZVN / 2 - 1] = z2.y;
                                        } else {
                                            zp[0] = *reinterpret_cast<const unsigned long long*>(zrow + o);
                                        }
#pragma unroll
                                        for (int u = 0; u < ZVN / 2; ++u)
#pragma unroll
                                            for (int hh = 0; hh < RB; ++hh)
                                                acc[hh][l][o / 2 + u] = f32x2_fma(lb[hh], zp[u], acc[hh][l][o / 2 + u]);
                                    }
                                } else {
#pragma unroll
                                    for (int o = 0; o < CBP; o += ZVN) {
                                        ZV z4 = *reinterpret_cast<const ZV*>(zrow + o);
                                        T zz[ZVN];
                                        memcpy(zz, &z4, sizeof(ZV));
#pragma unroll
                                        for (int u = 0; u < ZVN; ++u)
#pragma unroll
                                            for (int hh = 0; hh < RB; ++hh)
                                                acc[hh][l][o + u] = fma(lv[hh], zz[u], acc[hh][l][o + u]);
                                    }
                                }
                            }
                        }
                    }
                } else {
                    // column-owner: columns rp + RPT hh of tile (j, i); k = local rows KW kq + e
#pragma unroll
                    for (int e = 0; e < KW; ++e) {
                        const int kk = kq * KW + e;
                        T lv[RB][LG];
#pragma unroll
                        for (int hh = 0; hh < RB; ++hh) {
                            const int col = rp + RPT * hh;
                            const int coff = TMA ? rowhalf_off_f32(kk, col)
                                                 : kk * TB * ESZ + ((((col * ESZ) >> 4) ^ (kk & 7)) << 4) +
                                                       ((col * ESZ) & 15);
                            T ve[NPS];
#pragma unroll
                            for (int m = 0; m < NPS; ++m) ve[m] = *reinterpret_cast<const T*>(pl + m * HPB + coff);
#pragma unroll
                            for (int l = 0; l < LG; ++l) lv[hh][l] = evalv(ve, l);
                        }
#pragma unroll
                        for (int l = 0; l < LG; ++l) {
                            const T* zrow = zs + (l * HT + kk) * CBP;
                            if constexpr (PAIRED) {
                                unsigned long long lb[RB];
#pragma unroll
                                for (int hh = 0; hh < RB; ++hh) lb[hh] = f32x2_pack(lv[hh][l], lv[hh][l]);
#pragma unroll
                                for (int o = 0; o < CBP; o += ZVN) {
                                    unsigned long long zp[ZVN >= 2 ? ZVN / 2 : 1];
                                    if constexpr (ZVN == 4) {
                                        const ulonglong2 z2 = *reinterpret_cast<const ulonglong2*>(zrow + o);
                                        zp[0] = z2.x;
                                        zp[ZVN / 2 - 1] = z2.y;
                                    } else {
                                        zp[0] = *reinterpret_cast<const unsigned long long*>(zrow + o);
                                    }
#pragma unroll
                                    for (int u = 0; u < ZVN / 2; ++u)
#pragma unroll
                                        for (int hh = 0; hh < RB; ++hh)
                                            acc[hh][l][o / 2 + u] = f32x2_fma(lb[hh], zp[u], acc[hh][l][o / 2 + u]);
                                }
                            } else {
#pragma unroll
                                for (int o = 0; o < CBP; o += ZVN) {
                                    ZV z4 = *reinterpret_cast<const ZV*>(zrow + o);
                                    T zz[ZVN];
                                    memcpy(zz, &z4, sizeof(ZV));
#pragma unroll
                                    for (int u = 0; u < ZVN; ++u)
#pragma unroll
                                        for (int hh = 0; hh < RB; ++hh)
                                            acc[hh][l][o + u] = fma(lv[hh][l], zz[u], acc[hh][l][o + u]);
                                }
                            }
                        }
                    }
                }
                if (it + 1 < nit) store_z((it + 1) & 1);
                if constexpr (!TMA) __syncthreads();
            }
            // stage the LG diagonal inverses (the ring is free once every thread has
            // finished the last half tile) while the k-slice partial sums are combined
            if constexpr (TMA) __syncthreads();
#pragma unroll
            for (int l = 0; l < LG; ++l)
                stage_planes<T>(planes + l * TB * TB * ESZ,
                                dinv + (((int64_t)f * a.q + tl[l]) * a.nt + i) * TILE_ELEMS, 1, TB, TILE_ELEMS);
            cp_async_commit();
            // combine the k slices: slot s = kq & 3; with eight slices the upper four
            // write first and the lower four add (slot s = a[s + 4] + a[s]); the four
            // slots are then summed in order
            constexpr int ROUNDS = C::NKQ / 4;
#pragma unroll 1
            for (int round = 0; round < ROUNDS; ++round) {
                if ((kq >> 2) == ROUNDS - 1 - round) {
                    T* slot = Rs + (kq & 3) * LG * TB * CBP;
#pragma unroll
                    for (int hh = 0; hh < RB; ++hh)
#pragma unroll
                        for (int l = 0; l < LG; ++l)
#pragma unroll
                            for (int o = 0; o < CBP; ++o) {
                                T* dst = slot + (l * TB + rp + RPT * hh) * CBP + o;
                                T av;
                                if constexpr (PAIRED) {
                                    const float2 pr = f32x2_unpack(acc[hh][l][o >> 1]);
                                    av = (o & 1) ? pr.y : pr.x;
                                } else {
                                    av = acc[hh][l][o];
                                }
                                *dst = (round == 0) ? av : *dst + av;
                            }
                }
                __syncthreads();
            }
            // right-hand side of the diagonal solve (threads 0 .. LG*64-1: row rr, system l),
            // written into slot 0
            if (tid < LG * TB) {
                const int l = tid >> 6, rr = tid & 63;
#pragma unroll
                for (int o = 0; o < CBP; ++o) {
                    if (o < c) {
                        const int64_t row = (int64_t)i * TB + rr;
                        T b;
                        if (back) b = zb[sys_base(l) + row * c + o];
                        else if (a.rhs_per_system) b = rhs[sys_base(l) + row * c + o];
                        else b = rhs[(int64_t)f * dp * c + row * c + o];
                        const int idx = (l * TB + rr) * CBP + o;
                        const int sl = LG * TB * CBP;
                        const T sum = ((Rs[idx] + Rs[sl + idx]) + Rs[2 * sl + idx]) + Rs[3 * sl + idx];
                        Rs[idx] = b - sum;
                    }
                }
            }
            cp_async_wait<0>();
            __syncthreads();
            if (tid < LG * TB) {
                const int l = tid >> 6, rr = tid & 63;
                T x[CBP];
#pragma unroll
                for (int o = 0; o < CBP; ++o) x[o] = T(0);
                const unsigned char* pl = planes + l * TB * TB * ESZ;
                const T* rsl = Rs + l * TB * CBP;
                if (!back) {
#pragma unroll 2
                    for (int kc = 0; kc < TB / VN; ++kc) {
                        V dv4 = *reinterpret_cast<const V*>(pl + rr * TB * ESZ + ((kc ^ (rr & 7)) << 4));
                        T dv[VN];
                        memcpy(dv, &dv4, 16);
#pragma unroll
                        for (int e = 0; e < VN; ++e) {
                            const T* zrow = rsl + (kc * VN + e) * CBP;
#pragma unroll
                            for (int o = 0; o < CBP; ++o) x[o] = fma(dv[e], zrow[o], x[o]);
                        }
                    }
                } else {
#pragma unroll 2
                    for (int kk = 0; kk < TB; ++kk) {
                        const T dv = sm_elem<T>(pl, kk, rr);
                        const T* zrow = rsl + kk * CBP;
#pragma unroll
                        for (int o = 0; o < CBP; ++o) x[o] = fma(dv, zrow[o], x[o]);
                    }
                }
                if (live[l]) {
                    T* dstb = (back ? out : zb) + sys_base(l) + ((int64_t)i * TB + rr) * c;
#pragma unroll
                    for (int o = 0; o < CBP; ++o)
                        if (o < c) dstb[o] = x[o];
                }
            }
            if constexpr (TMA) fence_proxy_async();   // the inverses' ring before the next TMA fill
            __syncthreads();
        }
    }
}

// output columns a solve CTA carries for c outputs
inline int pick_cb(int64_t c) { return c <= 4 ? 4 : (c == 9 || c == 10 ? 10 : (c <= 12 ? 12 : 32)); }

// fp32 plane map (rows of 64 elements, 32 x 32 boxes, 128-byte swizzle) over
// `planes` 64 x 64 planes starting at buf
cudaError_t plane_map(CUtensorMap* m, const void* buf, int64_t planes);
// pass 0: (uhi, ulo) = L~^T W; pass 1: R = B - L~ u, for systems t0 .. t0 + tcount - 1
cudaError_t launch_resid_pass(pichol_ctx* ctx, const ResidArgs& ra, int pass, cudaStream_t s);

template <typename T, int LG, int CB, int NP, bool EXACT>
inline cudaError_t run_solve(pichol_ctx* ctx, const SolveArgs& sa, cudaStream_t s)
{
    using C = SolveCfg<T, LG, CB, NP, EXACT>;
    static std::atomic<unsigned long long> set{0};
    {
        const cudaError_t e = smem_limit_once(k_solve<T, LG, CB, NP, EXACT>, C::SMEM, set);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)((sa.tcount + LG - 1) / LG), ctx->cfg.k);
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    if constexpr (C::TMA) {
        const int64_t planes = EXACT ? ctx->nfac * ctx->ntiles : (int64_t)ctx->cfg.k * ctx->ntiles * ctx->p;
        cudaError_t e = plane_map(&map, sa.src, planes);
        if (e != cudaSuccess) return e;
    }
    {
        StageScope sc_(ctx, ST_SOLVE, s);
        k_solve<T, LG, CB, NP, EXACT><<<grid, 256, C::SMEM, s>>>(sa, map);
    }
    ctx->launches++;
    return cudaGetLastError();
}

template <typename T, int LG, int CB, bool EXACT>
inline cudaError_t solve_np(pichol_ctx* ctx, const SolveArgs& sa, cudaStream_t s)
{
    if (EXACT) return run_solve<T, LG, CB, 1, EXACT>(ctx, sa, s);
    switch (ctx->p) {
    case 1: return run_solve<T, LG, CB, 1, EXACT>(ctx, sa, s);
    case 2: return run_solve<T, LG, CB, 2, EXACT>(ctx, sa, s);
    case 3: return run_solve<T, LG, CB, 3, EXACT>(ctx, sa, s);
    case 4: return run_solve<T, LG, CB, 4, EXACT>(ctx, sa, s);
    case 5: return run_solve<T, LG, CB, 5, EXACT>(ctx, sa, s);
    case 6: return run_solve<T, LG, CB, 6, EXACT>(ctx, sa, s);
    default: return cudaErrorInvalidValue;
    }
}

// the solves of a few systems with one-lambda CTAs (exact: factor tiles)
cudaError_t launch_solve_single(pichol_ctx* ctx, const SolveArgs& sa, bool exact, cudaStream_t s);
// few systems as a wavefront over tile rows (solve_wave.cu); cudaErrorNotSupported
// where it does not apply
cudaError_t launch_solve_wave(pichol_ctx* ctx, const SolveArgs& sa, bool exact, cudaStream_t s);

}  // namespace pichol
