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
//   k_resid    : refinement residual r = B - L~ (L~^T W) with double-float
//                accumulation (error-free products, compensated sums).
//   k_score    : E partials <W_I, (G_f W)_I> - 2 <Bv_I, W_I> per tile row.
//   k_select   : E_f(t), mean over folds, first argmin.
#include "internal.cuh"
#include "tma.cuh"

#include <algorithm>
#include <cfloat>
#include <cstring>

namespace pichol {

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int N = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int N = 2; };


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

template <typename T, bool EXACT>
__global__ void __launch_bounds__(128)
k_diag_inv(DiagArgs a)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    T (*Ls)[TB + 1] = reinterpret_cast<T (*)[TB + 1]>(dsm);
    T (*Xs)[TB + 1] = reinterpret_cast<T (*)[TB + 1]>(dsm + sizeof(T) * TB * (TB + 1));
    __shared__ float rmax[TB], rmin[TB];
    __shared__ int rbad[TB];
    __shared__ T rinv[TB];
    const int i = blockIdx.x, t = a.t0 + blockIdx.y, f = blockIdx.z, tid = threadIdx.x;
    const int64_t ti = tile_index(i, i);
    T w[MAX_P];
    const int np = EXACT ? 1 : a.p;
    if constexpr (!EXACT) {
        for (int m = 0; m < a.p; ++m) w[m] = (T)a.phi[(int64_t)t * a.p + m];
    }
    const T* base;
    if constexpr (EXACT) {
        const int pr = f * a.per + (t - a.t0);
        base = (const T*)a.src + ((int64_t)pr * a.ntiles + ti) * TILE_ELEMS;
    } else {
        base = (const T*)a.src + ((int64_t)f * a.ntiles + ti) * a.p * TILE_ELEMS;
    }
    for (int e = tid; e < TILE_ELEMS; e += 128) {
        const int r = e / TB, c = e % TB;
        T v;
        if constexpr (EXACT) {
            v = base[e];
        } else {
            // phi_0 = 1 for both bases: start at Theta_0, then FMAs in m (the solve's order)
            v = base[e];
            for (int m = 1; m < np; ++m) v = fma(w[m], base[(int64_t)m * TILE_ELEMS + e], v);
        }
        Ls[r][c] = (c <= r) ? v : T(0);
        Xs[r][c] = T(0);
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
    if (tid < TB) {
        // inverse column c = tid by forward substitution on e_c:
        //   X[r][c] = -(sum_{c <= q < r} L[r][q] X[q][c]) / L[r][r],
        // each sum as two interleaved partial sums (even and odd q)
        const int c = tid;
        Xs[c][c] = rinv[c];
        for (int r = c + 1; r < TB; ++r) {
            T s0 = T(0), s1 = T(0);
            int qq = c;
            for (; qq + 1 < r; qq += 2) {
                s0 = fma(Ls[r][qq], Xs[qq][c], s0);
                s1 = fma(Ls[r][qq + 1], Xs[qq + 1][c], s1);
            }
            if (qq < r) s0 = fma(Ls[r][qq], Xs[qq][c], s0);
            Xs[r][c] = -(s0 + s1) * rinv[r];
        }
    }
    __syncthreads();
    T* out = (T*)a.dinv + (((int64_t)f * a.q + t) * a.nt + i) * TILE_ELEMS;
    for (int e = tid; e < TILE_ELEMS; e += 128) out[e] = Xs[e / TB][e % TB];
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
    static constexpr int CBP = (CB + VN - 1) / VN * VN;
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
    static constexpr int NSTAGE = 2;
    static constexpr int RING_LOOP = NSTAGE * STAGE_BYTES;
    static constexpr int RING_AFTER = DINV_BYTES + (TMA ? R_BYTES : 0);
    static constexpr int PLANE_BYTES = RING_LOOP > RING_AFTER ? RING_LOOP : RING_AFTER;
    static constexpr int R_OFFSET = TMA ? DINV_BYTES : PLANE_BYTES + ZS_BYTES;
    static constexpr int SMEM = PLANE_BYTES + ZS_BYTES + (TMA ? 1024 : R_BYTES);   // fp32: + alignment
    static constexpr int ZPER = (LG * (TB / 2) * CB + 255) / 256;      // staged values per thread
};

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
    constexpr int VN = C::VN, CBP = C::CBP, NPS = C::NPS, ESZ = C::ESZ;
    constexpr int RB = C::RB, RPT = C::RPT, KW = C::KW, HPB = C::HPB, ZPER = C::ZPER;
    constexpr int HT = TB / 2;
    constexpr bool TMA = C::TMA;
    using V = typename Vec16<T>::type;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw;
    if constexpr (TMA) smem += (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;   // 128-byte swizzle atoms
    __shared__ uint64_t tbar[3];
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

    T acc[RB][LG][CBP];
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
                    for (int o = 0; o < CBP; ++o) acc[hh][l][o] = T(0);
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
#pragma unroll
                                for (int o = 0; o < CBP; o += VN) {
                                    V z4 = *reinterpret_cast<const V*>(zrow + o);
                                    T zz[VN];
                                    memcpy(zz, &z4, 16);
#pragma unroll
                                    for (int u = 0; u < VN; ++u)
#pragma unroll
                                        for (int hh = 0; hh < RB; ++hh)
                                            acc[hh][l][o + u] = fma(lv[hh], zz[u], acc[hh][l][o + u]);
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
#pragma unroll
                            for (int o = 0; o < CBP; o += VN) {
                                V z4 = *reinterpret_cast<const V*>(zrow + o);
                                T zz[VN];
                                memcpy(zz, &z4, 16);
#pragma unroll
                                for (int u = 0; u < VN; ++u)
#pragma unroll
                                    for (int hh = 0; hh < RB; ++hh)
                                        acc[hh][l][o + u] = fma(lv[hh][l], zz[u], acc[hh][l][o + u]);
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
                                *dst = (round == 0) ? acc[hh][l][o] : *dst + acc[hh][l][o];
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

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// n consecutive fp32 values of shared memory in 16- or 8-byte loads when n
// allows (the row start is then aligned to match).
template <int N>
__device__ __forceinline__ void load_row(float (&dst)[N], const float* src)
{
    if constexpr (N % 4 == 0) {
#pragma unroll
        for (int o = 0; o < N; o += 4) {
            const float4 t = *reinterpret_cast<const float4*>(src + o);
            dst[o] = t.x; dst[o + 1] = t.y; dst[o + 2] = t.z; dst[o + 3] = t.w;
        }
    } else if constexpr (N % 2 == 0) {
#pragma unroll
        for (int o = 0; o < N; o += 2) {
            const float2 t = *reinterpret_cast<const float2*>(src + o);
            dst[o] = t.x; dst[o + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int o = 0; o < N; ++o) dst[o] = src[o];
    }
}

template <int LG, int CB, int NP, int PASS>
__global__ void __launch_bounds__(256, 2)
k_resid(ResidArgs a, const __grid_constant__ CUtensorMap tmap)
{
    constexpr int CBP = CB;                     // exact column count (no vector loads of Z here)
    constexpr int HT = TB / 2;
    constexpr int HPB = HT * TB * 4;            // half plane, fp32
    constexpr int STAGE = NP * HPB;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    __shared__ uint64_t tbar[2];
    uint32_t phase = 0;                         // bit s: parity of the next completion of stage s
    unsigned char* planes = smem;                                          // 2 stages (TMA)
    float* Zh = reinterpret_cast<float*>(smem + 2 * STAGE);                // [2][LG][32][CBP]
    float* Zl = Zh + 2 * LG * HT * CBP;                                    // [2][LG][32][CBP]
    double* Rd = reinterpret_cast<double*>(Zl + 2 * LG * HT * CBP);       // [LG][64][CBP]
    const int i = blockIdx.x, f = blockIdx.z, tid = threadIdx.x;
    const int r = tid & 63, kq = tid >> 6;      // row (PASS 1) / column (PASS 0) r, k slice [8 kq, 8 kq + 8)
    const int64_t c = a.c, dp = a.dp;
    int tl[LG];
    bool live[LG];
#pragma unroll
    for (int l = 0; l < LG; ++l) {
        const int li = blockIdx.y * LG + l;
        live[l] = li < a.tcount;
        tl[l] = a.t0 + (live[l] ? li : a.tcount - 1);
    }
    float w[LG][NP];
#pragma unroll
    for (int l = 0; l < LG; ++l)
#pragma unroll
        for (int m = 0; m < NP; ++m) w[l][m] = (float)a.phi[(int64_t)tl[l] * a.p + m];
    float sh[LG][CBP], sl[LG][CBP];
#pragma unroll
    for (int l = 0; l < LG; ++l)
#pragma unroll
        for (int o = 0; o < CBP; ++o) { sh[l][o] = 0.0f; sl[l][o] = 0.0f; }
    for (int e = tid; e < 2 * 2 * LG * HT * CBP; e += 256) Zh[e] = 0.0f;   // Zh and Zl, both buffers
    if (tid == 0) {
        mbar_init(&tbar[0], 1);
        mbar_init(&tbar[1], 1);
        mbar_init_fence();
    }
    __syncthreads();
    // staged values of this thread (precomputed offsets): system l, row kk, output o
    constexpr int ZPER = (LG * HT * CB + 255) / 256;
    int64_t zg[ZPER];
    int zoff[ZPER];
#pragma unroll
    for (int u = 0; u < ZPER; ++u) {
        const int e = tid + 256 * u;
        if (e < LG * HT * (int)c) {
            const int l = e / (HT * (int)c), rem = e % (HT * (int)c);
            zg[u] = ((int64_t)f * a.q + tl[l]) * dp * c + rem;
            zoff[u] = (l * HT + rem / (int)c) * CBP + rem % (int)c;
        } else {
            zg[u] = -1;
            zoff[u] = 0;
        }
    }
    const int jlo = PASS == 0 ? i : 0, jhi = PASS == 0 ? a.nt - 1 : i;
    const int nit = 2 * (jhi - jlo + 1);
    auto issue = [&](int it) {
        const int j = jlo + (it >> 1), h = it & 1;
        const int64_t tix = PASS == 0 ? tile_index(j, i) : tile_index(i, j);
        // PASS 0 reads columns r of tile (j, i): its k are the tile's rows (half = rows);
        // PASS 1 reads rows r of tile (i, j): its k are the tile's columns (half = columns)
        if (tid == 0)
            tma_stage_half<NP>(planes + (it & 1) * STAGE, &tmap, &tbar[it & 1], h, PASS == 1, [&](int pl) -> int {
                return (int)((((int64_t)f * a.ntiles + tix) * a.p + pl) * TB);
            });
    };
    float zr[2][ZPER];
    auto load_z = [&](int it) {
        const int j = jlo + (it >> 1), h = it & 1;
        const int64_t blk = ((int64_t)j * TB + h * HT) * c;
#pragma unroll
        for (int u = 0; u < ZPER; ++u) {
            if (zg[u] >= 0) {
                if (PASS == 0) {
                    zr[0][u] = a.W[zg[u] + blk];
                } else {
                    zr[0][u] = a.uhi[zg[u] + blk];
                    zr[1][u] = a.ulo[zg[u] + blk];
                }
            }
        }
    };
    auto store_z = [&](int buf) {
#pragma unroll
        for (int u = 0; u < ZPER; ++u) {
            if (zg[u] >= 0) {
                Zh[buf * LG * HT * CBP + zoff[u]] = zr[0][u];
                Zl[buf * LG * HT * CBP + zoff[u]] = (PASS == 1) ? zr[1][u] : 0.0f;
            }
        }
    };
    issue(0);
    load_z(0);
    store_z(0);
#pragma unroll 1
    for (int it = 0; it < nit; ++it) {
        const int stage = it & 1;
        // one barrier per half tile: the next stage is refilled after it, when every
        // thread has finished reading that stage (previous half tile)
        const bool ok = mbar_wait(&tbar[stage], (phase >> stage) & 1u);
        fence_proxy_async();
        if (__syncthreads_or(!ok)) {
            // a bounded copy wait ran out: latch, wait (bounded) for the copy still
            // in flight, and let every thread return
            if (tid == 0) {
                latch_error(a.st, PICHOL_ERR_TIMEOUT, f, (int)blockIdx.x, -1);
                mbar_wait(&tbar[stage], (phase >> stage) & 1u);
            }
            return;
        }
        phase ^= 1u << stage;
        if (it + 1 < nit) issue(it + 1);
        if (it + 1 < nit) load_z(it + 1);
        const unsigned char* pl = planes + (it & 1) * STAGE;
        const float* zhb = Zh + (it & 1) * LG * HT * CBP;
        const float* zlb = Zl + (it & 1) * LG * HT * CBP;
#pragma unroll 1
        for (int ch = 0; ch < 2; ++ch) {
            float v4[NP][4];
            const int k0 = kq * 8 + ch * 4;     // local k (0..31) of the half
#pragma unroll
            for (int m = 0; m < NP; ++m) {
                if (PASS == 0) {
                    // column r of the staged rows k0..k0+3 (two 32-column boxes)
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        v4[m][e] = *reinterpret_cast<const float*>(pl + m * HPB + rowhalf_off_f32(k0 + e, r));
                } else {
                    // row r, columns k0..k0+3 of the staged 32-wide rows: one 16-byte chunk
                    const int kc = k0 >> 2;
                    float4 x = *reinterpret_cast<const float4*>(pl + m * HPB + r * HT * 4 + ((kc ^ (r & 7)) << 4));
                    v4[m][0] = x.x; v4[m][1] = x.y; v4[m][2] = x.z; v4[m][3] = x.w;
                }
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int kk = k0 + e;
#pragma unroll
                for (int l = 0; l < LG; ++l) {
                    // same evaluation as the solve: phi_0 = 1, then FMAs in m
                    float lv = v4[0][e];
#pragma unroll
                    for (int m = 1; m < NP; ++m) lv = fmaf(w[l][m], v4[m][e], lv);
                    // the staged values of row kk (rows are 8- or 16-byte aligned when CBP is even)
                    float zh[CBP], zl[CBP];
                    load_row<CBP>(zh, zhb + (l * HT + kk) * CBP);
                    if (PASS == 1) load_row<CBP>(zl, zlb + (l * HT + kk) * CBP);
#pragma unroll
                    for (int o = 0; o < CBP; ++o) {
                        const float pp = lv * zh[o];
                        const float pe = fmaf(lv, zh[o], -pp);
                        float s2, e2;
                        two_sum(sh[l][o], pp, s2, e2);
                        sh[l][o] = s2;
                        sl[l][o] += e2 + pe + (PASS == 1 ? lv * zl[o] : 0.0f);
                    }
                }
            }
        }
        if (it + 1 < nit) store_z((it + 1) & 1);
    }
    // combine the four k slices in double
#pragma unroll 1
    for (int qq = 3; qq >= 0; --qq) {
        if (kq == qq) {
#pragma unroll
            for (int l = 0; l < LG; ++l)
#pragma unroll
                for (int o = 0; o < CBP; ++o) {
                    const double v = (double)sh[l][o] + (double)sl[l][o];
                    double* dst = Rd + (l * TB + r) * CBP + o;
                    *dst = (qq == 3) ? v : *dst + v;
                }
        }
        __syncthreads();
    }
    for (int e = tid; e < LG * TB * c; e += 256) {
        const int l = e / (TB * (int)c), rem = e % (TB * (int)c);
        if (!live[l]) continue;
        const int rr = rem / (int)c, o = rem % (int)c;
        const double v = Rd[(l * TB + rr) * CBP + o];
        const int64_t g = ((int64_t)f * a.q + tl[l]) * dp * c + (int64_t)i * TB * c + rem;
        if (PASS == 0) {
            const float hi = (float)v;
            a.ohi[g] = hi;
            a.olo[g] = (float)(v - (double)hi);
        } else {
            const double b = (double)a.B[(int64_t)f * dp * c + (int64_t)i * TB * c + rem];
            a.R[g] = (float)(b - v);
        }
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
static int pick_cb(int64_t c) { return c <= 4 ? 4 : (c <= 12 ? 12 : 32); }

// Dynamic shared memory the solve kernel needs for a mode (element bytes eb),
// p coefficient planes and c outputs; mirrors SolveCfg.
size_t solve_smem_bytes(int eb, int p, int64_t c)
{
    const int LG = 2, cb = pick_cb(c), vn = 16 / eb;
    const int cbp = (cb + vn - 1) / vn * vn;
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
static cudaError_t plane_map(CUtensorMap* m, const void* buf, int64_t planes)
{
    const int64_t rows = planes * TB;
    if (rows > INT32_MAX) return cudaErrorInvalidValue;   // TMA coordinates are 32-bit
    return make_map_f32(m, (const float*)buf, TB, (uint64_t)rows, TB, 32, 32) ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename T, int LG, int CB, int NP, bool EXACT>
static cudaError_t run_solve(pichol_ctx* ctx, const SolveArgs& sa, cudaStream_t s)
{
    using C = SolveCfg<T, LG, CB, NP, EXACT>;
    static bool done = false;
    if (!done) {
        cudaError_t e = cudaFuncSetAttribute(k_solve<T, LG, CB, NP, EXACT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e != cudaSuccess) return e;
        done = true;
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
static cudaError_t solve_np(pichol_ctx* ctx, const SolveArgs& sa, cudaStream_t s)
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

template <typename T, bool EXACT>
static cudaError_t solve_dispatch(pichol_ctx* ctx, const SolveArgs& sa, cudaStream_t s)
{
    constexpr int LG = 2;
    switch (pick_cb(ctx->cfg.c)) {
    case 4: return solve_np<T, LG, 4, EXACT>(ctx, sa, s);
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
    static bool done = false;
    if (!done) {
        cudaError_t e = cudaFuncSetAttribute(k_score<T, LG, CB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        done = true;
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
    case 12: return run_score<T, 2, 12>(ctx, sc, s);
    default: return run_score<T, 1, 32>(ctx, sc, s);
    }
}

template <int LG, int CB, int NP, int PASS>
static cudaError_t run_resid(pichol_ctx* ctx, const ResidArgs& ra, cudaStream_t s)
{
    const int smem = 2 * NP * (TB / 2) * TB * 4 + 2 * 2 * LG * (TB / 2) * CB * 4 + LG * TB * CB * 8 + 1024;
    static bool done = false;
    if (!done) {
        cudaError_t e = cudaFuncSetAttribute(k_resid<LG, CB, NP, PASS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        done = true;
    }
    CUtensorMap map;
    cudaError_t e = plane_map(&map, ra.theta, (int64_t)ctx->cfg.k * ctx->ntiles * ctx->p);
    if (e != cudaSuccess) return e;
    dim3 grid(ctx->nt, (unsigned)((ra.tcount + LG - 1) / LG), ctx->cfg.k);
    {
        StageScope sc_(ctx, ST_RESID, s);
        k_resid<LG, CB, NP, PASS><<<grid, 256, smem, s>>>(ra, map);
    }
    ctx->launches++;
    return cudaGetLastError();
}

template <int LG, int CB, int PASS>
static cudaError_t resid_np(pichol_ctx* ctx, const ResidArgs& ra, cudaStream_t s)
{
    switch (ctx->p) {
    case 1: return run_resid<LG, CB, 1, PASS>(ctx, ra, s);
    case 2: return run_resid<LG, CB, 2, PASS>(ctx, ra, s);
    case 3: return run_resid<LG, CB, 3, PASS>(ctx, ra, s);
    case 4: return run_resid<LG, CB, 4, PASS>(ctx, ra, s);
    case 5: return run_resid<LG, CB, 5, PASS>(ctx, ra, s);
    case 6: return run_resid<LG, CB, 6, PASS>(ctx, ra, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int PASS>
static cudaError_t resid_dispatch(pichol_ctx* ctx, const ResidArgs& ra, cudaStream_t s)
{
    // the residual reads its staged values one at a time, so it carries exactly
    // the columns it needs: 1, 4, 10, 12 or 32 (a larger count pads with zeros)
    const int64_t c = ctx->cfg.c;
    if (c <= 1) return resid_np<2, 1, PASS>(ctx, ra, s);
    if (c <= 4) return resid_np<2, 4, PASS>(ctx, ra, s);
    if (c <= 10) return resid_np<2, 10, PASS>(ctx, ra, s);
    if (c <= 12) return resid_np<2, 12, PASS>(ctx, ra, s);
    return resid_np<1, 32, PASS>(ctx, ra, s);
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
    const int dsm = 2 * (int)sizeof(T) * TB * (TB + 1);
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t ea = cudaFuncSetAttribute(k_diag_inv<T, EXACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsm);
        if (ea != cudaSuccess) return ea;
        attr_done = true;
    }
    {
        StageScope sc_(ctx, ST_DIAG_INV, s);
        k_diag_inv<T, EXACT><<<dim3(ctx->nt, tcount, cf.k), 128, dsm, s>>>(da);
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
        cudaError_t er = solve_dispatch<T, EXACT>(ctx, sa, st);
        if (er == cudaSuccess && solved) er = cudaEventRecord(solved, st);
        if (er != cudaSuccess) return er;
        if constexpr (std::is_same<T, float>::value && !EXACT) {
            for (int it = 0; it < cf.refine_steps; ++it) {
                // the residual of the system this step refines (see refine_target)
                if (cf.refine_target == PICHOL_REFINE_EXACT) {
                    if ((er = launch_resid_exact(ctx, t0h, tch, st)) != cudaSuccess) return er;
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
                    if ((er = resid_dispatch<0>(ctx, ra, st)) != cudaSuccess) return er;
                    if ((er = resid_dispatch<1>(ctx, ra, st)) != cudaSuccess) return er;
                }
                SolveArgs sc = sa;
                sc.rhs = ctx->Rres;
                sc.rhs_per_system = 1;
                sc.zbuf = ctx->Rres;
                sc.out = ctx->Rres;
                if ((er = solve_dispatch<T, EXACT>(ctx, sc, st)) != cudaSuccess) return er;
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
        const int dsm = 2 * (int)sizeof(T) * TB * (TB + 1);
        cudaError_t ea = cudaFuncSetAttribute(k_diag_inv<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsm);
        if (ea != cudaSuccess) return ea;
        {
            StageScope sc_(ctx, ST_DIAG_INV, s);
            k_diag_inv<T, false><<<dim3(ctx->nt, 1, cf.k), 128, dsm, s>>>(da);
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
