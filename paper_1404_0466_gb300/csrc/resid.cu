// Refinement residual of the interpolated system in double-float arithmetic
// (error-free products and compensated sums on the FP32 pipes), two passes:
//   pass 0: u_i = sum_{j >= i} L~_ji^T W_j      -> (uhi, ulo)
//   pass 1: r_i = B_i - sum_{j <= i} L~_ij u_j  -> R (rounded to float)
// with the coefficient planes of L~ staged by TMA, as in the solve.
#include "internal.cuh"
#include "solve_common.cuh"
#include "tma.cuh"

#include <cstring>

namespace pichol {


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

template <int LG, int CB, int NP, int PASS>
static cudaError_t run_resid(pichol_ctx* ctx, const ResidArgs& ra, cudaStream_t s)
{
    const int smem = 2 * NP * (TB / 2) * TB * 4 + 2 * 2 * LG * (TB / 2) * CB * 4 + LG * TB * CB * 8 + 1024;
    static std::atomic<unsigned long long> set{0};
    {
        const cudaError_t e = smem_limit_once(k_resid<LG, CB, NP, PASS>, smem, set);
        if (e != cudaSuccess) return e;
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

cudaError_t launch_resid_pass(pichol_ctx* ctx, const ResidArgs& ra, int pass, cudaStream_t s)
{
    return pass == 0 ? resid_dispatch<0>(ctx, ra, s) : resid_dispatch<1>(ctx, ra, s);
}

}  // namespace pichol
