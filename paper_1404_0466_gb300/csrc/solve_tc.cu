// Interpolated triangular solves on the tensor cores (mixed mode; Sec. 3.2's
// two substitutions with Sec. 3.3's evaluated polynomials):
//   forward  L~(t) Z(t) = B,      Z_i = Dinv_i(t) (B_i - sum_{j<i} L~_ij(t) Z_j)
//   backward L~(t)^T W(t) = Z,    W_i = Dinv_i(t)^T (Z_i - sum_{j>i} L~_ji(t)^T W_j)
// for every fold f and every lambda t of a call at once.  With
// L~_ij(t) = sum_m phi_m(t) Theta_{m,ij}, the off-diagonal part of a tile row is
// sum_m phi_m(t) [sum_j Theta_{m,ij} Z_j(t)]: one product per coefficient
// plane over all lambdas' columns (N = q c), scaled by phi_m(t) per column
// when the tensor-memory accumulators are drained.  Theta is read once per
// column block instead of once per lambda, and L~ is never formed.
//
// One CTA owns one fold and BN consecutive columns (lambda t = t0 + n / c,
// output o = n mod c) and walks the tile rows two at a time (M = 128):
//   1. warps 0 / 1: TMA + split-TF32 MMAs of the rows' products with the
//      blocks solved so far (read back as S^T, hi / lo, from a scratch buffer
//      this CTA writes), one accumulator per plane, drained every 32 rows of
//      K into compensated totals by warps 2..9;
//   2. warps 2..9: the two diagonal blocks in fp32 through the precomputed
//      inverses Dinv_i(t) (k_diag_inv), with the tile between the two rows
//      evaluated from its planes; the solved rows go to the output and, split,
//      to the scratch for the following rows' products.
// No CTA waits on another.  Every mbarrier wait is bounded; a wait that runs
// out latches PICHOL_ERR_TIMEOUT and the CTA stops, waits (bounded) for its
// copies, frees its tensor memory and returns.
#include "internal.cuh"
#include "tcgen05.cuh"
#include "tma.cuh"

#include <cstring>

namespace pichol {

namespace stc {

constexpr int BM = 128, BK = 32;
constexpr int NA = 5;                          // A ring stages (one coefficient plane, hi + lo)
constexpr int NB = 2;                          // B ring stages (one k-block of S^T, hi + lo)
constexpr int A_BYTES = 2 * BM * BK * 4;       // 32 KB
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 32 * (2 + EPI_WARPS);
constexpr int TMEM_COLS = 512;

template <int BN> struct Cfg {
    static constexpr int B_BYTES = 2 * BN * BK * 4;
    static constexpr int PHI_BYTES = MAX_P * BN * 4;
    // The diagonal steps' buffers live in the A ring: the producer loads nothing for a
    // step before the previous step's solved blocks are published, so the ring is idle
    // from the step's last drain to that point.
    static constexpr int V_BYTES = BM * BN * 4;    // drained products, then the two right-hand sides
    static constexpr int Z_BYTES = TB * BN * 4;    // the first solved block of a pair
    static constexpr int T_BYTES = 2 * TB * (TB + 1) * 4;   // a staged inverse block and the pair's tile
    static_assert(V_BYTES + Z_BYTES + T_BYTES <= NA * A_BYTES, "diagonal-step buffers exceed the A ring");
    static constexpr int SMEM = NA * A_BYTES + NB * B_BYTES + PHI_BYTES + 1024 + 256;
};

}  // namespace stc

struct SolveTcArgs {
    const double* phi;        // [t][p]
    const float* theta;       // [f][tile][m][64 x 64] (tiles between the two rows of a pair)
    const float* dinv;        // [f][t][i][64 x 64]
    const float* rhs;         // forward: [f][dp][c] (per fold) or [f][t][dp][c]; backward: the forward output
    float* out;               // [f][t][dp][c]
    float* Sh;                // scratch [f][q c][dp]: solved blocks transposed, TF32 hi
    float* Sl;                //                                                remainder lo
    int p, nt, q, t0, tcount, rhs_per_system;
    int64_t ntiles, dp, c, qc;
    int zero_row;             // first row of the zero plane in the Theta maps
    DevStatus* st;
};

// Row of the Theta map holding the block that multiplies K tile column j for
// tile row i, plane m: Theta_{ij} (forward, j < i) or Theta_{ji}^T (backward,
// j > i); the zero plane for a row past the last tile row.
template <int DIR>
__device__ __forceinline__ int s_row(const SolveTcArgs& a, int f, int i, int j, int m)
{
    if (i >= a.nt || j >= a.nt) return a.zero_row;
    const int64_t tile = DIR == 0 ? tile_index(i, j) : tile_index(j, i);
    return (int)((((int64_t)f * a.ntiles + tile) * a.p + m) * TB);
}

// Tile rows (i0, i0 + 1) of step s and the K range [jlo, jhi) of their products.
template <int DIR>
__device__ __forceinline__ void s_step(const SolveTcArgs& a, int s, int& i0, int& jlo, int& jhi)
{
    const int nS = (a.nt + 1) / 2;
    const int pr = DIR == 0 ? s : nS - 1 - s;
    i0 = 2 * pr;
    if (DIR == 0) { jlo = 0; jhi = i0; }
    else { jlo = i0 + 2; jhi = a.nt; }
    if (jhi < jlo) jhi = jlo;
}

// Warps 2..9 of k_solve_tc.  Per step: drain the products of tile rows
// (i0, i0 + 1) into V (rows 0..63: i0, 64..127: i0 + 1), then solve the two
// diagonal blocks column by column, thread (r, g) = (row, column group).
template <int DIR, int BN>
__device__ __forceinline__ void k_solve_tc_epilogue(const SolveTcArgs& a, uint32_t tmem, float* Vs, float* Zs,
                                                    float* Ds, float* Ls, const float* phis, uint64_t* tfull, uint64_t* tempty,
                                                    uint64_t* zready, volatile int* abort_flag, int f, int64_t n0,
                                                    int64_t N)
{
    constexpr int HC = BN / 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int qtr = warp & 3, chalf = (warp - 2) >> 2;
    const int et = threadIdx.x - 64;            // 0 .. 255
    const int p = a.p, nS = (a.nt + 1) / 2;
    const int64_t c = a.c, dp = a.dp;
    int cg = 0;
    auto epi_sync = [] { asm volatile("bar.sync 1, 256;\n" ::: "memory"); };
    // element (row rr of tile row i, column n) of the right-hand side and of the solution
    auto in_at_r = [&](int i, int64_t n, int rr) -> float {
        const int64_t t = a.t0 + n / c, o = n % c, row = (int64_t)i * TB + rr;
        if (DIR == 1 || a.rhs_per_system) return a.rhs[(((int64_t)f * a.q + t) * dp + row) * c + o];
        return a.rhs[((int64_t)f * dp + row) * c + o];
    };
    auto put_r = [&](int i, int64_t n, int rr, float v) {
        const int64_t t = a.t0 + n / c, o = n % c, row = (int64_t)i * TB + rr;
        a.out[(((int64_t)f * a.q + t) * dp + row) * c + o] = v;
        const int64_t so = ((int64_t)f * a.qc + (int64_t)a.t0 * c + n) * dp + row;
        const float h = tc5::tf32_round(v);
        a.Sh[so] = h;
        a.Sl[so] = v - h;
    };
    // A 64 x 64 tile is moved global -> registers (four 16-byte loads per thread,
    // all issued before the first use) -> shared rows of 65 (conflict-free column
    // reads), so each staging costs one memory latency.
    auto fetch_tile = [&](float4 (&v)[4], const float* src) {
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = reinterpret_cast<const float4*>(src)[et + 256 * u];
    };
    auto store_tile = [&](float* dst, const float4 (&v)[4]) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = 4 * (et + 256 * u);
            float* d = dst + (e / TB) * (TB + 1) + e % TB;
            d[0] = v[u].x;
            d[1] = v[u].y;
            d[2] = v[u].z;
            d[3] = v[u].w;
        }
    };
    const float* dinv_f = a.dinv + (int64_t)f * a.q * a.nt * TILE_ELEMS;
    auto dinv_at = [&](int t, int i) { return dinv_f + ((int64_t)t * a.nt + i) * TILE_ELEMS; };
    constexpr int PR = 2;                   // planes of the coupling tile kept in registers
    for (int s = 0; s < nS; ++s) {
        int i0, jlo, jhi;
        s_step<DIR>(a, s, i0, jlo, jhi);
        const int i1 = i0 + 1;
        const int nkb = 2 * (jhi - jlo);
        float tot[HC], cmp[HC];
#pragma unroll
        for (int u = 0; u < HC; ++u) { tot[u] = 0.0f; cmp[u] = 0.0f; }
        for (int kb = 0; kb < nkb; ++kb, ++cg) {
            const int b = cg & 1;
            if (!mbar_wait(&tfull[b], (cg >> 1) & 1)) { *abort_flag = 1; break; }
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
        if (*abort_flag) break;
        const bool two = i1 < a.nt;
        const int ia = DIR == 0 ? i0 : (two ? i1 : i0);   // solved first: i0 forward, i0 + 1 backward
        const int va = DIR == 0 ? 0 : (two ? TB : 0);     // its rows in V
        const int ib = DIR == 0 ? i1 : i0, vb = DIR == 0 ? TB : 0;
        // the lambdas of this CTA's columns
        const int64_t nlast = (n0 + BN < N ? n0 + BN : N) - 1;
        const int tfirst = a.t0 + (int)(n0 / c), tlast = a.t0 + (int)(nlast / c);
        // loads in flight during the drain's stores: the first lambda's inverse, and
        // the first PR planes of the tile between the pair's rows (the same for every
        // lambda, held in registers; the others are read per lambda, from L2)
        float4 pa[4], pb[4], thr[PR][4];
        fetch_tile(pa, dinv_at(tfirst, ia));
        const float* th = a.theta + ((int64_t)f * a.ntiles + tile_index(i1 < a.nt ? i1 : i0, i0)) * p * TILE_ELEMS;
        if (two) {
#pragma unroll
            for (int m = 0; m < PR; ++m)
                if (m < p) fetch_tile(thr[m], th + (int64_t)m * TILE_ELEMS);
        }
        // products of the pair's rows, V[row][col]; then R = rhs - V in place
#pragma unroll
        for (int u = 0; u < HC; ++u) Vs[(qtr * 32 + lane) * BN + chalf * HC + u] = tot[u];
        epi_sync();
        // (consecutive threads take consecutive columns: runs of c contiguous values)
        for (int e = et; e < TB * BN; e += 256) {
            const int rr = e / BN, col = e % BN;
            const int64_t n = n0 + col;
            if (n >= N) continue;
            Vs[(va + rr) * BN + col] = in_at_r(ia, n, rr) - Vs[(va + rr) * BN + col];
            if (two) Vs[(vb + rr) * BN + col] = in_at_r(ib, n, rr) - Vs[(vb + rr) * BN + col];
        }
        for (int t = tfirst; t <= tlast; ++t) {
            const int64_t ca = (int64_t)(t - a.t0) * c, cb = ca + c;
            const int cl0 = (int)((ca > n0 ? ca : n0) - n0), cl1 = (int)((cb < n0 + BN ? cb : n0 + BN) - n0);
            const int ncol = cl1 - cl0;
            epi_sync();                                     // Ds / Ls / V rows free, R of all columns ready
            store_tile(Ds, pa);
            if (two) fetch_tile(pb, dinv_at(t, ib));
            epi_sync();
            // Z = Dinv R (forward) or Dinv^T R (backward) for the columns of t
            for (int e = et; e < TB * ncol; e += 256) {
                const int col = cl0 + e / TB, rr = e % TB;
                float acc = 0.0f;
#pragma unroll 16
                for (int k = 0; k < TB; ++k)
                    acc = fmaf(DIR == 0 ? Ds[rr * (TB + 1) + k] : Ds[k * (TB + 1) + rr], Vs[(va + k) * BN + col], acc);
                Zs[rr * BN + col] = acc;
            }
            if (t < tlast) fetch_tile(pa, dinv_at(t + 1, ia));
            if (!two) continue;
            // the other row's R minus the tile between the rows times Z, then its Dinv
            float ph[MAX_P];
            for (int m = 0; m < p; ++m) ph[m] = (float)a.phi[(int64_t)t * p + m];
            float4 lv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                lv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int m = 0; m < PR; ++m)
                    if (m < p) {
                        lv[u].x = fmaf(ph[m], thr[m][u].x, lv[u].x);
                        lv[u].y = fmaf(ph[m], thr[m][u].y, lv[u].y);
                        lv[u].z = fmaf(ph[m], thr[m][u].z, lv[u].z);
                        lv[u].w = fmaf(ph[m], thr[m][u].w, lv[u].w);
                    }
            }
            for (int m = PR; m < p; m += 2) {          // two planes per memory latency
                float4 tv[2][4];
                const int m2 = m + 1 < p ? 2 : 1;
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    if (h < m2) fetch_tile(tv[h], th + (int64_t)(m + h) * TILE_ELEMS);
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    if (h < m2) {
                        const float w = ph[m + h];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            lv[u].x = fmaf(w, tv[h][u].x, lv[u].x);
                            lv[u].y = fmaf(w, tv[h][u].y, lv[u].y);
                            lv[u].z = fmaf(w, tv[h][u].z, lv[u].z);
                            lv[u].w = fmaf(w, tv[h][u].w, lv[u].w);
                        }
                    }
            }
            epi_sync();                                     // Z complete, Ds read
            store_tile(Ls, lv);
            store_tile(Ds, pb);
            epi_sync();
            for (int e = et; e < TB * ncol; e += 256) {
                const int col = cl0 + e / TB, rr = e % TB;
                float acc = Vs[(vb + rr) * BN + col];
#pragma unroll 16
                for (int k = 0; k < TB; ++k)
                    acc = fmaf(-(DIR == 0 ? Ls[rr * (TB + 1) + k] : Ls[k * (TB + 1) + rr]), Zs[k * BN + col], acc);
                Vs[(vb + rr) * BN + col] = acc;
            }
            epi_sync();
            for (int e = et; e < TB * ncol; e += 256) {
                const int col = cl0 + e / TB, rr = e % TB;
                float acc = 0.0f;
#pragma unroll 16
                for (int k = 0; k < TB; ++k)
                    acc = fmaf(DIR == 0 ? Ds[rr * (TB + 1) + k] : Ds[k * (TB + 1) + rr], Vs[(vb + k) * BN + col], acc);
                put_r(ib, n0 + col, rr, acc);
            }
        }
        epi_sync();
        for (int e = et; e < TB * BN; e += 256) {
            const int col = e / TB, rr = e % TB;
            if (n0 + col < N) put_r(ia, n0 + col, rr, Zs[rr * BN + col]);
        }
        // the solved rows feed the next steps' products through TMA (async proxy), and
        // the next step's copies overwrite the buffers above in the A ring
        asm volatile("fence.proxy.async.global;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        epi_sync();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(zready)) : "memory");
    }
}

template <int DIR, int BN>
__global__ void __launch_bounds__(320, 1)
k_solve_tc(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
           const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl, const SolveTcArgs a)
{
    using namespace stc;
    using C = Cfg<BN>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* aring = smem;
    unsigned char* bring = aring + NA * A_BYTES;
    float* Vs = (float*)aring;                             // [128][BN]   (in the A ring, see Cfg)
    float* Zs = Vs + BM * BN;                              // [64][BN]
    float* Ds = Zs + TB * BN;                              // [64][65]: an inverse diagonal block
    float* Ls = Ds + TB * (TB + 1);                        // [64][65]: the tile between a pair's rows
    float* phis = (float*)(bring + NB * C::B_BYTES);       // [m][BN]
    uint64_t* afull = (uint64_t*)(phis + MAX_P * BN);
    uint64_t* aempty = afull + NA;
    uint64_t* bfull = aempty + NA;
    uint64_t* bempty = bfull + NB;
    uint64_t* tfull = bempty + NB;
    uint64_t* tempty = tfull + 2;
    uint64_t* zready = tempty + 2;
    uint64_t* mdone = zready + 1;          // every MMA of the issuer complete (its exit)
    uint32_t* tmem_slot = (uint32_t*)(mdone + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    volatile int* aconsumed = abort_flag + 1;   // A / B stages whose copies the MMA issuer waited for
    volatile int* bconsumed = aconsumed + 1;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int f = blockIdx.y, nb = blockIdx.x;
    const int64_t N = (int64_t)a.tcount * a.c;
    const int64_t n0 = (int64_t)nb * BN;
    const int p = a.p;
    const int nS = (a.nt + 1) / 2;
    const int brow = (int)((int64_t)f * a.qc + (int64_t)a.t0 * a.c + n0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < NA; ++s) { mbar_init(&afull[s], 1); mbar_init(&aempty[s], 1); }
        for (int s = 0; s < NB; ++s) { mbar_init(&bfull[s], 1); mbar_init(&bempty[s], 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], EPI_WARPS); }
        mbar_init(zready, EPI_WARPS);
        mbar_init(mdone, 1);
        *abort_flag = 0;
        *aconsumed = 0;
        *bconsumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    for (int e = threadIdx.x; e < p * BN; e += blockDim.x) {
        const int m = e / BN, col = e % BN;
        const int64_t n = n0 + col;
        phis[e] = n < N ? (float)a.phi[(int64_t)(a.t0 + n / a.c) * p + m] : 0.0f;
    }
    if (warp == 0) tc5::alloc(tmem_slot, TMEM_COLS);
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- producer ----
            int kbg = 0, qg = 0, aiss = 0, biss = 0;
            for (int s = 0; s < nS && !*abort_flag; ++s) {
                int i0, jlo, jhi;
                s_step<DIR>(a, s, i0, jlo, jhi);
                const int nkb = 2 * (jhi - jlo);
                // the newest blocks of the product were solved in step s - 1
                if (nkb > 0 && s > 0 && !mbar_wait(zready, (s - 1) & 1)) { *abort_flag = 1; break; }
                for (int kb = 0; kb < nkb && !*abort_flag; ++kb, ++kbg) {
                    const int j = jlo + kb / 2, x = j * TB + (kb & 1) * BK, sb = kbg % NB;
                    if (!mbar_wait(&bempty[sb], ((kbg / NB) & 1) ^ 1)) { *abort_flag = 1; break; }
                    unsigned char* bs = bring + sb * C::B_BYTES;
                    mbar_expect_tx(&bfull[sb], C::B_BYTES);
                    tma_load_2d(bs, &mBh, &bfull[sb], x, brow);
                    tma_load_2d(bs + C::B_BYTES / 2, &mBl, &bfull[sb], x, brow);
                    ++biss;
                    const int xa = (kb & 1) * BK;
                    for (int m = 0; m < p; ++m, ++qg) {
                        const int sa = qg % NA;
                        if (!mbar_wait(&aempty[sa], ((qg / NA) & 1) ^ 1)) { *abort_flag = 1; break; }
                        unsigned char* as = aring + sa * A_BYTES;
                        mbar_expect_tx(&afull[sa], A_BYTES);
                        const int y0 = s_row<DIR>(a, f, i0, j, m), y1 = s_row<DIR>(a, f, i0 + 1, j, m);
                        tma_load_2d(as, &mAh, &afull[sa], xa, y0);
                        tma_load_2d(as + BM / 2 * 128, &mAh, &afull[sa], xa, y1);
                        tma_load_2d(as + BM * 128, &mAl, &afull[sa], xa, y0);
                        tma_load_2d(as + BM * 128 + BM / 2 * 128, &mAl, &afull[sa], xa, y1);
                        ++aiss;
                    }
                }
            }
            // wait (bounded) for copies that were issued but never consumed (at most one per
            // stage, so no phase parity is ambiguous)
            for (int q = *aconsumed; q < aiss; ++q) mbar_wait(&afull[q % NA], (q / NA) & 1);
            for (int kb = *bconsumed; kb < biss; ++kb) mbar_wait(&bfull[kb % NB], (kb / NB) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer: every k-block is one chunk, into accumulator set cg & 1 ----
            constexpr uint32_t idesc = tc5::idesc_tf32(BM, BN);
            int kbg = 0, qg = 0, cg = 0;
            for (int s = 0; s < nS && !*abort_flag; ++s) {
                int i0, jlo, jhi;
                s_step<DIR>(a, s, i0, jlo, jhi);
                const int nkb = 2 * (jhi - jlo);
                for (int kb = 0; kb < nkb && !*abort_flag; ++kb, ++kbg, ++cg) {
                    const int b = cg & 1, sb = kbg % NB;
                    if (!mbar_wait(&tempty[b], ((cg >> 1) & 1) ^ 1) || !mbar_wait(&bfull[sb], (kbg / NB) & 1)) {
                        *abort_flag = 1;
                        break;
                    }
                    tc5::fence_after();
                    const uint32_t bh = smem_u32(bring + sb * C::B_BYTES), bl = bh + C::B_BYTES / 2;
                    for (int m = 0; m < p; ++m, ++qg) {
                        const int sa = qg % NA;
                        if (!mbar_wait(&afull[sa], (qg / NA) & 1)) { *abort_flag = 1; break; }
                        tc5::fence_after();
                        const uint32_t ah = smem_u32(aring + sa * A_BYTES), al = ah + BM * 128;
                        const uint32_t acc = tmem + (uint32_t)((b * p + m) * BN);
                        tc5::mma_split3_k32(acc, ah, al, bh, bl, idesc, true);
                        tc5::commit(&aempty[sa]);
                        *aconsumed = qg + 1;
                    }
                    tc5::commit(&bempty[sb]);
                    *bconsumed = kbg + 1;
                    tc5::commit(&tfull[b]);
                }
            }
            // every MMA issued has completed before the tensor memory is freed
            tc5::commit(mdone);
            mbar_wait(mdone, 0);
        }
    } else {
        k_solve_tc_epilogue<DIR, BN>(a, tmem, Vs, Zs, Ds, Ls, phis, tfull, tempty, zready, abort_flag, f, n0, N);
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
template <int DIR, int BN>
static cudaError_t solve_pass(pichol_ctx* ctx, const CUtensorMap& ah, const CUtensorMap& al, const CUtensorMap& bh,
                              const CUtensorMap& bl, const SolveTcArgs& sa, cudaStream_t s)
{
    static std::atomic<unsigned long long> set{0};
    cudaError_t e = smem_limit_once(k_solve_tc<DIR, BN>, stc::Cfg<BN>::SMEM, set);
    if (e != cudaSuccess) return e;
    const int64_t N = (int64_t)sa.tcount * sa.c;
    {
        StageScope sc_(ctx, ST_SOLVE, s);
        k_solve_tc<DIR, BN><<<dim3((unsigned)((N + BN - 1) / BN), ctx->cfg.k), stc::THREADS, stc::Cfg<BN>::SMEM, s>>>(
            ah, al, bh, bl, sa);
    }
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t launch_solve_tc(pichol_ctx* ctx, int t0, int tcount, const void* rhs, int rhs_per_system, void* out,
                            cudaStream_t s)
{
    const pichol_config& c = ctx->cfg;
    const int64_t dp = ctx->dp, qc = (int64_t)c.q * c.c;
    const int p = ctx->p;
    if (p * 32 > 256 || !ctx->Th || !ctx->Sh) return cudaErrorInvalidValue;
    const int BN = p <= 4 ? 64 : 32;
    const uint64_t trows = (uint64_t)(c.k * ctx->ntiles * p + 1) * TB;
    CUtensorMap th, tl, tth, ttl, sh, sl;
    if (!make_map_f32(&th, ctx->Th, TB, trows, TB, stc::BK, TB) || !make_map_f32(&tl, ctx->Tl, TB, trows, TB, stc::BK, TB) ||
        !make_map_f32(&tth, ctx->TTh, TB, trows, TB, stc::BK, TB) ||
        !make_map_f32(&ttl, ctx->TTl, TB, trows, TB, stc::BK, TB) ||
        !make_map_f32(&sh, ctx->Sh, (uint64_t)dp, (uint64_t)(c.k * qc), (uint64_t)dp, stc::BK, BN) ||
        !make_map_f32(&sl, ctx->Sl, (uint64_t)dp, (uint64_t)(c.k * qc), (uint64_t)dp, stc::BK, BN))
        return cudaErrorInvalidValue;
    SolveTcArgs sa;
    memset(&sa, 0, sizeof(sa));
    sa.phi = ctx->phi;
    sa.theta = (const float*)ctx->Theta;
    sa.dinv = (const float*)ctx->Dinv;
    sa.rhs = (const float*)rhs;
    sa.out = (float*)out;
    sa.Sh = ctx->Sh;
    sa.Sl = ctx->Sl;
    sa.p = p;
    sa.nt = ctx->nt;
    sa.q = c.q;
    sa.t0 = t0;
    sa.tcount = tcount;
    sa.rhs_per_system = rhs_per_system;
    sa.ntiles = ctx->ntiles;
    sa.dp = dp;
    sa.c = c.c;
    sa.qc = qc;
    sa.zero_row = (int)((int64_t)c.k * ctx->ntiles * p * TB);
    sa.st = ctx->status;
    SolveTcArgs sb = sa;                 // backward: from the forward result, in place
    sb.rhs = (const float*)out;
    sb.rhs_per_system = 1;
    cudaError_t e;
    if (BN == 64) {
        if ((e = solve_pass<0, 64>(ctx, th, tl, sh, sl, sa, s)) != cudaSuccess) return e;
        return solve_pass<1, 64>(ctx, tth, ttl, sh, sl, sb, s);
    }
    if ((e = solve_pass<0, 32>(ctx, th, tl, sh, sl, sa, s)) != cudaSuccess) return e;
    return solve_pass<1, 32>(ctx, tth, ttl, sh, sl, sb, s);
}

}  // namespace pichol
