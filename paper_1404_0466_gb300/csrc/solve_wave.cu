// Interpolated triangular solves of few systems as a wavefront over tile rows
// (Sec. 3.2's two substitutions, with Sec. 3.3's evaluated factor):
//   forward   Z_i = Dinv_i (B_i - sum_{j<i} L~_ij Z_j)
//   backward  W_i = Dinv_i^T (Z_i - sum_{j>i} L~_ji^T W_j)
// When a call has few systems (the hold-out gradient's one lambda per fold, an
// MChol level's three, PINRMSE's samples), one CTA per system leaves most SMs
// idle and each system's tile rows form one long chain.  Here every (system,
// tile row) is a CTA: it evaluates its row's off-diagonal tiles from the
// coefficient planes (the next tile's planes prefetched into registers while
// the current one is applied) and adds each tile's product as soon as the
// solved block it multiplies is published, then solves its diagonal block
// through the precomputed inverse and publishes its own block.
//
// Scheduling: a CTA takes a ticket from a counter; ticket tk is row step
// tk / S of system tk mod S (forward rows in increasing order, backward rows in
// decreasing order), so every block a CTA waits for belongs to a smaller
// ticket, held by a CTA that is already running.  The wait is therefore never
// on a CTA that has not started, whatever the number of CTAs resident.
//
// Publication: besides the solution itself, every solved value is written once
// more into an exchange buffer with a relaxed GPU-scope store; the buffer is
// filled with the bit pattern NOT_READY (a NaN that arithmetic never produces:
// the GPU's computed NaN is 0x7fffffff, and a value with either reserved pattern
// is stored as that NaN) before each launch.  A waiting CTA polls the block it
// needs with relaxed GPU-scope 16-byte loads (each element an aligned 32-bit
// access, single-copy atomic, so an element that is not NOT_READY is the value
// itself) until no element reads NOT_READY: no fence, no flag and no second load
// lie between a value being stored and being used.  Every wait is bounded: a
// thread whose wait runs out latches PICHOL_ERR_TIMEOUT, and a CTA that timed out
// or read the pattern FAILED stops and writes its own block as FAILED, so a
// failure ends every dependent CTA at once.
#include "internal.cuh"
#include "solve_common.cuh"

#include <cstdint>
#include <cstring>

namespace pichol {

namespace {

constexpr int WT = 256;           // threads per CTA
constexpr int WNP = 4;            // coefficient planes held per tile (p <= 4)
constexpr int WNJ = 8;            // output columns per thread: c <= 32
constexpr int LSS = TB + 4;        // row stride of the staged tiles: 16-byte rows, 8 rows on distinct banks
constexpr unsigned NOT_READY = 0xffffffffu, FAILED = 0xfffffffeu;   // the buffer's fill: bytes 0xff

__device__ __forceinline__ uint4 block_poll(const unsigned* p)
{
    uint4 v;
    asm volatile("ld.relaxed.gpu.global.v4.b32 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p)
                 : "memory");
    return v;
}
__device__ __forceinline__ void value_publish(unsigned* p, unsigned v)
{
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

}  // namespace

// NJ values from shared memory at p (16-byte aligned when NJ is a multiple of 4)
template <int NJ>
__device__ __forceinline__ void lds_cols(const float* p, float (&z)[NJ])
{
    if constexpr (NJ % 4 == 0) {
#pragma unroll
        for (int j = 0; j < NJ; j += 4) {
            const float4 v = *reinterpret_cast<const float4*>(p + j);
            z[j] = v.x;
            z[j + 1] = v.y;
            z[j + 2] = v.z;
            z[j + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < NJ; ++j) z[j] = p[j];
    }
}

// acc[j] += sum_k A(r, k) Z[k][j] over the 64 k of a staged tile, A = the tile
// forward and its transpose backward; z points at this thread's columns of row 0
// of the staged block.  The k order is ascending in both directions.
template <int DIR, int NJ, int NJP>
__device__ __forceinline__ void apply_tile(const float* Ts, const float* z, int r, float (&acc)[NJ])
{
#pragma unroll 4
    for (int k0 = 0; k0 < TB; k0 += 4) {
        float l4[4];
        if constexpr (DIR == 0) {
            const float4 v = *reinterpret_cast<const float4*>(Ts + r * LSS + k0);
            l4[0] = v.x;
            l4[1] = v.y;
            l4[2] = v.z;
            l4[3] = v.w;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) l4[q] = Ts[(k0 + q) * LSS + r];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float zv[NJP];
            lds_cols<NJP>(z + (k0 + q) * 4 * NJP, zv);
#pragma unroll
            for (int j = 0; j < NJ; ++j) acc[j] = fmaf(l4[q], zv[j], acc[j]);
        }
    }
}

// One (system, tile row) per CTA; `ticket` starts at zero and `xw` (this pass's
// S x dp x c exchange values) at NOT_READY.  Tickets are numbered from tk0 (0,
// except in the wait check, which leaves out the first row step); `wait` is the
// limit of one wait in SM clocks.  NJ: output columns per thread (columns g, g + 4,
// ..: 4 NJ >= c).
//
// Shared memory: the tile and the diagonal inverse as stored (row-major, row
// stride LSS), read as L[r][k] forward and as L[k][r] (the transpose) backward;
// the solved block as [k][g][NJP], so that a thread's columns g + 4 j of one row
// k are adjacent (one 16-byte read for NJ = 3).
template <bool EXACT, int DIR, int NJ>
__global__ void __launch_bounds__(WT)
k_solve_wave(const SolveArgs a, int* __restrict__ ticket, unsigned* __restrict__ xw, int tk0, long long wait)
{
    constexpr int NJP = NJ == 1 ? 1 : (NJ + 3) / 4 * 4;   // padded columns per thread
    constexpr int ZR = 4 * NJP;                            // floats per row of the staged block
    __shared__ __align__(16) float Ls[TB * LSS];           // the tile applied to the solved block
    __shared__ __align__(16) float Zs[TB * ZR];            // a solved block, [k][g][j]
    __shared__ __align__(16) float Ds[TB * LSS];           // the diagonal block's inverse
    __shared__ int sh_tk;
    const int tid = threadIdx.x;
    const int S = (int)(a.tcount * (int64_t)gridDim.y);   // gridDim.y = k folds
    if (tid == 0) sh_tk = tk0 + atomicAdd(ticket, 1);
    __syncthreads();
    const int tk = sh_tk, step = tk / S, sidx = tk % S;
    const int f = sidx / a.tcount, tloc = sidx % a.tcount, t = a.t0 + tloc;
    const int nt = a.nt;
    const int I = DIR == 0 ? step : nt - 1 - step;
    const int c = (int)a.c;
    const int np = EXACT ? 1 : a.p;
    const int64_t sysb = ((int64_t)f * a.q + t) * a.dp * a.c;
    unsigned* xs = xw + (int64_t)sidx * a.dp * a.c;    // this system's exchanged blocks
    float* dst = (float*)(DIR == 0 ? a.zbuf : a.out);
    const float* src = (const float*)a.src;
    float w[WNP];
#pragma unroll
    for (int m = 0; m < WNP; ++m) w[m] = (!EXACT && m < np) ? (float)a.phi[(int64_t)t * a.p + m] : 0.0f;

    // tile (row, col) of this system's factor: plane base
    auto tile_base = [&](int ti, int tj) -> const float* {
        const int64_t tix = tile_index(ti, tj);
        if constexpr (EXACT) return src + ((int64_t)(f * a.per + tloc) * a.ntiles + tix) * TILE_ELEMS;
        return src + ((int64_t)f * a.ntiles + tix) * a.p * TILE_ELEMS;
    };
    // J of the jj-th off-diagonal tile, in the order the blocks are solved
    const int nj = DIR == 0 ? I : nt - 1 - I;
    auto jof = [&](int jj) { return DIR == 0 ? jj : nt - 1 - jj; };
    // this thread's 16 entries of a tile: four 16-byte groups, e = 4 (tid + 256 u) ..
    float4 cur[WNP][4], nxt[WNP][4];
    auto fetch = [&](float4 (&v)[WNP][4], int jj) {
        const int J = jof(jj);
        const float* b = DIR == 0 ? tile_base(I, J) : tile_base(J, I);
#pragma unroll
        for (int m = 0; m < WNP; ++m)
            if (m < np)
#pragma unroll
                for (int u = 0; u < 4; ++u) v[m][u] = reinterpret_cast<const float4*>(b + (int64_t)m * TILE_ELEMS)[tid + WT * u];
    };
    // output ownership: row r, columns g + 4 j
    const int r = tid >> 2, g = tid & 3;
    float acc[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[j] = 0.0f;
    // what the diagonal step needs and no wait guards, loaded first so that the step
    // after the last wait costs no memory round trip for it: the inverse (into Ds)
    // and the right-hand side of this thread's outputs (forward only; backward, the
    // forward solution, written by the previous launch)
    const int64_t row = (int64_t)I * TB + r;
    {
        const float4* dv = reinterpret_cast<const float4*>((const float*)a.dinv +
                                                           (((int64_t)f * a.q + t) * nt + I) * TILE_ELEMS);
        float4 dq[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) dq[u] = dv[tid + WT * u];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = 4 * (tid + WT * u);
            *reinterpret_cast<float4*>(&Ds[(e / TB) * LSS + e % TB]) = dq[u];
        }
    }
    // a block is 64 c values, 16 c groups of four; this thread polls groups tid + WT u,
    // and value e of the block, (row k, column o), goes to Zs[k][o & 3][o >> 2]
    constexpr int NV = (NJ + 3) / 4;
    int zdst[NV][4];
#pragma unroll
    for (int u = 0; u < NV; ++u)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int e = 4 * (tid + WT * u) + i, k = e / c, o = e - k * c;
            zdst[u][i] = k * ZR + (o & 3) * NJP + (o >> 2);
        }
    float bv[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int o = g + 4 * j;
        bv[j] = 0.0f;
        if (o < c) {
            const float* rhs = (const float*)a.rhs;
            if (DIR == 1) bv[j] = __ldcg((const float*)a.zbuf + sysb + row * c + o);
            else if (a.rhs_per_system) bv[j] = rhs[sysb + row * c + o];
            else bv[j] = rhs[((int64_t)f * a.dp + row) * c + o];
        }
    }

    bool bad = false;
    if (nj > 0) fetch(cur, 0);
    for (int jj = 0; jj < nj; ++jj) {
        if (jj + 1 < nj) fetch(nxt, jj + 1);       // in flight while this tile is applied
        // evaluate L~ = Theta_0 + sum_m phi_m Theta_m (phi_0 = 1) into Ls (the backward
        // pass applies its transpose)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float4 v = cur[0][u];
            if constexpr (!EXACT) {
#pragma unroll
                for (int m = 1; m < WNP; ++m)
                    if (m < np) {
                        v.x = fmaf(w[m], cur[m][u].x, v.x);
                        v.y = fmaf(w[m], cur[m][u].y, v.y);
                        v.z = fmaf(w[m], cur[m][u].z, v.z);
                        v.w = fmaf(w[m], cur[m][u].w, v.w);
                    }
            }
            const int e = 4 * (tid + WT * u);
            *reinterpret_cast<float4*>(&Ls[(e / TB) * LSS + e % TB]) = v;
        }
        // block J: poll (bounded) this thread's groups of it until none reads NOT_READY
        const int J = jof(jj);
        {
            const unsigned* xb = xs + (int64_t)J * TB * c;
            const int ng = 16 * c;
            uint4 wv[NV];
            unsigned pend = 0;
#pragma unroll
            for (int u = 0; u < NV; ++u)
                if (tid + WT * u < ng) pend |= 1u << u;
            const long long t0 = clock64();
            bool timeout = false;
            while (pend) {
#pragma unroll
                for (int u = 0; u < NV; ++u)
                    if (pend >> u & 1u) wv[u] = block_poll(xb + 4 * (tid + WT * u));
#pragma unroll
                for (int u = 0; u < NV; ++u)
                    if ((pend >> u & 1u) && wv[u].x != NOT_READY && wv[u].y != NOT_READY && wv[u].z != NOT_READY &&
                        wv[u].w != NOT_READY)
                        pend &= ~(1u << u);
                if (pend && clock64() - t0 > wait) {
                    timeout = true;
                    break;
                }
            }
            bool mine_bad = timeout;
#pragma unroll
            for (int u = 0; u < NV; ++u)
                if (tid + WT * u < ng) {
                    const unsigned vv[4] = {wv[u].x, wv[u].y, wv[u].z, wv[u].w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        if (vv[i] >= FAILED) mine_bad = true;
                        Zs[zdst[u][i]] = __uint_as_float(vv[i]);
                    }
                }
            if (timeout) latch_error(a.st, PICHOL_ERR_TIMEOUT, f, I, J);
            if (__syncthreads_or(mine_bad)) {
                bad = true;
                break;
            }
        }
        apply_tile<DIR, NJ, NJP>(Ls, Zs + g * NJP, r, acc);
        __syncthreads();                             // Ls and Zs are refilled next
        if (jj + 1 < nj) {
#pragma unroll
            for (int m = 0; m < WNP; ++m)
#pragma unroll
                for (int u = 0; u < 4; ++u) cur[m][u] = nxt[m][u];
        }
    }
    float x[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) x[j] = 0.0f;
    if (!bad) {
        // R = rhs_I - acc (rows of this tile row), then the diagonal inverse
#pragma unroll
        for (int j = 0; j < NJP; ++j) Zs[r * ZR + g * NJP + j] = j < NJ ? bv[j] - acc[j] : 0.0f;
        __syncthreads();
        apply_tile<DIR, NJ, NJP>(Ds, Zs + g * NJP, r, x);
#pragma unroll
        for (int j = 0; j < NJ; ++j)
            if (g + 4 * j < c) dst[sysb + row * c + g + 4 * j] = x[j];
    }
    // publish this thread's values of block I (FAILED when the CTA stopped)
#pragma unroll
    for (int j = 0; j < NJ; ++j)
        if (g + 4 * j < c) {
            unsigned v = __float_as_uint(x[j]);
            if (v >= FAILED) v = 0x7fffffffu;       // a value never reads as a reserved pattern
            value_publish(xs + row * c + g + 4 * j, bad ? FAILED : v);
        }
}

template <int NJ>
static void launch_wave_nj(bool exact, dim3 grid, cudaStream_t s, const SolveArgs& sa, int* ticket,
                           unsigned* xw, size_t nvals)
{
    if (exact) {
        k_solve_wave<true, 0, NJ><<<grid, WT, 0, s>>>(sa, ticket, xw, 0, WAIT_CYCLES);
        k_solve_wave<true, 1, NJ><<<grid, WT, 0, s>>>(sa, ticket + 1, xw + nvals, 0, WAIT_CYCLES);
    } else {
        k_solve_wave<false, 0, NJ><<<grid, WT, 0, s>>>(sa, ticket, xw, 0, WAIT_CYCLES);
        k_solve_wave<false, 1, NJ><<<grid, WT, 0, s>>>(sa, ticket + 1, xw + nvals, 0, WAIT_CYCLES);
    }
}

// The wavefront form applies when the systems are few (k tcount <= SMs), the
// mode is fp32 with at most four coefficient planes and at most 32 outputs;
// `sa` as for k_solve.  Returns cudaErrorNotSupported otherwise.
cudaError_t launch_solve_wave(pichol_ctx* ctx, const SolveArgs& sa, bool exact, cudaStream_t s)
{
    const pichol_config& cf = ctx->cfg;
    const int S = cf.k * sa.tcount;
    if (cf.mode != PICHOL_MODE_MIXED || !ctx->wave || (!exact && ctx->p > WNP) || cf.c > 4 * WNJ ||
        S > ctx->nsm || S > ctx->wave_sys)
        return cudaErrorNotSupported;
    const size_t nvals = (size_t)S * ctx->dp * cf.c;
    int* ticket = ctx->wave;                           // two tickets, then (at 256 bytes) [2][S][dp][c] values
    unsigned* xw = reinterpret_cast<unsigned*>(ctx->wave + WAVE_HEAD_INTS);
    cudaError_t e = cudaMemsetAsync(ticket, 0, 2 * sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(xw, 0xff, 2 * nvals * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)(sa.tcount * ctx->nt), cf.k);
    {
        StageScope sc_(ctx, ST_SOLVE, s);
        if (cf.c <= 4) launch_wave_nj<1>(exact, grid, s, sa, ticket, xw, nvals);
        else if (cf.c <= 12) launch_wave_nj<3>(exact, grid, s, sa, ticket, xw, nvals);
        else launch_wave_nj<WNJ>(exact, grid, s, sa, ticket, xw, nvals);
    }
    ctx->launches += 2;
    return cudaGetLastError();
}

// The failure path of the wavefront's waits: one forward pass over the
// gradient's buffers (one system per fold) whose first row step is never
// scheduled.  Block 0 is the first block every row waits for, so every CTA waits
// until `limit` SM clocks run out, latches PICHOL_ERR_TIMEOUT (fold, its row,
// block 0), publishes its block as FAILED and returns.  Nothing is written to
// the solution.  cudaErrorNotSupported where the wavefront does not
// apply (FP64 mode, p > 4, c > 32, d <= 64, or more folds than SMs).
cudaError_t launch_wave_check(pichol_ctx* ctx, long long limit, cudaStream_t s)
{
    const pichol_config& cf = ctx->cfg;
    const int S = cf.k;
    if (cf.mode != PICHOL_MODE_MIXED || !ctx->wave || ctx->p > WNP || cf.c > 4 * WNJ || ctx->nt < 2 ||
        S > ctx->nsm || S > ctx->wave_sys)
        return cudaErrorNotSupported;
    SolveArgs sa;
    sa.src = ctx->Theta;
    sa.dinv = ctx->gDinv;
    sa.rhs = ctx->Btr;
    sa.zbuf = ctx->gW;
    sa.out = ctx->gW;
    sa.phi = ctx->gphi;
    sa.p = ctx->p;
    sa.nt = ctx->nt;
    sa.q = 1;
    sa.t0 = 0;
    sa.tcount = 1;
    sa.per = 1;
    sa.rhs_per_system = 0;
    sa.ntiles = ctx->ntiles;
    sa.dp = ctx->dp;
    sa.c = cf.c;
    sa.st = ctx->status;
    const size_t nvals = (size_t)S * ctx->dp * cf.c;
    int* ticket = ctx->wave;
    unsigned* xw = reinterpret_cast<unsigned*>(ctx->wave + WAVE_HEAD_INTS);
    cudaError_t e = cudaMemsetAsync(ticket, 0, 2 * sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(xw, 0xff, nvals * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    // rows 1 .. nt-1 of every fold: tickets S .. S nt - 1
    const dim3 grid((unsigned)(ctx->nt - 1), cf.k);
    if (cf.c <= 4) k_solve_wave<false, 0, 1><<<grid, WT, 0, s>>>(sa, ticket, xw, S, limit);
    else if (cf.c <= 12) k_solve_wave<false, 0, 3><<<grid, WT, 0, s>>>(sa, ticket, xw, S, limit);
    else k_solve_wave<false, 0, WNJ><<<grid, WT, 0, s>>>(sa, ticket, xw, S, limit);
    ctx->launches++;
    return cudaGetLastError();
}

}  // namespace pichol
