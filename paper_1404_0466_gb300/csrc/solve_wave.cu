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
// more as a 64-bit word {tag, value bits} with one relaxed GPU-scope store; the
// word is read with one relaxed GPU-scope load, and an aligned 64-bit access is
// single-copy atomic, so a reader that sees the tag also sees the value.  A
// waiting CTA polls the words of the block it needs (each thread its own few,
// all in flight at once) until every tag is set: no fence, no flag and no second
// load lie between a value being stored and being used.  Tags: 0 not yet
// written (the buffer is cleared before each launch), 1 valid, 2 failed.  Every
// wait is bounded: a thread whose wait runs out latches PICHOL_ERR_TIMEOUT, and a
// CTA that timed out or read a failed tag stops and writes its own block with the
// failed tag, so a failure ends every dependent CTA at once.
#include "internal.cuh"
#include "solve_common.cuh"

#include <cstdint>
#include <cstring>

namespace pichol {

namespace {

constexpr int WT = 256;           // threads per CTA
constexpr int WNP = 4;            // coefficient planes held per tile (p <= 4)
constexpr int WNJ = 8;            // output columns per thread: c <= 32
constexpr unsigned long long TAG_VALID = 1ull << 32, TAG_FAILED = 2ull << 32;

__device__ __forceinline__ unsigned long long word_poll(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];\n" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void word_publish(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;\n" ::"l"(p), "l"(v) : "memory");
}

}  // namespace

// One (system, tile row) per CTA; `ticket` and `xw` (this pass's S x dp x c
// tagged words) start at zero.  NJ: output columns per thread (columns g, g + 4,
// ..: 4 NJ >= c).
template <bool EXACT, int DIR, int NJ>
__global__ void __launch_bounds__(WT)
k_solve_wave(const SolveArgs a, int* __restrict__ ticket, unsigned long long* __restrict__ xw)
{
    __shared__ float Ls[TB][TB + 1];                  // tile applied to the solved block, as L[row][k]
    __shared__ __align__(16) float Zs[TB * NJ * 4];   // a solved block, row-major with row stride c
    __shared__ float Ds[TB][TB + 1];                  // the diagonal block's inverse (transposed backward)
    __shared__ int sh_tk;
    const int tid = threadIdx.x;
    const int S = (int)(a.tcount * (int64_t)gridDim.y);   // gridDim.y = k folds
    if (tid == 0) sh_tk = atomicAdd(ticket, 1);
    __syncthreads();
    const int tk = sh_tk, step = tk / S, sidx = tk % S;
    const int f = sidx / a.tcount, tloc = sidx % a.tcount, t = a.t0 + tloc;
    const int nt = a.nt;
    const int I = DIR == 0 ? step : nt - 1 - step;
    const int c = (int)a.c;
    const int np = EXACT ? 1 : a.p;
    const int64_t sysb = ((int64_t)f * a.q + t) * a.dp * a.c;
    unsigned long long* xs = xw + (int64_t)sidx * a.dp * a.c;    // this system's tagged blocks
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
        const float* dv = (const float*)a.dinv + (((int64_t)f * a.q + t) * nt + I) * TILE_ELEMS;
        for (int e = tid; e < TILE_ELEMS; e += WT) {
            const float x = dv[e];
            if (DIR == 0) Ds[e / TB][e % TB] = x;
            else Ds[e % TB][e / TB] = x;
        }
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
        // evaluate L~ = Theta_0 + sum_m phi_m Theta_m (phi_0 = 1) into Ls, transposed for
        // the backward pass (which applies L~_ji^T)
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
            const int e = 4 * (tid + WT * u), rr = e / TB, cc = e % TB;
            const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (DIR == 0) Ls[rr][cc + q] = vv[q];
                else Ls[cc + q][rr] = vv[q];
            }
        }
        // block J: poll (bounded) this thread's words of it until every tag is set
        const int J = jof(jj);
        {
            const unsigned long long* xb = xs + (int64_t)J * TB * c;
            const int nw = TB * c;
            unsigned long long wv[NJ];
            unsigned pend = 0;
#pragma unroll
            for (int u = 0; u < NJ; ++u)
                if (tid + WT * u < nw) pend |= 1u << u;
            const long long t0 = clock64();
            bool timeout = false;
            while (pend) {
#pragma unroll
                for (int u = 0; u < NJ; ++u)
                    if (pend >> u & 1u) wv[u] = word_poll(xb + tid + WT * u);
#pragma unroll
                for (int u = 0; u < NJ; ++u)
                    if ((pend >> u & 1u) && (wv[u] >> 32) != 0) pend &= ~(1u << u);
                if (pend && clock64() - t0 > WAIT_CYCLES) {
                    timeout = true;
                    break;
                }
            }
            bool mine_bad = timeout;
#pragma unroll
            for (int u = 0; u < NJ; ++u)
                if (tid + WT * u < nw) {
                    if ((wv[u] >> 32) != 1u) mine_bad = true;
                    Zs[tid + WT * u] = __uint_as_float((unsigned)wv[u]);
                }
            if (timeout) latch_error(a.st, PICHOL_ERR_TIMEOUT, f, I, J);
            if (__syncthreads_or(mine_bad)) {
                bad = true;
                break;
            }
        }
#pragma unroll 8
        for (int k = 0; k < TB; ++k) {
            const float lv = Ls[r][k];
#pragma unroll
            for (int j = 0; j < NJ; ++j)
                if (g + 4 * j < c) acc[j] = fmaf(lv, Zs[k * c + g + 4 * j], acc[j]);
        }
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
        for (int j = 0; j < NJ; ++j)
            if (g + 4 * j < c) Zs[r * c + g + 4 * j] = bv[j] - acc[j];
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < TB; ++k) {
            const float lv = Ds[r][k];
#pragma unroll
            for (int j = 0; j < NJ; ++j)
                if (g + 4 * j < c) x[j] = fmaf(lv, Zs[k * c + g + 4 * j], x[j]);
        }
#pragma unroll
        for (int j = 0; j < NJ; ++j)
            if (g + 4 * j < c) dst[sysb + row * c + g + 4 * j] = x[j];
    }
    // publish this thread's words of block I (failed: tag 2 and no value)
#pragma unroll
    for (int j = 0; j < NJ; ++j)
        if (g + 4 * j < c)
            word_publish(xs + row * c + g + 4 * j,
                         bad ? TAG_FAILED : (TAG_VALID | (unsigned long long)__float_as_uint(x[j])));
}

template <int NJ>
static void launch_wave_nj(bool exact, dim3 grid, cudaStream_t s, const SolveArgs& sa, int* ticket,
                           unsigned long long* xw, size_t nwords)
{
    if (exact) {
        k_solve_wave<true, 0, NJ><<<grid, WT, 0, s>>>(sa, ticket, xw);
        k_solve_wave<true, 1, NJ><<<grid, WT, 0, s>>>(sa, ticket + 1, xw + nwords);
    } else {
        k_solve_wave<false, 0, NJ><<<grid, WT, 0, s>>>(sa, ticket, xw);
        k_solve_wave<false, 1, NJ><<<grid, WT, 0, s>>>(sa, ticket + 1, xw + nwords);
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
    const size_t nwords = (size_t)S * ctx->dp * cf.c;
    int* ticket = reinterpret_cast<int*>(ctx->wave);   // word 0: two tickets; then [2][S][dp][c] words
    unsigned long long* xw = ctx->wave + 1;
    cudaError_t e = cudaMemsetAsync(ctx->wave, 0, (1 + 2 * nwords) * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)(sa.tcount * ctx->nt), cf.k);
    {
        StageScope sc_(ctx, ST_SOLVE, s);
        if (cf.c <= 4) launch_wave_nj<1>(exact, grid, s, sa, ticket, xw, nwords);
        else if (cf.c <= 12) launch_wave_nj<3>(exact, grid, s, sa, ticket, xw, nwords);
        else launch_wave_nj<WNJ>(exact, grid, s, sa, ticket, xw, nwords);
    }
    ctx->launches += 2;
    return cudaGetLastError();
}

}  // namespace pichol
