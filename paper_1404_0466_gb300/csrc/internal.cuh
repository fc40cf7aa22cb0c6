// Internal definitions shared by the CUDA translation units of libpichol.
//
// Data layout in device memory (all inside the caller's workspace):
//  * The matrix side d is padded to dp = 64 * nt (nt = ceil(d / 64)).  Padded
//    rows/columns of every Hessian are the identity, so the padded Cholesky
//    factor is diag(L, I) and padded solution rows are zero.
//  * Lower-triangular matrices (shifted Hessians, Cholesky factors and the
//    polynomial coefficients of Algorithm 1) are stored tile-major: the 64 x 64
//    tile (I, J), I >= J, is contiguous (row-major inside the tile) at tile
//    index I (I + 1) / 2 + J.  This is the GPU analogue of the recursive
//    vectorisation of Sec. 5: every tile is an aligned contiguous block.
//  * Theta of fold f is [tile][m][64 x 64]: the (r+1) coefficient planes of one
//    tile are adjacent, so the solve streams one tile's planes as one block.
//  * Dense d x d Gram blocks G_j are row-major with leading dimension dp.
//  * Right-hand sides and solutions are [system][dp][c] row-major.
#pragma once

#include <atomic>
#include <cstdint>
#include <cstddef>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <type_traits>

#include "../../include/pichol.h"

namespace pichol {

constexpr int TB = 64;                   // tile side
constexpr int TILE_ELEMS = TB * TB;
constexpr int MAX_P = 8;                 // r + 1 <= 8
constexpr int MAX_G = 32;                // sampled lambdas
constexpr int MAX_K = 64;                // folds
constexpr int GRAD_CHUNKS = 8;           // chunks of a tile row in the gradient's triangular products
constexpr int64_t WAVE_SYS_CAP = 160;    // systems of one wavefront solve (at least the SM count)
constexpr int WAVE_HEAD_INTS = 64;       // the wavefront buffer's head (tickets), 256 bytes
// Debug build (-DPICHOL_DEBUG): every workspace section is followed by a guard
// band of GUARD_BYTES filled with GUARD_FILL when the workspace is attached;
// pichol_get_info checks them and reports a write past a section's end.
#ifdef PICHOL_DEBUG
constexpr size_t GUARD_BYTES = 4096;
#else
constexpr size_t GUARD_BYTES = 0;
#endif
constexpr unsigned char GUARD_FILL = 0xA5;
constexpr int MAX_GUARDS = 128;
constexpr int LAM_CHUNK = 448;           // caller lambdas passed per kernel launch (as arguments)

// Caller-supplied lambdas travel to the device as kernel arguments (3.5 KB, inside
// the classic 4 KB parameter space with the other arguments), so
// the calls that take them need no copy from host memory and stay capturable.
struct LamValues {
    double v[LAM_CHUNK];
};

struct DevStatus {
    int code;
    int fold;
    int index;
    int unusable;
    long long pivot;
    long long pad[3];
};

__host__ __device__ inline int64_t tile_index(int I, int J) {
    return (int64_t)I * (I + 1) / 2 + J;
}
__host__ __device__ inline int64_t num_tiles(int nt) {
    return (int64_t)nt * (nt + 1) / 2;
}

// Recover (I, J), J <= I, from a lower-triangular tile index.
__host__ __device__ inline void tile_coords(int64_t e, int& I, int& J) {
    int i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);   // estimate, fixed up below
    while ((int64_t)(i + 1) * (i + 2) / 2 <= e) ++i;
    while ((int64_t)i * (i + 1) / 2 > e) --i;
    I = i;
    J = (int)(e - (int64_t)i * (i + 1) / 2);
}

// A named NVTX range around one call of the C ABI, for timelines in a profiler
// (header-only NVTX; without a profiler attached the calls do nothing).
struct CallRange {
    explicit CallRange(const char* name) { nvtxRangePushA(name); }
    ~CallRange() { nvtxRangePop(); }
    CallRange(const CallRange&) = delete;
    CallRange& operator=(const CallRange&) = delete;
};

// Raises a kernel's dynamic shared-memory limit to `bytes` on the current
// device, once per device: the attribute belongs to the device's context, so a
// process that drives several GPUs needs it on each.  `set` is the caller's
// mask of devices (ordinal mod 64) done for this kernel.
template <typename Kernel>
inline cudaError_t smem_limit_once(Kernel* kernel, int bytes, std::atomic<unsigned long long>& set)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (set.load(std::memory_order_acquire) & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) set.fetch_or(bit, std::memory_order_release);
    return e;
}

#ifdef __CUDACC__
// 16-byte asynchronous global -> shared copies (cp.async, L2 only) and their groups.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    unsigned saddr = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// Two fp32 values as one 64-bit register pair, and the packed FMA on such pairs
// (fma.rn.f32x2: two independent round-to-nearest FMAs, bit for bit the scalar
// ones, in one issue slot).
__device__ __forceinline__ unsigned long long f32x2_pack(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 f32x2_unpack(unsigned long long v)
{
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ unsigned long long f32x2_fma(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// First error wins; the extra fields describe it.
__device__ inline void latch_error(DevStatus* st, int code, int fold, int index, long long pivot) {
    if (atomicCAS(&st->code, 0, code) == 0) {
        st->fold = fold;
        st->index = index;
        st->pivot = pivot;
    }
}
#endif

// Byte offset of element (row, col) of a 64 x 64 plane of elements of `esz`
// bytes in shared memory, with the 16-byte chunks of each row permuted by
// XOR with (row & 7).  Row-owner 16-byte reads along a row and column-owner
// scalar reads down a column are both free of bank conflicts.
__host__ __device__ inline int swz_off(int row, int col, int esz) {
    int byte = col * esz;
    int chunk = byte >> 4;
    return row * (TB * esz) + (((chunk ^ (row & 7)) << 4) | (byte & 15));
}

}  // namespace pichol

// Host-side context.
struct pichol_ctx {
    pichol_config cfg;
    int64_t dp;          // padded side
    int nt;              // tiles per side
    int64_t ntiles;      // lower tiles
    int p;               // r + 1
    int eb;              // element bytes of the mode's working type
    int64_t offs[pichol::MAX_K + 1];
    int64_t exact_batch; // lambdas per exact batch
    int64_t nfac;        // factor slots in the factor buffer

    char* ws;
    size_t ws_bytes;
    size_t need_bytes;

    // workspace sections (device pointers once the workspace is set)
    pichol::DevStatus* status;
    double* scal;        // [0] tau, [1] ln min lambda_s, [2] ln max lambda_s, [3] max lambda_s
    double* lam;         // q: the evaluation lambdas (the grid, or the caller's)
    double* lam_grid;    // q: the grid of pichol_hessian (or of MChol's final range)
    double* mlam;        // MChol state: [0..2] the level's lambdas, [4] c, [5] s, [6..7] final window
    double* lam_s;       // g
    double* pinv;        // p x g
    double* lam_w;       // g': warm-start lambdas (warm_samples > 0)
    double* pinv_w;      // min(g', p) x g': V'^+ of the warm start
    double* vw;          // g' x p: basis values at the warm-start lambdas
    double* phi;         // q x p
    double* dphi;        // q x p
    void* G;             // k x dp x dp
    void* Bv;            // k x dp x c
    double* yy;          // k
    void* Btr;           // k x dp x c
    double* xpart;       // k x XTY_SPLITS x dp x c partial sums of X_j^T Y_j
    void* Hf;            // k x ntiles x TB^2: H_f, tile-major lower
    void* F;             // nfac x ntiles x TB^2
    float* Ph;           // mixed mode: 2 x nfac x nt x TB^2, the panel tiles L_IJ of tile column J in
    float* Pl;           //   buffer J & 1, split TF32 hi / remainder lo (tensor-core trailing update)
    void* Theta;         // k x ntiles x p x TB^2
    void* Dinv;          // k x q x nt x TB^2
    void* W;             // k x q x dp x c
    void* U;             // 2 x k x q x dp x c floats: L~^T W as (hi, lo) (refinement); with the
                         // tensor-core residual [2][f][q c][dp], i.e. (L~^T W)^T split hi / lo
    float* Th;           // (k x ntiles x p + 1) x TB^2: Theta split TF32 hi (tensor-core residual;
    float* Tl;           //   the last plane is zero), remainder lo,
    float* TTh;          //   and the same with every tile transposed
    float* TTl;
    float* Sh;           // mixed mode: [2 halves: hi, lo] x k x (q c) x dp, solved blocks transposed
    float* Sl;           //   (tensor-core interpolated solve)
    void* Rres;          // k x q x dp x c (residual / correction)
    int64_t* nfc;        // k: n_f * c
    // tensor-core operands (mixed mode)
    int64_t kpad;        // columns of the transposed, fold-padded X (this fold split)
    int64_t kpad_cap;    // the most any fold split can need: floor((n + 31 k) / 32) * 32
    int64_t ldu;         // leading dimension of U2 (q c rounded up to 4)
    float* Xh;           // dp x kpad: X^T split, TF32 part
    float* Xl;           // dp x kpad: remainder
    float* Yh;           // c x kpad: Y^T split (fold-padded like X^T)
    float* Yl;
    const float* Yin;    // the caller's Y during pichol_hessian
    float* Gh;           // k x dp x dp: G_j split
    float* Gl;
    float* Wth;          // k x (q c) x dp: W^T split
    float* Wtl;
    float* U2;           // k x dp x ldu: G_f W for every lambda (exact-system refinement)
    float* Xrh;          // n x dp: X split row-major, TF32 part (direct hold-out scores)
    float* Xrl;          // n x dp: remainder
    float* Ycp;          // n x c: copy of Y (direct hold-out scores)
    double* Escore;      // k x mt_cap x ldu: per-(row tile, column) sums of squared residuals
    int mt_cap;          // row tiles of 128 in the largest possible fold
    float* Gah;          // dp x dp: G_all = sum_j G_j split (exact-system refinement only)
    float* Gal;
    float* U3;           // k x dp x ldu: G_all W for every lambda (exact-system refinement only)
    // gradient in log(lambda) at one lambda (pichol_holdout_grad)
    void* gW;            // 3 x k x dp x c: W, U, V
    void* gDinv;         // k x nt x TB^2
    double* gP;          // GRAD_CHUNKS x 4 x k x dp x c: chunks of L~^T W, L~^T U, L~'^T W, L~'^T U
    void* gL;            // 2 x k x ntiles x TB^2: L~ and L~' at the gradient's lambda
    double* gphi;        // phi (MAX_P), phi' (MAX_P), lambda
    int* gflags;         // k x nt
    float* gdmax;
    float* gdmin;
    double* Epart;       // k x q x nt
    double* E;           // k x q
    int* flags;          // k x q x nt (per-tile diagonal checks: bit0 nonpositive)
    int* wave;                  // wavefront solve: 2 tickets, then (at WAVE_HEAD_INTS) 2 x wave_sys x dp x c values
    int64_t wave_sys;           // systems the wavefront buffer holds: min(k q, WAVE_SYS_CAP)
    float* dmax;         // k x q x nt max |diag| of the tile
    float* dmin;         // k x q x nt min |diag| of the tile

    int nguard;          // debug build: guard bands after the workspace sections
    size_t guard_off[pichol::MAX_GUARDS];

    bool have_hessian, have_factors, have_fit;
    long long launches;

    // factorisation look-ahead: diagonal tiles, panels and the next tile column
    // run on `aux` (the device's highest stream priority) while the rest of each
    // trailing update runs on the caller's stream (created with the workspace)
    cudaStream_t aux;
    cudaEvent_t ev_fork, ev_panel, ev_upd, ev_join;
    int nsm;             // SMs of the device the workspace lives on
    pichol_tuning tune;  // factorisation launch shapes (pichol_set_tuning)

    // optional per-stage timing: pairs of events recorded around launches
    int timing;
    int ev_cap, ev_used;
    cudaEvent_t* ev;     // 2 * ev_cap events
    int* ev_stage;       // stage of each pair
};

namespace pichol {

// Stages reported by pichol_stage_times (order matters: it is the ABI's).
enum Stage {
    ST_GRAM = 0, ST_XTY, ST_SETUP, ST_CHOL_INIT, ST_CHOL_DIAG, ST_CHOL_PANEL, ST_CHOL_UPDATE, ST_FIT,
    ST_DIAG_INV, ST_SOLVE, ST_RESID, ST_SCORE, ST_SELECT, ST_MISC, NSTAGE
};

// Records a start event on construction and a stop event on destruction
// when timing is enabled on the context (and the event pool has room).  Under
// stream capture the records are external, so they become event-record nodes
// that every replay of the graph re-records.
struct StageScope {
    pichol_ctx* ctx;
    cudaStream_t s;
    int slot;
    unsigned flags;
    StageScope(pichol_ctx* c, int stage, cudaStream_t st) : ctx(c), s(st), slot(-1), flags(cudaEventRecordDefault) {
        if (ctx->timing && ctx->ev_used < ctx->ev_cap) {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
                flags = cudaEventRecordExternal;
            slot = ctx->ev_used++;
            ctx->ev_stage[slot] = stage;
            cudaEventRecordWithFlags(ctx->ev[2 * slot], s, flags);
        }
    }
    ~StageScope() {
        if (slot >= 0) cudaEventRecordWithFlags(ctx->ev[2 * slot + 1], s, flags);
    }
};

// Launch helpers implemented per translation unit; each returns a cudaError_t.
cudaError_t launch_gram(pichol_ctx* ctx, const void* X, const void* Y, cudaStream_t s);
cudaError_t launch_factor(pichol_ctx* ctx, int count, int exact, int t0, cudaStream_t s);
cudaError_t launch_fit(pichol_ctx* ctx, cudaStream_t s);
cudaError_t launch_eval(pichol_ctx* ctx, int exact, int t0, int tcount, cudaStream_t s);
cudaError_t launch_finish(pichol_ctx* ctx, double* E_out, int32_t* t_star, cudaStream_t s);
cudaError_t launch_export_tiles(pichol_ctx* ctx, const void* tiles, int64_t plane_stride_elems,
                                int64_t tile_stride_elems, double* out, cudaStream_t s);
cudaError_t launch_export_hessian(pichol_ctx* ctx, int f, double* H, double* B, cudaStream_t s);
cudaError_t launch_copy_w(pichol_ctx* ctx, void* W_out, cudaStream_t s);
size_t solve_smem_bytes(int eb, int p, int64_t c);
size_t xty_part_bytes(int k, int64_t dp, int64_t c);
int64_t tc_kpad(const pichol_ctx* ctx);
cudaError_t launch_gram_tc(pichol_ctx* ctx, const float* X, cudaStream_t s);
cudaError_t launch_grad(pichol_ctx* ctx, double log_lam, double* E_out, double* dE_out, cudaStream_t s);
cudaError_t launch_score_tc(pichol_ctx* ctx, int t0, int tcount, cudaStream_t s);
cudaError_t launch_gall_split(pichol_ctx* ctx, cudaStream_t s);
cudaError_t launch_wait_check(pichol_ctx* ctx, long long limit, cudaStream_t s);
cudaError_t launch_wave_check(pichol_ctx* ctx, long long limit, cudaStream_t s);
cudaError_t launch_resid_exact(pichol_ctx* ctx, int t0, int tcount, cudaStream_t s);
// W^T of systems [t0, t0 + tcount) split into TF32 parts (Wth / Wtl)
cudaError_t launch_split_wt(pichol_ctx* ctx, int t0, int tcount, int stage, cudaStream_t s);
// Theta split (and transposed) for the tensor-core residual, after the fit
cudaError_t launch_theta_split(pichol_ctx* ctx, cudaStream_t s);
// refinement residual of the interpolated system on tensor cores, into Rres
cudaError_t launch_resid_tc(pichol_ctx* ctx, int t0, int tcount, cudaStream_t s);
// interpolated solves of systems [t0, t0 + tcount) on tensor cores (mixed mode): rhs per fold
// [f][dp][c] or per system [f][t][dp][c]; the solution into out [f][t][dp][c]
cudaError_t launch_solve_tc(pichol_ctx* ctx, int t0, int tcount, const void* rhs, int rhs_per_system, void* out,
                            cudaStream_t s);
// bulk trailing update of tile column J on tensor cores (mixed mode; panel J split into Ph / Pl)
cudaError_t launch_update_tc(pichol_ctx* ctx, int per, int count, int warm, int nprob, int J, int first, int ncols,
                             int chunk, cudaStream_t s);
// grid, samples and V^+ from the Gram blocks; window (device, nullable) holds
// (lo, hi) replacing the configured range
cudaError_t launch_setup(pichol_ctx* ctx, const double* window, cudaStream_t s);
// the sampled lambdas (host values or NULL for the grid samples), V^+ and the basis normalisation
cudaError_t launch_set_samples(pichol_ctx* ctx, const double* lam_s_host, cudaStream_t s);
// the evaluation lambdas (host values or NULL for the grid) and their basis values
cudaError_t launch_set_evals(pichol_ctx* ctx, const double* lam_t_host, cudaStream_t s);
cudaError_t launch_mchol(pichol_ctx* ctx, double c, double s, int levels, double* trace_out, cudaStream_t st);
int mchol_levels(double s, double s_min);
cudaError_t launch_pinrmse(pichol_ctx* ctx, double* E_out, int32_t* t_star, cudaStream_t s);
cudaError_t launch_check_rsqrt(int64_t n, uint64_t seed, double* max_rel, cudaStream_t s);
// debug build: latch PICHOL_ERR_WORKSPACE (index = guard, pivot = byte) for a guard band byte that changed
cudaError_t launch_check_guards(pichol_ctx* ctx, cudaStream_t s);

}  // namespace pichol
