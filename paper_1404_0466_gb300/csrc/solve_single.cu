// The interpolated block substitutions of a single lambda per fold (the
// gradient's solves) with one-lambda CTAs: a separate translation unit so the
// solve kernels compile in parallel.
#include "internal.cuh"
#include "solve_common.cuh"
#include "tma.cuh"

namespace pichol {

template <typename T>
static cudaError_t single_dispatch(pichol_ctx* ctx, const SolveArgs& sa, cudaStream_t s)
{
    switch (pick_cb(ctx->cfg.c)) {
    case 4: return solve_np<T, 1, 4, false>(ctx, sa, s);
    case 12: return solve_np<T, 1, 12, false>(ctx, sa, s);
    default: return solve_np<T, 1, 32, false>(ctx, sa, s);
    }
}

cudaError_t launch_solve_single(pichol_ctx* ctx, const SolveArgs& sa, cudaStream_t s)
{
    if (ctx->cfg.mode == PICHOL_MODE_FP64) return single_dispatch<double>(ctx, sa, s);
    return single_dispatch<float>(ctx, sa, s);
}

}  // namespace pichol
