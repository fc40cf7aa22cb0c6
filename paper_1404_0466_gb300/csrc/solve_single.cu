// The block substitutions of few systems (a single lambda per fold, as in the
// gradient, or the three of an MChol level) with one-lambda CTAs and a deeper
// copy ring: a separate translation unit so the solve kernels compile in
// parallel.
#include "internal.cuh"
#include "solve_common.cuh"
#include "tma.cuh"

namespace pichol {

template <typename T, bool EXACT>
static cudaError_t single_dispatch(pichol_ctx* ctx, const SolveArgs& sa, cudaStream_t s)
{
    switch (pick_cb(ctx->cfg.c)) {
    case 4: return solve_np<T, 1, 4, EXACT>(ctx, sa, s);
    case 10:
    case 12: return solve_np<T, 1, 12, EXACT>(ctx, sa, s);
    default: return solve_np<T, 1, 32, EXACT>(ctx, sa, s);
    }
}

cudaError_t launch_solve_single(pichol_ctx* ctx, const SolveArgs& sa, bool exact, cudaStream_t s)
{
    if (ctx->cfg.mode == PICHOL_MODE_FP64)
        return exact ? single_dispatch<double, true>(ctx, sa, s) : single_dispatch<double, false>(ctx, sa, s);
    return exact ? single_dispatch<float, true>(ctx, sa, s) : single_dispatch<float, false>(ctx, sa, s);
}

}  // namespace pichol
