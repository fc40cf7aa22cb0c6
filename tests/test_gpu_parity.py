"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Tolerances:
  * double-precision mode: factor entries and coefficients within 1e-10 of the
    matrix scale, hold-out errors within 1e-10 relative, identical argmin;
  * mixed mode: hold-out errors within 1e-4 relative; the selected lambda must
    be the oracle's, or one whose oracle score is within 1e-4 of the oracle's
    minimum (the argmin is decided in each side's own precision).
"""
import numpy as np
import pytest

import oracle
import tolerances
from paper_1404_0466_gb300 import synth

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 1e-4


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    from paper_1404_0466_gb300 import build
    build.build()
    return torch


def _ctx(prob, **kw):
    from paper_1404_0466_gb300 import binding
    n, d = prob.X.shape
    c = prob.Y.shape[1]
    return binding.Context(n=n, d=d, c=c, **kw)


def _dev(torch, a, mode):
    dt = torch.float64 if mode == "fp64" else torch.float32
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)


def _check_selected(t_gpu, ref, tol):
    if t_gpu == ref.t_star:
        return
    Eb = ref.Ebar
    assert 0 <= t_gpu < len(Eb) and np.isfinite(Eb[t_gpu]), (t_gpu, ref.t_star)
    assert Eb[t_gpu] <= Eb[ref.t_star] * (1 + tol), (t_gpu, ref.t_star, Eb[t_gpu], Eb[ref.t_star])


# ---------------------------------------------------------------------------
# double-precision mode, the small case (n=2048, d=256, k=5, g=4, r=2, q=31)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def fp64_small(torch_mod):
    torch = torch_mod
    cfg = synth.FP64_SMALL
    prob = synth.fp64_small()
    ref = oracle.cv(prob.X, prob.Y, k=cfg["k"], g=cfg["g"], r=cfg["r"], q=cfg["q"], basis="mono", keep=True)
    ctx = _ctx(prob, k=cfg["k"], g=cfg["g"], r=cfg["r"], q=cfg["q"], basis="mono", mode="fp64")
    X, Y = _dev(torch, prob.X, "fp64"), _dev(torch, prob.Y, "fp64")
    ctx.hessian(X, Y)
    ctx.factor_samples()
    ctx.fit()
    out = ctx.eval_holdout(want_w=True)
    torch.cuda.synchronize()
    return dict(prob=prob, ref=ref, ctx=ctx, out=out, X=X, Y=Y)


def test_fp64_hessian_blocks(fp64_small):
    ctx, ref = fp64_small["ctx"], fp64_small["ref"]
    for f in range(5):
        H, B = ctx.export_hessian(f)
        H, B = H.cpu().numpy(), B.cpu().numpy()
        assert np.max(np.abs(H - ref.H[f])) <= 1e-12 * np.max(np.abs(ref.H[f]))
        assert np.max(np.abs(B - ref.B[f])) <= 1e-12 * np.max(np.abs(ref.B[f]))


def test_fp64_lambda_grid(fp64_small):
    lam = fp64_small["ctx"].lambdas().cpu().numpy()
    np.testing.assert_allclose(lam, fp64_small["ref"].lam, rtol=1e-13)


def test_fp64_sampled_factors(fp64_small):
    ctx, ref = fp64_small["ctx"], fp64_small["ref"]
    for f in range(5):
        for s in range(4):
            L = ctx.export_factor(f, s).cpu().numpy()
            Lr = ref.factors[(f, s)]
            assert np.max(np.abs(L - Lr)) <= FP64_TOL * np.max(np.abs(Lr)), (f, s)


def test_fp64_coefficients(fp64_small):
    ctx, ref = fp64_small["ctx"], fp64_small["ref"]
    d = 256
    for f in range(5):
        Th = ctx.export_theta(f).cpu().numpy()
        for m in range(3):
            Tr = oracle.unvec_lower(ref.theta[f][m], d)
            scale = max(np.max(np.abs(oracle.unvec_lower(ref.theta[f][mm], d))) for mm in range(3))
            assert np.max(np.abs(Th[m] - Tr)) <= 1e-9 * scale, (f, m)


def test_fp64_holdout_and_selection(fp64_small):
    out, ref = fp64_small["out"], fp64_small["ref"]
    E = out.E.cpu().numpy()
    np.testing.assert_allclose(E, ref.E, rtol=FP64_TOL, atol=0)
    assert int(out.t_star.cpu().item()) == ref.t_star


def test_fp64_solutions(fp64_small):
    out, ref = fp64_small["out"], fp64_small["ref"]
    W = out.W.cpu().numpy()
    for (f, t), Wr in list(ref.W.items())[::17]:
        assert np.max(np.abs(W[f, t] - Wr)) <= 1e-9 * np.max(np.abs(Wr)), (f, t)


def test_fp64_device_status_clean(fp64_small):
    info = fp64_small["ctx"].info()
    assert info.code == 0 and info.unusable == int(fp64_small["ref"].unusable.sum())
    assert fp64_small["ctx"].launch_count() > 10


def test_fp64_exact_cv(fp64_small, torch_mod):
    prob = fp64_small["prob"]
    ref = oracle.cv(prob.X, prob.Y, k=5, g=4, r=2, q=31, exact=True)
    ctx = _ctx(prob, k=5, g=4, r=2, q=31, mode="fp64", exact_batch=8)
    ctx.hessian(fp64_small["X"], fp64_small["Y"])
    out = ctx.eval_holdout_exact()
    np.testing.assert_allclose(out.E.cpu().numpy(), ref.E, rtol=FP64_TOL)
    assert int(out.t_star.cpu().item()) == ref.t_star
    assert ctx.info().code == 0


# ---------------------------------------------------------------------------
# ragged shapes and edge cases, double precision
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,d,c,k,g,r,q,basis", [
    (517, 100, 1, 3, 3, 2, 7, "mono"),        # d not a multiple of 64, uneven folds, one output
    (300, 37, 4, 7, 5, 3, 11, "cheb_log"),    # d smaller than one tile
    (900, 129, 12, 2, 2, 1, 5, "cheb_log"),   # two folds, 3 tiles with a 1-wide edge
    (260, 64, 2, 4, 1, 0, 1, "mono"),         # a single lambda, constant polynomial
])
def test_fp64_ragged_shapes(torch_mod, n, d, c, k, g, r, q, basis):
    torch = torch_mod
    prob = synth.spectral_gaussian(n, d, c, seed=100 + d)
    ref = oracle.cv(prob.X, prob.Y, k=k, g=g, r=r, q=q, basis=basis)
    ctx = _ctx(prob, k=k, g=g, r=r, q=q, basis=basis, mode="fp64")
    out = ctx.run(_dev(torch, prob.X, "fp64"), _dev(torch, prob.Y, "fp64"))
    E = out.E.cpu().numpy()
    np.testing.assert_allclose(E, ref.E, rtol=1e-9)
    assert int(out.t_star.cpu().item()) == ref.t_star
    ex = ctx.eval_holdout_exact()
    refx = oracle.cv(prob.X, prob.Y, k=k, g=g, r=r, q=q, exact=True)
    np.testing.assert_allclose(ex.E.cpu().numpy(), refx.E, rtol=1e-9)


def test_nan_input_latches_not_spd(torch_mod):
    """A NaN in X makes a pivot non-positive: the factorisation latches
    PICHOL_ERR_NOT_SPD with its fold, sample and row (absolute grid, so the
    grid itself stays finite)."""
    torch = torch_mod
    prob = synth.spectral_gaussian(200, 20, 2, seed=5)
    X = prob.X.copy()
    X[3, 7] = np.nan
    ctx = _ctx(prob, k=4, g=3, r=2, q=5, mode="fp64", scale_by_trace=False)
    ctx.hessian(_dev(torch, X, "fp64"), _dev(torch, prob.Y, "fp64"))
    ctx.factor_samples()
    info = ctx.info()
    assert info.code == 2 and 0 <= info.fold < 4 and 0 <= info.index < 3 and 0 <= info.pivot < 20
    ctx.clear_status()
    assert ctx.info().code == 0


def test_bounded_wait_runs_out_and_the_context_recovers(torch_mod):
    """A bounded copy wait that nothing completes (about 1 ms of clocks) latches
    PICHOL_ERR_TIMEOUT without a fault or a hang; after clearing the status the
    same context runs a cross-validation that matches the oracle."""
    torch = torch_mod
    prob = synth.spectral_gaussian(300, 40, 2, seed=6)
    ctx = _ctx(prob, k=3, g=3, r=2, q=5, mode="fp64")
    ctx.check_timeout(2_000_000)
    info = ctx.info()
    assert info.code == 5 and info.fold == -1 and info.index == -1
    ctx.clear_status()
    out = ctx.run(_dev(torch, prob.X, "fp64"), _dev(torch, prob.Y, "fp64"))
    assert ctx.info().code == 0
    ref = oracle.cv(prob.X, prob.Y, k=3, g=3, r=2, q=5)
    np.testing.assert_allclose(out.E.cpu().numpy(), ref.E, rtol=1e-10)


def test_nan_input_with_trace_scaled_grid_latches_invalid(torch_mod):
    """With the grid scaled by tr(X^T X)/d a NaN makes the grid itself
    non-finite; the set-up latches PICHOL_ERR_INVALID_ARG first."""
    torch = torch_mod
    prob = synth.spectral_gaussian(200, 20, 2, seed=5)
    X = prob.X.copy()
    X[3, 7] = np.nan
    ctx = _ctx(prob, k=4, g=3, r=2, q=5, mode="fp64")
    ctx.hessian(_dev(torch, X, "fp64"), _dev(torch, prob.Y, "fp64"))
    ctx.factor_samples()
    assert ctx.info().code == 1


# ---------------------------------------------------------------------------
# mixed precision
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def mixed_small(torch_mod):
    # the mixed case's generator and method parameters at n = 4096, d = 200
    prob = synth.mixed_ecc(n=4096, d=200)
    ref = oracle.cv(prob.X, prob.Y, k=5, g=6, r=3, q=101, basis="cheb_log")
    return prob, ref


@pytest.mark.parametrize("refine,residual,solve", [(0, "tensor", 1), (1, "tensor", 1), (1, "double_float", 1),
                                                  (2, "tensor", 1), (0, "tensor", 0), (1, "tensor", 0)])
def test_mixed_holdout_and_selection(torch_mod, mixed_small, refine, residual, solve):
    """Mixed mode against the oracle: refinement steps, the residual on the
    tensor cores or in double-float, the solves on the CUDA cores (solve 1) or
    the tensor cores (solve 0)."""
    torch = torch_mod
    prob, ref = mixed_small
    ctx = _ctx(prob, k=5, g=6, r=3, q=101, basis="cheb_log", mode="mixed", refine_steps=refine,
               refine_residual=residual)
    ctx.set_tuning(solve_engine=solve)
    out = ctx.run(_dev(torch, prob.X, "mixed"), _dev(torch, prob.Y, "mixed"))
    E = out.E.cpu().numpy()
    rel = np.max(np.abs(E - ref.E) / ref.E)
    assert rel <= MIXED_TOL, rel
    _check_selected(int(out.t_star.cpu().item()), ref, MIXED_TOL)
    assert ctx.info().code == 0


@pytest.mark.parametrize("strip", [1, 2, 4])
def test_tensor_core_trailing_update_option(torch_mod, mixed_small, strip):
    """update_engine = 0 runs the bulk trailing updates of the factorisation on
    the tensor cores (split TF32, pairs of 128 output rows per MMA).  Its
    factors satisfy the Cholesky backward-error bound of a split-TF32 product
    per update, and on this well-conditioned data the hold-out errors stay
    within 1e-4 of the oracle."""
    torch = torch_mod
    prob, ref = mixed_small
    kw = dict(k=5, g=6, r=3, q=101, basis="cheb_log")
    ctx = _ctx(prob, mode="mixed", refine_steps=1, **kw)
    ctx.set_tuning(update_engine=0, update_strip=strip)
    out = ctx.run(_dev(torch, prob.X, "mixed"), _dev(torch, prob.Y, "mixed"))
    torch.cuda.synchronize()
    assert ctx.info().code == 0
    E = out.E.cpu().numpy()
    assert np.max(np.abs(E - ref.E) / ref.E) <= MIXED_TOL
    H, _ = (t.cpu().numpy() for t in ctx.export_hessian(1))
    lam_s = ctx.lambdas().cpu().numpy()[oracle.sample_indices(101, 6)]
    d = H.shape[0]
    for s in (0, 5):
        L = ctx.export_factor(1, s).cpu().numpy()
        A = H + lam_s[s] * np.eye(d)
        bound = (d + 1) * 2.0 ** -21 * (np.abs(L) @ np.abs(L.T)) + 2.0 ** -22 * np.abs(A)
        assert np.all(np.abs(L @ L.T - A) <= bound), float(np.max(np.abs(L @ L.T - A) / bound))
    ctx.close()


@pytest.mark.parametrize("r", [2, 5])
def test_tensor_core_residual_equals_double_float_residual(torch_mod, r):
    """The refinement residual B - L~ (L~^T W) formed on the tensor cores (all
    lambdas at once, one product per coefficient plane; degree 5 takes the
    narrower column tiles) against the double-float one on the FP32 pipes:
    after one step the solutions agree to about an fp32 rounding of the
    solve, and both scores are within 1e-4 of the oracle."""
    torch = torch_mod
    prob = synth.spectral_gaussian(1500, 150, 4, seed=41, decay=1.5, dtype=np.float32)
    kw = dict(k=5, g=8, r=r, q=33, basis="cheb_log")
    ref = oracle.cv(prob.X, prob.Y, **kw)
    outs = {}
    for residual in ("tensor", "double_float"):
        ctx = _ctx(prob, mode="mixed", refine_steps=1, refine_residual=residual, **kw)
        out = ctx.run(_dev(torch, prob.X, "mixed"), _dev(torch, prob.Y, "mixed"), want_w=True)
        torch.cuda.synchronize()
        assert ctx.info().code == 0
        outs[residual] = (out.E.cpu().numpy(), out.W.cpu().numpy().astype(np.float64))
        rel = np.abs(outs[residual][0] - ref.E) / ref.E
        assert np.all(rel <= MIXED_TOL), (residual, float(rel.max()))
        ctx.close()
    Wa, Wb = outs["tensor"][1], outs["double_float"][1]
    scale = np.max(np.abs(Wb), axis=(2, 3), keepdims=True)
    assert np.max(np.abs(Wa - Wb) / scale) <= 1e-4


def test_mixed_exact_system_refinement(torch_mod, mixed_small):
    """One refinement step against H_f + lambda I (the interpolated factor as a
    preconditioner): the oracle's refined errors, and closer to exact CV than
    the interpolated solution itself."""
    torch = torch_mod
    prob, ref0 = mixed_small
    kw = dict(k=5, g=6, r=3, q=101, basis="cheb_log")
    ref = oracle.cv(prob.X, prob.Y, precond_steps=1, **kw)
    ex = oracle.cv(prob.X, prob.Y, exact=True, **kw)
    ctx = _ctx(prob, mode="mixed", refine_steps=1, refine_target="exact", **kw)
    out = ctx.run(_dev(torch, prob.X, "mixed"), _dev(torch, prob.Y, "mixed"))
    E = out.E.cpu().numpy()
    tol = tolerances.MIXED_RTOL
    assert np.all(np.abs(E - ref.E) <= tol * ref.E), float(np.max(np.abs(E - ref.E) / ref.E))
    _check_selected(int(out.t_star.cpu().item()), ref, tol)
    gap = np.max(np.abs(E - ex.E) / ex.E)
    gap0 = np.max(np.abs(ref0.E - ex.E) / ex.E)
    assert gap < gap0 / 3, (gap, gap0)
    assert ctx.info().code == 0


def test_tuning_leaves_every_result_bit_identical(torch_mod, mixed_small):
    """Launch-shape tunings change scheduling only: scores, selection and solutions
    are bit-identical."""
    torch = torch_mod
    prob, _ = mixed_small
    ctx = _ctx(prob, k=5, g=6, r=3, q=101, basis="cheb_log", mode="mixed", refine_steps=1)
    X, Y = _dev(torch, prob.X, "mixed"), _dev(torch, prob.Y, "mixed")
    outs = []
    for tune in (dict(update_strip=4, diag_threads=512, diag_exclusive=1, eval_overlap=0),
                 dict(update_strip=1, diag_threads=256, diag_exclusive=0, eval_overlap=1),
                 dict(update_strip=8, diag_threads=512, diag_exclusive=0, eval_overlap=0),
                 dict(update_strip=2, diag_threads=256, diag_exclusive=1, eval_overlap=1)):
        ctx.set_tuning(**tune)
        assert {k: ctx.tuning()[k] for k in tune} == tune
        out = ctx.run(X, Y, want_w=True)
        outs.append((out.E.clone(), out.t_star.clone(), out.W.clone()))
    for E, t, W in outs[1:]:
        assert torch.equal(E, outs[0][0]) and torch.equal(t, outs[0][1]) and torch.equal(W, outs[0][2])
    assert ctx.info().code == 0


def test_mixed_exact_cv(torch_mod, mixed_small):
    torch = torch_mod
    prob, _ = mixed_small
    ref = oracle.cv(prob.X, prob.Y, k=5, g=6, r=3, q=101, exact=True, lam_idx=range(0, 101, 10))
    ctx = _ctx(prob, k=5, g=6, r=3, q=101, basis="cheb_log", mode="mixed", exact_batch=17)
    ctx.hessian(_dev(torch, prob.X, "mixed"), _dev(torch, prob.Y, "mixed"))
    out = ctx.eval_holdout_exact()
    E = out.E.cpu().numpy()
    cols = list(range(0, 101, 10))
    rel = np.max(np.abs(E[:, cols] - ref.E[:, cols]) / ref.E[:, cols])
    assert rel <= MIXED_TOL, rel


@pytest.mark.parametrize("n,d,passes", [
    (1500, 200, 3),    # 2 tensor-core tiles per side, 56 padded rows, uneven folds
    (2999, 300, 3),    # 3 tiles per side
    (1500, 200, 1),    # plain TF32 products
])
def test_mixed_hessian_on_tensor_cores(torch_mod, n, d, passes):
    """H_f formed by the tcgen05 Gram (split TF32 or plain TF32) against the
    FP64 oracle's direct sum over the training rows (Eq. 2).

    Tolerance, relative to max |H|: split TF32 products are exact to ~2^-22
    and the fp32 accumulation of n_train terms adds ~sqrt(n_train) 2^-24; the
    bound used is 8 sqrt(n_train) 2^-24.  Plain TF32 rounds each operand to 11
    bits, so a product is off by up to ~2^-10."""
    torch = torch_mod
    tol = 8 * np.sqrt(n) * 2.0 ** -24 if passes == 3 else 2.0 ** -10
    prob = synth.mixture_ecc(n, d, 10, seed=40 + d)
    ctx = _ctx(prob, k=5, g=4, r=2, q=9, basis="cheb_log", mode="mixed", gram_passes=passes)
    ctx.hessian(_dev(torch, prob.X, "mixed"), _dev(torch, prob.Y, "mixed"))
    offs = oracle.fold_offsets(n, 5)
    for f in (0, 3):
        H, B = ctx.export_hessian(f)
        Hr, Br = oracle.normal_blocks(prob.X, prob.Y, offs[f], offs[f + 1])
        err = np.max(np.abs(H.cpu().numpy() - Hr)) / np.max(np.abs(Hr))
        assert err <= tol, (f, err)
        # X_f^T Y_f runs on the same tensor-core path with the same tolerance
        errb = np.max(np.abs(B.cpu().numpy() - Br)) / np.max(np.abs(Br))
        assert errb <= tol, (f, errb)
    assert ctx.info().code == 0


def test_pivot_rsqrt_matches_library_within_a_few_ulps(torch_mod):
    """The pivots' 1/sqrt (float seed from the high word, one third-order step)
    against the library's 1.0 / sqrt on 2^22 values spread over 2^-110..2^110
    (seeded range and both fallbacks): within 4 units of 2^-53 relative."""
    from paper_1404_0466_gb300 import binding
    err = binding.check_rsqrt(1 << 22, seed=3)
    assert 0.0 <= err <= 4 * 2.0 ** -53, err


def test_fma_probe_reports_plausible_pipe_rates(torch_mod):
    """The FP32 pipes are tens of TFLOP/s on this part and the FP64 pipes a
    small fraction of that (GB300: one FP64 warp instruction per 64 cycles per
    sub-partition)."""
    from paper_1404_0466_gb300 import binding
    f32 = binding.probe_fma(False, 1 << 12)
    f64 = binding.probe_fma(True, 1 << 10)
    assert 10.0 < f32 < 200.0, f32
    assert 0.05 < f64 < f32 / 8, (f64, f32)


def test_mma_probe_reports_plausible_tensor_rates(torch_mod):
    """tcgen05.mma kind::tf32 at M = 128, K = 8: hundreds of TFLOP/s on this part,
    and a wider N is never slower per flop than a narrower one."""
    from paper_1404_0466_gb300 import binding
    r64 = binding.probe_mma(64, 1 << 12)
    r128 = binding.probe_mma(128, 1 << 12)
    r256 = binding.probe_mma(256, 1 << 12)
    assert 100.0 < r64 < 5000.0 and 100.0 < r128 < 5000.0 and 100.0 < r256 < 5000.0, (r64, r128, r256)
    assert r256 > 0.9 * r128 and r128 > 0.9 * r64, (r64, r128, r256)


def test_unusable_interpolated_diagonal_scores_inf(torch_mod):
    """Over twelve decades with g = r + 1 = 3 the interpolated factor's diagonal
    turns negative on part of the grid: the oracle flags 27 of the 63 (fold,
    lambda) pairs, each with min diag = -max |diag|, while every other pair keeps
    min diag >= 0.24 max |diag|.  The device scores exactly those pairs +inf,
    counts them, matches the oracle elsewhere (double precision) and picks the
    same lambda; nothing is latched as an error."""
    torch = torch_mod
    prob = synth.spectral_gaussian(300, 24, 2, seed=0, decay=2.0)
    kw = dict(k=3, g=3, r=2, q=21, basis="cheb_log")
    ref = oracle.cv(prob.X, prob.Y, lo=1e-9, hi=1e3, **kw)
    assert ref.unusable.sum() == 27
    ctx = _ctx(prob, lam_lo=1e-9, lam_hi=1e3, mode="fp64", **kw)
    out = ctx.run(_dev(torch, prob.X, "fp64"), _dev(torch, prob.Y, "fp64"))
    E = out.E.cpu().numpy()
    info = ctx.info()
    assert info.code == 0
    assert np.array_equal(np.isinf(E), ref.unusable)
    assert info.unusable == 27
    fin = ~ref.unusable
    assert np.max(np.abs(E[fin] - ref.E[fin]) / ref.E[fin]) <= 1e-9
    assert int(out.t_star.cpu().item()) == ref.t_star
