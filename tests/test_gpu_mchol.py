"""GPU parity of the multi-level range search (MChol, Sec. 6.2) and of
piCholesky on the range it returns, through the C ABI, against the oracle.

Every level of the device trace is checked along the device's own path: the
three lambdas against tau 10^(c + (i-1) s) from the previous level's (c, s),
their mean exact hold-out errors against the oracle at the same lambdas, the
choice against the oracle's errors (the first argmin of the device's values,
and a valid minimum of the oracle's), and the update of (c, s).  In double
precision the path must also be the oracle's own.  Tolerances: 1e-10 relative
in double precision; in mixed precision the conditioning-derived tolerance of
the other mixed tests (max(1e-4, 16 kappa u32) per fold and lambda) on the
errors and 1e-5 on lambdas (tau comes from the split-TF32 Gram diagonal).
"""
import numpy as np
import pytest

import oracle
import tolerances
from paper_1404_0466_gb300 import synth

pytestmark = pytest.mark.gpu

K, G, R, Q = 5, 5, 3, 31
C0, S0, SMIN = -1.0, 2.0, 0.1          # [1e-3, 1e1] tau, five levels, final half-width 1/16 decade


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    from paper_1404_0466_gb300 import build
    build.build()
    return torch


def _ctx(prob, mode, **kw):
    from paper_1404_0466_gb300 import binding
    n, d = prob.X.shape
    args = dict(n=n, d=d, c=prob.Y.shape[1], k=K, g=G, r=R, q=Q, basis="cheb_log", mode=mode)
    args.update(kw)
    return binding.Context(**args)


def _dev(torch, a, mode):
    dt = torch.float64 if mode == "fp64" else torch.float32
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)


def _follow(trace, X, k, Y, tau, tol_E, tol_lam):
    """Checks each level of a device trace along its own path; returns the
    device's choices."""
    c, s = C0, S0
    choices = []
    for lv, row in enumerate(trace):
        lams, Eb, c_new, s_new = row[:3], row[3:6], row[6], row[7]
        want = tau * 10.0 ** (c + np.array([-1.0, 0.0, 1.0]) * s)
        assert np.all(np.abs(lams / want - 1.0) <= tol_lam), (lv, lams, want)
        ref = oracle.holdout_exact_at(X, Y, k=k, lams=lams)
        Eref = ref.mean(axis=0)
        tol = tol_E(lams)
        assert np.all(np.abs(Eb - Eref) <= tol * Eref), (lv, Eb, Eref)
        b = oracle.argmin_first(Eb)
        assert b >= 0
        assert Eref[b] <= Eref.min() * (1.0 + 2.0 * tol.max()), (lv, b, Eref)
        assert abs(c_new - (c + (b - 1) * s)) <= 1e-12 * max(1.0, abs(c_new)), (lv, c_new, c, b, s)
        assert s_new == s / 2.0
        choices.append(b)
        c, s = c_new, s_new
    return choices


def _run(torch, prob, mode, **kw):
    ctx = _ctx(prob, mode, **kw)
    ctx.hessian(_dev(torch, prob.X, mode), _dev(torch, prob.Y, mode))
    tr = ctx.mchol(C0, S0, SMIN)
    lam = ctx.lambdas()
    ctx.factor_samples()
    ctx.fit()
    out = ctx.eval_holdout()
    torch.cuda.synchronize()
    assert ctx.info().code == 0
    return ctx, tr.cpu().numpy(), lam.cpu().numpy(), out


def test_mchol_fp64_follows_the_oracle_and_pichol_searches_its_window(torch_mod):
    torch = torch_mod
    prob = synth.fp64_small()
    ctx, tr, lam, out = _run(torch, prob, "fp64")
    from paper_1404_0466_gb300 import binding
    assert tr.shape == (binding.mchol_levels(S0, SMIN), 8) == (5, 8)
    tau = oracle.trace_scale(prob.X)
    choices = _follow(tr, prob.X, K, prob.Y, tau, lambda lams: np.full(3, 1e-10), 1e-12)
    ref = oracle.mchol(prob.X, prob.Y, k=K, c=C0, s=S0, s_min=SMIN)
    assert choices == ref.best
    assert abs(tr[-1, 6] - ref.c) <= 1e-12 and tr[-1, 7] == ref.s
    # piCholesky over the final range
    lo, hi = ref.window
    cv = oracle.cv(prob.X, prob.Y, k=K, g=G, r=R, q=Q, lo=lo, hi=hi, basis="cheb_log")
    np.testing.assert_allclose(lam, cv.lam, rtol=1e-12)
    E = out.E.cpu().numpy()
    assert np.max(np.abs(E - cv.E) / cv.E) <= 1e-10
    assert int(out.t_star.cpu().item()) == cv.t_star
    ctx.close()


def test_mchol_mixed_levels_and_window(torch_mod):
    torch = torch_mod
    prob = synth.mixed_ecc(n=4096, d=200)
    ctx, tr, lam, out = _run(torch, prob, "mixed")
    tau = oracle.trace_scale(prob.X)
    X64 = prob.X.astype(np.float64)
    tol_E = lambda lams: np.full(len(lams), tolerances.MIXED_RTOL)
    _follow(tr, prob.X, K, prob.Y, tau, tol_E, 1e-5)
    lo, hi = 10.0 ** (tr[-1, 6] - tr[-1, 7]), 10.0 ** (tr[-1, 6] + tr[-1, 7])
    cv = oracle.cv(prob.X, prob.Y, k=K, g=G, r=R, q=Q, lo=lo, hi=hi, basis="cheb_log")
    np.testing.assert_allclose(lam, cv.lam, rtol=1e-5)
    E = out.E.cpu().numpy()
    rel = np.abs(E - cv.E) / cv.E
    assert np.all(rel <= tolerances.MIXED_RTOL), float(rel.max())
    t = int(out.t_star.cpu().item())
    assert tolerances.same_choice(cv.Ebar, t, cv.t_star), (t, cv.t_star)
    ctx.close()


def test_mchol_batches_of_one_and_no_trace_give_identical_results(torch_mod):
    """With exact_batch = 1 and g = 1 the factor buffer holds one problem per
    fold, so the three lambdas of a level are factored and scored one at a
    time; the results are bit-identical to batches of three, and so is a run
    without a trace buffer."""
    torch = torch_mod
    prob = synth.fp64_small(n=1024, d=130)
    _, tr_a, lam_a, out_a = _run(torch, prob, "fp64", g=1, r=0)
    _, tr_b, lam_b, out_b = _run(torch, prob, "fp64", g=1, r=0, exact_batch=1)
    assert np.array_equal(tr_a, tr_b) and np.array_equal(lam_a, lam_b)
    assert torch.equal(out_a.E, out_b.E)
    ctx = _ctx(prob, "fp64", g=1, r=0)
    ctx.hessian(_dev(torch, prob.X, "fp64"), _dev(torch, prob.Y, "fp64"))
    assert ctx.mchol(C0, S0, SMIN, trace=False) is None
    assert np.array_equal(ctx.lambdas().cpu().numpy(), lam_a)
    ctx.close()


def test_mchol_state_rules(torch_mod):
    """pichol_mchol needs the Gram step and q >= 3, and invalidates the fit."""
    torch = torch_mod
    from paper_1404_0466_gb300 import binding
    prob = synth.fp64_small(n=600, d=40)
    ctx = _ctx(prob, "fp64", g=2, r=1, q=2)
    with pytest.raises(binding.PicholError) as ei:
        ctx.mchol(C0, S0, SMIN)
    assert ei.value.code == 7                      # PICHOL_ERR_STATE: no Gram blocks yet
    ctx.hessian(_dev(torch, prob.X, "fp64"), _dev(torch, prob.Y, "fp64"))
    with pytest.raises(binding.PicholError) as ei:
        ctx.mchol(C0, S0, SMIN)
    assert ei.value.code == 6                      # PICHOL_ERR_UNSUPPORTED: q < 3
    ctx.close()
    ctx = _ctx(prob, "fp64")
    ctx.hessian(_dev(torch, prob.X, "fp64"), _dev(torch, prob.Y, "fp64"))
    ctx.factor_samples()
    ctx.fit()
    ctx.mchol(C0, S0, SMIN)
    with pytest.raises(binding.PicholError) as ei:
        ctx.eval_holdout()
    assert ei.value.code == 7
    torch.cuda.synchronize()
    assert ctx.info().code == 0
    ctx.close()


def test_mchol_on_nan_input_latches_an_error_and_returns(torch_mod):
    """A NaN in X reaches every exact factorisation of the search: the status
    word reports the first error (NOT_SPD, or INVALID_ARG from the trace-scaled
    range), every call returns, and the context still works afterwards."""
    torch = torch_mod
    prob = synth.fp64_small(n=600, d=40)
    X = prob.X.copy()
    X[5, 3] = np.nan
    ctx = _ctx(prob, "fp64", q=9, g=4, r=2)
    ctx.hessian(_dev(torch, X, "fp64"), _dev(torch, prob.Y, "fp64"))
    ctx.mchol(C0, S0, SMIN)
    torch.cuda.synchronize()
    assert ctx.info().code in (1, 2)
    ctx.clear_status()
    ctx.hessian(_dev(torch, prob.X, "fp64"), _dev(torch, prob.Y, "fp64"))
    tr = ctx.mchol(C0, 1.0, 0.5).cpu().numpy()
    torch.cuda.synchronize()
    assert ctx.info().code == 0 and np.all(np.isfinite(tr))
    ctx.close()
