"""GPU parity of PINRMSE (pichol_eval_pinrmse), the supplementary comparator
that interpolates the g sampled exact hold-out errors directly, against the
oracle's PINRMSE through the C ABI.

The interpolated error is a fixed linear combination of the sampled errors,
E(t) = sum_s w[t, s] t_s with w = Phi V^+, so each sample's tolerance carries
over as |dE(t)| <= sum_s |w[t, s]| tol_s t_s: 1e-10 per sample in double
precision, the mixed tests' conditioning tolerance per sample in mixed
precision.
"""
import numpy as np
import pytest

import oracle
import tolerances
from paper_1404_0466_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    from paper_1404_0466_gb300 import build
    build.build()
    return torch


def _ctx(prob, **kw):
    from paper_1404_0466_gb300 import binding
    n, d = prob.X.shape
    return binding.Context(n=n, d=d, c=prob.Y.shape[1], **kw)


def _dev(torch, a, mode):
    dt = torch.float64 if mode == "fp64" else torch.float32
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)


def _weights(ref, basis, g, r):
    lam_s = ref.lam[ref.sample_idx]
    V = oracle.basis_values(basis, lam_s, lam_s, r + 1)
    Phi = oracle.basis_values(basis, ref.lam, lam_s, r + 1)
    return Phi @ np.linalg.pinv(V)                       # q x g


def _check(torch, prob, mode, k, g, r, q, basis, sample_tol):
    ref = oracle.pinrmse(prob.X, prob.Y, k=k, g=g, r=r, q=q, basis=basis)
    ctx = _ctx(prob, k=k, g=g, r=r, q=q, basis=basis, mode=mode)
    ctx.hessian(_dev(torch, prob.X, mode), _dev(torch, prob.Y, mode))
    ctx.factor_samples()
    out = ctx.eval_pinrmse()
    torch.cuda.synchronize()
    assert ctx.info().code == 0
    E = out.E.cpu().numpy()
    lam_s = ref.lam[ref.sample_idx]
    ts = oracle.holdout_exact_at(prob.X, prob.Y, k=k, lams=lam_s)             # k x g
    w = np.abs(_weights(ref, basis, g, r))
    tol = sample_tol(lam_s)                                                     # k x g
    bound = (tol * ts) @ w.T                                                    # k x q
    assert np.all(np.abs(E - ref.E) <= bound), np.max(np.abs(E - ref.E) / bound)
    t = int(out.t_star.cpu().item())
    if t != ref.t_star:
        assert ref.Ebar[t] <= ref.Ebar[ref.t_star] + bound.mean(axis=0)[t] + bound.mean(axis=0)[ref.t_star]
    return ctx, ref, E


def test_pinrmse_fp64_small_case(torch_mod):
    cfg = synth.FP64_SMALL
    prob = synth.fp64_small()
    ctx, ref, _ = _check(torch_mod, prob, "fp64", cfg["k"], cfg["g"], cfg["r"], cfg["q"], "mono",
                         lambda lam_s: np.full((cfg["k"], len(lam_s)), 1e-10))
    ctx.close()


def test_pinrmse_mixed_case_and_the_fit_stays_valid(torch_mod):
    torch = torch_mod
    prob = synth.mixed_ecc(n=4096, d=200)
    X64 = prob.X.astype(np.float64)
    ctx, ref, _ = _check(torch, prob, "mixed", 5, 6, 3, 101, "cheb_log",
                         lambda lam_s: np.full((5, len(lam_s)), tolerances.MIXED_RTOL))
    # piCholesky before and after PINRMSE on the same context: identical
    ctx.fit()
    a = ctx.eval_holdout()
    torch.cuda.synchronize()
    Ea = a.E.clone()
    ctx.eval_pinrmse()
    b = ctx.eval_holdout()
    torch.cuda.synchronize()
    assert torch.equal(Ea, b.E)
    ctx.close()


def test_pinrmse_needs_the_sampled_factors(torch_mod):
    from paper_1404_0466_gb300 import binding
    prob = synth.fp64_small(n=400, d=30)
    ctx = _ctx(prob, k=4, g=4, r=2, q=9, mode="fp64")
    ctx.hessian(_dev(torch_mod, prob.X, "fp64"), _dev(torch_mod, prob.Y, "fp64"))
    with pytest.raises(binding.PicholError) as ei:
        ctx.eval_pinrmse()
    assert ei.value.code == 7
    ctx.close()


def test_pinrmse_interpolates_the_exact_errors_at_the_nodes(torch_mod):
    """g = r + 1 in the Chebyshev basis: at the sampled grid points PINRMSE is
    exact CV (the device's own exact path), to the solves' precision."""
    torch = torch_mod
    prob = synth.fp64_small(n=800, d=70)
    k, g, r, q = 4, 4, 3, 13
    ctx = _ctx(prob, k=k, g=g, r=r, q=q, basis="cheb_log", mode="fp64")
    ctx.hessian(_dev(torch, prob.X, "fp64"), _dev(torch, prob.Y, "fp64"))
    ctx.factor_samples()
    pin = ctx.eval_pinrmse().E.cpu().numpy()
    ex = ctx.eval_holdout_exact().E.cpu().numpy()
    torch.cuda.synchronize()
    idx = oracle.sample_indices(q, g)
    np.testing.assert_allclose(pin[:, idx], ex[:, idx], rtol=1e-9)
    ctx.close()
