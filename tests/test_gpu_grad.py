"""Derivative of the hold-out error in log(lambda) through the interpolated
factor (pichol_holdout_grad), against the FP64 oracle's gradient, central
differences, and the exact-Cholesky gradient; the autograd wrapper; gradient
steps on log(lambda)."""
import math

import numpy as np
import pytest

import oracle
from paper_1404_0466_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    from paper_1404_0466_gb300 import build
    build.build()
    return torch


def _setup(torch, prob, mode, **kw):
    from paper_1404_0466_gb300 import binding
    n, d = prob.X.shape
    c = prob.Y.shape[1]
    ctx = binding.Context(n=n, d=d, c=c, mode=mode, **kw)
    dt = torch.float64 if mode == "fp64" else torch.float32
    X = torch.from_numpy(prob.X).to(device="cuda", dtype=dt).contiguous()
    Y = torch.from_numpy(prob.Y).to(device="cuda", dtype=dt).contiguous()
    ctx.hessian(X, Y)
    ctx.factor_samples()
    ctx.fit()
    return ctx


@pytest.mark.parametrize("basis", ["mono", "cheb_log"])
def test_fp64_gradient_matches_oracle_and_central_differences(torch_mod, basis):
    torch = torch_mod
    prob = synth.spectral_gaussian(600, 100, 3, seed=60)
    kw = dict(k=4, g=4, r=2, q=9, basis=basis)
    ctx = _setup(torch, prob, "fp64", **kw)
    tau = oracle.trace_scale(prob.X)
    for rel in (0.01, 0.3):
        ll = math.log(rel * tau)
        E, dE = (t.cpu().numpy() for t in ctx.holdout_grad(ll))
        ref = oracle.holdout_grad(prob.X, prob.Y, log_lam=ll, **kw)
        np.testing.assert_allclose(E, ref.E, rtol=1e-10)
        np.testing.assert_allclose(dE, ref.dE, rtol=1e-8, atol=1e-12 * np.abs(E).max())
        h = 1e-4
        Ep = ctx.holdout_grad(ll + h)[0].cpu().numpy()
        Em = ctx.holdout_grad(ll - h)[0].cpu().numpy()
        np.testing.assert_allclose(dE, (Ep - Em) / (2 * h), rtol=1e-5, atol=1e-10 * np.abs(E).max())
    assert ctx.info().code == 0


def test_mixed_gradient_matches_oracle(torch_mod):
    torch = torch_mod
    prob = synth.mixed_ecc(n=4096, d=200)
    kw = dict(k=5, g=5, r=3, q=51, basis="cheb_log")
    ctx = _setup(torch, prob, "mixed", **kw)
    tau = oracle.trace_scale(prob.X)
    for rel in (0.02, 0.5):
        ll = math.log(rel * tau)
        E, dE = (t.cpu().numpy() for t in ctx.holdout_grad(ll))
        ref = oracle.holdout_grad(prob.X, prob.Y, log_lam=ll, **kw)
        np.testing.assert_allclose(E, ref.E, rtol=1e-4)
        # the derivative is a difference of O(E) terms computed in fp32
        np.testing.assert_allclose(dE, ref.dE, rtol=1e-3, atol=1e-4 * np.abs(ref.E).max())


def test_wavefront_wait_runs_out_and_the_context_recovers(torch_mod):
    """The few-system solve's waits on blocks of other CTAs are bounded: a pass
    whose first tile row never runs latches PICHOL_ERR_TIMEOUT (some fold, a
    waiting row >= 1, block 0) without a fault or a hang, writes none of the
    context's results, and after clearing the status the gradient is the same as
    before."""
    torch = torch_mod
    prob = synth.mixed_ecc(n=2048, d=200)
    kw = dict(k=5, g=5, r=3, q=21, basis="cheb_log")
    ctx = _setup(torch, prob, "mixed", **kw)
    ll = math.log(0.3 * oracle.trace_scale(prob.X))
    E0, dE0 = (t.cpu().numpy().copy() for t in ctx.holdout_grad(ll))
    assert ctx.info().code == 0
    ctx.check_wave_timeout(2_000_000)
    info = ctx.info()
    assert info.code == 5 and 0 <= info.fold < 5 and 1 <= info.index < 4 and info.pivot == 0
    ctx.clear_status()
    E1, dE1 = (t.cpu().numpy() for t in ctx.holdout_grad(ll))
    assert ctx.info().code == 0
    np.testing.assert_allclose(E1, E0, rtol=1e-6)
    np.testing.assert_allclose(dE1, dE0, rtol=1e-6, atol=1e-9 * np.abs(E0).max())


def test_wavefront_wait_check_is_unsupported_in_fp64(torch_mod):
    from paper_1404_0466_gb300 import binding
    prob = synth.spectral_gaussian(300, 100, 2, seed=7)
    ctx = _setup(torch_mod, prob, "fp64", k=3, g=3, r=2, q=5)
    with pytest.raises(binding.PicholError) as err:
        ctx.check_wave_timeout(1000)
    assert err.value.code == 6                                       # PICHOL_ERR_UNSUPPORTED
    assert ctx.info().code == 0


def test_interpolated_gradient_is_close_to_exact_cholesky_gradient(torch_mod):
    """Near the sampled lambdas the polynomial follows the exact factor, so the
    gradient through it stays close to the exact-Cholesky gradient (FP64 oracle)."""
    torch = torch_mod
    prob = synth.spectral_gaussian(800, 64, 4, seed=61)
    kw = dict(k=4, g=5, r=3, q=5, lo=0.05, hi=0.5, basis="cheb_log")
    ctx = _setup(torch, prob, "fp64", k=4, g=5, r=3, q=5, lam_lo=0.05, lam_hi=0.5, basis="cheb_log")
    tau = oracle.trace_scale(prob.X)
    ll = math.log(0.15 * tau)
    _, dE = ctx.holdout_grad(ll)
    ex = oracle.holdout_grad(prob.X, prob.Y, log_lam=ll, exact=True, **kw)
    dE = dE.cpu().numpy()
    assert np.all(np.sign(dE) == np.sign(ex.dE))
    np.testing.assert_allclose(dE, ex.dE, rtol=0.05)


def test_autograd_and_gradient_steps_on_log_lambda(torch_mod):
    torch = torch_mod
    from paper_1404_0466_gb300 import binding
    prob = synth.spectral_gaussian(1000, 64, 4, seed=62)
    ctx = _setup(torch, prob, "fp64", k=5, g=5, r=3, q=21, basis="cheb_log")
    tau = oracle.trace_scale(prob.X)
    ll = torch.tensor(math.log(0.3 * tau), dtype=torch.float64, requires_grad=True)
    loss = binding.holdout_loss(ctx, ll)
    loss.backward()
    E, dE = ctx.holdout_grad(float(ll.detach()))
    assert abs(float(ll.grad) - float(dE.mean())) <= 1e-12 * abs(float(dE.mean())) + 1e-15
    assert abs(float(loss.detach()) - float(E.mean())) <= 1e-14
    # 20 gradient steps on log(lambda) lower the mean hold-out error
    opt = torch.optim.SGD([ll], lr=0.5 / max(1e-12, abs(float(ll.grad)) * 10))
    first = float(loss.detach())
    for _ in range(20):
        opt.zero_grad()
        loss = binding.holdout_loss(ctx, ll)
        loss.backward()
        opt.step()
    assert float(binding.holdout_loss(ctx, ll).detach()) <= first
