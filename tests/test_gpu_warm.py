"""GPU parity of the warm start across folds (warm_samples = g'): fold 0 fitted
from its g sampled factors, every other fold from g' exact factors and fold
0's coefficients, against the oracle's cv(..., warm=g') through the C ABI.

Tolerances as in the other parity tests: double precision 1e-10 of the
matrix scale for factors, 1e-9 for coefficients, 1e-10 relative for hold-out
errors with the same argmin; mixed precision the conditioning tolerance.
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


@pytest.mark.parametrize("warm", [2, 3])
def test_warm_start_fp64_factors_coefficients_and_errors(torch_mod, warm):
    torch = torch_mod
    cfg = synth.FP64_SMALL
    k, g, r, q = cfg["k"], cfg["g"], cfg["r"], cfg["q"]
    prob = synth.fp64_small()
    d = prob.X.shape[1]
    ref = oracle.cv(prob.X, prob.Y, k=k, g=g, r=r, q=q, basis="mono", warm=warm, keep=True)
    ctx = _ctx(prob, k=k, g=g, r=r, q=q, basis="mono", mode="fp64", warm_samples=warm)
    out = ctx.run(_dev(torch, prob.X, "fp64"), _dev(torch, prob.Y, "fp64"))
    torch.cuda.synchronize()
    assert ctx.info().code == 0
    for f in range(k):
        for s in range(g if f == 0 else warm):
            L = ctx.export_factor(f, s).cpu().numpy()
            Lr = ref.factors[(f, s)]
            assert np.max(np.abs(L - Lr)) <= 1e-10 * np.max(np.abs(Lr)), (f, s)
        Th = ctx.export_theta(f).cpu().numpy()
        scale = max(np.max(np.abs(oracle.unvec_lower(ref.theta[f][m], d))) for m in range(r + 1))
        for m in range(r + 1):
            Tr = oracle.unvec_lower(ref.theta[f][m], d)
            assert np.max(np.abs(Th[m] - Tr)) <= 1e-9 * scale, (f, m)
    E = out.E.cpu().numpy()
    assert np.max(np.abs(E - ref.E) / ref.E) <= 1e-10
    assert int(out.t_star.cpu().item()) == ref.t_star
    ctx.close()


def test_warm_start_mixed_case(torch_mod):
    torch = torch_mod
    prob = synth.mixed_ecc(n=4096, d=200)
    k, g, r, q = 5, 6, 3, 101
    ref = oracle.cv(prob.X, prob.Y, k=k, g=g, r=r, q=q, basis="cheb_log", warm=2)
    ctx = _ctx(prob, k=k, g=g, r=r, q=q, basis="cheb_log", mode="mixed", refine_steps=1, warm_samples=2)
    out = ctx.run(_dev(torch, prob.X, "mixed"), _dev(torch, prob.Y, "mixed"))
    torch.cuda.synchronize()
    assert ctx.info().code == 0
    E = out.E.cpu().numpy()
    rel = np.abs(E - ref.E) / ref.E
    assert np.all(rel <= tolerances.MIXED_RTOL), float(rel.max())
    t = int(out.t_star.cpu().item())
    assert tolerances.same_choice(ref.Ebar, t, ref.t_star), (t, ref.t_star)
    ctx.close()


def test_warm_start_rules(torch_mod):
    """Folds f > 0 export only their g' factors, and PINRMSE needs common samples."""
    from paper_1404_0466_gb300 import binding
    torch = torch_mod
    prob = synth.fp64_small(n=600, d=40)
    ctx = _ctx(prob, k=4, g=5, r=3, q=21, mode="fp64", warm_samples=2)
    ctx.hessian(_dev(torch, prob.X, "fp64"), _dev(torch, prob.Y, "fp64"))
    ctx.factor_samples()
    ctx.export_factor(0, 4)
    ctx.export_factor(1, 1)
    with pytest.raises(binding.PicholError) as ei:
        ctx.export_factor(1, 2)
    assert ei.value.code == 1
    with pytest.raises(binding.PicholError) as ei:
        ctx.eval_pinrmse()
    assert ei.value.code == 6
    torch.cuda.synchronize()
    assert ctx.info().code == 0
    ctx.close()


def test_warm_start_with_every_sample_matches_the_plain_fit(torch_mod):
    """g' = g: Theta_0 + V^+ (T - V Theta_0) = V^+ T, so the device's warm-started
    errors equal its plain piCholesky errors up to rounding."""
    torch = torch_mod
    prob = synth.fp64_small(n=1000, d=90)
    kw = dict(k=4, g=5, r=3, q=21, basis="cheb_log", mode="fp64")
    X, Y = _dev(torch, prob.X, "fp64"), _dev(torch, prob.Y, "fp64")
    a = _ctx(prob, **kw).run(X, Y).E.cpu().numpy()
    b = _ctx(prob, warm_samples=5, **kw).run(X, Y).E.cpu().numpy()
    torch.cuda.synchronize()
    np.testing.assert_allclose(b, a, rtol=1e-10)
