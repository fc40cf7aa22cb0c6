"""The C ABI's caller inputs against the FP64 oracle given the same inputs:
lambdas off the grid (sampled and evaluated; Sec. 3.3: the interpolant is
evaluated at any lambda without a new factorisation), caller fold offsets
(Sec. 1 leaves the split to the user), the coefficients copied out by
pichol_fit, a checkpoint resumed in a new context, and the degenerate sizes
d = 1 (a scalar ridge) and n = k (one held-out row per fold)."""
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


def _off_grid(prob, g, q, seed):
    """g sampled and q evaluation lambdas, drawn log-uniformly inside
    [2e-3, 5] tau, the evaluation ones unsorted and none on the default grid."""
    rng = np.random.default_rng(seed)
    tau = oracle.trace_scale(prob.X)
    lam_s = np.sort(tau * 10.0 ** rng.uniform(np.log10(2e-3), np.log10(5.0), size=g))
    lam_t = tau * 10.0 ** rng.uniform(np.log10(2e-3), np.log10(5.0), size=q)
    lam_t[0] = lam_s[1]                      # one evaluation lambda on a node
    return lam_s, lam_t


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_caller_lambdas_against_the_oracle(torch_mod, mode):
    torch = torch_mod
    if mode == "fp64":
        prob, kw, tol = synth.fp64_small(n=1024, d=130), dict(k=5, g=4, r=2, q=23, basis="mono"), 1e-10
    else:
        prob, kw, tol = synth.mixed_ecc(n=4096, d=200), dict(k=5, g=6, r=3, q=37, basis="cheb_log"), \
            tolerances.MIXED_RTOL
    lam_s, lam_t = _off_grid(prob, kw["g"], kw["q"], seed=11)
    ctx = _ctx(prob, mode=mode, refine_steps=1 if mode == "mixed" else 0, **kw)
    out = ctx.run(_dev(torch, prob.X, mode), _dev(torch, prob.Y, mode), lam_s=lam_s, lam_t=lam_t)
    torch.cuda.synchronize()
    assert ctx.info().code == 0
    np.testing.assert_array_equal(ctx.lambdas().cpu().numpy(), lam_t)
    ref = oracle.cv(prob.X, prob.Y, lams=lam_t, lam_samples=lam_s, **kw)
    E = out.E.cpu().numpy()
    # pairs whose interpolated diagonal is unusable score +inf on both sides
    fin = np.isfinite(ref.E)
    assert np.array_equal(np.isfinite(E), fin) and fin.sum() > fin.size // 2
    rel = np.abs(E[fin] - ref.E[fin]) / ref.E[fin]
    assert np.all(rel <= tol), float(rel.max())
    assert tolerances.same_choice(ref.Ebar, int(out.t_star.cpu().item()), ref.t_star, tol)
    # exact CV at the same lambdas, and the grid again when no lambdas are given
    ex = ctx.eval_holdout_exact(lam_t=lam_t)
    refx = oracle.cv(prob.X, prob.Y, exact=True, lams=lam_t, **kw)
    relx = np.abs(ex.E.cpu().numpy() - refx.E) / refx.E
    assert np.all(relx <= tol), float(relx.max())
    ctx.close()


def test_no_lambdas_restore_the_grid_bit_for_bit(torch_mod):
    torch = torch_mod
    prob = synth.mixed_ecc(n=4096, d=200)
    kw = dict(k=5, g=6, r=3, q=37, basis="cheb_log", mode="mixed", refine_steps=1)
    ctx = _ctx(prob, **kw)
    X, Y = _dev(torch, prob.X, "mixed"), _dev(torch, prob.Y, "mixed")
    a = ctx.run(X, Y)
    Ea, ta = a.E.clone(), a.t_star.clone()
    grid = ctx.lambdas().clone()
    lam_s, lam_t = _off_grid(prob, 6, 37, seed=12)
    ctx.run(X, Y, lam_s=lam_s, lam_t=lam_t)
    b = ctx.run(X, Y)
    torch.cuda.synchronize()
    assert torch.equal(Ea, b.E) and torch.equal(ta, b.t_star)
    assert torch.equal(grid, ctx.lambdas())
    ctx.close()


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_caller_fold_offsets_against_the_oracle(torch_mod, mode):
    torch = torch_mod
    prob = synth.fp64_small(n=1000, d=100) if mode == "fp64" else synth.mixed_ecc(n=3000, d=150)
    n = prob.X.shape[0]
    offs = [0, 37, 400, 401, 700 if n == 1000 else 2100, n]
    kw = dict(k=5, g=4, r=2, q=15, basis="cheb_log")
    ctx = _ctx(prob, mode=mode, **kw)
    out = ctx.run(_dev(torch, prob.X, mode), _dev(torch, prob.Y, mode), fold_offsets=offs)
    torch.cuda.synchronize()
    assert ctx.info().code == 0
    ref = oracle.cv(prob.X, prob.Y, offsets=offs, **kw)
    tol = 1e-10 if mode == "fp64" else tolerances.MIXED_RTOL
    # the one-row fold's error can be near zero: measured against the larger of
    # it and the fold mean at that lambda
    rel = np.abs(out.E.cpu().numpy() - ref.E) / np.maximum(ref.E, ref.Ebar[None, :])
    assert np.all(rel <= tol), float(rel.max())
    assert tolerances.same_choice(ref.Ebar, int(out.t_star.cpu().item()), ref.t_star, tol)
    # the Hessian of the one-row fold leaves exactly that row out
    H, B = (t.cpu().numpy() for t in ctx.export_hessian(2))
    Hr, Br = oracle.normal_blocks(prob.X, prob.Y, 400, 401)
    scale = np.max(np.abs(np.diag(Hr)))
    assert np.max(np.abs(H - Hr)) <= (1e-12 if mode == "fp64" else 1e-5) * scale
    ctx.close()


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_fit_copies_the_coefficients_out(torch_mod, mode):
    torch = torch_mod
    prob = synth.fp64_small(n=600, d=70)
    ctx = _ctx(prob, k=4, g=4, r=2, q=9, mode=mode, basis="cheb_log")
    ctx.hessian(_dev(torch, prob.X, mode), _dev(torch, prob.Y, mode))
    ctx.factor_samples()
    dt = torch.float64 if mode == "fp64" else torch.float32
    theta = torch.full((ctx.theta_elems(),), float("nan"), dtype=dt, device="cuda")
    ctx.fit(theta_out=theta)
    torch.cuda.synchronize()
    d, p, nt = 70, 3, 2
    th = theta.cpu().numpy().astype(np.float64).reshape(4, nt * (nt + 1) // 2, p, 64, 64)
    for f in range(4):
        dense = ctx.export_theta(f).cpu().numpy()            # p x d x d
        for i in range(nt):
            for j in range(i + 1):
                blk = th[f, i * (i + 1) // 2 + j]              # p x 64 x 64
                r0, c0 = 64 * i, 64 * j
                rr, cc = min(64, d - r0), min(64, d - c0)
                np.testing.assert_array_equal(blk[:, :rr, :cc], dense[:, r0:r0 + rr, c0:c0 + cc])
        # padding: the fit of the identity's constant 1 on the padded diagonal
        last = th[f, nt * (nt + 1) // 2 - 1]
        for a in range(d - 64, 64):
            assert abs(last[0, a, a] - 1.0) < 1e-5 and np.all(np.abs(last[1:, a, a]) < 1e-5)
    ctx.close()


def test_checkpoint_resumes_in_a_new_context(torch_mod):
    """state_dict after the fit, a new context of the same configuration,
    load_state_dict, then pichol_eval_holdout without the earlier steps: the
    same scores and choice as the original context, bit for bit."""
    torch = torch_mod
    prob = synth.mixed_ecc(n=4096, d=200)
    kw = dict(k=5, g=6, r=3, q=41, basis="cheb_log", mode="mixed", refine_steps=1)
    a = _ctx(prob, **kw)
    out_a = a.run(_dev(torch, prob.X, "mixed"), _dev(torch, prob.Y, "mixed"))
    torch.cuda.synchronize()
    sd = a.state_dict()
    Ea, ta = out_a.E.clone(), out_a.t_star.clone()
    a.close()
    b = _ctx(prob, **kw)
    b.load_state_dict(sd)
    out_b = b.eval_holdout()
    torch.cuda.synchronize()
    assert b.info().code == 0
    assert torch.equal(Ea, out_b.E) and torch.equal(ta, out_b.t_star)
    ref = oracle.cv(prob.X, prob.Y, k=5, g=6, r=3, q=41, basis="cheb_log")
    assert np.max(np.abs(out_b.E.cpu().numpy() - ref.E) / ref.E) <= tolerances.MIXED_RTOL
    b.close()


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_scalar_ridge_d1(torch_mod, mode):
    """d = 1: every factor is the scalar sqrt(h + lambda) in a 64 x 64 tile
    whose other 63 rows are padding."""
    torch = torch_mod
    prob = synth.spectral_gaussian(200, 1, 2, seed=31)
    kw = dict(k=4, g=4, r=2, q=11, basis="cheb_log")
    ctx = _ctx(prob, mode=mode, **kw)
    out = ctx.run(_dev(torch, prob.X, mode), _dev(torch, prob.Y, mode))
    torch.cuda.synchronize()
    assert ctx.info().code == 0
    ref = oracle.cv(prob.X, prob.Y, **kw)
    tol = 1e-10 if mode == "fp64" else tolerances.MIXED_RTOL
    rel = np.abs(out.E.cpu().numpy() - ref.E) / ref.E
    assert np.all(rel <= tol), float(rel.max())
    assert tolerances.same_choice(ref.Ebar, int(out.t_star.cpu().item()), ref.t_star, tol)
    ctx.close()


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_one_held_out_row_per_fold(torch_mod, mode):
    """n = k: leave-one-out cross-validation, each fold a single row."""
    torch = torch_mod
    prob = synth.spectral_gaussian(40, 12, 3, seed=32)
    kw = dict(k=40, g=4, r=2, q=9, basis="mono")
    ctx = _ctx(prob, mode=mode, **kw)
    out = ctx.run(_dev(torch, prob.X, mode), _dev(torch, prob.Y, mode))
    torch.cuda.synchronize()
    assert ctx.info().code == 0
    ref = oracle.cv(prob.X, prob.Y, **kw)
    fin = np.isfinite(ref.E)
    E = out.E.cpu().numpy()
    assert np.array_equal(np.isfinite(E), fin)
    tol = 1e-9 if mode == "fp64" else tolerances.MIXED_RTOL
    # one row's error can be near zero: measured against the larger of it and
    # the fold mean at that lambda
    scale = np.maximum(ref.E, ref.Ebar[None, :])
    rel = np.abs(E[fin] - ref.E[fin]) / scale[fin]
    assert np.all(rel <= tol), float(rel.max())
    assert tolerances.same_choice(ref.Ebar, int(out.t_star.cpu().item()), ref.t_star, tol)
    ctx.close()
