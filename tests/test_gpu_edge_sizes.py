"""The largest sizes the C ABI accepts: q = 4096 grid points, g = 32 samples,
degree r = 5 and c = 32 outputs (against the oracle; FP64 mode up to the
largest degree and output count its shared memory holds), and d = 16384
features (256 tiles per side; mixed mode, checked on sampled Gram and factor
entries and on hold-out errors recomputed from the returned solutions)."""
import math

import numpy as np
import pytest

import oracle
import tolerances
from paper_1404_0466_gb300 import synth

pytestmark = pytest.mark.gpu
U32 = tolerances.U32


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    from paper_1404_0466_gb300 import build
    build.build()
    return torch


def _vs_oracle(torch, mode, tol_fn, *, c, r):
    from paper_1404_0466_gb300 import binding
    prob = synth.spectral_gaussian(1000, 96, c, seed=80)
    kw = dict(k=5, g=32, r=r, q=4096, basis="cheb_log")
    ref = oracle.cv(prob.X, prob.Y, **kw)
    ctx = binding.Context(n=1000, d=96, c=c, mode=mode, **kw)
    dt = torch.float64 if mode == "fp64" else torch.float32
    out = ctx.run(torch.from_numpy(prob.X).to("cuda", dt), torch.from_numpy(prob.Y).to("cuda", dt))
    E = out.E.cpu().numpy()
    fin = np.isfinite(ref.E)
    assert np.array_equal(np.isfinite(E), fin)
    tol = tol_fn(prob, ref)
    assert np.all(np.abs(E[fin] - ref.E[fin]) <= tol * ref.E[fin]), float(np.max(np.abs(E[fin] - ref.E[fin]) / ref.E[fin]))
    t = int(out.t_star.cpu().item())
    assert tolerances.same_choice(ref.Ebar, t, ref.t_star, tol), (t, ref.t_star)
    assert ctx.info().code == 0


def test_largest_grid_samples_and_degree_fp64(torch_mod):
    """q = 4096, g = 32, r = 5 in FP64 mode with c = 4 (with degree 5 the FP64
    solve's double-buffered planes leave room for at most 4 outputs)."""
    _vs_oracle(torch_mod, "fp64", lambda prob, ref: 1e-10, c=4, r=5)


def test_largest_grid_samples_degree_and_outputs_mixed(torch_mod):
    """q = 4096, g = 32, r = 5, c = 32 in mixed mode (1e-4)."""
    _vs_oracle(torch_mod, "mixed", lambda prob, ref: tolerances.MIXED_RTOL, c=32, r=5)


def test_largest_dimension_mixed(torch_mod):
    torch = torch_mod
    from paper_1404_0466_gb300 import binding
    n, d, c, k, g = 2000, 16384, 2, 5, 4
    prob = synth.random_fourier(n, d, c, seed=81)
    ctx = binding.Context(n=n, d=d, c=c, k=k, g=g, r=2, q=7, lam_lo=0.1, lam_hi=10.0, basis="cheb_log",
                          mode="mixed", exact_batch=g)
    out = ctx.run(torch.from_numpy(prob.X).cuda(), torch.from_numpy(prob.Y).cuda(), want_w=True)
    torch.cuda.synchronize()
    assert ctx.info().code == 0
    E = out.E.cpu().numpy()
    t_star = int(out.t_star.cpu().item())
    lam = ctx.lambdas().cpu().numpy()
    lam_s = lam[oracle.sample_indices(7, g)]
    offs = oracle.fold_offsets(n, k)
    rng = np.random.default_rng(81)
    # Gram: sampled entries of H_0 against dot products over fold 0's training rows
    H, B = (t.cpu().numpy() for t in ctx.export_hessian(0))
    Xtr = prob.X[offs[1]:].astype(np.float64)
    cols = np.unique(rng.integers(0, d, size=64))
    Hs = Xtr[:, cols].T @ Xtr[:, cols]
    err = np.max(np.abs(H[np.ix_(cols, cols)] - Hs)) / np.max(np.abs(np.diag(H)))
    assert err <= 8 * math.sqrt(Xtr.shape[0]) * U32, err
    # factor at the smallest sample: |A - L L^T| <= gamma_{d+1} |L| |L^T| (+ fp32 rounding of H)
    L = ctx.export_factor(0, 0).cpu().numpy()
    gam = (d + 1) * U32 / (1 - (d + 1) * U32)
    pairs = np.sort(rng.integers(0, d, size=(64, 2)), axis=1)[:, ::-1]
    for a, b in np.vstack([pairs, np.stack([cols, cols], axis=1)]):
        llt = float(L[a, : b + 1] @ L[b, : b + 1])
        ref = H[a, b] + (lam_s[0] if a == b else 0.0)
        bound = gam * float(np.abs(L[a, : b + 1]) @ np.abs(L[b, : b + 1])) + U32 * abs(H[a, b])
        assert abs(llt - ref) <= bound, (a, b, llt, ref, bound)
    del L, H
    # hold-out errors recomputed from the returned solutions
    X0 = prob.X[: offs[1]].astype(np.float64)
    Y0 = prob.Y[: offs[1]].astype(np.float64)
    assert np.isfinite(E[0, t_star])
    for t in sorted({0, t_star}):
        if not np.isfinite(E[0, t]):
            continue
        W = out.W[0, t].cpu().numpy().astype(np.float64)
        Eh = float(np.sum((Y0 - X0 @ W) ** 2)) / (Y0.shape[0] * c)
        assert abs(E[0, t] - Eh) <= 1e-4 * Eh, (t, E[0, t], Eh)
