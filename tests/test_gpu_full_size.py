"""Parity at the full sizes of the GPU workloads, in the launch configuration
the benchmark uses, on outputs the oracle can compute one by one or on
properties that hold at any size.

* Mixed case (n = 32768, d = 2048, c = 10, k = 5, g = 6, r = 3, q = 101,
  one refinement step): every hold-out error and the selected lambda against
  the FP64 oracle.
* Large random-Fourier case (n = 131072, d = 8192, c = 32): sampled Gram
  entries against direct dot products; sampled entries of L L^T against
  H_f + lambda_s I (Cholesky backward error); sampled coefficient vectors
  against the oracle's least-squares fit of the exported factors; the
  interpolated system's residual (backward error of the triangular solves);
  the hold-out error recomputed from the returned solutions.
* Batched case (64 problems of uneven size, one CUDA graph replay): four
  problems spread over the size range against the oracle.
* Differentiation case (n = 16384, d = 1024): the error and its derivative in
  log(lambda) against the oracle's interpolated gradient, the oracle's central
  differences (h = 1e-4) and the exact-Cholesky gradient; 20 gradient steps.
"""
import math
import os

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


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to("cuda")


def _ctx(cfg, **kw):
    from paper_1404_0466_gb300 import binding
    return binding.Context(n=cfg["n"], d=cfg["d"], c=cfg["c"], k=cfg["k"], g=cfg["g"], r=cfg["r"], q=cfg["q"],
                           lam_lo=cfg["lo"], lam_hi=cfg["hi"], basis="cheb_log", mode="mixed",
                           exact_batch=cfg["g"], **kw)


def test_mixed_ecc_full_size(torch_mod):
    torch = torch_mod
    cfg = synth.MIXED_ECC
    prob = synth.mixed_ecc()
    ctx = _ctx(cfg, refine_steps=1)
    out = ctx.run(_dev(torch, prob.X), _dev(torch, prob.Y))
    E = out.E.cpu().numpy()
    t_star = int(out.t_star.cpu().item())
    assert ctx.info().code == 0
    ref = oracle.cv(prob.X, prob.Y, k=cfg["k"], g=cfg["g"], r=cfg["r"], q=cfg["q"], lo=cfg["lo"], hi=cfg["hi"],
                    basis="cheb_log")
    rel = np.abs(E - ref.E) / ref.E
    assert np.all(rel <= tolerances.MIXED_RTOL), float(rel.max())
    assert tolerances.same_choice(ref.Ebar, t_star, ref.t_star), (t_star, ref.t_star)


def test_large_rff_full_size_properties(torch_mod):
    torch = torch_mod
    cfg = synth.LARGE_RFF
    prob = synth.large_rff()
    n, d, c, k, g, r, q = (cfg[x] for x in ("n", "d", "c", "k", "g", "r", "q"))
    p = r + 1
    ctx = _ctx(cfg, refine_steps=1)
    out = ctx.run(_dev(torch, prob.X), _dev(torch, prob.Y), want_w=True)
    torch.cuda.synchronize()
    assert ctx.info().code == 0
    E = out.E.cpu().numpy()
    t_star = int(out.t_star.cpu().item())
    lam = ctx.lambdas().cpu().numpy()
    # tau = tr(H)/d carries the Gram's error bound (positive diagonal terms)
    np.testing.assert_allclose(lam, oracle.lambda_grid(oracle.trace_scale(prob.X), q, cfg["lo"], cfg["hi"]),
                               rtol=8 * math.sqrt(n) * U32)
    lam_s = lam[oracle.sample_indices(q, g)]
    offs = oracle.fold_offsets(n, k)
    rng = np.random.default_rng(2024)

    # (a) Gram: sampled entries of H_0 and B_0 against dot products over fold 0's training rows
    H, B = (t.cpu().numpy() for t in ctx.export_hessian(0))
    Xtr, Ytr = prob.X[offs[1]:], prob.Y[offs[1]:].astype(np.float64)
    ntr = Xtr.shape[0]
    cols = np.unique(rng.integers(0, d, size=96))
    Xs = Xtr[:, cols].astype(np.float64)
    Hs = Xs.T @ Xs
    tol_h = 8 * math.sqrt(ntr) * U32
    err = np.max(np.abs(H[np.ix_(cols, cols)] - Hs)) / np.max(np.abs(np.diag(H)))
    assert err <= tol_h, err
    errb = np.max(np.abs(B[cols] - Xs.T @ Ytr)) / np.max(np.abs(B))
    assert errb <= tol_h, errb
    del Xs, Hs

    # (b) factors: |A - L L^T| <= gamma_{d+1} |L| |L^T| (+ the fp32 rounding of H), sampled entries
    pairs = rng.integers(0, d, size=(256, 2))
    pairs = np.sort(pairs, axis=1)[:, ::-1]                    # a >= b
    pairs = np.vstack([pairs, np.stack([cols, cols], axis=1)])
    gam = (d + 1) * U32 / (1 - (d + 1) * U32)
    T = np.empty((g, len(pairs)))
    for s in range(g):
        L = ctx.export_factor(0, s).cpu().numpy()
        T[s] = L[pairs[:, 0], pairs[:, 1]]
        if s in (0, g - 1):
            for a, b in pairs[:64]:
                llt = float(L[a, : b + 1] @ L[b, : b + 1])
                ref = H[a, b] + (lam_s[s] if a == b else 0.0)
                bound = gam * float(np.abs(L[a, : b + 1]) @ np.abs(L[b, : b + 1])) + U32 * abs(H[a, b])
                assert abs(llt - ref) <= bound, (s, a, b, llt, ref, bound)
        del L

    # (c) fit: Theta = V^+ T per entry; fp32 contraction with P = V^+ rounded to fp32
    Theta = ctx.export_theta(0).cpu().numpy()
    V = oracle.basis_values("cheb_log", lam_s, lam_s, p)
    th_ref = oracle.lstsq(V, T)
    P = oracle.lstsq(V, np.eye(g))
    bound = (g + 2) * U32 * (np.abs(P) @ np.abs(T)) + 1e-12 * np.max(np.abs(T))
    got = Theta[:, pairs[:, 0], pairs[:, 1]]
    assert np.all(np.abs(got - th_ref) <= bound), float(np.max(np.abs(got - th_ref) / bound))

    # (d) solves and scoring at the smallest lambda and the selected one
    X0 = prob.X[: offs[1]].astype(np.float64)
    Y0 = prob.Y[: offs[1]].astype(np.float64)
    assert np.isfinite(E[0, t_star])
    for t in sorted({0, t_star}):
        if not np.isfinite(E[0, t]):
            continue                          # flagged unusable: scored +inf by design
        phi = oracle.basis_values("cheb_log", [lam[t]], lam_s, p)[0]
        Lt = np.tril(np.tensordot(phi, Theta, axes=1))
        S = np.tril(np.tensordot(np.abs(phi), np.abs(Theta), axes=1))
        W = out.W[0, t].cpu().numpy().astype(np.float64)
        R = B - Lt @ (Lt.T @ W)
        scale = np.linalg.norm(S @ (S.T @ np.abs(W)))
        # backward error of the two fp32 triangular solves (gamma_d each), the fp32
        # evaluation of L~ from Theta ((p + 1) u32 per entry, twice) and W's rounding
        back = (2 * d + 2 * (p + 1) + 4) * U32
        assert np.linalg.norm(R) <= back * scale, (t, np.linalg.norm(R) / scale)
        Eh = float(np.sum((Y0 - X0 @ W) ** 2)) / (Y0.shape[0] * c)
        assert abs(E[0, t] - Eh) <= 1e-4 * Eh, (t, E[0, t], Eh)


def _golden_large_rff():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "large_rff_fold0.txt")
    out = {"idx": [], "lam": [], "E": []}
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            if key in ("tau", "y_sum"):
                out[key] = float(vals[0])
            elif key == "fingerprint_rows":
                out[key] = [int(v) for v in vals]
            elif key == "fingerprint_sums":
                out[key] = [float(v) for v in vals]
            else:
                out["idx"].append(int(key))
                out["lam"].append(float(vals[0]))
                out["E"].append(float(vals[1]))
    return out


def test_large_rff_holdout_errors_against_the_oracle(torch_mod):
    """Fold 0 of the large random-Fourier case at five grid lambdas against the
    FP64 oracle's hold-out errors (stored in tests/golden by a script that runs
    only the oracle: its Gram step is ~3.5e12 multiply-adds of plain loops).
    The regenerated inputs are first checked against the stored fingerprint."""
    torch = torch_mod
    gold = _golden_large_rff()
    cfg = synth.LARGE_RFF
    prob = synth.large_rff()
    for r, s in zip(gold["fingerprint_rows"], gold["fingerprint_sums"]):
        assert abs(float(np.sum(prob.X[r].astype(np.float64))) - s) <= 1e-6 * max(1.0, abs(s)), r
    assert abs(float(np.sum(prob.Y.astype(np.float64))) - gold["y_sum"]) <= 1e-6 * abs(gold["y_sum"])
    ctx = _ctx(cfg, refine_steps=1)
    out = ctx.run(_dev(torch, prob.X), _dev(torch, prob.Y))
    torch.cuda.synchronize()
    assert ctx.info().code == 0
    lam = ctx.lambdas().cpu().numpy()
    idx = gold["idx"]
    np.testing.assert_allclose(lam[idx], gold["lam"], rtol=8 * math.sqrt(cfg["n"]) * U32)
    E = out.E.cpu().numpy()[0, idx]
    ref = np.array(gold["E"])
    rel = np.abs(E - ref) / ref
    assert np.all(rel <= tolerances.MIXED_RTOL), rel
    assert int(np.argmin(E)) == int(np.argmin(ref))
    ctx.close()


def test_batched_uneven_full_size(torch_mod):
    torch = torch_mod
    from paper_1404_0466_gb300 import binding
    K, G, R, Q, lo, hi = 5, 5, 3, 51, 1e-3, 1e1
    probs = synth.batched_uneven(64, seed=3, dtype=np.float32)
    specs = [dict(n=pb.X.shape[0], d=pb.X.shape[1], c=pb.Y.shape[1], k=K, g=G, r=R, q=Q, lam_lo=lo, lam_hi=hi,
                  basis="cheb_log", mode="mixed", refine_steps=1) for pb in probs]
    b = binding.Batch(specs, nstreams=16)
    Xs = [_dev(torch, pb.X) for pb in probs]
    Ys = [_dev(torch, pb.Y) for pb in probs]
    b.run(Xs, Ys)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        b.run(Xs, Ys)
    for e in b.E:
        e.fill_(-1.0)
    graph.replay()
    torch.cuda.synchronize()
    by_size = sorted(range(len(probs)), key=lambda i: probs[i].X.shape[1])
    pick = [by_size[(2 * j + 1) * len(probs) // 8] for j in range(4)]
    idx = [0, Q // 4, Q // 2, 3 * Q // 4, Q - 1]
    for i in pick:
        pb = probs[i]
        ref = oracle.cv(pb.X, pb.Y, k=K, g=G, r=R, q=Q, lo=lo, hi=hi, basis="cheb_log", folds=[0], lam_idx=idx)
        got = b.E[i][0].cpu().numpy()[idx]
        rel = np.abs(got - ref.E[0, idx]) / ref.E[0, idx]
        assert np.all(rel <= tolerances.MIXED_RTOL), (i, pb.X.shape[1], rel)
    for i in range(len(probs)):
        assert b.info(i).code == 0, i
    b.close()


def test_differentiation_full_size(torch_mod):
    torch = torch_mod
    from paper_1404_0466_gb300 import binding
    cfg = synth.DIFFERENTIATION
    prob = synth.differentiation()
    k, g, r, q = cfg["k"], cfg["g"], cfg["r"], cfg["q"]
    ctx = _ctx(cfg)
    ctx.hessian(_dev(torch, prob.X), _dev(torch, prob.Y))
    ctx.factor_samples()
    ctx.fit()
    tau = oracle.trace_scale(prob.X)
    ll = math.log(0.113 * tau)
    kw = dict(k=k, g=g, r=r, q=q, lo=cfg["lo"], hi=cfg["hi"], basis="cheb_log", folds=[0])
    E, dE = (t.cpu().numpy() for t in ctx.holdout_grad(ll))
    assert ctx.info().code == 0
    ref = oracle.holdout_grad(prob.X, prob.Y, log_lam=ll, **kw)
    tolE = tolerances.MIXED_RTOL
    assert abs(E[0] - ref.E[0]) <= tolE * ref.E[0], (E[0], ref.E[0])
    # the derivative is a difference of O(E) terms computed in fp32 after two solves
    tolD = 1e-3
    assert abs(dE[0] - ref.dE[0]) <= tolD * abs(ref.dE[0]) + 1e-4 * abs(ref.E[0]), (dE[0], ref.dE[0])
    # central differences of the oracle's interpolated error, h = 1e-4
    h = 1e-4
    fd = (oracle.holdout_grad(prob.X, prob.Y, log_lam=ll + h, **kw).E[0]
          - oracle.holdout_grad(prob.X, prob.Y, log_lam=ll - h, **kw).E[0]) / (2 * h)
    assert abs(ref.dE[0] - fd) <= 1e-6 * abs(fd) + 1e-9 * ref.E[0], (ref.dE[0], fd)
    assert abs(dE[0] - fd) <= tolD * abs(fd) + 1e-4 * abs(ref.E[0]), (dE[0], fd)
    # the exact-Cholesky gradient: inside this window the interpolated factor
    # follows the exact one, so the two derivatives agree in sign and to a few %
    ex = oracle.holdout_grad(prob.X, prob.Y, log_lam=ll, exact=True, **kw)
    assert np.sign(dE[0]) == np.sign(ex.dE[0])
    assert abs(dE[0] - ex.dE[0]) <= 0.05 * abs(ex.dE[0]), (dE[0], ex.dE[0])
    # 20 gradient steps on log(lambda) lower the mean hold-out error
    x = torch.tensor(ll, dtype=torch.float64, requires_grad=True)
    loss = binding.holdout_loss(ctx, x)
    loss.backward()
    first = float(loss.detach())
    opt = torch.optim.SGD([x], lr=0.05 / max(1e-12, abs(float(x.grad))))
    for _ in range(20):
        opt.zero_grad()
        loss = binding.holdout_loss(ctx, x)
        loss.backward()
        opt.step()
    last = float(binding.holdout_loss(ctx, x).detach())
    assert last < first, (first, last)
    lo_ll, hi_ll = math.log(cfg["lo"] * tau), math.log(cfg["hi"] * tau)
    assert lo_ll - 1.0 <= float(x.detach()) <= hi_ll + 1.0
