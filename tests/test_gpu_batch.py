"""Batches of independent problems of uneven size (pichol_batch_run): every
problem against the FP64 oracle, and a CUDA-graph replay of the whole batch
against the eager run."""
import numpy as np
import pytest

import oracle
import tolerances
from paper_1404_0466_gb300 import synth

pytestmark = pytest.mark.gpu

K, G, R, Q = 5, 5, 3, 51


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    from paper_1404_0466_gb300 import build
    build.build()
    return torch


def _batch(torch, probs, mode):
    from paper_1404_0466_gb300 import binding
    specs = [dict(n=p.X.shape[0], d=p.X.shape[1], c=p.Y.shape[1], k=K, g=G, r=R, q=Q, basis="cheb_log", mode=mode)
             for p in probs]
    b = binding.Batch(specs, nstreams=3)
    dt = torch.float64 if mode == "fp64" else torch.float32
    Xs = [torch.from_numpy(p.X).to(device="cuda", dtype=dt).contiguous() for p in probs]
    Ys = [torch.from_numpy(p.Y).to(device="cuda", dtype=dt).contiguous() for p in probs]
    return b, Xs, Ys


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_batch_matches_oracle_per_problem(torch_mod, mode):
    torch = torch_mod
    probs = synth.batched_uneven(6, seed=7, d_lo=40, d_hi=200)
    b, Xs, Ys = _batch(torch, probs, mode)
    E, t_star = b.run(Xs, Ys)
    torch.cuda.synchronize()
    ts = t_star.cpu().numpy()
    for i, p in enumerate(probs):
        ref = oracle.cv(p.X, p.Y, k=K, g=G, r=R, q=Q, basis="cheb_log")
        got = E[i].cpu().numpy()
        tol = 1e-9 if mode == "fp64" else tolerances.MIXED_RTOL
        rel = np.abs(got - ref.E) / np.abs(ref.E)
        assert np.all(rel <= tol), (i, float(rel.max()))
        assert tolerances.same_choice(ref.Ebar, int(ts[i]), ref.t_star, tol), (i, ts[i], ref.t_star)
        assert b.info(i).code == 0
    assert b.launch_count() > 0
    b.close()


def test_batch_graph_replay_equals_eager_run(torch_mod):
    torch = torch_mod
    probs = synth.batched_uneven(5, seed=8, d_lo=64, d_hi=300)
    b, Xs, Ys = _batch(torch, probs, "mixed")
    b.run(Xs, Ys)                                  # creates streams and kernel attributes
    torch.cuda.synchronize()
    eager = [e.clone() for e in b.E]
    t_eager = b.t_star.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.run(Xs, Ys)
    for e in b.E:
        e.zero_()
    b.t_star.fill_(-7)
    g.replay()
    torch.cuda.synchronize()
    for a, e in zip(eager, b.E):
        assert torch.equal(a, e)
    assert torch.equal(t_eager, b.t_star)
    b.close()


def test_batch_stage_timing_per_problem(torch_mod):
    torch = torch_mod
    probs = synth.batched_uneven(3, seed=9, d_lo=64, d_hi=160)
    b, Xs, Ys = _batch(torch, probs, "mixed")
    b.set_streams(1)
    b.set_timing(256)
    b.run(Xs, Ys)
    torch.cuda.synchronize()
    for i in range(len(probs)):
        st, complete = b.stage_times(i)
        assert complete
        for stage in ("gram", "chol_diag", "fit", "solve", "score"):
            ms, launches = st[stage]
            assert launches > 0 and ms > 0.0, (i, stage)
    b.set_timing(0)
    b.close()
