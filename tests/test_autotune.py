"""Host logic of the launch-shape autotuner (paper_1404_0466_gb300.autotune) on
CPU: a fake context or batch records the tuning each run sees, and a fake timer
returns a cost from a table, so the stages, the argmin, the cache and the
agreement across gloo ranks are checked without a GPU."""
import json
import os
import socket
from types import SimpleNamespace

import pytest

from paper_1404_0466_gb300 import autotune
from paper_1404_0466_gb300.binding import PICHOL_MODE_FP64, PICHOL_MODE_MIXED

KEYS = ("update_strip", "diag_threads", "diag_exclusive", "eval_overlap")


def _cfg(**kw):
    base = dict(n=32768, d=2048, c=10, k=5, g=6, r=3, q=101, mode=PICHOL_MODE_MIXED, basis=1,
                refine_steps=1, refine_target=0, exact_batch=0, warm_samples=0, gram_passes=3)
    base.update(kw)
    return SimpleNamespace(**base)


class FakeContext:
    def __init__(self, cfg):
        self.cfg = cfg
        self._t = dict(update_strip=4, diag_threads=512, diag_exclusive=1, eval_overlap=0, update_engine=1)
        self.runs = []

    def tuning(self):
        return dict(self._t)

    def set_tuning(self, **kw):
        assert set(kw) <= set(KEYS), kw
        self._t.update(kw)

    def _outputs(self, want_w):
        return (None, None, None)

    def run(self, X, Y, out=None, stream=None):
        assert out == (None, None, None)
        self.runs.append(self.tuning())


class FakeBatch:
    def __init__(self, cfgs):
        self.cfgs = cfgs
        self.streams = 8
        self.strip = 4
        self.runs = []

    def set_streams(self, ns):
        self.streams = ns

    def set_tuning(self, update_strip=4, diag_threads=512, diag_exclusive=0, eval_overlap=0):
        self.strip = update_strip

    def run(self, Xs, Ys, stream=None):
        self.runs.append((self.streams, self.strip))


def _ctx_cost(t):
    """A cost with a unique minimum at strip 2, 256 threads, exclusive off and
    overlap on, each stage's choice independent of the others."""
    ms = 20.0
    ms += {1: 3.0, 2: 0.0, 4: 0.5, 8: 2.0}[t["update_strip"]]
    ms += {256: 0.0, 512: 0.25}[t["diag_threads"]]
    ms += {1: 0.3, 0: 0.0}[t["diag_exclusive"]]
    ms += {0: 0.2, 1: 0.0}[t["eval_overlap"]]
    return ms


def _timer_for(obj, cost, calls=None):
    def timer(fn, reps, stream):
        fn()                                # the untimed run
        for _ in range(reps):
            fn()
        if calls is not None:
            calls.append(reps)
        return cost(obj)
    return timer


def test_context_stages_pick_each_fastest_candidate():
    ctx = FakeContext(_cfg())
    calls = []
    res = autotune.tune_context(ctx, "X", "Y", reps=3, timer=_timer_for(ctx, lambda c: _ctx_cost(c.tuning()), calls),
                                device="fake")
    assert res.choice == dict(update_strip=2, diag_threads=256, diag_exclusive=0, eval_overlap=1, update_engine=1)
    assert ctx.tuning() == res.choice and not res.cached
    # 8 shapes, then 2 exclusivity settings, then 2 overlap settings, each 1 + reps runs
    assert calls == [3] * 12 and len(ctx.runs) == 12 * 4
    seen = {(t["update_strip"], t["diag_threads"]) for t in ctx.runs[:32]}
    assert seen == {(a, b) for a in autotune.UPDATE_STRIPS for b in autotune.DIAG_THREADS}
    # the later stages start from the earlier stages' choices
    assert all((t["update_strip"], t["diag_threads"]) == (2, 256) for t in ctx.runs[32:])
    assert all(t["diag_exclusive"] == 0 for t in ctx.runs[40:])
    assert set(res.timings) == {"shapes", "diag_exclusive", "eval_overlap"}
    assert res.timings["shapes"]["strip2_diag256"] == pytest.approx(20.5)


@pytest.mark.parametrize("cfg", [_cfg(mode=PICHOL_MODE_FP64), _cfg(refine_steps=0)])
def test_context_overlap_is_tuned_only_with_mixed_refinement(cfg):
    ctx = FakeContext(cfg)
    res = autotune.tune_context(ctx, "X", "Y", timer=_timer_for(ctx, lambda c: _ctx_cost(c.tuning())), device="fake")
    assert res.choice["eval_overlap"] == 0
    assert "eval_overlap" not in res.timings
    assert len(ctx.runs) == 10 * 3


def test_equal_times_keep_the_first_listed_candidate():
    ctx = FakeContext(_cfg())
    res = autotune.tune_context(ctx, "X", "Y", timer=_timer_for(ctx, lambda c: 1.0), device="fake")
    assert res.choice == dict(update_strip=autotune.UPDATE_STRIPS[0], diag_threads=autotune.DIAG_THREADS[0],
                              diag_exclusive=autotune.DIAG_EXCLUSIVE[0], eval_overlap=autotune.EVAL_OVERLAP[0],
                              update_engine=1)


def test_context_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    ctx = FakeContext(_cfg())
    first = autotune.tune_context(ctx, "X", "Y", cache=path, timer=_timer_for(ctx, lambda c: _ctx_cost(c.tuning())),
                                  device="GB300")
    stored = json.load(open(path))
    # the cache keeps the tuned launch shapes (the update engine is the caller's choice)
    assert stored == {first.key: {k: v for k, v in first.choice.items() if not k.endswith("_engine")}}
    assert first.key.startswith("GB300|context|n=32768,d=2048,c=10,k=5,g=6,r=3,q=101,")

    def no_timing(fn, reps, stream):
        raise AssertionError("a cached choice must not be timed")

    again = FakeContext(_cfg())
    res = autotune.tune_context(again, "X", "Y", cache=path, timer=no_timing, device="GB300")
    assert res.cached and res.choice == first.choice and again.tuning() == first.choice
    assert again.runs == []
    # another device or another configuration is a different key
    other = FakeContext(_cfg(q=51))
    res = autotune.tune_context(other, "X", "Y", cache=path, timer=_timer_for(other, lambda c: 1.0), device="GB300")
    assert not res.cached and len(json.load(open(path))) == 2
    res = autotune.tune_context(FakeContext(_cfg()), "X", "Y", cache=path, timer=_timer_for(other, lambda c: 1.0),
                                device="B200")
    assert not res.cached and len(json.load(open(path))) == 3
    assert not [f for f in os.listdir(tmp_path) if f.endswith(".tmp")]


def test_bad_arguments_and_a_bad_cache(tmp_path):
    ctx = FakeContext(_cfg())
    with pytest.raises(ValueError):
        autotune.tune_context(ctx, "X", "Y", reps=0, timer=_timer_for(ctx, lambda c: 1.0), device="fake")
    path = tmp_path / "bad.json"
    path.write_text("[1, 2]")
    with pytest.raises(ValueError):
        autotune.tune_context(ctx, "X", "Y", cache=str(path), timer=_timer_for(ctx, lambda c: 1.0), device="fake")
    with pytest.raises(ValueError):
        autotune.tune_batch(FakeBatch([_cfg()]), [], [], reps=0, timer=lambda *a: 1.0, device="fake")


def _batch_cost(b):
    return {4: 5.0, 8: 4.0, 16: 3.5, 32: 3.6}[b.streams] + {1: 0.4, 2: 0.0, 4: 0.1}[b.strip]


def test_batch_grid_and_cache(tmp_path):
    cfgs = [_cfg(n=1000 + 10 * i, d=64 + i) for i in range(5)]
    b = FakeBatch(cfgs)
    path = str(tmp_path / "tune.json")
    res = autotune.tune_batch(b, [], [], cache=path, timer=_timer_for(b, _batch_cost), device="GB300")
    assert res.choice == dict(streams=16, update_strip=2) and (b.streams, b.strip) == (16, 2)
    assert set(b.runs) == {(a, s) for a in autotune.BATCH_STREAMS for s in autotune.BATCH_STRIPS}
    assert res.key.startswith("GB300|batch|5|")
    b2 = FakeBatch(cfgs)
    res2 = autotune.tune_batch(b2, [], [], cache=path, timer=None, device="GB300")
    assert res2.cached and (b2.streams, b2.strip) == (16, 2) and b2.runs == []
    # the key depends on every problem, in order
    assert autotune.batch_key(cfgs[::-1], "GB300") != res.key
    assert autotune.batch_key(cfgs[:4] + [_cfg(n=1040, d=68, q=51)], "GB300") != res.key


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, cache_dir, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pg = dist.group.WORLD
    try:
        # each rank's timings favour a different shape; all must apply rank 0's
        ctx = FakeContext(_cfg())
        bias = {0: (2, 256), 1: (8, 512)}[rank]
        cost = lambda c: 1.0 if (c.tuning()["update_strip"], c.tuning()["diag_threads"]) == bias else 2.0
        path = os.path.join(cache_dir, f"rank{rank}.json")
        res = autotune.tune_context(ctx, "X", "Y", cache=path, pg=pg, timer=_timer_for(ctx, cost), device="fake")
        first = (res.choice["update_strip"], res.choice["diag_threads"], os.path.exists(path))
        # now rank 0 alone has the choice cached: no rank times
        def no_timing(fn, reps, stream):
            raise AssertionError("rank 0's cached choice must be applied without timing")
        shared = os.path.join(cache_dir, "rank0.json")
        again = FakeContext(_cfg())
        res2 = autotune.tune_context(again, "X", "Y", cache=shared if rank == 0 else path + ".none", pg=pg,
                                     timer=no_timing, device="fake")
        second = (res2.cached, res2.choice["update_strip"], res2.choice["diag_threads"])
        b = FakeBatch([_cfg()])
        bcost = lambda x: 1.0 if (x.streams, x.strip) == ({0: (32, 1), 1: (4, 4)}[rank]) else 2.0
        res3 = autotune.tune_batch(b, [], [], pg=pg, timer=_timer_for(b, bcost), device="fake")
        out.put((rank, first, second, (res3.choice["streams"], res3.choice["update_strip"])))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_apply_rank_zeros_choice(tmp_path):
    import torch.multiprocessing as mp
    mpctx = mp.get_context("spawn")
    out = mpctx.Queue()
    port = _free_port()
    procs = [mpctx.Process(target=_rank, args=(r, 2, port, str(tmp_path), out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, first0, second0, batch0), (r1, first1, second1, batch1) = got
    assert first0 == (2, 256, True)            # rank 0 writes its cache
    assert first1 == (2, 256, False)           # rank 1 takes rank 0's choice and writes none
    assert second0 == second1 == (True, 2, 256)
    assert batch0 == batch1 == (32, 1)


def test_tuner_drives_the_real_binding_methods(monkeypatch):
    """The tuner against binding.Context and binding.Batch themselves (their
    tuning calls reach a fake C library), so the method names, keywords and
    the Tuning struct are the ones the tuner uses."""
    import ctypes
    from paper_1404_0466_gb300 import binding as B

    lib_state = {"t": B.Tuning(4, 512, 1, 0, 1, 2), "bt": None, "streams": 8}

    class FakeLib:
        def pichol_get_tuning(self, h, ref):
            ctypes.memmove(ctypes.addressof(ref._obj), ctypes.addressof(lib_state["t"]), ctypes.sizeof(B.Tuning))
            return 0

        def pichol_set_tuning(self, h, ref):
            ctypes.memmove(ctypes.addressof(lib_state["t"]), ctypes.addressof(ref._obj), ctypes.sizeof(B.Tuning))
            return 0

        def pichol_batch_set_tuning(self, h, ref):
            lib_state["bt"] = (ref._obj.update_strip, ref._obj.diag_threads)
            return 0

        def pichol_batch_set_streams(self, h, n):
            lib_state["streams"] = n
            return 0

    monkeypatch.setattr(B, "lib", lambda: FakeLib())
    ctx = B.Context.__new__(B.Context)
    ctx._h = None                     # a null handle: nothing for the real library to free later
    ctx.cfg = B.Config()
    ctx.cfg.mode, ctx.cfg.refine_steps = B.PICHOL_MODE_MIXED, 1
    ran = []
    ctx._outputs = lambda want_w: (None, None, None)
    ctx.run = lambda X, Y, out=None, stream=None: ran.append(ctx.tuning())

    def timer(fn, reps, stream):
        fn()
        t = ctx.tuning()
        return _ctx_cost(t)

    res = autotune.tune_context(ctx, "X", "Y", timer=timer, device="fake")
    assert res.choice == dict(update_strip=2, diag_threads=256, diag_exclusive=0, eval_overlap=1, update_engine=1,
                              solve_engine=2)
    t = lib_state["t"]
    assert (t.update_strip, t.diag_threads, t.diag_exclusive, t.eval_overlap) == (2, 256, 0, 1)
    assert len(ran) == 12

    b = B.Batch.__new__(B.Batch)
    b._h = None
    b.n = 2
    b.cfgs = (B.Config * 2)()
    b.run = lambda Xs, Ys, stream=None: None
    costs = {(16, 2): 1.0}
    res = autotune.tune_batch(b, [], [], device="fake",
                              timer=lambda fn, reps, s: costs.get((lib_state["streams"], lib_state["bt"][0]), 2.0))
    assert res.choice == dict(streams=16, update_strip=2)
    assert lib_state["streams"] == 16 and lib_state["bt"] == (2, 512)
