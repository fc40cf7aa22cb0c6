"""Launch-shape autotuner for a piCholesky context or batch.

No tuning changes a result: every kernel's sums run in the same order under
every launch shape, so the tuner only times.  It runs each candidate on the
caller's own inputs, once untimed and then ``reps`` times between two CUDA
events on the launching stream, and keeps the fastest.

One problem (``tune_context``), in this order, each stage starting from the
previous stage's choice:

1. output tiles per trailing-update CTA (``update_strip``) x threads per
   diagonal-tile CTA (``diag_threads``);
2. whether the diagonal-tile CTAs keep their SMs to themselves
   (``diag_exclusive``);
3. in mixed precision with refinement only: whether the interpolated solves
   and their refinement run as two overlapped halves (``eval_overlap``).

A batch (``tune_batch``): concurrent streams x ``update_strip``.

With ``cache=path`` a choice is stored in a JSON file under a key made of the
device name and the problem's configuration, and a later call with the same
key applies it without timing.  With a process group ``pg``, every rank
applies rank 0's choice, so that all ranks run the same launch shapes.
"""
from __future__ import annotations

import hashlib
import json
import os
from dataclasses import dataclass, field

from .binding import PICHOL_MODE_MIXED

UPDATE_STRIPS = (1, 2, 4, 8)
DIAG_THREADS = (256, 512)
DIAG_EXCLUSIVE = (1, 0)
EVAL_OVERLAP = (0, 1)
BATCH_STREAMS = (4, 8, 16, 32)
BATCH_STRIPS = (1, 2, 4)

_CFG_FIELDS = ("n", "d", "c", "k", "g", "r", "q", "mode", "basis", "refine_steps", "refine_target",
               "exact_batch", "warm_samples", "gram_passes")


@dataclass
class TuneResult:
    choice: dict                                   # the tuning applied at the end
    timings: dict = field(default_factory=dict)    # stage -> {candidate label: ms per run}
    cached: bool = False                           # True when taken from the cache without timing
    key: str = ""


def event_timer(fn, reps: int, stream=None) -> float:
    """Milliseconds per call of ``fn``: one untimed call, then ``reps`` calls
    between two CUDA events recorded on ``stream`` (default: the current one)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    fn()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(s)
    for _ in range(reps):
        fn()
    b.record(s)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _device_name() -> str:
    import torch
    return torch.cuda.get_device_name()


def _cfg_values(cfg) -> list:
    return [getattr(cfg, f, None) for f in _CFG_FIELDS]


def context_key(cfg, device: str) -> str:
    """Cache key of one problem: the device name and the configuration fields
    that change the launches."""
    return f"{device}|context|" + ",".join(f"{f}={v}" for f, v in zip(_CFG_FIELDS, _cfg_values(cfg)))


def batch_key(cfgs, device: str) -> str:
    """Cache key of a batch: the device name, the problem count and a digest of
    every problem's configuration in order."""
    rows = [",".join(str(v) for v in _cfg_values(c)) for c in cfgs]
    digest = hashlib.sha1("\n".join(rows).encode()).hexdigest()[:16]
    return f"{device}|batch|{len(rows)}|{digest}"


def _load(path):
    if path is None or not os.path.exists(path):
        return {}
    with open(path) as f:
        data = json.load(f)
    if not isinstance(data, dict):
        raise ValueError(f"tuning cache {path} does not hold a JSON object")
    return data


def _store(path, key, choice, pg):
    if path is None or _rank(pg) != 0:
        return
    data = _load(path)
    data[key] = choice
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _argmin(times: dict):
    """Fastest candidate; the first listed among equal times."""
    best = None
    for cand, ms in times.items():
        if best is None or ms < times[best]:
            best = cand
    return best


def _rank(pg) -> int:
    if pg is None:
        return 0
    import torch.distributed as dist
    return dist.get_rank(pg)


def _agree(values: list, pg) -> list:
    """Rank 0's integers on every rank of ``pg`` (unchanged without one)."""
    if pg is None:
        return values
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend(pg) == "nccl" else "cpu"
    t = torch.tensor(values, dtype=torch.int64, device=dev)
    dist.broadcast(t, dist.get_global_rank(pg, 0), group=pg)
    return [int(v) for v in t.tolist()]


def tune_context(ctx, X, Y, *, reps: int = 2, stream=None, cache=None, pg=None, timer=None,
                 device: str | None = None) -> TuneResult:
    """Time the launch-shape candidates of one problem on (X, Y) and apply the
    fastest to ``ctx``.  Leaves ``ctx`` holding the results of its last run."""
    if reps < 1:
        raise ValueError("reps must be at least 1")
    timer = timer or event_timer
    key = context_key(ctx.cfg, device or _device_name())
    names = ("update_strip", "diag_threads", "diag_exclusive", "eval_overlap")
    # rank 0's cache decides for every rank, so that all of them time or none does
    hit = _load(cache).get(key) if _rank(pg) == 0 else None
    vals = _agree([1] + [int(hit[n]) for n in names] if hit is not None else [0] * 5, pg)
    if vals[0]:
        ctx.set_tuning(**dict(zip(names, vals[1:])))
        return TuneResult(choice=ctx.tuning(), cached=True, key=key)

    out = ctx._outputs(False)

    def step():
        ctx.run(X, Y, out=out, stream=stream)

    timings = {}
    shapes = {}
    for strip in UPDATE_STRIPS:
        for dt in DIAG_THREADS:
            ctx.set_tuning(update_strip=strip, diag_threads=dt)
            shapes[(strip, dt)] = timer(step, reps, stream)
    strip, dt = _argmin(shapes)
    ctx.set_tuning(update_strip=strip, diag_threads=dt)
    timings["shapes"] = {f"strip{a}_diag{b}": ms for (a, b), ms in shapes.items()}

    excl = {}
    for ex in DIAG_EXCLUSIVE:
        ctx.set_tuning(diag_exclusive=ex)
        excl[ex] = timer(step, reps, stream)
    ex = _argmin(excl)
    ctx.set_tuning(diag_exclusive=ex)
    timings["diag_exclusive"] = {f"diag_exclusive{v}": ms for v, ms in excl.items()}

    ov = 0
    if ctx.cfg.mode == PICHOL_MODE_MIXED and ctx.cfg.refine_steps > 0:
        over = {}
        for v in EVAL_OVERLAP:
            ctx.set_tuning(eval_overlap=v)
            over[v] = timer(step, reps, stream)
        ov = _argmin(over)
        timings["eval_overlap"] = {f"eval_overlap{v}": ms for v, ms in over.items()}

    strip, dt, ov, ex = _agree([strip, dt, ov, ex], pg)
    choice = dict(update_strip=strip, diag_threads=dt, diag_exclusive=ex, eval_overlap=ov)
    ctx.set_tuning(**choice)
    _store(cache, key, choice, pg)
    return TuneResult(choice=ctx.tuning(), timings=timings, key=key)


def tune_batch(batch, Xs, Ys, *, reps: int = 2, stream=None, cache=None, pg=None, timer=None,
               device: str | None = None) -> TuneResult:
    """Time concurrent streams x update strip for a batch on (Xs, Ys) and apply
    the fastest to ``batch``."""
    if reps < 1:
        raise ValueError("reps must be at least 1")
    timer = timer or event_timer
    key = batch_key(batch.cfgs, device or _device_name())
    hit = _load(cache).get(key) if _rank(pg) == 0 else None
    use, ns, strip = _agree([1, int(hit["streams"]), int(hit["update_strip"])] if hit is not None else [0, 0, 0], pg)
    if use:
        batch.set_streams(ns)
        batch.set_tuning(update_strip=strip)
        return TuneResult(choice=dict(streams=ns, update_strip=strip), cached=True, key=key)

    def step():
        batch.run(Xs, Ys, stream=stream)

    grid = {}
    for ns in BATCH_STREAMS:
        for strip in BATCH_STRIPS:
            batch.set_streams(ns)
            batch.set_tuning(update_strip=strip)
            grid[(ns, strip)] = timer(step, reps, stream)
    ns, strip = _agree(list(_argmin(grid)), pg)
    batch.set_streams(ns)
    batch.set_tuning(update_strip=strip)
    choice = dict(streams=ns, update_strip=strip)
    _store(cache, key, choice, pg)
    return TuneResult(choice=choice, timings={"streams_strip": {f"{a}x{b}": ms for (a, b), ms in grid.items()}},
                      key=key)
