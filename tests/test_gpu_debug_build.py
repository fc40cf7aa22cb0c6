"""The bounds-checked build (libpichol_debug.so, -DPICHOL_DEBUG): every
workspace section is followed by a guard band that pichol_get_info checks.
The odd-size cases (a single partial tile, ragged last tiles, uneven folds,
one held-out row per fold) run through every kernel variant of the path --
double precision, mixed precision with the tensor-core and double-float
residuals, the tensor-core trailing update and the tensor-core solve -- and
must leave every band untouched and match the FP64 oracle.  A byte changed
from the host inside a band (no kernel involved) must be reported.

Runs in a child process with PICHOL_DEBUG=1, so that the binding loads the
debug library; it is compiled first (a minute or two)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np, torch
import oracle
from paper_1404_0466_gb300 import binding, synth
assert binding.lib().pichol_debug_build() == 1
runs = 0
for (n, d, c, k, mode, tune, resid) in [
        (300, 37, 3, 4, "fp64", {}, "tensor"),
        (700, 129, 2, 5, "mixed", {}, "tensor"),
        (700, 129, 2, 5, "mixed", {"update_engine": 0, "solve_engine": 0}, "tensor"),
        (650, 100, 12, 5, "mixed", {"solve_engine": 0}, "double_float"),
        (40, 12, 3, 40, "mixed", {}, "tensor"),
        (1100, 200, 5, 3, "mixed", {"update_engine": 0, "update_strip": 4, "solve_engine": 0}, "tensor")]:
    prob = synth.spectral_gaussian(n, d, c, seed=d + n)
    kw = dict(k=k, g=5, r=3, q=17, basis="cheb_log")
    ctx = binding.Context(n=n, d=d, c=c, mode=mode, refine_steps=0 if mode == "fp64" else 1,
                          refine_residual=resid, **kw)
    assert len(ctx.guard_offsets()) > 20
    if tune:
        ctx.set_tuning(**tune)
    dt = torch.float64 if mode == "fp64" else torch.float32
    out = ctx.run(torch.from_numpy(prob.X).to("cuda", dt), torch.from_numpy(prob.Y).to("cuda", dt))
    ex = ctx.eval_holdout_exact()
    info = ctx.info()
    assert info.code == 0, (n, d, mode, tune, binding.STATUS.get(info.code), info.index, info.pivot)
    ref = oracle.cv(prob.X, prob.Y, **kw)
    tol = 1e-9 if mode == "fp64" else 1e-4
    scale = np.maximum(ref.E, ref.Ebar[None, :])
    fin = np.isfinite(ref.E)
    rel = np.abs(out.E.cpu().numpy()[fin] - ref.E[fin]) / scale[fin]
    assert rel.max() <= tol, (n, d, mode, tune, float(rel.max()))
    runs += 1
    ctx.close()
# a byte changed inside a guard band from the host is reported, with its band
prob = synth.spectral_gaussian(300, 37, 3, seed=5)
ctx = binding.Context(n=300, d=37, c=3, k=4, g=4, r=2, q=9, mode="fp64")
ctx.run(torch.from_numpy(prob.X).cuda(), torch.from_numpy(prob.Y).cuda())
assert ctx.info().code == 0
offs = ctx.guard_offsets()
ctx._ws[offs[7] + 100] = 0
info = ctx.info()
assert info.code == 4 and info.index == 7 and info.pivot == 100, (info.code, info.index, info.pivot)
print("debug build ok", runs)
"""


def test_debug_build_guard_bands_and_odd_sizes():
    from paper_1404_0466_gb300 import build
    build.build(debug=True)
    env = dict(os.environ, PICHOL_DEBUG="1", PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "debug build ok 6" in r.stdout
