"""Host-side checks of the C ABI: the library builds, loads without a GPU,
exports every symbol include/pichol.h declares, and validates arguments."""
import ctypes
import os
import re

import pytest

from paper_1404_0466_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return binding.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "pichol.h")).read()
    return sorted(set(re.findall(r"PICHOL_API\s+[\w\s\*]*?\b(pichol_\w+)\s*\(", src)))


def test_header_declares_every_binding_export():
    assert _declared() == sorted(binding.EXPORTS)


def test_library_exports_every_declared_symbol(L):
    for name in _declared():
        assert hasattr(L, name), name


def _cfg(L, **kw):
    cfg = binding.Config()
    L.pichol_config_default(ctypes.byref(cfg))
    base = dict(n=1000, d=100, c=3, k=5, g=4, r=2, q=31)
    base.update(kw)
    for k, v in base.items():
        setattr(cfg, k, v)
    return cfg


def _create(L, cfg):
    h = ctypes.c_void_p()
    rc = L.pichol_create(ctypes.byref(cfg), ctypes.byref(h))
    return rc, h


def test_defaults(L):
    cfg = binding.Config()
    L.pichol_config_default(ctypes.byref(cfg))
    assert cfg.lam_lo == 1e-3 and cfg.lam_hi == 1e1 and cfg.scale_by_trace == 1
    assert cfg.mode == binding.PICHOL_MODE_FP64 and cfg.basis == binding.PICHOL_BASIS_MONO
    assert cfg.gram_passes == 3 and cfg.refine_steps == 0


@pytest.mark.parametrize("bad", [
    dict(k=1), dict(k=65), dict(n=3, k=5), dict(d=0), dict(d=16385), dict(c=0), dict(c=33),
    dict(q=0), dict(q=4097), dict(r=6), dict(r=-1), dict(g=2, r=2), dict(g=40, q=50), dict(g=8, q=5),
    dict(refine_target=2), dict(refine_target=-1), dict(refine_residual=2), dict(refine_residual=-1),
    dict(lam_lo=0.0), dict(lam_lo=2.0, lam_hi=1.0), dict(lam_hi=float("inf")), dict(lam_lo=float("nan")),
    dict(lam_hi=float("nan")), dict(basis=7), dict(mode=5),
    dict(refine_steps=9), dict(gram_passes=2), dict(exact_batch=99), dict(scale_by_trace=2),
])
def test_create_rejects_bad_config(L, bad):
    rc, h = _create(L, _cfg(L, **bad))
    assert rc == 1 and not h.value


def test_create_rejects_nonzero_reserved(L):
    cfg = _cfg(L)
    cfg.reserved[2] = 1
    rc, h = _create(L, cfg)
    assert rc == 1


def test_workspace_size_and_state_errors(L):
    rc, h = _create(L, _cfg(L, d=130, mode=binding.PICHOL_MODE_MIXED, refine_steps=1))
    assert rc == 0 and h.value
    n = ctypes.c_size_t()
    assert L.pichol_workspace_size(h, ctypes.byref(n)) == 0
    # d = 130 pads to 192 = 3 tiles; the dense Gram blocks alone are 5 * 192^2 floats
    assert n.value >= 5 * 192 * 192 * 4
    # calls before a workspace is attached fail without touching the GPU
    assert L.pichol_factor_samples(h, None, None) == 4
    assert L.pichol_hessian(h, None, None, None, None) == 1
    # a misaligned or short workspace is refused before any CUDA call
    assert L.pichol_set_workspace(h, ctypes.c_void_p(0x1001), n.value) == 4
    assert L.pichol_set_workspace(h, ctypes.c_void_p(0x1000), n.value - 1) == 4
    assert L.pichol_launch_count(h) == 0
    L.pichol_destroy(h)


def test_caller_offsets_and_lambdas_are_checked_before_any_cuda_call(L):
    """pichol_hessian's fold offsets (host, k+1: 0, increasing, n) and the
    sampled and evaluation lambdas (host, finite and positive) are checked
    before anything else, so bad values fail here without a GPU; good ones
    reach the workspace check."""
    rc, h = _create(L, _cfg(L))
    assert rc == 0
    cfg = _cfg(L)
    k, n, g, q = cfg.k, cfg.n, cfg.g, cfg.q
    I64 = ctypes.c_int64 * (k + 1)
    x = ctypes.c_void_p(1)
    good = [f * n // k for f in range(k + 1)]
    for bad in ([1] + good[1:], good[:-1] + [n - 1], good[:2] + [good[1]] + good[3:], list(reversed(good))):
        assert L.pichol_hessian(h, x, x, I64(*bad), None) == 1, bad
    assert L.pichol_hessian(h, x, x, I64(*good), None) == 4          # valid: no workspace yet
    uneven = [0, 1, 2, 3, 4, n]
    assert L.pichol_hessian(h, x, x, I64(*uneven[:k] + [n]), None) == 4
    D_g, D_q = ctypes.c_double * g, ctypes.c_double * q
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        vals = [1.0] * g
        vals[g // 2] = bad
        assert L.pichol_factor_samples(h, D_g(*vals), None) == 1, bad
        tv = [1.0] * q
        tv[-1] = bad
        E = ctypes.c_void_p(8)
        assert L.pichol_eval_holdout(h, D_q(*tv), E, E, None, None) == 1, bad
        assert L.pichol_eval_holdout_exact(h, D_q(*tv), E, E, None, None) == 1, bad
    assert L.pichol_factor_samples(h, D_g(*[0.5 + i for i in range(g)]), None) == 4
    assert L.pichol_eval_holdout(h, D_q(*[1.0] * q), ctypes.c_void_p(8), ctypes.c_void_p(8), None, None) == 4
    assert L.pichol_fit(h, None, None) == 4
    L.pichol_destroy(h)


def test_workspace_grows_with_exact_batch(L):
    sizes = []
    for eb in (1, 31):
        rc, h = _create(L, _cfg(L, exact_batch=eb))
        n = ctypes.c_size_t()
        L.pichol_workspace_size(h, ctypes.byref(n))
        sizes.append(n.value)
        L.pichol_destroy(h)
    assert sizes[1] > sizes[0]


def test_status_strings(L):
    assert L.pichol_status_string(0) == b"ok"
    assert b"positive definite" in L.pichol_status_string(2)


def test_exact_system_refinement_needs_mixed_mode(L):
    rc, h = _create(L, _cfg(L, refine_target=binding.REFINE_TARGETS["exact"], refine_steps=1))
    assert rc == 6 and not h.value        # PICHOL_ERR_UNSUPPORTED in FP64 mode
    rc, h = _create(L, _cfg(L, refine_target=1, refine_steps=1, mode=binding.PICHOL_MODE_MIXED))
    assert rc == 0
    L.pichol_destroy(h)


def test_fp64_shapes_beyond_shared_memory_are_unsupported(L):
    """The FP64 solve double-buffers p = r + 1 coefficient half-planes of 16 KB
    beside its staged blocks and reduction slots: degree 5 fits in a CTA's
    227 KB with up to 4 outputs (212 KB) but not with 12 (252 KB)."""
    rc, h = _create(L, _cfg(L, r=5, g=8, q=31, c=12))
    assert rc == 6 and not h.value
    for r, c in ((5, 4), (3, 12)):
        rc, h = _create(L, _cfg(L, r=r, g=8, q=31, c=c))
        assert rc == 0, (r, c)
        L.pichol_destroy(h)


def test_tuning_defaults_and_validation(L):
    rc, h = _create(L, _cfg(L))
    assert rc == 0
    t = binding.Tuning()
    assert L.pichol_get_tuning(h, ctypes.byref(t)) == 0
    assert (t.update_strip, t.diag_threads, t.diag_exclusive, t.eval_overlap) == (4, 512, 1, 0)
    assert (t.update_engine, t.solve_engine) == (1, 2)       # CUDA-core updates, automatic solve engine
    for bad in (dict(update_strip=0), dict(update_strip=9), dict(diag_threads=384), dict(diag_exclusive=2),
                dict(eval_overlap=2), dict(update_engine=2), dict(solve_engine=3), dict(solve_engine=-1)):
        b = binding.Tuning(**{**dict(update_strip=4, diag_threads=512, diag_exclusive=1, update_engine=1), **bad})
        assert L.pichol_set_tuning(h, ctypes.byref(b)) == 1, bad
    good = binding.Tuning(update_strip=2, diag_threads=256, diag_exclusive=0, eval_overlap=1, update_engine=0,
                          solve_engine=0)
    assert L.pichol_set_tuning(h, ctypes.byref(good)) == 0
    assert L.pichol_get_tuning(h, ctypes.byref(t)) == 0
    assert (t.update_strip, t.diag_threads, t.diag_exclusive, t.eval_overlap) == (2, 256, 0, 1)
    L.pichol_destroy(h)


def test_mchol_levels_and_argument_checks(L):
    """Level counts (the paper's s = 1.5, s0 = 0.0025 give ten) and the checks
    pichol_mchol makes before any CUDA call."""
    n = ctypes.c_int32()
    for s, s_min, want in [(1.5, 0.0025, 10), (1.5, 0.1, 4), (1.5, 0.75, 1), (0.1, 0.2, 1), (1.0, 0.5, 1)]:
        assert L.pichol_mchol_levels(s, s_min, ctypes.byref(n)) == 0
        assert n.value == want, (s, s_min)
    for s, s_min in [(0.0, 0.1), (-1.0, 0.1), (1.0, 0.0), (float("nan"), 0.1), (1.0, float("inf")),
                     (300.0, 1e-30)]:                   # the last needs more than 64 levels
        assert L.pichol_mchol_levels(s, s_min, ctypes.byref(n)) == 1, (s, s_min)
    assert L.pichol_mchol_levels(1.0, 0.1, None) == 1
    rc, h = _create(L, _cfg(L))
    assert L.pichol_mchol(h, float("nan"), 1.0, 0.1, None, None) == 1
    assert L.pichol_mchol(h, 0.0, 1.0, 0.0, None, None) == 1
    assert L.pichol_mchol(h, 0.0, 1.0, 0.1, None, None) == 4      # no workspace yet
    assert L.pichol_mchol(None, 0.0, 1.0, 0.1, None, None) == 1
    L.pichol_destroy(h)


def test_warm_samples_validation(L):
    """warm_samples: 0, or 2 <= g' <= min(g, 8)."""
    for ws, want in [(0, 0), (2, 0), (4, 0), (1, 1), (5, 1), (-1, 1)]:
        rc, h = _create(L, _cfg(L, g=4, r=2, warm_samples=ws))
        assert rc == want, (ws, rc)
        if rc == 0:
            L.pichol_destroy(h)
    rc, h = _create(L, _cfg(L, g=12, r=3, q=31, warm_samples=9))
    assert rc == 1
    rc, h = _create(L, _cfg(L, g=12, r=3, q=31, warm_samples=8))
    assert rc == 0
    L.pichol_destroy(h)


def test_new_entry_points_check_arguments_without_a_gpu(L):
    """Argument and state checks that return before any CUDA call."""
    E = ctypes.c_void_p(0x1000)
    assert L.pichol_eval_pinrmse(None, E, E, None) == 1
    rc, h = _create(L, _cfg(L))
    assert L.pichol_eval_pinrmse(h, None, E, None) == 1
    assert L.pichol_eval_pinrmse(h, E, E, None) == 4                 # no workspace yet
    for check in (L.pichol_check_timeout, L.pichol_check_wave_timeout):
        assert check(None, 1000, None) == 1
        assert check(h, 0, None) == 1
        assert check(h, (1 << 34) + 1, None) == 1
        assert check(h, 1000, None) == 4                             # no workspace yet
    L.pichol_destroy(h)
    out = ctypes.c_double()
    assert L.pichol_probe_fma(2, 1024, ctypes.byref(out)) == 1
    assert L.pichol_probe_fma(0, 0, ctypes.byref(out)) == 1
    assert L.pichol_probe_fma(1, (1 << 24) + 1, ctypes.byref(out)) == 1
    assert L.pichol_probe_fma(0, 1024, None) == 1
    for n_cols, iters in ((32, 1024), (96, 1024), (128, 0), (256, (1 << 22) + 1)):
        assert L.pichol_probe_mma(n_cols, iters, ctypes.byref(out)) == 1
    assert L.pichol_probe_mma(128, 1024, None) == 1
    assert L.pichol_check_rsqrt(0, 1, E, None) == 1
    assert L.pichol_check_rsqrt((1 << 32) + 1, 1, E, None) == 1
    assert L.pichol_check_rsqrt(1024, 1, None, None) == 1


def test_context_and_batch_close_on_leaving_a_with_block(monkeypatch):
    """The with-statement frees the C handle once, also when the block raises."""
    from paper_1404_0466_gb300 import binding
    freed = []

    class FakeLib:
        def pichol_destroy(self, h):
            freed.append(("ctx", h))

        def pichol_batch_destroy(self, h):
            freed.append(("batch", h))

    monkeypatch.setattr(binding, "lib", lambda: FakeLib())
    for cls, tag in ((binding.Context, "ctx"), (binding.Batch, "batch")):
        obj = cls.__new__(cls)
        obj._h = 17
        with pytest.raises(KeyError):
            with obj as o:
                assert o is obj
                raise KeyError("inside")
        assert obj._h is None
        obj.close()
        assert freed.count((tag, 17)) == 1


def test_tensor_arguments_are_checked_before_any_call(monkeypatch):
    """Wrong device, dtype, shape or layout raise before the C library is
    reached (the kernels would read or write out of bounds); without assert,
    so the checks hold under python -O.  CPU tensors stand in for the CUDA
    ones: the device is the first thing checked."""
    import torch
    from types import SimpleNamespace
    from paper_1404_0466_gb300 import binding as B

    def no_lib():
        raise AssertionError("the C library must not be reached")

    monkeypatch.setattr(B, "lib", no_lib)
    ctx = B.Context.__new__(B.Context)
    ctx._h = None
    ctx.cfg = SimpleNamespace(n=8, d=3, c=2, k=2, q=5)
    ctx.dtype = torch.float64
    X, Y = torch.zeros(8, 3, dtype=torch.float64), torch.zeros(8, 2, dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA"):
        ctx.hessian(X, Y)
    with pytest.raises(TypeError):
        ctx.hessian(X.numpy(), Y)
    # the remaining checks, each with the device check passed
    monkeypatch.setattr(torch.Tensor, "is_cuda", property(lambda self: True))
    with pytest.raises(ValueError, match="float64"):
        ctx.hessian(X.float(), Y)
    with pytest.raises(ValueError, match=r"shape \(8, 3\)"):
        ctx.hessian(X[:7], Y)
    with pytest.raises(ValueError, match="contiguous"):
        ctx.hessian(torch.zeros(3, 8, dtype=torch.float64).t(), Y)
    E, t = torch.zeros(2, 5, dtype=torch.float64), torch.zeros(1, dtype=torch.int32)
    with pytest.raises(ValueError, match="E must have shape"):
        ctx._given_outputs((torch.zeros(2, 4, dtype=torch.float64), t, None), False)
    with pytest.raises(ValueError, match="t_star"):
        ctx._given_outputs((E, torch.zeros(1, dtype=torch.int64), None), False)
    with pytest.raises(ValueError, match="W must have shape"):
        ctx._given_outputs((E, t, torch.zeros(2, 5, 3, 1, dtype=torch.float64)), True)
    assert ctx._given_outputs((E, t, None), False)[0] is E
    # a batch checks every problem against its own configuration and mode
    b = B.Batch.__new__(B.Batch)
    b._h = None
    b.n = 2
    b.cfgs = [SimpleNamespace(n=8, d=3, c=2, mode=B.PICHOL_MODE_FP64),
              SimpleNamespace(n=6, d=4, c=1, mode=B.PICHOL_MODE_MIXED)]
    good_x = [X, torch.zeros(6, 4)]
    good_y = [Y, torch.zeros(6, 1)]
    with pytest.raises(ValueError, match="expected 2"):
        b.run(good_x[:1], good_y[:1])
    with pytest.raises(ValueError, match=r"X\[1\] must be torch.float32"):
        b.run([X, torch.zeros(6, 4, dtype=torch.float64)], good_y)
    with pytest.raises(ValueError, match=r"Y\[0\] must have shape"):
        b.run(good_x, [torch.zeros(8, 1, dtype=torch.float64), good_y[1]])


def test_unknown_names_are_value_errors():
    from paper_1404_0466_gb300 import binding as B
    assert B._choice("mode", "mixed", B.MODES) == B.PICHOL_MODE_MIXED
    with pytest.raises(ValueError, match="basis must be one of"):
        B._choice("basis", "legendre", B.BASES)
    with pytest.raises(ValueError, match="refine_target"):
        B._choice("refine_target", "both", B.REFINE_TARGETS)


C_CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "pichol.h"

int main(void)
{
    pichol_config cfg;
    pichol_ctx* ctx = NULL;
    int32_t levels = 0;
    pichol_config_default(&cfg);
    cfg.n = 1000; cfg.d = 100; cfg.c = 3; cfg.k = 5; cfg.g = 4; cfg.r = 2; cfg.q = 31;
    cfg.lam_lo = 2.0; cfg.lam_hi = 1.0;                      /* lo > hi: refused */
    printf("%d ", (int)pichol_create(&cfg, &ctx));
    printf("%d ", ctx == NULL);
    printf("%d ", (int)pichol_mchol_levels(1.5, 0.0025, &levels));
    printf("%d ", (int)levels);
    printf("%s\n", pichol_status_string(PICHOL_ERR_NOT_SPD));
    return 0;
}
"""


def test_plain_c_client_compiles_links_and_runs(L, tmp_path):
    """The header is C (pedantic C99, no C++), and a C program links against
    libpichol.so and calls its host-only entry points without a GPU."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(str(binding.LIB_PATH))
    subprocess.check_call(["gcc", "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror",
                           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                           "-L", libdir, "-lpichol", "-Wl,-rpath," + libdir])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    assert out.strip() == "1 1 0 10 matrix not positive definite"


def test_state_and_resume_rules_without_a_gpu(L):
    h = _create(L, _cfg(L))[1]
    st = ctypes.c_int32(-1)
    assert L.pichol_get_state(h, ctypes.byref(st)) == 0 and st.value == 0
    assert L.pichol_get_state(None, ctypes.byref(st)) == 1
    assert L.pichol_get_state(h, None) == 1
    assert L.pichol_resume(None, 0) == 1
    assert L.pichol_resume(h, 8) == 1          # unknown bit
    assert L.pichol_resume(h, 2) == 1          # factors without the Hessian
    assert L.pichol_resume(h, 4) == 1          # fit without the Hessian
    assert L.pichol_resume(h, 7) == 4          # no workspace yet
    # a workspace whose CUDA setup fails (no GPU here) is not taken
    n = ctypes.c_size_t()
    assert L.pichol_workspace_size(h, ctypes.byref(n)) == 0
    rc = L.pichol_set_workspace(h, ctypes.c_void_p(0x100000), n.value)
    if rc != 0:
        assert rc == 3
        assert L.pichol_resume(h, 7) == 4
        assert L.pichol_hessian(h, ctypes.c_void_p(1), ctypes.c_void_p(1), None, None) == 4
    L.pichol_destroy(h)


def test_load_state_dict_checks_the_configuration(monkeypatch):
    import torch
    from paper_1404_0466_gb300 import binding as B

    def no_lib():
        raise AssertionError("the C library must not be reached")

    monkeypatch.setattr(B, "lib", no_lib)
    ctx = B.Context.__new__(B.Context)
    ctx._h = None
    ctx.cfg = B.Config()
    ctx.cfg.n, ctx.cfg.d = 10, 4
    ctx._ws = torch.zeros(512, dtype=torch.uint8)
    other = B.Config()
    other.n, other.d = 10, 5
    with pytest.raises(ValueError, match="another configuration"):
        ctx.load_state_dict({"config": bytes(other), "tuning": {}, "state": 7, "workspace": ctx._ws})
    with pytest.raises(ValueError, match="workspace does not match"):
        ctx.load_state_dict({"config": bytes(ctx.cfg), "tuning": {}, "state": 7,
                             "workspace": torch.zeros(256, dtype=torch.uint8)})


def test_check_raises_the_latched_device_error(monkeypatch):
    from paper_1404_0466_gb300 import binding as B
    ctx = B.Context.__new__(B.Context)
    ctx._h = None
    monkeypatch.setattr(B.Context, "info", lambda self, stream=None: B.Info(0, -1, -1, -1, 0))
    ctx.check()
    monkeypatch.setattr(B.Context, "info", lambda self, stream=None: B.Info(2, 3, 1, 417, 0))
    with pytest.raises(B.PicholError, match="PICHOL_ERR_NOT_SPD") as ei:
        ctx.check()
    assert ei.value.code == 2 and "fold 3" in str(ei.value) and "pivot 417" in str(ei.value)


def test_regular_build_has_no_guard_bands(L):
    """Only the -DPICHOL_DEBUG build places guard bands in the workspace."""
    assert L.pichol_debug_build() == 0
    rc, h = _create(L, _cfg(L))
    n = ctypes.c_int32(-1)
    arr = (ctypes.c_int64 * 4)()
    assert L.pichol_debug_guards(h, arr, 4, ctypes.byref(n)) == 0 and n.value == 0
    assert L.pichol_debug_guards(h, None, 4, ctypes.byref(n)) == 1
    L.pichol_destroy(h)


def test_interface_version_agrees(L):
    src = open(os.path.join(ROOT, "include", "pichol.h")).read()
    major = int(re.search(r"#define PICHOL_VERSION_MAJOR (\d+)", src).group(1))
    minor = int(re.search(r"#define PICHOL_VERSION_MINOR (\d+)", src).group(1))
    assert (major, minor) == binding.INTERFACE
    assert L.pichol_version() == 100 * major + minor
