"""The allocation-free entry point pichol_fold_rhs_noalloc.

It serves callers that cannot allocate device memory (a plug-in inside a
framework that owns the whole GPU through its own pool, a real-time path that
cannot pay for cudaMalloc's implicit synchronisation): its partial sums live in
a fixed array inside the library.  This file checks, through the C ABI, that
after a call on other data of a larger shape, two calls in a row give the
training right-hand sides B_f that the regular workspace path (pichol_hessian,
read back with pichol_export_hessian) forms and that the FP64 oracle forms,
within the test tolerance of the mode, and that sizes beyond the fixed array
are refused.  It is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_1404_0466_gb300 import synth

pytestmark = pytest.mark.gpu


def _noalloc(lib, torch, mode, X, Y, k):
    n, d = X.shape
    c = Y.shape[1]
    Bv = torch.empty((k, d, c), dtype=X.dtype, device="cuda")
    B = torch.empty((k, d, c), dtype=X.dtype, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.pichol_fold_rhs_noalloc(mode, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                     n, d, c, k, ctypes.c_void_p(Bv.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                     stream)
    torch.cuda.synchronize()
    return rc, Bv, B


@pytest.mark.parametrize("mode_name,n,d,c,k", [("fp64", 700, 130, 3, 5), ("mixed", 1500, 200, 10, 4)])
def test_noalloc_matches_workspace_path_twice(mode_name, n, d, c, k):
    """A first call on other data of a larger shape leaves its partial sums in
    the shared array; the next two calls on the test shape must not see them.
    Both are compared with the workspace path and with the FP64 oracle's
    right-hand sides of each fold."""
    import torch

    import oracle
    from paper_1404_0466_gb300 import binding, build
    build.build()
    lib = binding.lib()
    mode = binding.PICHOL_MODE_FP64 if mode_name == "fp64" else binding.PICHOL_MODE_MIXED
    dt = torch.float64 if mode_name == "fp64" else torch.float32
    prob = synth.spectral_gaussian(n, d, c, seed=31 + d)
    X = torch.from_numpy(prob.X).to(device="cuda", dtype=dt).contiguous()
    Y = torch.from_numpy(prob.Y).to(device="cuda", dtype=dt).contiguous()
    big = synth.spectral_gaussian(n + 300, d + 70, c + 2, seed=77)
    Xb = torch.from_numpy(big.X).to(device="cuda", dtype=dt).contiguous()
    Yb = (-3.0 * torch.from_numpy(big.Y)).to(device="cuda", dtype=dt).contiguous()
    rc, _, _ = _noalloc(lib, torch, mode, Xb, Yb, k + 1)
    assert rc == 0, binding.STATUS.get(rc)

    ctx = binding.Context(n=n, d=d, c=c, k=k, g=2, r=1, q=3, mode=mode_name)
    ctx.hessian(X, Y)
    ref = [ctx.export_hessian(f)[1].cpu().numpy() for f in range(k)]
    offs = oracle.fold_offsets(n, k)
    orc = [oracle.normal_blocks(prob.X, prob.Y, offs[f], offs[f + 1])[1] for f in range(k)]
    tol = 1e-12 if mode_name == "fp64" else 1e-6

    for call in range(2):
        rc, Bv, B = _noalloc(lib, torch, mode, X, Y, k)
        assert rc == 0, binding.STATUS.get(rc)
        B = B.double().cpu().numpy()
        Bv = Bv.double().cpu().numpy()
        for f in range(k):
            scale = np.max(np.abs(orc[f]))
            assert np.max(np.abs(B[f] - ref[f])) <= tol * scale, (call, f)
            assert np.max(np.abs(B[f] - orc[f])) <= tol * scale, (call, f)
            # Bv_f is fold f's own X_f^T Y_f
            Xf, Yf = prob.X[offs[f]:offs[f + 1]], prob.Y[offs[f]:offs[f + 1]]
            np.testing.assert_allclose(Bv[f], Xf.T @ Yf, rtol=0, atol=tol * scale)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch

    from paper_1404_0466_gb300 import binding, build
    build.build()
    lib = binding.lib()
    n, d, c, k = 200, 2048, 32, 8          # 8 * 16 * 2048 * 32 doubles > 2^20
    X = torch.zeros((n, d), dtype=torch.float32, device="cuda")
    Y = torch.zeros((n, c), dtype=torch.float32, device="cuda")
    rc, _, _ = _noalloc(lib, torch, binding.PICHOL_MODE_MIXED, X, Y, k)
    assert rc == 4   # PICHOL_ERR_WORKSPACE
