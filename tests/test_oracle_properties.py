"""The oracle's pins over random small shapes (hypothesis): d down to 1, a
single lambda, folds of one row, uneven folds and several outputs.

- Exact cross-validation equals an independent pipeline: numpy.linalg.solve
  on each fold's training normal equations (Eq. 2) and the hold-out mean
  squared error, on the log-spaced grid scaled by tr(X^T X) / d.
- piCholesky equals exact cross-validation when every grid lambda is a
  sampled node (g = q, r = g - 1), in either basis.
"""
import numpy as np
import pytest

import oracle as orc

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import assume, given, settings, strategies as st  # noqa: E402


def _library_cv(X, Y, k, q, lo=1e-3, hi=1e1):
    n, d = X.shape
    c = Y.shape[1]
    bounds = [(f * n) // k for f in range(k + 1)]
    tau = float(np.sum(X * X)) / d
    lam = tau * lo * (hi / lo) ** (np.arange(q) / (q - 1)) if q > 1 else np.array([tau * lo])
    E = np.empty((k, q))
    for f in range(k):
        keep = np.r_[0:bounds[f], bounds[f + 1]:n]
        H, B = X[keep].T @ X[keep], X[keep].T @ Y[keep]
        Xv, Yv = X[bounds[f]:bounds[f + 1]], Y[bounds[f]:bounds[f + 1]]
        for t in range(q):
            W = np.linalg.solve(H + lam[t] * np.eye(d), B)
            E[f, t] = np.sum((Yv - Xv @ W) ** 2) / (Yv.shape[0] * c)
    return E


@settings(max_examples=30, deadline=None, derandomize=True)
@given(n=st.integers(2, 40), d=st.integers(1, 8), c=st.integers(1, 3), k=st.integers(2, 6),
       q=st.integers(1, 5), seed=st.integers(0, 2 ** 32 - 1))
def test_exact_cv_equals_a_library_pipeline(n, d, c, k, q, seed):
    assume(n >= k)
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d))
    Y = rng.standard_normal((n, c))
    res = orc.cv(X, Y, k=k, g=1, r=0, q=q, exact=True)
    np.testing.assert_allclose(res.E, _library_cv(X, Y, k, q), rtol=1e-8, atol=1e-12)
    assert res.t_star == int(np.argmin(res.E.mean(axis=0)))


@settings(max_examples=20, deadline=None, derandomize=True)
@given(n=st.integers(12, 40), d=st.integers(1, 6), c=st.integers(1, 2), k=st.integers(2, 4),
       q=st.integers(2, 5), basis=st.sampled_from([orc.BASIS_MONO, orc.BASIS_CHEB_LOG]),
       seed=st.integers(0, 2 ** 32 - 1))
def test_pichol_at_nodes_equals_exact_cv(n, d, c, k, q, basis, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d))
    Y = rng.standard_normal((n, c))
    a = orc.cv(X, Y, k=k, g=q, r=q - 1, q=q, basis=basis)
    b = orc.cv(X, Y, k=k, g=q, r=q - 1, q=q, exact=True)
    np.testing.assert_allclose(a.E, b.E, rtol=1e-7)


@settings(max_examples=40, deadline=None, derandomize=True)
@given(g=st.integers(1, 12), p=st.integers(1, 6), D=st.integers(1, 30), seed=st.integers(0, 2 ** 32 - 1))
def test_householder_fit_equals_library_least_squares(g, p, D, seed):
    assume(g >= p)
    rng = np.random.default_rng(seed)
    V = rng.standard_normal((g, p))
    T = rng.standard_normal((g, D))
    np.testing.assert_allclose(orc.lstsq(V, T), np.linalg.lstsq(V, T, rcond=None)[0], rtol=1e-9, atol=1e-9)


@settings(max_examples=40, deadline=None, derandomize=True)
@given(lo=st.floats(-6, 3), span=st.floats(0.1, 8), g=st.integers(2, 8), p=st.integers(1, 6),
       seed=st.integers(0, 2 ** 32 - 1))
def test_log_chebyshev_basis_equals_chebvander(lo, span, g, p, seed):
    rng = np.random.default_rng(seed)
    lam_s = np.sort(10.0 ** rng.uniform(lo, lo + span, g))
    assume(lam_s[-1] > lam_s[0] * (1 + 1e-9))
    lam = 10.0 ** rng.uniform(lo, lo + span, 17)
    u = 2 * (np.log(lam) - np.log(lam_s[0])) / (np.log(lam_s[-1]) - np.log(lam_s[0])) - 1
    np.testing.assert_allclose(orc.basis_values(orc.BASIS_CHEB_LOG, lam, lam_s, p),
                               np.polynomial.chebyshev.chebvander(u, p - 1), rtol=1e-10, atol=1e-10)


@settings(max_examples=30, deadline=None, derandomize=True)
@given(d=st.integers(1, 40), seed=st.integers(0, 2 ** 32 - 1))
def test_vectorisation_round_trip_any_size(d, seed):
    L = np.tril(np.random.default_rng(seed).standard_normal((d, d)))
    v = orc.vec_lower(L)
    assert v.size == d * (d + 1) // 2
    np.testing.assert_array_equal(orc.unvec_lower(v, d), L)
    np.testing.assert_array_equal(v, L[np.tril_indices(d)])       # row by row


@settings(max_examples=60, deadline=None, derandomize=True)
@given(n=st.integers(1, 10 ** 6), k=st.integers(1, 64))
def test_fold_boundaries_partition_the_rows(n, k):
    assume(n >= k)
    o = orc.fold_offsets(n, k)
    assert o[0] == 0 and o[-1] == n and all(o[f] == (f * n) // k for f in range(k + 1))
    sizes = np.diff(o)
    assert sizes.min() >= n // k and sizes.max() <= -(-n // k)


@settings(max_examples=15, deadline=None, derandomize=True)
@given(n=st.integers(20, 60), d=st.integers(1, 6), c=st.integers(1, 2), r=st.integers(1, 3),
       basis=st.sampled_from([orc.BASIS_MONO, orc.BASIS_CHEB_LOG]), pos=st.floats(0.1, 0.9),
       seed=st.integers(0, 2 ** 32 - 1))
def test_interpolated_gradient_equals_central_differences(n, d, c, r, basis, pos, seed):
    """dE/dlog(lambda) through the interpolated factor against central
    differences of the same function (h = 1e-4 in log lambda), inside the
    sampled range."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d))
    Y = X @ rng.standard_normal((d, c)) + 0.3 * rng.standard_normal((n, c))
    kw = dict(k=3, g=r + 2, r=r, q=9, basis=basis, lo=0.05, hi=5.0)
    tau = orc.trace_scale(X)
    ll = np.log(tau * 0.05) + pos * np.log(100.0)
    g0 = orc.holdout_grad(X, Y, log_lam=ll, **kw)
    h = 1e-4
    fd = (orc.holdout_grad(X, Y, log_lam=ll + h, **kw).E - orc.holdout_grad(X, Y, log_lam=ll - h, **kw).E) / (2 * h)
    np.testing.assert_allclose(g0.dE, fd, rtol=1e-5, atol=1e-9 * np.abs(g0.E).max())
