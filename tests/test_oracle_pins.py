"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these compares the oracle with itself: each check uses a closed form,
a hand-derived fixture, an invariant, a library routine for a special case, or
a bound stated in the paper (Kuang, Gittens, Hamid, arXiv 1404.0466).
"""
import math
import os

import numpy as np
import pytest

import oracle as orc
from paper_1404_0466_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EPS = np.finfo(np.float64).eps


def _spd(rng, d, cond=100.0):
    Q = synth.haar_orthogonal(rng, d)
    ev = np.geomspace(1.0, 1.0 / cond, d)
    return (Q * ev) @ Q.T


def _golden_chol():
    rows = []
    with open(os.path.join(GOLDEN, "chol_closed_form.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, d, lam, A, L = [s.strip() for s in line.split("|")]
            d = int(d)
            rows.append((name, d, float(lam),
                         np.array(A.split(), dtype=float).reshape(d, d),
                         np.array(L.split(), dtype=float).reshape(d, d)))
    return rows


# --------------------------------------------------------------------------
# Cholesky factor and triangular solves (Sec. 3.2)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", _golden_chol(), ids=lambda c: c[0])
def test_cholesky_closed_form(case):
    name, d, lam, A, L_ref = case
    L = orc.cholesky(A + lam * np.eye(d))
    np.testing.assert_allclose(L, L_ref, rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("d", [1, 7, 64, 131])
def test_cholesky_residual_and_structure(d):
    rng = np.random.default_rng(10 + d)
    A = _spd(rng, d, cond=1e4)
    L = orc.cholesky(A)
    assert np.all(np.triu(L, 1) == 0.0)
    assert np.all(np.diag(L) > 0)
    res = np.linalg.norm(L @ L.T - A) / np.linalg.norm(A)
    assert res <= 4 * d * EPS, res


def test_cholesky_matches_library():
    rng = np.random.default_rng(3)
    A = _spd(rng, 90, cond=1e6)
    np.testing.assert_allclose(orc.cholesky(A), np.linalg.cholesky(A), rtol=0, atol=1e-12)


def test_cholesky_rejects_indefinite():
    rng = np.random.default_rng(4)
    Q = synth.haar_orthogonal(rng, 12)
    ev = np.linspace(1.0, 2.0, 12)
    ev[5] = -0.5
    A = (Q * ev) @ Q.T
    with pytest.raises(orc.NotSPD) as ei:
        orc.cholesky(A)
    assert 0 <= ei.value.pivot < 12


def test_triangular_solves_match_library():
    rng = np.random.default_rng(5)
    d, c = 77, 6
    A = _spd(rng, d, cond=1e3)
    L = np.linalg.cholesky(A)
    B = rng.standard_normal((d, c))
    Z = orc.forward(L, B)
    np.testing.assert_allclose(L @ Z, B, rtol=0, atol=1e-12 * np.abs(B).max() * d)
    W = orc.backward(L, Z)
    np.testing.assert_allclose(L.T @ W, Z, rtol=0, atol=1e-12 * np.abs(Z).max() * d)
    np.testing.assert_allclose(orc.solve_factored(L, B), np.linalg.solve(A, B), rtol=1e-9, atol=1e-12)


# --------------------------------------------------------------------------
# ridge solution (Eq. 1-2) against closed forms
# --------------------------------------------------------------------------

def test_ridge_matches_eigendecomposition_closed_form():
    """Eq. `reg_normal_equation_svd` restated on H = Q diag(mu) Q^T:
    W(lambda) = Q diag(1 / (mu + lambda)) Q^T B."""
    p = synth.spectral_gaussian(300, 40, 3, seed=11)
    H, B = orc.normal_blocks(p.X, p.Y)
    mu, Q = np.linalg.eigh(p.X.T @ p.X)
    for lam in [1e-3, 0.1, 10.0, 1e3]:
        W = orc.solve_factored(orc.cholesky(H + lam * np.eye(40)), B)
        W_ref = Q @ ((Q.T @ (p.X.T @ p.Y)) / (mu + lam)[:, None])
        np.testing.assert_allclose(W, W_ref, rtol=1e-10, atol=1e-12 * np.abs(W_ref).max())


def test_ridge_matches_augmented_least_squares():
    """Eq. 1 is the least-squares problem [X; sqrt(lambda) I] W ~ [Y; 0]."""
    rng = np.random.default_rng(12)
    n, d, c, lam = 40, 9, 2, 0.37
    X = rng.standard_normal((n, d))
    Y = rng.standard_normal((n, c))
    H, B = orc.normal_blocks(X, Y)
    W = orc.solve_factored(orc.cholesky(H + lam * np.eye(d)), B)
    Xa = np.vstack([X, math.sqrt(lam) * np.eye(d)])
    Ya = np.vstack([Y, np.zeros((d, c))])
    W_ref = np.linalg.lstsq(Xa, Ya, rcond=None)[0]
    np.testing.assert_allclose(W, W_ref, rtol=1e-11, atol=1e-13)


def test_normal_blocks_leave_out_rows():
    """H_f = X^T X - X_f^T X_f = sum_{j != f} X_j^T X_j (Eq. 2 on the training rows)."""
    rng = np.random.default_rng(13)
    n, d, c, k = 103, 17, 4, 5
    X = rng.standard_normal((n, d))
    Y = rng.standard_normal((n, c))
    offs = orc.fold_offsets(n, k)
    for f in range(k):
        H, B = orc.normal_blocks(X, Y, offs[f], offs[f + 1])
        keep = np.r_[0:offs[f], offs[f + 1]:n]
        np.testing.assert_allclose(H, X[keep].T @ X[keep], rtol=1e-13, atol=1e-12)
        np.testing.assert_allclose(B, X[keep].T @ Y[keep], rtol=1e-13, atol=1e-12)
        G = sum(X[offs[j]:offs[j + 1]].T @ X[offs[j]:offs[j + 1]] for j in range(k) if j != f)
        np.testing.assert_allclose(H, G, rtol=1e-12, atol=1e-12)
        assert np.array_equal(H, H.T)


def test_holdout_sse_direct_and_expansion():
    """||Y - X W||^2 directly, and the expansion
    ||Y||^2 - 2 <X^T Y, W> + <W, X^T X W> that the device path uses."""
    rng = np.random.default_rng(14)
    X = rng.standard_normal((57, 11))
    Y = rng.standard_normal((57, 3))
    W = rng.standard_normal((11, 3))
    sse = orc.holdout_sse(X, Y, W)
    ref = float(np.sum((Y - X @ W) ** 2))
    assert abs(sse - ref) <= 1e-12 * ref
    G, Bv = X.T @ X, X.T @ Y
    expn = float(np.sum(Y * Y) - 2 * np.sum(Bv * W) + np.sum(W * (G @ W)))
    assert abs(expn - ref) <= 1e-10 * ref


# --------------------------------------------------------------------------
# Algorithm 1: basis, observation matrix, least-squares fit
# --------------------------------------------------------------------------

def test_lstsq_matches_library_and_pseudoinverse():
    rng = np.random.default_rng(15)
    V = rng.standard_normal((6, 4))
    T = rng.standard_normal((6, 33))
    np.testing.assert_allclose(orc.lstsq(V, T), np.linalg.lstsq(V, T, rcond=None)[0],
                               rtol=1e-12, atol=1e-13)
    P = orc.lstsq(V, np.eye(6))        # V^+ (p x g)
    np.testing.assert_allclose(P @ V, np.eye(4), atol=1e-13)


def test_chebyshev_basis_matches_library():
    lam_s = np.geomspace(0.02, 50.0, 6)
    lam = np.geomspace(0.02, 50.0, 41)
    Phi = orc.basis_values(orc.BASIS_CHEB_LOG, lam, lam_s, 5)
    u = 2 * (np.log(lam) - np.log(0.02)) / (np.log(50.0) - np.log(0.02)) - 1
    np.testing.assert_allclose(Phi, np.polynomial.chebyshev.chebvander(u, 4), atol=1e-14)
    assert np.allclose(Phi[[0, -1], 1], [-1.0, 1.0])


def test_basis_derivatives_match_finite_differences():
    lam_s = np.geomspace(0.3, 30.0, 5)
    lam = np.array([0.5, 2.0, 17.0])
    for kind in (orc.BASIS_MONO, orc.BASIS_CHEB_LOG):
        dPhi = orc.basis_derivs(kind, lam, lam_s, 4)
        h = 1e-6 * lam
        fd = (orc.basis_values(kind, lam + h, lam_s, 4) - orc.basis_values(kind, lam - h, lam_s, 4)) / (2 * h[:, None])
        np.testing.assert_allclose(dPhi, fd, rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("kind", [orc.BASIS_MONO, orc.BASIS_CHEB_LOG])
def test_fit_reproduces_polynomials(kind):
    """If every column of T is a polynomial of degree <= r in the basis, the
    least-squares fit of Algorithm 1 returns its coefficients exactly."""
    rng = np.random.default_rng(16)
    lam_s = np.geomspace(0.1, 10.0, 6)
    V = orc.basis_values(kind, lam_s, lam_s, 4)
    Theta_star = rng.standard_normal((4, 50))
    np.testing.assert_allclose(orc.lstsq(V, V @ Theta_star), Theta_star, rtol=1e-10, atol=1e-10)


def test_monomial_scaling_leaves_the_fit_unchanged():
    """Algorithm 1 uses raw monomials 1, lambda, lambda^2; dividing lambda by the
    largest sample spans the same space, so the fitted values agree with a
    library polynomial fit in the raw variable."""
    rng = np.random.default_rng(17)
    lam_s = np.array([0.2, 0.9, 2.5, 4.0])
    T = rng.standard_normal((4, 7))
    Theta = orc.lstsq(orc.basis_values(orc.BASIS_MONO, lam_s, lam_s, 3), T)
    lam = np.array([0.3, 1.7, 3.3])
    got = orc.basis_values(orc.BASIS_MONO, lam, lam_s, 3) @ Theta
    for j in range(7):
        coef = np.polyfit(lam_s, T[:, j], 2)
        np.testing.assert_allclose(got[:, j], np.polyval(coef, lam), rtol=1e-10, atol=1e-12)


def test_vectorisation_round_trip():
    rng = np.random.default_rng(18)
    L = np.tril(rng.standard_normal((9, 9)))
    v = orc.vec_lower(L)
    assert v.size == 45
    assert v[0] == L[0, 0] and v[1] == L[1, 0] and v[2] == L[1, 1] and v[3] == L[2, 0]
    np.testing.assert_array_equal(orc.unvec_lower(v, 9), L)


# --------------------------------------------------------------------------
# small host-side steps
# --------------------------------------------------------------------------

def test_fold_offsets_partition_rows():
    for n, k in [(10, 3), (2048, 5), (7, 7), (103, 5)]:
        o = orc.fold_offsets(n, k)
        assert o[0] == 0 and o[-1] == n and len(o) == k + 1
        sizes = np.diff(o)
        assert sizes.min() >= n // k and sizes.max() <= n // k + 1
    # the split's convention (the paper leaves it open): boundaries floor(f n / k),
    # so the longer folds come last
    assert orc.fold_offsets(10, 3) == [0, 3, 6, 10]
    assert orc.fold_offsets(103, 5) == [0, 20, 41, 61, 82, 103]


def test_sample_indices_and_grid():
    assert orc.sample_indices(31, 4) == [0, 10, 20, 30]
    assert orc.sample_indices(101, 6) == [0, 20, 40, 60, 80, 100]
    assert orc.sample_indices(51, 5) == [0, 13, 25, 38, 50]   # 12.5 and 37.5 round up
    lam = orc.lambda_grid(2.0, 31, 1e-3, 1e1)
    assert np.isclose(lam[0], 2e-3) and np.isclose(lam[-1], 20.0)
    np.testing.assert_allclose(np.diff(np.log(lam)), np.log(1e4) / 30, rtol=1e-12)
    # degenerate grids: one lambda (the low end), one sample (index 0)
    assert np.allclose(orc.lambda_grid(2.0, 1, 1e-3, 1e1), [2e-3])
    assert orc.sample_indices(1, 1) == [0] and orc.sample_indices(9, 1) == [0]
    assert orc.sample_indices(2, 2) == [0, 1]


def test_trace_scale():
    rng = np.random.default_rng(19)
    X = rng.standard_normal((30, 8))
    assert np.isclose(orc.trace_scale(X), np.trace(X.T @ X) / 8, rtol=1e-14)


def test_argmin_first_ties_and_inf():
    assert orc.argmin_first(np.array([3.0, 1.0, 1.0, 2.0])) == 1
    assert orc.argmin_first(np.array([np.inf, 5.0, np.inf])) == 1
    assert orc.argmin_first(np.array([np.inf, np.nan])) == -1


def test_unusable_diagonal_rule():
    assert orc.diag_unusable(np.array([1.0, -1e-3, 2.0]))
    assert orc.diag_unusable(np.array([1.0, 1e-20, 2.0]))
    assert not orc.diag_unusable(np.array([1.0, 1e-3, 2.0]))
    # the threshold is 1e3 eps max|diag| = 4.44e-13 here: either side of it
    assert orc.diag_unusable(np.array([1.0, 1e-14, 2.0]))
    assert orc.diag_unusable(np.array([1.0, 4.4e-13, 2.0]))
    assert not orc.diag_unusable(np.array([1.0, 4.5e-13, 2.0]))


# --------------------------------------------------------------------------
# interpolation: nodes, exact cases and the paper's bounds (Sec. 4)
# --------------------------------------------------------------------------

def test_fit_reproduces_factors_at_nodes_when_g_equals_r_plus_1():
    """With g = r + 1 the observation matrix V is square and invertible
    (Algorithm 1 allows g > r), so the polynomials interpolate the sampled
    factors: L_tilde(lambda_s) = L_s."""
    p = synth.spectral_gaussian(200, 12, 2, seed=20)
    for kind in (orc.BASIS_MONO, orc.BASIS_CHEB_LOG):
        res = orc.cv(p.X, p.Y, k=4, g=3, r=2, q=9, basis=kind, keep=True, folds=[1])
        lam_s = res.lam[res.sample_idx]
        Phi = orc.basis_values(kind, lam_s, lam_s, 3)
        for s in range(3):
            Lt = orc.unvec_lower(Phi[s] @ res.theta[1], 12)
            np.testing.assert_allclose(Lt, res.factors[(1, s)], rtol=1e-9, atol=1e-11)


def test_pichol_equals_exact_cv_when_every_lambda_is_a_node():
    """Sampling every grid lambda with r = g - 1 makes the fit interpolate each
    exact factor, so piCholesky CV equals exact CV (Sec. 6.2, Chol)."""
    p = synth.spectral_gaussian(160, 10, 3, seed=21)
    a = orc.cv(p.X, p.Y, k=4, g=4, r=3, q=4, basis=orc.BASIS_CHEB_LOG)
    b = orc.cv(p.X, p.Y, k=4, g=4, r=3, q=4, exact=True)
    np.testing.assert_allclose(a.E, b.E, rtol=1e-8)
    assert a.t_star == b.t_star


def test_exact_cv_matches_independent_library_pipeline():
    """Exact CV hold-out errors against np.linalg.solve on every fold and lambda."""
    p = synth.spectral_gaussian(150, 14, 2, seed=22)
    res = orc.cv(p.X, p.Y, k=5, g=1, r=0, q=7, exact=True)
    X, Y = p.X, p.Y
    offs = orc.fold_offsets(150, 5)
    tau = np.trace(X.T @ X) / 14
    lam = tau * 1e-3 * (1e4) ** (np.arange(7) / 6)
    for f in range(5):
        keep = np.r_[0:offs[f], offs[f + 1]:150]
        H = X[keep].T @ X[keep]
        B = X[keep].T @ Y[keep]
        Xv, Yv = X[offs[f]:offs[f + 1]], Y[offs[f]:offs[f + 1]]
        for t in range(7):
            W = np.linalg.solve(H + lam[t] * np.eye(14), B)
            ref = np.mean((Yv - Xv @ W) ** 2)
            assert abs(res.E[f, t] - ref) <= 1e-10 * ref
    Ebar = res.E.mean(axis=0)
    assert res.t_star == int(np.argmin(Ebar))


def test_caller_lambdas_and_offsets_equal_to_the_defaults_change_nothing():
    """Passing the grid, its samples and the floor split explicitly gives the
    default run bit for bit (the options only replace where the values come from)."""
    p = synth.spectral_gaussian(150, 14, 2, seed=23)
    kw = dict(k=5, g=4, r=2, q=9, basis=orc.BASIS_CHEB_LOG)
    a = orc.cv(p.X, p.Y, **kw)
    b = orc.cv(p.X, p.Y, lams=a.lam, lam_samples=a.lam[a.sample_idx], offsets=orc.fold_offsets(150, 5), **kw)
    assert np.array_equal(a.E, b.E) and a.t_star == b.t_star


def test_interpolant_at_caller_nodes_is_exact_at_those_lambdas():
    """Algorithm 1 at caller-chosen nodes off the grid, g = r + 1: the fitted
    polynomials pass through the exact factors there (Sec. 3.3), so piCholesky
    evaluated at the nodes gives exact CV's hold-out errors at those lambdas,
    while at a lambda between the nodes it differs."""
    p = synth.spectral_gaussian(160, 12, 3, seed=24)
    tau = orc.trace_scale(p.X)
    nodes = tau * np.array([0.0137, 0.41, 2.9])
    # the evaluation lambdas' own evenly spaced samples (indices 0, 2, 4) are not the nodes
    lams = np.array([nodes[0], nodes[1], 1.7 * tau, 5.0 * tau, nodes[2]])
    for kind in (orc.BASIS_MONO, orc.BASIS_CHEB_LOG):
        pi = orc.cv(p.X, p.Y, k=4, g=3, r=2, q=5, basis=kind, lams=lams, lam_samples=nodes)
        ex = orc.cv(p.X, p.Y, k=4, g=1, r=0, q=5, exact=True, lams=lams)
        for t in (0, 1, 4):
            np.testing.assert_allclose(pi.E[:, t], ex.E[:, t], rtol=1e-9)
        assert np.max(np.abs(pi.E[:, 2] - ex.E[:, 2]) / ex.E[:, 2]) > 1e-7
    # fitted at the evaluation lambdas' own samples instead, the factor at nodes[1] is interpolated
    own = orc.cv(p.X, p.Y, k=4, g=3, r=2, q=5, basis=orc.BASIS_CHEB_LOG, lams=lams)
    assert np.max(np.abs(own.E[:, 1] - ex.E[:, 1]) / ex.E[:, 1]) > 1e-7
    np.testing.assert_allclose(own.E[:, 2], ex.E[:, 2], rtol=1e-9)


def test_caller_fold_offsets_match_an_independent_pipeline():
    """Uneven caller folds: exact CV against np.linalg.solve on each fold's
    training rows (H_f, B_f left out by the caller's offsets), and the rows of
    one fold scored alone."""
    p = synth.spectral_gaussian(130, 9, 2, seed=25)
    offs = [0, 7, 50, 51, 130]
    lams = np.array([0.3, 2.0, 11.0])
    res = orc.cv(p.X, p.Y, k=4, g=1, r=0, q=3, exact=True, lams=lams, offsets=offs)
    X, Y = p.X, p.Y
    for f in range(4):
        keep = np.r_[0:offs[f], offs[f + 1]:130]
        H, B = X[keep].T @ X[keep], X[keep].T @ Y[keep]
        Xv, Yv = X[offs[f]:offs[f + 1]], Y[offs[f]:offs[f + 1]]
        for t, lam in enumerate(lams):
            W = np.linalg.solve(H + lam * np.eye(9), B)
            ref = np.mean((Yv - Xv @ W) ** 2)
            assert abs(res.E[f, t] - ref) <= 1e-10 * ref
    with pytest.raises(ValueError):
        orc.cv(p.X, p.Y, k=4, g=1, r=0, q=3, exact=True, offsets=[0, 7, 7, 51, 130])
    with pytest.raises(ValueError):
        orc.cv(p.X, p.Y, k=4, g=1, r=0, q=3, exact=True, lams=[1.0, -1.0, 2.0])


def _kron_sum(L):
    d = L.shape[0]
    I = np.eye(d)
    return np.kron(I, L) + np.kron(L, I)


def _vec(M):
    return M.reshape(-1, order="F")


def _unvec(v, d):
    return v.reshape(d, d, order="F")


def _R_and_pieces(h, s):
    """Quantities of Thm 4.4 at shift s for A = diag(h), built from the
    d^2 x d^2 Kronecker sums M_s = [[C(A + s I)]] and E_s."""
    d = h.size
    L = np.diag(np.sqrt(h + s))
    M = _kron_sum(L)
    Mi = np.linalg.inv(M)
    vI = _vec(np.eye(d))
    MivI = Mi @ vI
    E = _kron_sum(_unvec(MivI, d))
    MiE = Mi @ E
    R = (np.linalg.norm(MiE, 2) ** 2 * np.linalg.norm(MivI)
         + np.linalg.norm(Mi, 2) * np.linalg.norm(MiE, 2) * np.linalg.norm(MivI) ** 2)
    return L, Mi, MivI, E, R


def test_taylor_polynomial_and_bound_thm_4_4():
    """For diagonal A the entries of C(A + lambda I) are sqrt(h_i + lambda); the
    second-order Taylor polynomial of Thm 4.4 must equal the scalar Taylor
    polynomial of sqrt, and its error must respect the stated bound."""
    h = np.array([0.4, 1.3, 2.2])
    d = h.size
    D = d * (d + 1) / 2
    lc = 1.0
    L, Mi, MivI, E, _ = _R_and_pieces(h, lc)
    for lam in [0.6, 0.9, 1.25, 1.5]:
        dl = lam - lc
        pTS = L + _unvec(dl * MivI - 0.5 * dl ** 2 * (Mi @ E @ MivI), d)
        l0 = np.sqrt(h + lc)
        scalar = l0 + dl / (2 * l0) - dl ** 2 / (8 * l0 ** 3)
        np.testing.assert_allclose(np.diag(pTS), scalar, rtol=1e-12)
        exact = np.diag(np.sqrt(h + lam))
        lhs = np.linalg.norm(exact - pTS) / math.sqrt(D)
        Rmax = max(_R_and_pieces(h, s)[4] for s in np.linspace(min(lam, lc), max(lam, lc), 41))
        rhs = 2 * abs(dl) ** 3 / (3 * math.sqrt(D)) * Rmax
        assert lhs <= rhs, (lam, lhs, rhs)


def test_main_bound_thm_4_7_diagonal():
    """Thm 4.7 (r = 2, g = 4 > 3 samples within w of lambda_c, lambda_c > gamma >= w)
    on a diagonal A, where the derivative formulas of Thm 4.3 hold exactly.
    The left side uses the oracle's own fit (Algorithm 1)."""
    h = np.array([0.5, 1.1, 1.9])
    d = h.size
    D = d * (d + 1) / 2
    lc, w, gamma, g = 1.2, 0.3, 0.45, 4
    lam_s = lc + w * np.array([-1.0, -1 / 3, 1 / 3, 1.0])
    T = np.stack([orc.vec_lower(orc.cholesky(np.diag(h) + ls * np.eye(d))) for ls in lam_s])
    Theta = orc.lstsq(orc.basis_values(orc.BASIS_MONO, lam_s, lam_s, 3), T)
    V = np.stack([np.ones(g), lam_s, lam_s ** 2], axis=1)
    Vpinv = np.linalg.norm(np.linalg.pinv(V), 2)
    R = max(_R_and_pieces(h, s)[4] for s in np.linspace(lc - gamma, lc + gamma, 61))
    rhs = (gamma ** 3 + math.sqrt(g) * w ** 3 * (1 + gamma ** 2) * (lc + 1) * Vpinv) * R / math.sqrt(D)
    worst = 0.0
    for lam in np.linspace(lc - gamma, lc + gamma, 31):
        Lt = orc.unvec_lower(orc.basis_values(orc.BASIS_MONO, [lam], lam_s, 3)[0] @ Theta, d)
        lhs = np.linalg.norm(np.diag(np.sqrt(h + lam)) - Lt) / math.sqrt(D)
        worst = max(worst, lhs)
        assert lhs <= rhs, (lam, lhs, rhs)
    assert worst > 0.0


def test_diagonal_hessian_interpolation_error_is_small():
    """Diagonal H: the exact factor is diag(sqrt(h + lambda)) and off-diagonal
    entries stay zero; piCholesky over a narrow range must track it."""
    h = np.array([1.0, 2.0, 3.0, 5.0])
    lam_s = np.linspace(0.5, 1.5, 5)
    T = np.stack([orc.vec_lower(orc.cholesky(np.diag(h) + ls * np.eye(4))) for ls in lam_s])
    Theta = orc.lstsq(orc.basis_values(orc.BASIS_MONO, lam_s, lam_s, 3), T)
    # scale of the cubic Taylor remainder of sqrt(h + lambda) about the centre:
    # max |f'''| w^3 / 6 with f''' = (3/8) (h + lambda)^(-5/2), w = 0.5
    tol = (3 / 8) * (h + 0.5) ** -2.5 * 0.5 ** 3 / 6
    for lam in np.linspace(0.5, 1.5, 11):
        Lt = orc.unvec_lower(orc.basis_values(orc.BASIS_MONO, [lam], lam_s, 3)[0] @ Theta, 4)
        assert np.all(np.abs(np.diag(Lt) - np.sqrt(h + lam)) <= tol)
        assert np.abs(np.tril(Lt, -1)).max() < 1e-14


# --------------------------------------------------------------------------
# gradient of the hold-out error in log(lambda)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("exact,basis", [(True, "mono"), (False, orc.BASIS_CHEB_LOG), (False, orc.BASIS_MONO)])
def test_holdout_gradient_matches_central_differences(exact, basis):
    """dE/dlog(lambda) against central differences of E itself (h = 1e-4 in
    log lambda), for the exact factor and for the interpolated factor."""
    p = synth.spectral_gaussian(240, 16, 3, seed=50)
    kw = dict(k=4, g=4, r=2, q=9, basis=basis, exact=exact)
    for ll in (np.log(0.05), np.log(2.0)):
        tau = orc.trace_scale(p.X)
        ll = ll + np.log(tau)
        gr = orc.holdout_grad(p.X, p.Y, log_lam=ll, **kw)
        h = 1e-4
        ep = orc.holdout_grad(p.X, p.Y, log_lam=ll + h, **kw).E
        em = orc.holdout_grad(p.X, p.Y, log_lam=ll - h, **kw).E
        fd = (ep - em) / (2 * h)
        np.testing.assert_allclose(gr.dE, fd, rtol=1e-5, atol=1e-9 * np.abs(gr.E).max())


def test_exact_gradient_matches_eigen_closed_form():
    """For exact ridge, E(lambda) has the closed form through H = Q diag(mu) Q^T;
    its derivative in log(lambda) is lambda * sum over the eigenbasis."""
    p = synth.spectral_gaussian(200, 12, 2, seed=51)
    k = 4
    offs = orc.fold_offsets(200, k)
    lam = 0.3 * orc.trace_scale(p.X)
    gr = orc.holdout_grad(p.X, p.Y, k=k, g=2, r=1, q=3, log_lam=np.log(lam), exact=True)
    for f in range(k):
        keep = np.r_[0:offs[f], offs[f + 1]:200]
        H = p.X[keep].T @ p.X[keep]
        B = p.X[keep].T @ p.Y[keep]
        mu, Q = np.linalg.eigh(H)
        Xv, Yv = p.X[offs[f]:offs[f + 1]], p.Y[offs[f]:offs[f + 1]]
        Bq = Q.T @ B
        W = Q @ (Bq / (mu + lam)[:, None])
        dW = Q @ (-Bq / ((mu + lam) ** 2)[:, None])
        R = Yv - Xv @ W
        nvc = R.size
        assert abs(gr.E[f] - np.sum(R * R) / nvc) <= 1e-10 * gr.E[f]
        ref = lam * (-2.0 / nvc) * np.sum((Xv.T @ R) * dW)
        assert abs(gr.dE[f] - ref) <= 1e-8 * abs(ref) + 1e-14


# ---------------------------------------------------------------------------
# refinement against the exact system with the interpolated factor as the
# preconditioner (not in the paper)
# ---------------------------------------------------------------------------

def test_exact_system_refinement_step_is_the_preconditioned_iteration():
    """One step maps the error e0 = w0 - w* to (I - M^{-1} A) e0 with
    M = L~ L~^T and A = H_f + lambda I, both solved densely by numpy."""
    prob = synth.spectral_gaussian(300, 20, 2, seed=71)
    kw = dict(k=3, g=4, r=2, q=7, basis="cheb_log", folds=[1], lam_idx=[2], keep=True)
    r0 = orc.cv(prob.X, prob.Y, **kw)
    r1 = orc.cv(prob.X, prob.Y, precond_steps=1, **kw)
    f, t = 1, 2
    Hf, Bf = r0.H[f], r0.B[f]
    A = Hf + r0.lam[t] * np.eye(Hf.shape[0])
    lam_s = r0.lam[r0.sample_idx]
    phi = orc.basis_values("cheb_log", [r0.lam[t]], lam_s, 3)[0]
    Lt = orc.unvec_lower(orc.eval_poly(phi, r0.theta[f]), Hf.shape[0])
    M = Lt @ Lt.T
    w_star = np.linalg.solve(A, Bf)
    e0 = r0.W[(f, t)] - w_star
    e1 = r1.W[(f, t)] - w_star
    np.testing.assert_allclose(e1, e0 - np.linalg.solve(M, A @ e0), rtol=1e-8, atol=1e-12 * np.abs(w_star).max())


def test_exact_system_refinement_converges_to_exact_cv():
    """Where the interpolated factor is a good preconditioner (the mixed
    case's generator), each step shrinks the distance to exact CV."""
    prob = synth.mixed_ecc(n=2048, d=96)
    kw = dict(k=4, g=6, r=3, q=41, basis="cheb_log", folds=[0])
    ex = orc.cv(prob.X, prob.Y, exact=True, **kw)
    errs = [np.max(np.abs(orc.cv(prob.X, prob.Y, precond_steps=st, **kw).E[0] - ex.E[0]) / ex.E[0])
            for st in (0, 1, 2, 3)]
    assert errs[0] > 1e-4
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3 and errs[3] < errs[2] / 3, errs


def test_exact_system_refinement_is_idle_when_every_lambda_is_a_node():
    prob = synth.spectral_gaussian(200, 12, 2, seed=72)
    kw = dict(k=4, g=5, r=4, q=5, basis="cheb_log")
    ex = orc.cv(prob.X, prob.Y, exact=True, **kw)
    r1 = orc.cv(prob.X, prob.Y, precond_steps=1, **kw)
    np.testing.assert_allclose(r1.E, ex.E, rtol=1e-11)


# ----------------------------------------------------------------------------
# MChol (Sec. 6.2): multi-level narrowing of the lambda range
# ----------------------------------------------------------------------------

def test_exact_holdout_at_any_lambda_matches_eigen_closed_form():
    """Exact hold-out MSE at lambdas off any grid, against the spectral form
    W = Q diag(1 / (mu + lambda)) Q^T B on each fold's training rows."""
    p = synth.spectral_gaussian(180, 12, 3, seed=81)
    lams = np.array([3.7e-2, 1.0, 55.5])
    E = orc.holdout_exact_at(p.X, p.Y, k=4, lams=lams)
    offs = orc.fold_offsets(180, 4)
    for f in range(4):
        keep = np.r_[0:offs[f], offs[f + 1]:180]
        mu, Q = np.linalg.eigh(p.X[keep].T @ p.X[keep])
        B = p.X[keep].T @ p.Y[keep]
        Xv, Yv = p.X[offs[f]:offs[f + 1]], p.Y[offs[f]:offs[f + 1]]
        for i, lam in enumerate(lams):
            W = Q @ ((Q.T @ B) / (mu + lam)[:, None])
            ref = np.mean((Yv - Xv @ W) ** 2)
            assert abs(E[f, i] - ref) <= 1e-10 * ref
    assert np.all(np.isnan(orc.holdout_exact_at(p.X, p.Y, k=4, lams=lams, folds=[1])[[0, 2, 3]]))


def test_mchol_level_count():
    """The paper's parameters s = 1.5, s0 = 0.0025 (Sec. 6.3): 1.5 / 2^9 > s0
    and 1.5 / 2^10 <= s0, so ten levels; a start already below s0 still runs
    one level."""
    assert orc.mchol_levels(1.5, 0.0025) == 10
    assert orc.mchol_levels(1.5, 0.1) == 4
    assert orc.mchol_levels(1.5, 0.75) == 1
    assert orc.mchol_levels(0.1, 0.2) == 1
    with pytest.raises(ValueError):
        orc.mchol_levels(1.0, 0.0)


def test_mchol_search_hand_traced():
    """h(lambda) = (log10 lambda - 0.3)^2 from c = 0, s = 1.5, s0 = 0.0025,
    traced by hand: the nearest of the three points wins at each level.
      s=1.5     {-1.5, 0, 1.5}              -> 0
      s=0.75    {-0.75, 0, 0.75}            -> 0
      s=0.375   {-0.375, 0, 0.375}          -> 0.375
      s=0.1875  {0.1875, 0.375, 0.5625}     -> 0.375
      s=0.09375 {0.28125, 0.375, 0.46875}   -> 0.28125
      s=3/64    {0.234375, 0.28125, 0.328125} -> 0.28125
      s=3/128   {0.2578125, 0.28125, 0.3046875} -> 0.3046875
      s=3/256   {0.29296875, 0.3046875, 0.31640625} -> 0.3046875
      s=3/512   {0.298828125, 0.3046875, 0.310546875} -> 0.298828125
      s=3/1024  {0.2958984375, 0.298828125, 0.3017578125} -> 0.298828125
    final c = 153/512, s = 3/2048."""
    res = orc.mchol_search(lambda lam: (np.log10(lam) - 0.3) ** 2, 0.0, 1.5, 0.0025)
    assert res.best == [1, 1, 2, 1, 0, 1, 2, 1, 0, 1]
    assert abs(res.c - 153 / 512) < 1e-12
    assert res.s == 3 / 2048
    np.testing.assert_allclose(res.lams[4], 10.0 ** np.array([0.28125, 0.375, 0.46875]), rtol=1e-14)


def test_mchol_search_brackets_a_unimodal_minimum():
    """For h = (log10 lambda - c*)^2 the winner of a level is the point nearest
    c*, so |c - c*| <= 1.5 s before a level gives |c - c*| <= s after it; from
    c = 0, s = 1.5 every c* in [-2.25, 2.25] ends within the final s."""
    for cstar in np.linspace(-2.25, 2.25, 41):
        res = orc.mchol_search(lambda lam: (np.log10(lam) - cstar) ** 2, 0.0, 1.5, 0.01)
        assert abs(res.c - cstar) <= res.s + 1e-12, (cstar, res.c, res.s)


def test_mchol_search_ties_and_non_finite_values():
    """Equal errors pick the smallest lambda (first argmin): c drops by s at
    every level, c_final = c0 - 2 s0 (1 - 2^-n).  A level with no finite
    value keeps c and still halves s."""
    res = orc.mchol_search(lambda lam: np.ones_like(lam), 1.0, 1.0, 0.1)
    n = orc.mchol_levels(1.0, 0.1)
    assert res.best == [0] * n
    assert abs(res.c - (1.0 - 2.0 * (1.0 - 2.0 ** -n))) < 1e-12
    res = orc.mchol_search(lambda lam: np.full_like(lam, np.inf), 0.5, 1.0, 0.1)
    assert res.best == [-1] * n and res.c == 0.5 and res.s == 2.0 ** -n


def test_mchol_on_data_finds_the_dense_scan_minimum():
    """On data whose exact mean hold-out curve is unimodal in log lambda
    (checked on a dense scan), MChol ends within its final half-width plus
    one scan step of the scan's minimum, the best error never rises from one
    level to the next, and each level is centred on the previous winner."""
    p = synth.spectral_gaussian(240, 16, 2, seed=83)
    k = 4
    tau = orc.trace_scale(p.X)
    u = np.linspace(-4.0, 1.0, 201)
    Ebar = orc.holdout_exact_at(p.X, p.Y, k=k, lams=tau * 10.0 ** u).mean(axis=0)
    i0 = int(np.argmin(Ebar))
    assert 0 < i0 < u.size - 1
    assert np.all(np.diff(Ebar[:i0 + 1]) < 0) and np.all(np.diff(Ebar[i0:]) > 0)
    res = orc.mchol(p.X, p.Y, k=k, c=-1.5, s=1.5, s_min=0.01)
    assert abs(res.c - u[i0]) <= res.s + (u[1] - u[0])
    mins = [float(np.min(e)) for e in res.Ebar]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(mins, mins[1:]))
    for lv in range(1, len(res.lams)):
        prev = res.lams[lv - 1][res.best[lv - 1]]
        assert abs(res.lams[lv][1] / prev - 1.0) < 1e-12
    lo, hi = res.window
    assert abs(np.log10(hi / lo) - 2 * res.s) < 1e-12


# ----------------------------------------------------------------------------
# PINRMSE (supplementary comparator): the hold-out error interpolated directly
# ----------------------------------------------------------------------------

def test_pinrmse_matches_a_library_polynomial_fit_of_the_exact_errors():
    """With monomials the fitted curve is numpy's least-squares polynomial in
    lambda / max lambda_s through the exact errors at the sampled grid points."""
    p = synth.spectral_gaussian(200, 10, 2, seed=91)
    k, g, r, q = 4, 6, 2, 25
    res = orc.pinrmse(p.X, p.Y, k=k, g=g, r=r, q=q, basis="mono")
    tau = np.trace(p.X.T @ p.X) / 10
    lam = tau * 1e-3 * 1e4 ** (np.arange(q) / (q - 1))
    sidx = [round(i * (q - 1) / (g - 1) + 1e-9) for i in range(g)]
    assert sidx == orc.sample_indices(q, g)
    offs = orc.fold_offsets(200, k)
    for f in range(k):
        keep = np.r_[0:offs[f], offs[f + 1]:200]
        H, B = p.X[keep].T @ p.X[keep], p.X[keep].T @ p.Y[keep]
        Xv, Yv = p.X[offs[f]:offs[f + 1]], p.Y[offs[f]:offs[f + 1]]
        ts = [np.mean((Yv - Xv @ np.linalg.solve(H + lam[i] * np.eye(10), B)) ** 2) for i in sidx]
        x = lam / lam[sidx].max()
        coef = np.polyfit(x[sidx], ts, r)
        np.testing.assert_allclose(res.E[f], np.polyval(coef, x), rtol=1e-8, atol=1e-12)


@pytest.mark.parametrize("basis", ["mono", "cheb_log"])
def test_pinrmse_reproduces_the_exact_errors_at_the_nodes(basis):
    """g = r + 1: the polynomial interpolates, so at the sampled grid points
    PINRMSE equals exact CV; with every grid point a node it is exact CV."""
    p = synth.spectral_gaussian(160, 8, 2, seed=92)
    ex = orc.cv(p.X, p.Y, k=4, g=1, r=0, q=9, exact=True)
    res = orc.pinrmse(p.X, p.Y, k=4, g=5, r=4, q=9, basis=basis)
    sidx = orc.sample_indices(9, 5)
    np.testing.assert_allclose(res.E[:, sidx], ex.E[:, sidx], rtol=1e-9)
    full = orc.pinrmse(p.X, p.Y, k=4, g=5, r=4, q=5, basis=basis)
    ex5 = orc.cv(p.X, p.Y, k=4, g=1, r=0, q=5, exact=True)
    np.testing.assert_allclose(full.E, ex5.E, rtol=1e-9)
    assert full.t_star == ex5.t_star


def test_pinrmse_is_the_fit_of_the_fold_mean_and_rejects_too_few_samples():
    """The fit is linear in t, so the mean over folds of the interpolated errors
    is the interpolation of the mean sampled error; g <= r is refused."""
    p = synth.spectral_gaussian(150, 7, 1, seed=93)
    k, g, r, q = 3, 5, 3, 17
    res = orc.pinrmse(p.X, p.Y, k=k, g=g, r=r, q=q, basis="cheb_log")
    tau = orc.trace_scale(p.X)
    lam = orc.lambda_grid(tau, q, 1e-3, 1e1)
    sidx = orc.sample_indices(q, g)
    tbar = orc.holdout_exact_at(p.X, p.Y, k=k, lams=lam[sidx]).mean(axis=0)
    V = orc.basis_values("cheb_log", lam[sidx], lam[sidx], r + 1)
    Phi = orc.basis_values("cheb_log", lam, lam[sidx], r + 1)
    np.testing.assert_allclose(res.Ebar, Phi @ np.linalg.lstsq(V, tbar, rcond=None)[0], rtol=1e-9)
    with pytest.raises(ValueError):
        orc.pinrmse(p.X, p.Y, k=k, g=3, r=3, q=q)


# ----------------------------------------------------------------------------
# warm start across folds (the paper's future work, Sec. 7)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("basis", ["mono", "cheb_log"])
def test_warm_start_with_every_sample_is_the_plain_fit(basis):
    """g' = g uses fold 0's sample indices; with V of full column rank,
    Theta_0 + V^+ (T - V Theta_0) = V^+ T, the plain fit of Algorithm 1."""
    p = synth.spectral_gaussian(200, 12, 2, seed=101)
    kw = dict(k=4, g=5, r=3, q=21, basis=basis, keep=True)
    a = orc.cv(p.X, p.Y, **kw)
    b = orc.cv(p.X, p.Y, warm=5, **kw)
    for f in range(4):
        np.testing.assert_allclose(b.theta[f], a.theta[f], rtol=1e-8, atol=1e-10 * np.abs(a.theta[f]).max())
    np.testing.assert_allclose(b.E, a.E, rtol=1e-9)


def test_warm_start_interpolates_the_exact_factors_at_its_nodes():
    """g' <= r + 1: the correction interpolates, so at the warm nodes a warm
    fold's interpolated factor is its exact Cholesky factor; fold 0 is the
    plain fit; and the warm samples sit at round(i (q-1)/(g'-1))."""
    p = synth.spectral_gaussian(240, 10, 2, seed=102)
    k, g, r, q = 4, 5, 3, 21
    for warm in (2, 3, 4):
        res = orc.cv(p.X, p.Y, k=k, g=g, r=r, q=q, basis="cheb_log", warm=warm, keep=True)
        assert res.warm_idx == [round(i * (q - 1) / (warm - 1) + 1e-9) for i in range(warm)]
        lam_s = res.lam[res.sample_idx]
        for f in range(1, k):
            for s, t in enumerate(res.warm_idx):
                phi = orc.basis_values("cheb_log", [res.lam[t]], lam_s, r + 1)[0]
                L = orc.unvec_lower(orc.eval_poly(phi, res.theta[f]), 10)
                np.testing.assert_allclose(L, res.factors[(f, s)], rtol=1e-9, atol=1e-11)
        plain = orc.cv(p.X, p.Y, k=k, g=g, r=r, q=q, basis="cheb_log", folds=[0])
        np.testing.assert_allclose(res.E[0], plain.E[0], rtol=1e-12)


def test_warm_start_arguments():
    p = synth.spectral_gaussian(100, 6, 1, seed=103)
    for bad in (1, 6):
        with pytest.raises(ValueError):
            orc.cv(p.X, p.Y, k=3, g=5, r=2, q=11, warm=bad)
    with pytest.raises(ValueError):
        orc.cv(p.X, p.Y, k=3, g=5, r=2, q=11, warm=2, exact=True)


# ----------------------------------------------------------------------------
# NRMSE of the fit (Sec. 6.6 diagnostic)
# ----------------------------------------------------------------------------

def test_nrmse_is_zero_at_the_nodes_and_one_for_the_mean():
    """g = r + 1: the fit interpolates, so the NRMSE vanishes at the sampled
    grid points; and the normalisation makes a prediction by the targets' mean
    score exactly 1 (checked on the definition with the exact factor)."""
    p = synth.spectral_gaussian(200, 10, 2, seed=111)
    k, g, r, q = 4, 4, 3, 13
    curve = orc.nrmse_curve(p.X, p.Y, k=k, g=g, r=r, q=q, basis="cheb_log")
    idx = orc.sample_indices(q, g)
    assert np.all(curve[idx] < 1e-12)
    assert np.all(curve >= 0) and np.all(np.isfinite(curve))
    # the normalisation: the mean predictor's NRMSE is 1 by construction
    H, _ = orc.normal_blocks(p.X, p.Y, *orc.fold_offsets(200, k)[0:2])
    t = orc.vec_lower(np.linalg.cholesky(H + 0.5 * np.eye(10)))
    mean_pred = np.full_like(t, t.mean())
    assert abs(np.sqrt(np.mean((mean_pred - t) ** 2)) / np.sqrt(np.mean((t - t.mean()) ** 2)) - 1.0) < 1e-15


def test_nrmse_is_small_inside_a_well_sampled_range():
    """A narrow, well-sampled range fits the factors closely (the paper reports a
    maximum of 0.0457 on its data); a four-decade range with g = 3 samples fits
    them worse."""
    p = synth.spectral_gaussian(300, 16, 2, seed=112)
    narrow = orc.nrmse_curve(p.X, p.Y, k=4, g=5, r=3, q=21, lo=0.05, hi=0.5, basis="cheb_log")
    wide = orc.nrmse_curve(p.X, p.Y, k=4, g=3, r=2, q=21, lo=1e-3, hi=1e1, basis="cheb_log")
    assert narrow.max() < 1e-3
    assert wide.max() > 10 * narrow.max()


def test_oracle_is_the_same_from_run_to_run():
    """OpenMP in the oracle only runs independent units side by side, so two
    runs give identical bits (the hold-out error's row sums included)."""
    p = synth.spectral_gaussian(300, 20, 2, seed=71)
    for kw in (dict(), dict(warm=3), dict(precond_steps=2), dict(exact=True)):
        a = orc.cv(p.X, p.Y, k=3, g=5, r=3, q=15, basis="cheb_log", **kw)
        b = orc.cv(p.X, p.Y, k=3, g=5, r=3, q=15, basis="cheb_log", **kw)
        assert np.array_equal(a.E, b.E), kw


def test_nrmse_worked_by_hand():
    """pred = (1, 2, 3) for target = (1, 2, 4): the RMSE is sqrt(1/3); the
    target's mean is 7/3, so its RMS deviation is sqrt(14/9) = sqrt(14)/3,
    and the ratio is sqrt(3/14)."""
    assert abs(orc.nrmse([1.0, 2.0, 3.0], [1.0, 2.0, 4.0]) - math.sqrt(3.0 / 14.0)) <= 1e-15
    t = np.array([0.5, -1.0, 2.0, 3.5])
    assert orc.nrmse(t, t) == 0.0
    assert abs(orc.nrmse(np.full(4, t.mean()), t) - 1.0) <= 1e-15
