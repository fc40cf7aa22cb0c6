"""Plain FP64 CPU oracle of piCholesky k-fold cross-validation.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA library (``paper_1404_0466_gb300``) and never imports it; inputs
reach both sides only through the seeded generators in
``paper_1404_0466_gb300.synth``, which the callers pass in as arrays.

The steps follow the paper's method in its own order (Kuang, Gittens, Hamid,
arXiv 1404.0466):

1. k folds of contiguous rows (Sec. 1: k-fold cross-validation; the split
   itself is not specified, contiguous floor boundaries are used).
2. Training Hessian and right-hand side per fold, H_f = X_tr^T X_tr and
   B_f = X_tr^T Y_tr (Sec. 3.1, Eq. 2), by direct sums over the kept rows.
3. A grid of q log-spaced lambdas, scaled by tau = tr(X^T X) / d of the full
   data so one grid is shared by all folds (Sec. 6.3 uses a fixed range; the
   scale makes the range dimensionless).
4. g sampled lambdas at evenly spaced grid indices including both ends
   (Sec. 6.3 samples 4 of its 31 grid values; their positions are not given).
5. Exact Cholesky factors at the sampled lambdas (Algorithm 1, its first step).
6. Target matrix T (g x D) of vectorised lower triangles (Algorithm 1;
   Sec. 5: any ordering gives the same coefficients entrywise).
7. Observation matrix V (g x (r+1)) of a polynomial basis at the sampled
   lambdas (Algorithm 1; monomials, or Chebyshev polynomials which
   Sec. 3.3 names as the more stable choice).
8. Theta = argmin ||T - V Theta||_F (Algorithm 1's least squares) by Householder QR.
9. For each of the q lambdas: interpolated factor L_t = sum_m phi_m(lambda_t)
   Theta_m (Sec. 3.3, last paragraph), forward and back substitution for the c
   right-hand sides (Sec. 3.2), hold-out mean squared error.
10. Mean over folds, argmin over the grid (Sec. 3.1).

Exact cross-validation (``Chol`` of Sec. 6.2) is the same with the exact factor
at every lambda.

Around the method, each written from the paper's description:
  * ``holdout_grad``   : the hold-out error's derivative in log(lambda);
  * ``cv(precond_steps=...)``: refinement against H_f + lambda I (not in the paper);
  * ``cv(warm=...)``   : the warm start across folds of Sec. 7's future work;
  * ``holdout_exact_at``, ``mchol_search``, ``mchol``: MChol's range search (Sec. 6.2);
  * ``pinrmse``        : the supplementary comparator that interpolates the
    sampled hold-out errors themselves;
  * ``nrmse_curve``, ``nrmse``: the NRMSE of the fit per grid lambda (Sec. 6.6).
"""
from __future__ import annotations

import ctypes
import os
import pathlib
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = pathlib.Path(__file__).resolve().parent
_SRC = _HERE / "pichol_oracle.c"
_BUILD = _HERE / "_build"
_SO = _BUILD / "liboracle.so"
_lib = None

BASIS_MONO = "mono"          # phi_m(lambda) = (lambda / lambda_s_max)^m      (Algorithm 1)
BASIS_CHEB_LOG = "cheb_log"  # phi_m(lambda) = T_m(u), u affine in log lambda  (Sec. 3.3)


class NotSPD(RuntimeError):
    """Cholesky met a non-positive pivot (Sec. 3.2 needs H + lambda I > 0)."""

    def __init__(self, pivot: int):
        super().__init__(f"matrix not positive definite at pivot {pivot}")
        self.pivot = pivot


def build(force: bool = False) -> pathlib.Path:
    """Compile the C part of the oracle with gcc (plain -O2, IEEE arithmetic)."""
    _BUILD.mkdir(exist_ok=True)
    if force or not _SO.exists() or _SO.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _BUILD / f"liboracle.{os.getpid()}.so"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp",
                               "-o", str(tmp), str(_SRC), "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _get():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(str(build()))
        i64, dp = ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
        lib.orc_normal_blocks.argtypes = [i64, i64, i64, dp, dp, i64, i64, dp, dp]
        lib.orc_normal_blocks.restype = None
        lib.orc_cholesky.argtypes = [i64, dp, dp]
        lib.orc_cholesky.restype = i64
        lib.orc_forward.argtypes = [i64, i64, dp, dp, dp]
        lib.orc_forward.restype = None
        lib.orc_backward.argtypes = [i64, i64, dp, dp, dp]
        lib.orc_backward.restype = None
        lib.orc_holdout_sse.argtypes = [i64, i64, i64, dp, dp, dp]
        lib.orc_holdout_sse.restype = ctypes.c_double
        lib.orc_lstsq_householder.argtypes = [i64, i64, dp, i64, dp, dp]
        lib.orc_lstsq_householder.restype = ctypes.c_int
        lib.orc_vec_lower.argtypes = [i64, dp, dp]
        lib.orc_vec_lower.restype = None
        lib.orc_unvec_lower.argtypes = [i64, dp, dp]
        lib.orc_unvec_lower.restype = None
        lib.orc_eval_poly.argtypes = [i64, i64, dp, dp, dp]
        lib.orc_eval_poly.restype = None
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------------------
# primitives (thin wrappers over the C loops)
# ----------------------------------------------------------------------------

def normal_blocks(X, Y, skip0: int = 0, skip1: int = 0):
    """H = X_kept^T X_kept, B = X_kept^T Y_kept, rows [skip0, skip1) left out (Eq. 2)."""
    X, Y = _f64(X), _f64(Y)
    n, d = X.shape
    c = Y.shape[1]
    H = np.empty((d, d))
    B = np.empty((d, c))
    _get().orc_normal_blocks(n, d, c, _p(X), _p(Y), skip0, skip1, _p(H), _p(B))
    return H, B


def cholesky(A) -> np.ndarray:
    """Lower Cholesky factor of A (Sec. 3.2); raises NotSPD on a non-positive pivot."""
    A = _f64(A)
    d = A.shape[0]
    L = np.empty((d, d))
    piv = _get().orc_cholesky(d, _p(A), _p(L))
    if piv >= 0:
        raise NotSPD(int(piv))
    return L


def forward(L, B) -> np.ndarray:
    """Z with L Z = B (Sec. 3.2)."""
    L, B = _f64(L), _f64(B)
    d, c = B.shape
    Z = np.empty((d, c))
    _get().orc_forward(d, c, _p(L), _p(B), _p(Z))
    return Z


def backward(L, Z) -> np.ndarray:
    """W with L^T W = Z (Sec. 3.2)."""
    L, Z = _f64(L), _f64(Z)
    d, c = Z.shape
    W = np.empty((d, c))
    _get().orc_backward(d, c, _p(L), _p(Z), _p(W))
    return W


def solve_factored(L, B) -> np.ndarray:
    """W = (L L^T)^{-1} B by forward then back substitution (Sec. 3.2)."""
    return backward(L, forward(L, B))


def holdout_sse(Xv, Yv, W) -> float:
    """||Y_v - X_v W||_F^2 evaluated directly."""
    Xv, Yv, W = _f64(Xv), _f64(Yv), _f64(W)
    nv, d = Xv.shape
    return float(_get().orc_holdout_sse(nv, d, Yv.shape[1], _p(Xv), _p(Yv), _p(W)))


def lstsq(V, T) -> np.ndarray:
    """Theta = argmin ||T - V Theta||_F (Algorithm 1's least squares) by Householder QR."""
    V, T = _f64(V), _f64(T)
    g, p = V.shape
    D = T.shape[1]
    Theta = np.empty((p, D))
    rc = _get().orc_lstsq_householder(g, p, _p(V), D, _p(T), _p(Theta))
    if rc == 2:
        raise MemoryError("no memory for the least-squares scratch matrices")
    if rc:
        raise np.linalg.LinAlgError("observation matrix V is rank deficient")
    return Theta


def vec_lower(L) -> np.ndarray:
    """Row-wise vectorisation of the lower triangle (Sec. 5), length d(d+1)/2."""
    L = _f64(L)
    d = L.shape[0]
    v = np.empty(d * (d + 1) // 2)
    _get().orc_vec_lower(d, _p(L), _p(v))
    return v


def unvec_lower(v, d: int) -> np.ndarray:
    v = _f64(v)
    L = np.empty((d, d))
    _get().orc_unvec_lower(d, _p(v), _p(L))
    return L


def eval_poly(phi, Theta) -> np.ndarray:
    """sum_m phi[m] * Theta[m, :] (Sec. 3.3, evaluating the D polynomials)."""
    phi, Theta = _f64(phi), _f64(Theta)
    p, D = Theta.shape
    out = np.empty(D)
    _get().orc_eval_poly(p, D, _p(phi), _p(Theta), _p(out))
    return out


# ----------------------------------------------------------------------------
# the method's small host-side steps
# ----------------------------------------------------------------------------

def fold_offsets(n: int, k: int) -> list[int]:
    """Fold f holds rows [floor(f n / k), floor((f+1) n / k))."""
    return [(f * n) // k for f in range(k + 1)]


def trace_scale(X) -> float:
    """tau = tr(X^T X) / d = (sum of squares of all entries of X) / d."""
    X = _f64(X)
    s = 0.0
    for row in X:
        s += float(np.dot(row, row))
    return s / X.shape[1]


def lambda_grid(tau: float, q: int, lo: float, hi: float) -> np.ndarray:
    """lambda_t = tau * lo * (hi / lo)^(t / (q - 1)), t = 0..q-1 (log-spaced)."""
    if q == 1:
        return np.array([tau * lo])
    t = np.arange(q, dtype=np.float64)
    return tau * lo * (hi / lo) ** (t / (q - 1))


def sample_indices(q: int, g: int) -> list[int]:
    """g grid indices evenly spread over 0..q-1, both ends included,
    idx_i = round(i (q-1) / (g-1)) with halves rounded up."""
    if g == 1:
        return [0]
    return [(2 * i * (q - 1) + (g - 1)) // (2 * (g - 1)) for i in range(g)]


def basis_values(kind: str, lam, lam_s, p: int) -> np.ndarray:
    """Rows phi(lambda) = [phi_0 .. phi_{p-1}] for each lambda in ``lam``.

    mono     : phi_m = (lambda / max(lam_s))^m.  Dividing by the largest sampled
               lambda spans the same polynomial space as Algorithm 1's monomials
               and leaves the fitted function unchanged.
    cheb_log : phi_m = T_m(u), u = 2 (ln lambda - ln min lam_s) /
               (ln max lam_s - ln min lam_s) - 1, T_m the Chebyshev polynomials
               of the first kind (T_0 = 1, T_1 = u, T_{m+1} = 2 u T_m - T_{m-1}).
    """
    lam = np.atleast_1d(np.asarray(lam, dtype=np.float64))
    lam_s = np.asarray(lam_s, dtype=np.float64)
    out = np.empty((lam.size, p))
    if kind == BASIS_MONO:
        x = lam / lam_s.max()
        for m in range(p):
            out[:, m] = x ** m
    elif kind == BASIS_CHEB_LOG:
        a, b = np.log(lam_s.min()), np.log(lam_s.max())
        u = 2.0 * (np.log(lam) - a) / (b - a) - 1.0
        out[:, 0] = 1.0
        if p > 1:
            out[:, 1] = u
        for m in range(2, p):
            out[:, m] = 2.0 * u * out[:, m - 1] - out[:, m - 2]
    else:
        raise ValueError(f"unknown basis {kind!r}")
    return out


def basis_derivs(kind: str, lam, lam_s, p: int) -> np.ndarray:
    """d phi_m / d lambda at each lambda (for the hold-out gradient)."""
    lam = np.atleast_1d(np.asarray(lam, dtype=np.float64))
    lam_s = np.asarray(lam_s, dtype=np.float64)
    out = np.zeros((lam.size, p))
    if kind == BASIS_MONO:
        s = lam_s.max()
        x = lam / s
        for m in range(1, p):
            out[:, m] = m * x ** (m - 1) / s
    elif kind == BASIS_CHEB_LOG:
        a, b = np.log(lam_s.min()), np.log(lam_s.max())
        u = 2.0 * (np.log(lam) - a) / (b - a) - 1.0
        du = 2.0 / ((b - a) * lam)
        T = np.zeros((lam.size, p))
        dT = np.zeros((lam.size, p))
        T[:, 0] = 1.0
        if p > 1:
            T[:, 1] = u
            dT[:, 1] = 1.0
        for m in range(2, p):
            T[:, m] = 2.0 * u * T[:, m - 1] - T[:, m - 2]
            dT[:, m] = 2.0 * T[:, m - 1] + 2.0 * u * dT[:, m - 1] - dT[:, m - 2]
        out = dT * du[:, None]
    else:
        raise ValueError(f"unknown basis {kind!r}")
    return out


def diag_unusable(diag: np.ndarray) -> bool:
    """An interpolated factor whose diagonal has an entry <= 0, or one smaller
    than 1e3 * eps * max |diag|, does not define a usable solve; such a
    (fold, lambda) is scored +inf and left out of the argmin."""
    m = float(np.max(np.abs(diag))) if diag.size else 0.0
    thr = 1e3 * np.finfo(np.float64).eps * m
    return bool(np.any(diag <= 0.0) or np.any(np.abs(diag) <= thr))


def argmin_first(values: np.ndarray) -> int:
    """Index of the smallest finite value, ties to the smallest index; -1 if none."""
    best, best_t = np.inf, -1
    for t, v in enumerate(values):
        if np.isfinite(v) and v < best:
            best, best_t = v, t
    return best_t


def warm_fit(theta0, Vw, Tw, pw: int) -> np.ndarray:
    """Coefficients of a warm-started fold (the future work of Sec. 7, as read
    here): fold 0's coefficients plus the least-squares correction fitted to
    the residual of the warm fold's exact factors,
    Theta_f = Theta_0 + V'^+ (T'_f - V' Theta_0) on the first pw rows."""
    Theta = theta0.copy()
    Theta[:pw] += lstsq(Vw[:, :pw], Tw - Vw @ theta0)
    return Theta


def refine_exact_step(Hf, lam: float, Lt, Bf, W) -> np.ndarray:
    """One step of iterative refinement against the exact system, with the
    interpolated factor as the preconditioner (not in the paper):
    R = B_f - (H_f + lambda I) W, then W + (L~ L~^T)^{-1} R."""
    R = Bf - (Hf @ W + lam * W)
    return W + solve_factored(Lt, R)


# ----------------------------------------------------------------------------
# the full cross-validation
# ----------------------------------------------------------------------------

@dataclass
class CVResult:
    lam: np.ndarray                 # q lambda values
    sample_idx: list                # g grid indices that were factored exactly
    E: np.ndarray                   # k x q hold-out MSE
    Ebar: np.ndarray                # q, mean over folds
    t_star: int                     # argmin of Ebar
    unusable: np.ndarray            # k x q bool, interpolated diagonal unusable
    tau: float
    factors: dict = field(default_factory=dict)   # (f, s) -> L (keep=True)
    theta: dict = field(default_factory=dict)     # f -> Theta (p x D, row-wise vec)
    W: dict = field(default_factory=dict)         # (f, t) -> W (d x c)
    H: dict = field(default_factory=dict)         # f -> H_f
    B: dict = field(default_factory=dict)         # f -> B_f
    warm_idx: list = field(default_factory=list)  # grid indices of the warm-start samples


def cv(X, Y, *, k: int, g: int, r: int, q: int, lo: float = 1e-3, hi: float = 1e1,
       basis: str = BASIS_MONO, exact: bool = False, scale_by_trace: bool = True,
       folds=None, lam_idx=None, keep: bool = False, timings: dict | None = None,
       precond_steps: int = 0, warm: int = 0, lams=None, lam_samples=None, offsets=None) -> CVResult:
    """k-fold CV of ridge regression over q lambdas, piCholesky (default) or
    exact Cholesky at every lambda (``exact=True``, ``Chol`` of Sec. 6.2).

    ``precond_steps`` > 0 (piCholesky only; not in the paper) follows each
    interpolated solve with that many steps of iterative refinement against
    the exact system: R = B_f - (H_f + lambda I) W, W <- W + (L~ L~^T)^{-1} R,
    so the interpolated factor serves as a preconditioner.

    ``warm`` = g' (2 <= g' <= g; piCholesky only; the paper's future-work
    warm start, Sec. 7) fits fold 0 from its g sampled factors as above and
    every other fold f from g' exact factors only, at the grid indices
    round(i (q-1)/(g'-1)), starting from fold 0's coefficients:
    Theta_f = Theta_0 + V'^+ (T'_f - V' Theta_0), where V' holds the first
    p' = min(g', r+1) basis functions at those lambdas (the basis normalised
    by fold 0's samples) and the remaining rows of Theta_f are fold 0's.

    ``folds`` restricts the work to some folds and ``lam_idx`` to some grid
    indices (entries outside are NaN); the grid, the samples and the fit are
    unchanged by either.

    Caller choices (Sec. 3.3: the interpolant is evaluated at any lambda without
    a new factorisation; Sec. 1 leaves the fold split open): ``lams`` = the q
    evaluation lambdas (absolute values) in place of the grid; ``lam_samples``
    = the g sampled lambdas in place of the grid samples (they are the fit's
    nodes and set the basis normalisation); ``offsets`` = the k+1 row offsets
    of the folds in place of the floor split.  Not with ``warm``.  If ``timings`` is a dict, wall-clock seconds are
    added to its keys "setup" (grid scale), "fold" (per-fold Hessian, factors
    and fit) and "eval" (per-lambda work), and "n_eval" counts evaluations.
    """
    import time as _time
    tm = timings if timings is not None else {}
    for key in ("setup", "fold", "eval", "n_eval"):
        tm.setdefault(key, 0.0)
    _t0 = _time.perf_counter()
    X, Y = _f64(X), _f64(Y)
    n, d = X.shape
    c = Y.shape[1]
    p = r + 1
    if not exact and not (g > r):
        raise ValueError("piCholesky needs g > r sampled lambdas (Algorithm 1)")
    if warm and (exact or not (2 <= warm <= g)):
        raise ValueError("the warm start needs piCholesky and 2 <= warm <= g")
    if warm and (lams is not None or lam_samples is not None):
        raise ValueError("the warm start takes its samples from the grid")
    if offsets is None:
        offs = fold_offsets(n, k)
    else:
        offs = [int(o) for o in offsets]
        if len(offs) != k + 1 or offs[0] != 0 or offs[k] != n or any(b <= a for a, b in zip(offs, offs[1:])):
            raise ValueError("offsets must be k+1 increasing row offsets from 0 to n")
    tau = trace_scale(X) if scale_by_trace else 1.0
    if lams is None:
        lam = lambda_grid(tau, q, lo, hi)
    else:
        lam = np.asarray(lams, dtype=np.float64).reshape(-1).copy()
        if lam.shape[0] != q or not np.all(np.isfinite(lam)) or not np.all(lam > 0):
            raise ValueError("lams must be q finite positive values")
    sidx = sample_indices(q, g) if not exact else list(range(q))
    folds = list(range(k)) if folds is None else list(folds)
    tsel = list(range(q)) if lam_idx is None else list(lam_idx)
    tm["setup"] += _time.perf_counter() - _t0

    E = np.full((k, q), np.nan)
    bad = np.zeros((k, q), dtype=bool)
    res = CVResult(lam=lam, sample_idx=sidx, E=E, Ebar=None, t_star=-1, unusable=bad, tau=tau)
    theta0 = None
    if warm:
        # fold 0's coefficients start every other fold, whichever folds are asked for
        H0, _ = normal_blocks(X, Y, offs[0], offs[1])
        T0 = np.empty((g, d * (d + 1) // 2))
        for s_ in range(g):
            T0[s_] = vec_lower(cholesky(H0 + lam[sidx[s_]] * np.eye(d)))
        theta0 = lstsq(basis_values(basis, lam[sidx], lam[sidx], p), T0)
        widx = sample_indices(q, warm)
        pw = min(warm, p)
        Vw = basis_values(basis, lam[widx], lam[sidx], p)
        res.warm_idx = widx

    for f in folds:
        _tf = _time.perf_counter()
        r0, r1 = offs[f], offs[f + 1]
        nv = r1 - r0
        Hf, Bf = normal_blocks(X, Y, r0, r1)
        Xv, Yv = X[r0:r1], Y[r0:r1]
        if keep:
            res.H[f], res.B[f] = Hf, Bf
        if exact:
            tm["fold"] += _time.perf_counter() - _tf
            for t in tsel:
                _te = _time.perf_counter()
                L = cholesky(Hf + lam[t] * np.eye(d))
                W = solve_factored(L, Bf)
                E[f, t] = holdout_sse(Xv, Yv, W) / (nv * c)
                if keep:
                    res.W[(f, t)] = W
                tm["eval"] += _time.perf_counter() - _te
                tm["n_eval"] += 1
            continue
        if lam_samples is None:
            lam_s = lam[sidx]
        else:
            lam_s = np.asarray(lam_samples, dtype=np.float64).reshape(-1).copy()
            if lam_s.shape[0] != g or not np.all(np.isfinite(lam_s)) or not np.all(lam_s > 0):
                raise ValueError("lam_samples must be g finite positive values")
        if warm and f > 0:
            # warm start: g' exact factors, a degree-(p'-1) correction of fold 0's fit
            Tw = np.empty((warm, d * (d + 1) // 2))
            for s in range(warm):
                L = cholesky(Hf + lam[widx[s]] * np.eye(d))
                Tw[s] = vec_lower(L)
                if keep:
                    res.factors[(f, s)] = L
            Theta = warm_fit(theta0, Vw, Tw, pw)
        else:
            # Algorithm 1: exact factors at the samples, stacked as rows of T
            T = np.empty((g, d * (d + 1) // 2))
            for s in range(g):
                L = cholesky(Hf + lam_s[s] * np.eye(d))
                T[s] = vec_lower(L)
                if keep:
                    res.factors[(f, s)] = L
            # then the observation matrix and the least-squares coefficients
            V = basis_values(basis, lam_s, lam_s, p)
            Theta = lstsq(V, T)
        if keep:
            res.theta[f] = Theta
        # evaluation at every grid lambda, two triangular solves, hold-out error
        Phi = basis_values(basis, lam, lam_s, p)
        tm["fold"] += _time.perf_counter() - _tf
        for t in tsel:
            _te = _time.perf_counter()
            tm["n_eval"] += 1
            Lt = unvec_lower(eval_poly(Phi[t], Theta), d)
            if diag_unusable(np.diag(Lt)):
                bad[f, t] = True
                E[f, t] = np.inf
                tm["eval"] += _time.perf_counter() - _te
                continue
            W = solve_factored(Lt, Bf)
            for _ in range(precond_steps):
                W = refine_exact_step(Hf, lam[t], Lt, Bf, W)
            E[f, t] = holdout_sse(Xv, Yv, W) / (nv * c)
            if keep:
                res.W[(f, t)] = W
            tm["eval"] += _time.perf_counter() - _te
    if len(folds) == k:
        res.Ebar = E.mean(axis=0)
        res.t_star = argmin_first(res.Ebar)
    return res


# ----------------------------------------------------------------------------
# gradient of the mean hold-out error with respect to log(lambda)
# ----------------------------------------------------------------------------

@dataclass
class GradResult:
    E: np.ndarray        # k hold-out MSEs at lambda
    dE: np.ndarray       # k derivatives dE_f / d log(lambda)
    Ebar: float
    dEbar: float


def _holdout_and_grad(Xv, Yv, Bf, L, dL, lam):
    """E = ||Y_v - X_v W||^2 / (n_v c) with W = A^{-1} B_f, A = L L^T, and
    dE/dlog(lambda) = lambda dE/dlambda where dA/dlambda = dL L^T + L dL^T:
      dW = -A^{-1} (dA) W,   dE/dlambda = -(2 / (n_v c)) <X_v^T (Y_v - X_v W), dW>
    (chain rule on the definitions; no identity of the paper is needed)."""
    nv, c = Yv.shape
    W = solve_factored(L, Bf)
    R = Yv - Xv @ W
    E = float(np.sum(R * R)) / (nv * c)
    dA_W = dL @ (L.T @ W) + L @ (dL.T @ W)
    dW = -solve_factored(L, dA_W)
    dE = -2.0 / (nv * c) * float(np.sum((Xv.T @ R) * dW))
    return E, lam * dE


def holdout_grad(X, Y, *, k: int, g: int, r: int, q: int, log_lam: float, lo: float = 1e-3, hi: float = 1e1,
                 basis: str = BASIS_CHEB_LOG, exact: bool = False, scale_by_trace: bool = True,
                 folds=None) -> GradResult:
    """Hold-out MSE per fold at lambda = exp(log_lam) and its derivative with
    respect to log(lambda).  ``folds`` restricts the work to some folds (the
    others are NaN; Ebar and dEbar then average the computed folds only).

    exact=False: through the interpolated factor L(lambda) = sum_m phi_m(lambda)
    Theta_m of Algorithm 1 (sampled at the same grid indices as ``cv``), so
    dL/dlambda = sum_m phi_m'(lambda) Theta_m.
    exact=True: through the exact factor of H_f + lambda I, where
    dA/dlambda = I, so dW/dlambda = -A^{-1} W.
    """
    X, Y = _f64(X), _f64(Y)
    n, d = X.shape
    p = r + 1
    lam = float(np.exp(log_lam))
    offs = fold_offsets(n, k)
    tau = trace_scale(X) if scale_by_trace else 1.0
    grid = lambda_grid(tau, q, lo, hi)
    sidx = sample_indices(q, g)
    lam_s = grid[sidx]
    E = np.full(k, np.nan)
    dE = np.full(k, np.nan)
    for f in (range(k) if folds is None else folds):
        r0, r1 = offs[f], offs[f + 1]
        Hf, Bf = normal_blocks(X, Y, r0, r1)
        Xv, Yv = X[r0:r1], Y[r0:r1]
        nv, c = Yv.shape
        if exact:
            L = cholesky(Hf + lam * np.eye(d))
            W = solve_factored(L, Bf)
            R = Yv - Xv @ W
            E[f] = float(np.sum(R * R)) / (nv * c)
            dW = -solve_factored(L, W)                   # dA/dlambda = I
            dE[f] = lam * (-2.0 / (nv * c)) * float(np.sum((Xv.T @ R) * dW))
            continue
        T = np.empty((g, d * (d + 1) // 2))
        for s in range(g):
            T[s] = vec_lower(cholesky(Hf + lam_s[s] * np.eye(d)))
        Theta = lstsq(basis_values(basis, lam_s, lam_s, p), T)
        phi = basis_values(basis, [lam], lam_s, p)[0]
        dphi = basis_derivs(basis, [lam], lam_s, p)[0]
        L = unvec_lower(eval_poly(phi, Theta), d)
        dL = unvec_lower(eval_poly(dphi, Theta), d)
        E[f], dE[f] = _holdout_and_grad(Xv, Yv, Bf, L, dL, lam)
    return GradResult(E=E, dE=dE, Ebar=float(np.nanmean(E)), dEbar=float(np.nanmean(dE)))


# ----------------------------------------------------------------------------
# multi-level range narrowing (MChol, Sec. 6.2)
# ----------------------------------------------------------------------------

def holdout_exact_at(X, Y, *, k: int, lams, folds=None) -> np.ndarray:
    """k x m hold-out MSEs E[f, i] = ||Y_f - X_f W||^2 / (n_f c) with
    W = (H_f + lams[i] I)^{-1} B_f through the exact Cholesky factor, at any
    lambdas (not only grid points).  Folds outside ``folds`` are NaN."""
    X, Y = _f64(X), _f64(Y)
    n, d = X.shape
    lams = np.atleast_1d(np.asarray(lams, dtype=np.float64))
    offs = fold_offsets(n, k)
    E = np.full((k, lams.size), np.nan)
    for f in (range(k) if folds is None else folds):
        r0, r1 = offs[f], offs[f + 1]
        Hf, Bf = normal_blocks(X, Y, r0, r1)
        Xv, Yv = X[r0:r1], Y[r0:r1]
        for i, lam in enumerate(lams):
            W = solve_factored(cholesky(Hf + lam * np.eye(d)), Bf)
            E[f, i] = holdout_sse(Xv, Yv, W) / (Yv.shape[0] * Yv.shape[1])
    return E


def mchol_levels(s: float, s_min: float) -> int:
    """Number of levels the search runs: the three steps repeat, halving s
    each time, until s <= s_min (at least one level)."""
    if not (s > 0.0 and s_min > 0.0):
        raise ValueError("MChol needs s > 0 and s_min > 0")
    n = 0
    while True:
        n += 1
        s = s / 2.0
        if s <= s_min:
            return n


@dataclass
class MCholResult:
    lams: list          # per level: the three lambdas 10^(c-s), 10^c, 10^(c+s) (times tau)
    Ebar: list          # per level: their mean hold-out errors
    best: list          # per level: index 0..2 of the first smallest finite one, -1 if none
    c: float            # final centre (log10 of lambda / tau)
    s: float            # final half-width (decades)
    tau: float

    @property
    def window(self) -> tuple:
        """The final range [10^(c-s), 10^(c+s)], relative to tau."""
        return 10.0 ** (self.c - self.s), 10.0 ** (self.c + self.s)


def mchol_search(h, c: float, s: float, s_min: float, tau: float = 1.0) -> MCholResult:
    """The multi-level search of Sec. 6.2 over a hold-out function h that maps
    an array of lambdas to their mean hold-out errors:
      (a) evaluate h at lambda = tau 10^(c-s), tau 10^c, tau 10^(c+s);
      (b) lambda_opt = the first argmin of (a) over finite values;
      (c) c <- log10(lambda_opt / tau), s <- s / 2;
    repeated until s <= s_min.  tau = 1 is the paper's absolute range; a
    trace scale makes c relative, as for the grid of ``cv``.  If no value of a
    level is finite, c is kept."""
    res = MCholResult(lams=[], Ebar=[], best=[], c=c, s=s, tau=tau)
    for _ in range(mchol_levels(s, s_min)):
        lams = tau * 10.0 ** np.array([c - s, c, c + s])
        Ebar = np.asarray(h(lams), dtype=np.float64)
        best = argmin_first(Ebar)
        if best >= 0:
            c = float(np.log10(lams[best] / tau))
        s = s / 2.0
        res.lams.append(lams)
        res.Ebar.append(Ebar)
        res.best.append(best)
    res.c, res.s = c, s
    return res


def mchol(X, Y, *, k: int, c: float, s: float, s_min: float, scale_by_trace: bool = True) -> MCholResult:
    """MChol of Sec. 6.2 on k-fold cross-validation: the search of
    ``mchol_search`` with h = the mean over folds of the exact hold-out MSE
    (``holdout_exact_at``).  With scale_by_trace the range is relative to
    tau = tr(X^T X) / d, like the grid of ``cv``; piCholesky then searches
    the final window by ``cv(..., lo=window[0], hi=window[1])``."""
    tau = trace_scale(X) if scale_by_trace else 1.0
    return mchol_search(lambda lams: holdout_exact_at(X, Y, k=k, lams=lams).mean(axis=0), c, s, s_min, tau)


# ----------------------------------------------------------------------------
# PINRMSE: interpolating the sampled hold-out errors directly
# ----------------------------------------------------------------------------

def pinrmse(X, Y, *, k: int, g: int, r: int, q: int, lo: float = 1e-3, hi: float = 1e1,
            basis: str = BASIS_MONO, scale_by_trace: bool = True, folds=None) -> CVResult:
    """PINRMSE, the comparator of the paper's supplementary section: Algorithm
    1 with the g x D target matrix T replaced by the g x 1 vector t_f of exact
    hold-out errors at the sampled lambdas, so the fitted polynomial is the
    hold-out error itself: theta_f = argmin ||t_f - V theta||, then
    E[f, t] = phi(lambda_t) . theta_f on the whole grid.  Same grid, samples
    and basis as ``cv``.  A fold with a non-finite sampled error scores +inf
    everywhere."""
    X, Y = _f64(X), _f64(Y)
    n, d = X.shape
    p = r + 1
    if not (g > r):
        raise ValueError("PINRMSE needs g > r sampled lambdas (Algorithm 1)")
    tau = trace_scale(X) if scale_by_trace else 1.0
    lam = lambda_grid(tau, q, lo, hi)
    sidx = sample_indices(q, g)
    lam_s = lam[sidx]
    V = basis_values(basis, lam_s, lam_s, p)
    Phi = basis_values(basis, lam, lam_s, p)
    folds = list(range(k)) if folds is None else list(folds)
    t = holdout_exact_at(X, Y, k=k, lams=lam_s, folds=folds)          # k x g
    E = np.full((k, q), np.nan)
    for f in folds:
        if not np.all(np.isfinite(t[f])):
            E[f] = np.inf
            continue
        theta = lstsq(V, t[f][:, None])[:, 0]
        E[f] = Phi @ theta
    res = CVResult(lam=lam, sample_idx=sidx, E=E, Ebar=None, t_star=-1,
                   unusable=np.zeros((k, q), dtype=bool), tau=tau)
    if len(folds) == k:
        res.Ebar = E.mean(axis=0)
        res.t_star = argmin_first(res.Ebar)
    return res


# ----------------------------------------------------------------------------
# NRMSE of the fit (the paper's Sec. 6.6 diagnostic)
# ----------------------------------------------------------------------------

def nrmse_curve(X, Y, *, k: int, g: int, r: int, q: int, lo: float = 1e-3, hi: float = 1e1,
                basis: str = BASIS_MONO, scale_by_trace: bool = True, fold: int = 0) -> np.ndarray:
    """NRMSE of Algorithm 1's fit at every grid lambda of one fold (Sec. 6.6):
    the root mean squared difference between the interpolated and the exact
    factor entries (the D lower-triangular entries), divided by the root mean
    squared deviation of the exact entries from their mean, so that predicting
    the mean scores 1."""
    res = cv(X, Y, k=k, g=g, r=r, q=q, lo=lo, hi=hi, basis=basis, scale_by_trace=scale_by_trace,
             folds=[fold], lam_idx=[], keep=True)
    d = _f64(X).shape[1]
    Hf = normal_blocks(X, Y, fold_offsets(_f64(X).shape[0], k)[fold], fold_offsets(_f64(X).shape[0], k)[fold + 1])[0]
    lam_s = res.lam[res.sample_idx]
    Phi = basis_values(basis, res.lam, lam_s, r + 1)
    out = np.empty(q)
    for t in range(q):
        target = vec_lower(cholesky(Hf + res.lam[t] * np.eye(d)))
        pred = eval_poly(Phi[t], res.theta[fold])
        out[t] = nrmse(pred, target)
    return out


def nrmse(pred, target) -> float:
    """Root mean squared error of ``pred`` over the root mean squared deviation
    of ``target`` from its mean (Sec. 6.6's normalisation: the mean scores 1)."""
    pred, target = _f64(pred), _f64(target)
    return float(np.sqrt(np.mean((pred - target) ** 2)) / np.sqrt(np.mean((target - target.mean()) ** 2)))
