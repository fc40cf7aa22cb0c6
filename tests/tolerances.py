"""Tolerances derived from the arithmetic, shared by the GPU parity tests."""
import numpy as np

import oracle

U32 = 2.0 ** -24


def mixed_tolerance(X, lam, k, folds=None):
    """Per (fold, lambda) relative tolerance of a mixed-mode hold-out error:
    1e-4, or the fp32 forward-error scale 16 kappa u32 where
    kappa = (mu_max + lambda) / (mu_min + lambda) is the condition number of
    H_f + lambda I (mu = eigenvalues of H_f), whichever is larger.  Rows of
    folds not listed are NaN."""
    n = X.shape[0]
    offs = oracle.fold_offsets(n, k)
    tol = np.full((k, len(lam)), np.nan)
    for f in (range(k) if folds is None else folds):
        keep = np.r_[0:offs[f], offs[f + 1]:n]
        Xk = X[keep].astype(np.float64)
        mu = np.linalg.eigvalsh(Xk.T @ Xk)
        kappa = (mu.max() + lam) / (max(mu.min(), 0.0) + lam)
        tol[f] = np.maximum(1e-4, 16 * kappa * U32)
    return tol
