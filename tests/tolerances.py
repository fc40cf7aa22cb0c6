"""Tolerances of the GPU parity tests.

MIXED_RTOL is the mixed-precision bar the method is held to: a hold-out error
within 1e-4 relative of the FP64 oracle's, for every (fold, lambda) of every
workload.  fp32_forward_bound is a diagnostic only (printed beside failures,
never a pass criterion): the fp32 forward-error scale 16 kappa 2^-24 of
H_f + lambda I."""
import numpy as np

import oracle

U32 = 2.0 ** -24
MIXED_RTOL = 1e-4


def fp32_forward_bound(X, lam, k, folds=None):
    """Per (fold, lambda): 16 kappa u32 with kappa = (mu_max + lambda) /
    (mu_min + lambda), mu the eigenvalues of H_f.  Rows of folds not listed
    are NaN."""
    n = X.shape[0]
    offs = oracle.fold_offsets(n, k)
    out = np.full((k, len(lam)), np.nan)
    for f in (range(k) if folds is None else folds):
        keep = np.r_[0:offs[f], offs[f + 1]:n]
        Xk = X[keep].astype(np.float64)
        mu = np.linalg.eigvalsh(Xk.T @ Xk)
        out[f] = 16 * (mu.max() + lam) / (max(mu.min(), 0.0) + lam) * U32
    return out


def same_choice(Ebar_ref, t_gpu, t_ref, rtol=MIXED_RTOL):
    """The selected lambda is the oracle's, or the oracle's mean errors at the
    two indices differ by less than the tolerance (either is then a minimum
    within the stated accuracy)."""
    if t_gpu == t_ref:
        return True
    return t_gpu >= 0 and Ebar_ref[t_gpu] <= Ebar_ref[t_ref] * (1 + rtol)
