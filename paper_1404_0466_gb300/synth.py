"""Seeded synthetic inputs for ridge cross-validation workloads.

This module only draws data.  It holds none of the method's arithmetic (no
Gram matrix, factorisation, fit or solve) and imports nothing from the CUDA
library or the oracle, so both can be fed the same arrays from it.

The paper's datasets (MNIST, COIL-100, Caltech-101/256 projected to
h = 1024..16384 features, Sec. 6.1) are not available; these generators stand
in for them with the shapes and spectra of the workloads used here.  Every
generator uses NumPy's PCG64 with an explicit seed.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Problem:
    X: np.ndarray          # n x d design matrix, row-major
    Y: np.ndarray          # n x c targets, row-major
    name: str
    seed: int


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def haar_orthogonal(rng: np.random.Generator, d: int) -> np.ndarray:
    """Haar-random orthogonal d x d matrix: QR of a Gaussian matrix with the
    signs of R's diagonal moved into Q."""
    G = rng.standard_normal((d, d))
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))


def spectral_gaussian(n: int, d: int, c: int, *, seed: int, decay: float = 1.0,
                      noise: float = 0.1, dtype=np.float64, name: str = "") -> Problem:
    """Rows x ~ N(0, Sigma), Sigma = Q diag(i^-decay) Q^T with Q Haar-orthogonal;
    Y = X W* + noise * N(0, 1), W* ~ N(0, 1) (d x c)."""
    rng = _rng(seed)
    Q = haar_orthogonal(rng, d)
    ev = np.arange(1, d + 1, dtype=np.float64) ** (-decay)
    Z = rng.standard_normal((n, d))
    X = (Z * np.sqrt(ev)) @ Q.T
    Wstar = rng.standard_normal((d, c))
    Y = X @ Wstar + noise * rng.standard_normal((n, c))
    return Problem(np.ascontiguousarray(X, dtype=dtype), np.ascontiguousarray(Y, dtype=dtype),
                   name or f"spectral_gaussian_n{n}_d{d}_c{c}", seed)


def ecc_codebook(rng: np.random.Generator, classes: int, bits: int) -> np.ndarray:
    """Random +-1 code words (classes x bits) with no two rows equal: whole
    codebooks are drawn until one has distinct rows, and after 1000 draws (a
    codebook that nearly fills the 2^bits words) distinct words are drawn
    without replacement instead."""
    if classes > 2 ** bits:
        raise ValueError("not enough bits for distinct code words")
    for _ in range(1000):
        C = rng.choice(np.array([-1.0, 1.0]), size=(classes, bits))
        if len({tuple(row) for row in C}) == classes:
            return C
    words = rng.choice(2 ** bits, size=classes, replace=False)
    return np.where((words[:, None] >> np.arange(bits)) & 1, 1.0, -1.0)


def mixture_ecc(n: int, d: int, c: int = 10, *, seed: int, clusters: int = 10,
                mean_scale: float = 3.0, dtype=np.float32, name: str = "") -> Problem:
    """Gaussian-mixture features with error-correcting-code targets.

    Cluster means mu_j ~ N(0, (mean_scale^2 / d) I), so ||mu_j|| is about
    mean_scale; each row draws a cluster uniformly and adds N(0, I) noise.
    Each cluster has a distinct random +-1 code word of c bits, which is the
    row's target (multi-output regression onto codes, Sec. 1 item c).
    """
    rng = _rng(seed)
    means = rng.standard_normal((clusters, d)) * (mean_scale / np.sqrt(d))
    code = ecc_codebook(rng, clusters, c)
    labels = rng.integers(0, clusters, size=n)
    X = np.empty((n, d), dtype=dtype)
    step = 4096
    for r0 in range(0, n, step):
        r1 = min(n, r0 + step)
        X[r0:r1] = means[labels[r0:r1]] + rng.standard_normal((r1 - r0, d))
    Y = code[labels].astype(dtype)
    return Problem(X, np.ascontiguousarray(Y), name or f"mixture_ecc_n{n}_d{d}_c{c}", seed)


def random_fourier(n: int, d: int, c: int, *, seed: int, in_dim: int = 64, gamma: float = 64.0,
                   noise: float = 0.1, dtype=np.float32, name: str = "") -> Problem:
    """Random-Fourier features Phi = sqrt(2/d) cos(Z omega + b) of 64-dim
    Gaussian inputs Z, omega ~ N(0, I / gamma), b ~ U[0, 2 pi);
    Y = Phi W* + noise * N(0, 1), W* ~ N(0, 1) / sqrt(d)."""
    rng = _rng(seed)
    omega = rng.standard_normal((in_dim, d)) / np.sqrt(gamma)
    b = rng.uniform(0.0, 2.0 * np.pi, size=d)
    Wstar = rng.standard_normal((d, c)) / np.sqrt(d)
    X = np.empty((n, d), dtype=dtype)
    Y = np.empty((n, c), dtype=dtype)
    step = 2048
    for r0 in range(0, n, step):
        r1 = min(n, r0 + step)
        Z = rng.standard_normal((r1 - r0, in_dim))
        Phi = np.sqrt(2.0 / d) * np.cos(Z @ omega + b)
        X[r0:r1] = Phi
        Y[r0:r1] = Phi @ Wstar + noise * rng.standard_normal((r1 - r0, c))
    return Problem(X, Y, name or f"rff_n{n}_d{d}_c{c}", seed)


# ---------------------------------------------------------------------------
# the named workloads
# ---------------------------------------------------------------------------

# Small FP64 case: n = 2048, d = 256, Sigma eigenvalues i^-1, c = 10,
# k = 5, g = 4, r = 2, q = 31, lambda in [1e-3, 1e1] * tr(H)/d, seed 0.
FP64_SMALL = dict(n=2048, d=256, c=10, k=5, g=4, r=2, q=31, lo=1e-3, hi=1e1, seed=0)
# Mixed-precision case: n = 32768, d = 2048, 10-cluster mixture, c = 10 ECC
# targets, k = 5, g = 6, r = 3, q = 101.
MIXED_ECC = dict(n=32768, d=2048, c=10, k=5, g=6, r=3, q=101, lo=1e-3, hi=1e1, seed=1)
# Large single problem: n = 131072, d = 8192 random-Fourier features, c = 32.
LARGE_RFF = dict(n=131072, d=8192, c=32, k=5, g=6, r=3, q=101, lo=1e-3, hi=1e1, seed=2)
# Differentiation case: n = 16384, d = 1024, c = 10, Sigma eigenvalues i^-1,
# k = 5, g = 5, r = 3, fp32 data; lambda window [0.02, 0.5] tr(H)/d (q only
# fixes where the g samples sit).
DIFFERENTIATION = dict(n=16384, d=1024, c=10, k=5, g=5, r=3, q=51, lo=0.02, hi=0.5, seed=4)


def fp64_small(**over) -> Problem:
    cfg = {**FP64_SMALL, **over}
    return spectral_gaussian(cfg["n"], cfg["d"], cfg["c"], seed=cfg["seed"], decay=1.0,
                             dtype=np.float64, name="fp64_small")


def mixed_ecc(**over) -> Problem:
    cfg = {**MIXED_ECC, **over}
    return mixture_ecc(cfg["n"], cfg["d"], cfg["c"], seed=cfg["seed"], dtype=np.float32,
                       name="mixed_ecc")


def large_rff(**over) -> Problem:
    cfg = {**LARGE_RFF, **over}
    return random_fourier(cfg["n"], cfg["d"], cfg["c"], seed=cfg["seed"], name="large_rff")


def differentiation(**over) -> Problem:
    cfg = {**DIFFERENTIATION, **over}
    return spectral_gaussian(cfg["n"], cfg["d"], cfg["c"], seed=cfg["seed"], decay=1.0, dtype=np.float32,
                             name="differentiation")


def batched_uneven(count: int = 64, *, seed: int = 3, d_lo: int = 128, d_hi: int = 1536,
                   dtype=np.float64) -> list[Problem]:
    """``count`` independent problems, d ~ U[d_lo, d_hi], n = 8 d, c alternating
    1 and 10, Sigma eigenvalues i^-1.5."""
    rng = _rng(seed)
    ds = rng.integers(d_lo, d_hi + 1, size=count)
    out = []
    for i, d in enumerate(ds):
        c = 1 if i % 2 == 0 else 10
        out.append(spectral_gaussian(int(8 * d), int(d), c, seed=seed * 1000 + i, decay=1.5,
                                     dtype=dtype, name=f"batched_{i}"))
    return out
