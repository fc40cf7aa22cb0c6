"""The seeded generators draw what the input recipe states: shapes, dtypes,
seeds, spectra, code words, feature maps and the uneven batch.  Statistical
checks use enough rows that their tolerances are several standard errors."""
import numpy as np
import pytest

from paper_1404_0466_gb300 import synth


def test_haar_orthogonal_is_orthogonal():
    Q = synth.haar_orthogonal(np.random.default_rng(0), 40)
    np.testing.assert_allclose(Q.T @ Q, np.eye(40), atol=1e-13)


def test_spectral_gaussian_covariance_and_noise():
    n, d, c = 40000, 6, 2
    p = synth.spectral_gaussian(n, d, c, seed=5, decay=1.5)
    assert p.X.shape == (n, d) and p.Y.shape == (n, c) and p.X.dtype == np.float64
    ev = np.sort(np.linalg.eigvalsh(p.X.T @ p.X / n))[::-1]
    np.testing.assert_allclose(ev, np.arange(1, d + 1) ** -1.5, rtol=0.05)
    # Y = X W* + 0.1 N(0, 1): the least-squares residual has standard deviation 0.1
    W = np.linalg.lstsq(p.X, p.Y, rcond=None)[0]
    assert abs(np.std(p.Y - p.X @ W) - 0.1) < 0.005


def test_generators_are_seeded():
    a = synth.spectral_gaussian(50, 7, 2, seed=3)
    b = synth.spectral_gaussian(50, 7, 2, seed=3)
    c = synth.spectral_gaussian(50, 7, 2, seed=4)
    assert np.array_equal(a.X, b.X) and np.array_equal(a.Y, b.Y)
    assert not np.array_equal(a.X, c.X)
    m1, m2 = synth.mixture_ecc(300, 16, seed=9), synth.mixture_ecc(300, 16, seed=9)
    assert np.array_equal(m1.X, m2.X) and np.array_equal(m1.Y, m2.Y)


def test_ecc_codebook():
    C = synth.ecc_codebook(np.random.default_rng(1), 10, 10)
    assert C.shape == (10, 10) and set(np.unique(C)) == {-1.0, 1.0}
    assert len({tuple(r) for r in C}) == 10
    C = synth.ecc_codebook(np.random.default_rng(2), 4, 2)     # every code word of 2 bits
    assert len({tuple(r) for r in C}) == 4
    with pytest.raises(ValueError):
        synth.ecc_codebook(np.random.default_rng(3), 5, 2)
    C = synth.ecc_codebook(np.random.default_rng(4), 16, 4)    # all 16 words: drawn without replacement
    assert len({tuple(r) for r in C}) == 16 and set(np.unique(C)) == {-1.0, 1.0}


def test_mixture_ecc_targets_and_clusters():
    n, d = 20000, 32
    p = synth.mixture_ecc(n, d, 10, seed=11)
    assert p.X.dtype == np.float32 and p.Y.dtype == np.float32 and p.Y.shape == (n, 10)
    words, labels = np.unique(p.Y, axis=0, return_inverse=True)
    labels = labels.ravel()
    assert len(words) == 10 and set(np.unique(p.Y)) == {-1.0, 1.0}
    counts = np.bincount(labels, minlength=10)
    assert counts.min() > 0.8 * n / 10 and counts.max() < 1.2 * n / 10     # uniform labels
    # unit within-cluster covariance; means of norm about mean_scale = 3
    X = p.X.astype(np.float64)
    means = np.stack([X[labels == j].mean(axis=0) for j in range(10)])
    within = X - means[labels]
    assert abs(within.var() - 1.0) < 0.02
    assert 2.0 < np.median(np.linalg.norm(means, axis=1)) < 4.0


def test_random_fourier_features():
    n, d, c = 8192, 256, 4
    p = synth.random_fourier(n, d, c, seed=2)
    assert p.X.dtype == np.float32 and p.X.shape == (n, d) and p.Y.shape == (n, c)
    assert np.abs(p.X).max() <= np.sqrt(2.0 / d) * (1 + 1e-6)
    # E[(2/d) cos^2(.)] = 1/d with b uniform, so the mean squared entry is 1/d
    assert abs(np.mean(p.X.astype(np.float64) ** 2) * d - 1.0) < 0.02


def test_batched_uneven_recipe():
    probs = synth.batched_uneven(16, seed=3)
    assert len(probs) == 16
    for i, p in enumerate(probs):
        n, d = p.X.shape
        assert 128 <= d <= 1536 and n == 8 * d
        assert p.Y.shape[1] == (1 if i % 2 == 0 else 10)
        assert p.X.dtype == np.float64


def test_named_workloads():
    assert synth.FP64_SMALL["n"] == 2048 and synth.FP64_SMALL["d"] == 256 and synth.FP64_SMALL["q"] == 31
    assert (synth.MIXED_ECC["n"], synth.MIXED_ECC["d"], synth.MIXED_ECC["c"]) == (32768, 2048, 10)
    assert (synth.LARGE_RFF["n"], synth.LARGE_RFF["d"], synth.LARGE_RFF["c"]) == (131072, 8192, 32)
    assert (synth.DIFFERENTIATION["n"], synth.DIFFERENTIATION["d"]) == (16384, 1024)
    p = synth.fp64_small(n=64, d=16)
    assert p.X.shape == (64, 16) and p.X.dtype == np.float64 and p.seed == 0
    p = synth.mixed_ecc(n=64, d=16)
    assert p.X.dtype == np.float32 and p.Y.shape == (64, 10) and p.seed == 1
