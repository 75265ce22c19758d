"""Test-side helpers: minimum-image geometry computed directly from global
coordinates (independent of both the oracle's and the library's cell frames)."""
import numpy as np

FX = 16777216  # 2^24


def min_image_d2(xy, L):
    """All-pairs squared minimum-image distances (float64), diagonal = inf."""
    d = xy[:, None, :] - xy[None, :, :]
    d -= L * np.round(d / L)
    r2 = (d * d).sum(-1)
    np.fill_diagonal(r2, np.inf)
    return r2


def to_fixed(xy):
    """Global positions of the fixed-point form are exact multiples of 2^-24."""
    X = np.round(np.asarray(xy) * FX).astype(np.int64)
    assert np.array_equal(X.astype(np.float64) / FX, np.asarray(xy))
    return X


def min_image_d2_fixed(X, LF):
    """Exact all-pairs squared distances in (2^-24 sigma)^2 units (int64)."""
    d = X[:, None, :] - X[None, :, :]
    d = (d + LF // 2) % LF - LF // 2
    r2 = (d * d).sum(-1)
    np.fill_diagonal(r2, np.iinfo(np.int64).max)
    return r2


def batch_se(samples, nbatch=20):
    """Mean and batch-means standard error of a correlated series."""
    s = np.asarray(samples, dtype=np.float64)
    n = (len(s) // nbatch) * nbatch
    b = s[:n].reshape(nbatch, -1).mean(axis=1)
    return float(s.mean()), float(b.std(ddof=1) / np.sqrt(nbatch))
