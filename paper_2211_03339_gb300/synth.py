"""Seeded synthetic inputs shaped like the paper's experiments (Sec. 6).

This module only draws random inputs; it holds none of the method's
arithmetic.  Both the CUDA-path tests and the oracle tests take their inputs
from here, so the two sides always see identical matrices.

The paper builds its matrices with MATLAB's ``gallery('randsvd', ...)`` and
``orth(randn(n))`` (Examples 1-3).  Those random streams are not reproducible
here, so the matrices below are stand-ins with the same structure:

* ``A = Q diag(lam) Q^T`` with a Haar-distributed orthogonal ``Q`` (QR of a
  standard Gaussian matrix, columns signed so that ``diag(R) > 0``), made
  exactly symmetric by ``(A + A^T)/2``;
* spectra: ``uniform`` in [-1, 1]; ``gapped`` (uniform in [-1, 1], one eigenvalue per
  stratum of width 2/n, so the minimum gap is at least 0.8/n); ``geometric`` with ``|lam_i| =
  10^(-8 (i-1)/(n-1))`` and random signs; ``cluster``: 10 centres in
  ``linspace(-0.9, 0.9, 10)``, members uniform in ``centre +- 5e-7``;
  and the Example 1 modes 3/4/5 (geometric, arithmetic, log-uniform with
  condition number kappa, positive definite);
* ``A = U diag(sigma) V^T`` (m x n) with Haar ``U`` (m x n) and ``V``
  (n x n) and ``sigma`` geometric from 1 to ``sigma_min`` (Example 3).

Seeds follow ``seed = 1000 * config_id + matrix_index``.
"""
from __future__ import annotations

import numpy as np

SPECTRA = ("uniform", "geometric", "cluster", "mode3", "mode4", "mode5", "gapped")


def seed_for(config_id: int, index: int) -> int:
    return 1000 * int(config_id) + int(index)


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def haar(rng: np.random.Generator, m: int, n: int | None = None) -> np.ndarray:
    """m x n matrix with orthonormal columns, Haar distributed (n <= m)."""
    n = m if n is None else n
    G = rng.standard_normal((m, n))
    Q, R = np.linalg.qr(G)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return np.asfortranarray(Q * d[None, :])


def spectrum(kind: str, n: int, rng: np.random.Generator, kappa: float = 1e6) -> np.ndarray:
    if kind == "uniform":
        lam = rng.uniform(-1.0, 1.0, n)
    elif kind == "geometric":
        e = np.arange(n) / max(n - 1, 1)
        lam = 10.0 ** (-8.0 * e) * rng.choice([-1.0, 1.0], n)
    elif kind == "cluster":
        centres = np.linspace(-0.9, 0.9, 10)
        per = -(-n // 10)
        lam = np.concatenate([c + rng.uniform(-5e-7, 5e-7, per) for c in centres])[:n]
    elif kind == "gapped":     # uniform in [-1, 1], stratified: min gap >= 0.4 * 2/n (>= 1e-3 for n <= 800)
        h = 2.0 / n
        lam = -1.0 + h * (np.arange(n) + 0.5 + rng.uniform(-0.3, 0.3, n))
    elif kind == "mode3":      # geometric, lam_1 = 1 ... lam_n = 1/kappa
        e = np.arange(n) / max(n - 1, 1)
        lam = kappa ** (-e)
    elif kind == "mode4":      # arithmetic
        e = np.arange(n) / max(n - 1, 1)
        lam = 1.0 - (1.0 - 1.0 / kappa) * e
    elif kind == "mode5":      # log-uniform random
        lam = np.exp(rng.uniform(-np.log(kappa), 0.0, n))
    else:
        raise ValueError(f"unknown spectrum {kind!r}")
    return np.asarray(lam, dtype=np.float64)


def multiple_spectrum(s: int, r: int, mode: int, kappa: float, rng: np.random.Generator) -> np.ndarray:
    """Example 2: lam (length s) repeated r times (lam kron 1_r), modes 1-5.

    Modes 1, 2 and 4 follow the stated formulas.  The printed modes 3 and 5
    (kappa .* linspace(-1, 0, s) and kappa .* (-rand(s, 1))) would give a
    non-positive-definite A, contradicting the example's own statement; they are
    read as kappa .^ linspace(-1, 0, s) and kappa .^ (-rand(s, 1)) (geometric and
    log-uniform in [1/kappa, 1])."""
    if mode == 1:
        lam = np.concatenate([[1.0], np.ones(s - 1) / kappa])
    elif mode == 2:
        lam = np.concatenate([np.ones(s - 1), [1.0 / kappa]])
    elif mode == 3:
        lam = kappa ** np.linspace(-1.0, 0.0, s)
    elif mode == 4:
        lam = 1.0 - (1.0 - 1.0 / kappa) * np.linspace(0.0, 1.0, s)
    elif mode == 5:
        lam = kappa ** (-rng.uniform(0.0, 1.0, s))
    else:
        raise ValueError("mode must be 1..5")
    return np.kron(lam, np.ones(r))


def sym_matrix_multiple(r: int, s: int, mode: int, kappa: float = 1e4, seed: int = 0):
    """Example 2 stand-in: A = P diag(lam kron 1_r) P^T, n = r s, Haar P."""
    rng = rng_for(seed)
    lam = multiple_spectrum(s, r, mode, kappa, rng)
    P = haar(rng, r * s)
    A = (P * lam[None, :]) @ P.T
    A = 0.5 * (A + A.T)
    return np.asfortranarray(A), np.sort(lam)


def sym_matrix(n: int, kind: str = "uniform", seed: int = 0, kappa: float = 1e6):
    """Return (A, lam_sorted_ascending) with A = Q diag(lam) Q^T, column-major."""
    rng = rng_for(seed)
    lam = spectrum(kind, n, rng, kappa)
    Q = haar(rng, n)
    A = (Q * lam[None, :]) @ Q.T
    A = 0.5 * (A + A.T)
    return np.asfortranarray(A), np.sort(lam)


def svd_matrix(m: int, n: int, seed: int = 0, sigma_min: float = 1e-10):
    """Return (A, sigma_desc, U, V) with A = U diag(sigma) V^T (m >= n)."""
    rng = rng_for(seed)
    e = np.arange(n) / max(n - 1, 1)
    sigma = sigma_min ** e
    U = haar(rng, m, n)
    V = haar(rng, n)
    A = (U * sigma[None, :]) @ V.T
    return np.asfortranarray(A), sigma, U, V


def graded_matrix(m: int, n: int, seed: int = 0, decades: float = 12.0):
    """A = B D column-major: B m x n Gaussian (well conditioned for m well above n),
    D diagonal with entries 10^(-decades * k / (n - 1)) in a random column order."""
    rng = rng_for(seed)
    B = rng.standard_normal((m, n))
    d = 10.0 ** (-decades * np.arange(n) / max(n - 1, 1))
    return np.asfortranarray(B * rng.permutation(d)[None, :])


def batch_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Sizes n_i uniform in [lo, hi] for a batched workload."""
    return rng_for(seed).integers(lo, hi + 1, size=count)
