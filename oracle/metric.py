"""Local distance and Euclidean map of the DD method (FP64 oracle).

Eq. (3):  d_e^2(y, z) = C (eps - eps') . (eps - eps') + C^{-1} (sig - sig') . (sig - sig')
Sec. 3.2 (k-d tree search): the search runs on mapped coordinates
          q = (C^{1/2} eps, C^{-1/2} sig),
          here scaled by 1/sqrt(2) so that |q - q'|^2 = 1/2 d_e^2, the summand of
          the global distance Eq. (2) up to the weight w_e.

Pinned by tests/test_oracle_metric.py (closed-form spectrum of the isotropic
metric, C^{1/2} C^{1/2} = C, |dq|^2 = d_e^2 / 2 against the direct Eq. (3)).
"""
from __future__ import annotations

import numpy as np


def metric_roots(C: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Symmetric square root C^{1/2} and its inverse C^{-1/2} of the SPD
    metric, from the eigen-decomposition C = V diag(w) V^T."""
    C = np.asarray(C, dtype=np.float64)
    if not np.allclose(C, C.T, rtol=0, atol=1e-14 * np.abs(C).max()):
        raise ValueError("metric must be symmetric")
    w, V = np.linalg.eigh(C)
    if w.min() <= 0.0:
        raise ValueError("metric must be positive definite")
    r = np.sqrt(w)
    return (V * r) @ V.T, (V / r) @ V.T


def to_z(states: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Map states (eps, sig) [n, 12] to q = (C^{1/2} eps, C^{-1/2} sig)/sqrt(2)."""
    s = np.asarray(states, dtype=np.float64)
    Ch, Cmh = metric_roots(C)
    z = np.empty_like(s)
    z[:, :6] = s[:, :6] @ Ch.T
    z[:, 6:] = s[:, 6:] @ Cmh.T
    return z / np.sqrt(2.0)


def local_d2(y: np.ndarray, z: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Eq. (3) for paired rows of y and z, both (eps, sig) [n, 12]."""
    y = np.asarray(y, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    de = y[:, :6] - z[:, :6]
    ds = y[:, 6:] - z[:, 6:]
    Cinv = np.linalg.inv(C)
    return np.einsum("ni,ij,nj->n", de, C, de) + np.einsum("ni,ij,nj->n", ds, Cinv, ds)


def pca_metric(data: np.ndarray) -> np.ndarray:
    """The data-derived metric of Sec. 3.1: the 6 principal component vectors
    of the 12-d data (eigenvectors of its covariance with the 6 largest
    eigenvalues) are the columns of A (12 x 6); with A_eps its upper and
    A_sig its lower 6 x 6 block, C = sym(A_sig A_eps^{-1}).

    Reading: the paper writes sym(A_eps^{-1} A_sig); with the components as
    the *rows* of A that is the same matrix, and it is the one that returns C
    itself for data on a linear law sig = C eps (the columns of A span
    {(x, C x)}, so A_sig = C A_eps).  The covariance is taken about the mean.
    """
    d = np.asarray(data, dtype=np.float64)
    X = d - d.mean(axis=0)
    S = X.T @ X / len(d)
    w, V = np.linalg.eigh(S)
    A = V[:, np.argsort(w)[::-1][:6]]
    Ae, As = A[:6], A[6:]
    M = np.linalg.solve(Ae.T, As.T).T           # A_sig A_eps^{-1}
    return 0.5 * (M + M.T)
