"""Leverage scores and ridge leverage scores (Sec. 2, Sec. 4.1 Lemma 4.1, Sec. 4.2).

Oracle module: test infrastructure.  Only tests/, __graft_entry__.smoke() and
bench.py's cpu_baseline / reference leg may import anything under oracle/.
Plain FP64 numpy; every function is a definition of the paper written out.
"""
from __future__ import annotations

import numpy as np


def pinv_tol(n_rows: int, n_cols: int) -> float:
    """Relative eigenvalue cutoff for the pseudo-inverse of a Gram A^T A.

    The paper leaves the tolerance of "+" open (Eq. ridge_leverage_score_def);
    eigenvalues below max(I, R) * eps64 * lambda_max count as zero.
    """
    return max(int(n_rows), int(n_cols)) * np.finfo(np.float64).eps


def gram_pinv(A: np.ndarray, lam: float = 0.0):
    """(A^T A + lam I)^+ and the numerical rank of A^T A (FP64)."""
    A = np.asarray(A, dtype=np.float64)
    G = A.T @ A + lam * np.eye(A.shape[1])
    evals, evecs = np.linalg.eigh(G)
    top = float(evals.max()) if evals.size else 0.0
    keep = evals > pinv_tol(*A.shape) * top
    inv = np.where(keep, 1.0 / np.where(keep, evals, 1.0), 0.0)
    return (evecs * inv) @ evecs.T, int(keep.sum())


def ridge_leverage_scores(A: np.ndarray, lam: float = 0.0) -> np.ndarray:
    """l_i^lam(A) = a_i (A^T A + lam I)^+ a_i^T  (Eq. ridge_leverage_score_def, Sec. 2).

    lam = 0 gives the statistical leverage scores l(A) used by Alg. 3 line 1.
    """
    A = np.asarray(A, dtype=np.float64)
    P, _ = gram_pinv(A, lam)
    return np.einsum("ir,rs,is->i", A, P, A)


def leverage_scores(A: np.ndarray):
    """(l(A), rank(A)): statistical leverage scores of one factor (Alg. 3 line 1)."""
    A = np.asarray(A, dtype=np.float64)
    P, rank = gram_pinv(A, 0.0)
    return np.einsum("ir,rs,is->i", A, P, A), rank


def cross_ridge_leverage_scores(A: np.ndarray, lam: float = 0.0) -> np.ndarray:
    """Matrix L = A (A^T A + lam I)^+ A^T of cross ridge leverage scores (Sec. 2)."""
    A = np.asarray(A, dtype=np.float64)
    P, _ = gram_pinv(A, lam)
    return A @ P @ A.T


def effective_dimension(A: np.ndarray, lam: float) -> float:
    """d_eff = sum_i l_i^lam(A)  (Eq. d_eff_def)."""
    return float(ridge_leverage_scores(A, lam).sum())
