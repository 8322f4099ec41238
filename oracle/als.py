"""Regularised Tucker ALS (Alg. 2) and the Tucker loss (Sec. 2) in FP64.

Oracle module: test infrastructure.  Only tests/, __graft_entry__.smoke() and
bench.py's cpu_baseline / reference leg may import anything under oracle/.

Factor update of Alg. 2 for mode n: with K_n = G_(n) (x)_{k != n} A^(k)T and
B = X_(n), every row solves argmin_y ||y K_n - b_i||^2 + lam ||y||^2, i.e.
A^(n) = X_(n) W G_(n)^T (G_(n) W^T W G_(n)^T + lam I)^-1 where
W = (x)_{k != n} A^(k); X_(n) W is the mode-n unfolding of X x_{k != n} A^(k)T and
W^T W = (x)_{k != n} A^(k)T A^(k).  Unfoldings order the remaining indices
row-major (last fastest), matching the Kronecker order k = 1..N, k != n.
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np

from .core_update import (mode_product, kron_matrix, exact_core_kron_eig, sketched_core,
                          kt_x)


def unfold(T: np.ndarray, n: int) -> np.ndarray:
    """Mode-n unfolding X_(n): I_n x prod_{k != n} I_k (Sec. 2)."""
    return np.moveaxis(np.asarray(T), n, 0).reshape(T.shape[n], -1)


def tucker_model(core, factors) -> np.ndarray:
    """X-hat = G x_1 A^(1) ... x_N A^(N)  (Eq. tucker_decomposition_elementwise)."""
    t = np.asarray(core, dtype=np.float64)
    for n, A in enumerate(factors):
        t = mode_product(t, np.asarray(A, dtype=np.float64), n)
    return t


def tucker_loss(X, core, factors, lam) -> float:
    """L = ||X - X-hat||_F^2 + lam (||G||_F^2 + sum_n ||A^(n)||_F^2)  (Sec. 2)."""
    r = np.asarray(X, dtype=np.float64) - tucker_model(core, factors)
    reg = float(np.sum(np.asarray(core, dtype=np.float64) ** 2))
    reg += sum(float(np.sum(np.asarray(A, dtype=np.float64) ** 2)) for A in factors)
    return float(np.sum(r * r)) + lam * reg


def rmse(X, core, factors) -> float:
    """sqrt(mean squared residual over entries); with 1% of entries carrying
    N(0,1) noise the floor is 0.10 (Sec. 5)."""
    r = np.asarray(X, dtype=np.float64) - tucker_model(core, factors)
    return float(np.sqrt(np.mean(r * r)))


def factor_update(X, core, factors, n, lam) -> np.ndarray:
    """New A^(n) of Alg. 2 (all I_n row problems at once)."""
    N = len(factors)
    Y = np.asarray(X, dtype=np.float64)
    for k in range(N):
        if k != n:
            Y = mode_product(Y, np.asarray(factors[k], dtype=np.float64).T, k)
    B = unfold(Y, n)
    Gn = unfold(np.asarray(core, dtype=np.float64), n)
    H = np.ones((1, 1))
    for k in range(N):
        if k != n:
            A = np.asarray(factors[k], dtype=np.float64)
            H = np.kron(H, A.T @ A)
    lhs = Gn @ H @ Gn.T + lam * np.eye(Gn.shape[0])
    return np.linalg.solve(lhs, (B @ Gn.T).T).T


def factor_update_bruteforce(X, core, factors, n, lam) -> np.ndarray:
    """Alg. 2 factor update with K_n = G_(n) (x)_{k!=n} A^(k)T formed explicitly."""
    N = len(factors)
    W = kron_matrix([factors[k] for k in range(N) if k != n])
    Kn = unfold(np.asarray(core, dtype=np.float64), n) @ W.T
    B = unfold(np.asarray(X, dtype=np.float64), n)
    lhs = Kn @ Kn.T + lam * np.eye(Kn.shape[0])
    return np.linalg.solve(lhs, Kn @ B.T).T


def als_sweep(X, core, factors, lam, sketched: bool = False, m: int = 0, seed: int = 0,
              sweep: int = 0, reg: int = 0):
    """One repeat-loop pass of Alg. 2: factor updates n = 1..N, then the core update."""
    factors = [np.asarray(A, dtype=np.float64).copy() for A in factors]
    core = np.asarray(core, dtype=np.float64)
    for n in range(len(factors)):
        factors[n] = factor_update(X, core, factors, n, lam)
    R = core.shape
    if sketched:
        g = sketched_core(np.asarray(X), factors, lam, m, seed, sweep, reg)["g"]
    else:
        g = exact_core_kron_eig(X, factors, lam)
    return g.reshape(R), factors
