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

from . import sampling as S
from .core_update import (mode_product, kron_matrix, exact_core_kron_eig, sketched_core,
                          kt_x)
from .leverage import leverage_scores


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


# ------------------------------------------------ sketched factor update
# The factor update of mode n is the ridge regression min ||B_n A^T - X_(n)^T||^2 +
# lam ||A||^2 with the design B_n = W G_(n)^T, W = (x)_{k != n} A^(k) (rows indexed by
# the multi-index over the modes k != n, row-major).  The rows of B_n lie in the
# column space of W, so l_j(B_n) <= l_j(W) = prod_{k != n} l_{j_k}(A^(k)) (Lemma 4.1
# at lam = 0): the product distribution of the other modes' leverage scores is a
# (R_n / prod_{k != n} R_k)-overestimate of the leverage scores of B_n, and the same
# sampling, weights and normal equations as the core's sketch (Alg. 1) apply with
# B_n in place of K.  This is this library's design (the paper updates the factors
# exactly); its draws use Philox key word 1 = sweep + (n + 1) 2^32, apart from the
# core sampler's (seed, sweep).

def factor_sample_key(sweep: int, n: int) -> int:
    """Philox key word 1 of the mode-n factor sampler."""
    return int(sweep) + ((int(n) + 1) << 32)


def factor_design_rows(core, factors, n, idx) -> np.ndarray:
    """b_u = G_(n) (x)_{k != n} A^(k)[j_k] for the multi-indices idx (list over k != n):
    the rows of B_n, n_u x R_n."""
    others = [np.asarray(A, dtype=np.float64) for k, A in enumerate(factors) if k != n]
    rows = None
    for A, j in zip(others, idx):                   # Kronecker order: earlier modes outer
        a = A[np.asarray(j)]
        rows = a if rows is None else np.einsum("ua,ub->uab", rows, a).reshape(a.shape[0], -1)
    Gn = unfold(np.asarray(core, dtype=np.float64), n)
    return rows @ Gn.T


def factor_update_from_rows(X, core, factors, n, lam, keys, w) -> np.ndarray:
    """Alg. 2's factor update on the rows `keys` of B_n with weights w:
    A^(n) = Y M^-1, M = sum_u w_u b_u b_u^T + lam I, Y = sum_u w_u x_u b_u^T, with x_u
    the mode-n fiber of X at row u (column keys_u of X_(n))."""
    dims = [int(v) for k, v in enumerate(np.shape(X)) if k != n]
    keys = np.asarray(keys, dtype=np.uint64)
    b = factor_design_rows(core, factors, n, S.decode_keys(keys, dims))
    Xn = unfold(np.asarray(X, dtype=np.float64), n)[:, keys.astype(np.int64)]
    wb = np.asarray(w, dtype=np.float64)[:, None] * b
    M = wb.T @ b + lam * np.eye(b.shape[1])
    Y = Xn @ wb
    return np.linalg.solve(M, Y.T).T


def sketched_factor_update(X, core, factors, n, lam, m, seed, sweep=0):
    """Sketched factor update of mode n: m draws from the product of the leverage
    scores of A^(k), k != n (the core sampler's arithmetic over those modes, key word
    factor_sample_key(sweep, n)), dedupe, w = c / (m p), and the weighted normal
    equations of factor_update_from_rows."""
    others = [np.asarray(A, dtype=np.float64) for k, A in enumerate(factors) if k != n]
    dims = [int(v) for k, v in enumerate(np.shape(X)) if k != n]
    lev = [leverage_scores(A)[0] for A in others]
    keys, T = S.sample_keys(lev, dims, m, seed, factor_sample_key(sweep, n))
    ku, cu = S.dedupe(keys)
    p = S.row_probabilities(ku, lev, dims, S.REG_EXACT, 0)
    w = S.sample_weights(cu, p, T)
    A = factor_update_from_rows(X, core, factors, n, lam, ku, w)
    return {"A": A, "keys": ku, "counts": cu, "prob": p, "w": w}


def als_sweep(X, core, factors, lam, sketched: bool = False, m: int = 0, seed: int = 0,
              sweep: int = 0, reg: int = 0, m_factor: int = 0):
    """One repeat-loop pass of Alg. 2: factor updates n = 1..N (sketched with m_factor
    draws each when m_factor > 0), then the core update."""
    factors = [np.asarray(A, dtype=np.float64).copy() for A in factors]
    core = np.asarray(core, dtype=np.float64)
    for n in range(len(factors)):
        if m_factor > 0:
            factors[n] = sketched_factor_update(X, core, factors, n, lam, m_factor, seed,
                                                sweep)["A"]
        else:
            factors[n] = factor_update(X, core, factors, n, lam)
    R = core.shape
    if sketched:
        g = sketched_core(np.asarray(X), factors, lam, m, seed, sweep, reg)["g"]
    else:
        g = exact_core_kron_eig(X, factors, lam)
    return g.reshape(R), factors
