"""Regularised CP-ALS with sketched factor updates (the closing remark of Sec. 6:
the sampling of Sec. 4 extends the leverage-score-sampled CP-ALS of the cited
works to L2 regularisation; Sec. 4, remark before Alg. 2: Kronecker leverage
scores overestimate those of a Khatri-Rao design) in FP64.

Oracle module: test infrastructure.  Only tests/, __graft_entry__.smoke() and
bench.py's cpu_baseline / reference leg may import anything under oracle/.

CP model of rank R: X_hat[i_1, ..., i_N] = sum_r prod_n A^(n)[i_n, r].  The loss
is ||X - X_hat||^2 + lam sum_n ||A^(n)||_F^2 (the Tucker loss of Sec. 2 with the
superdiagonal core and the regulariser on the factors).  The factor update of
mode n is the ridge regression of every mode-n fiber on the Khatri-Rao design
Z_n (rows indexed row-major by the multi-index over the modes k != n, last
fastest), row j = the Hadamard product of A^(k)[j_k, :], k != n:
    A^(n) = X_(n) Z_n (Z_n^T Z_n + lam I)^-1,  Z_n^T Z_n = Hadamard_{k != n} A^(k)T A^(k).
Z_n's columns are the columns (r, ..., r) of the Kronecker product
(x)_{k != n} A^(k), so its column space lies in the Kronecker product's and
l_j(Z_n) <= prod_{k != n} l_{j_k}(A^(k)) (leverage scores of a subspace cannot
exceed those of a space containing it): the product distribution of the other
modes' leverage scores is an overestimate with beta = R / prod_{k != n} rank(A^(k)),
and Alg. 1's weighted sketch applies with Z_n in place of K.  The sketched update
uses the core sampler's arithmetic over the modes k != n (Philox key word 1 =
sweep + (n + 1) 2^32, as the sketched Tucker factor update), dedupe,
w = c / (m p), and the weighted normal equations
    M = sum_u w_u z_u z_u^T + lam I,  Y = sum_u w_u x_u z_u^T,  A^(n) = Y M^-1.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np

from . import sampling as S
from .leverage import leverage_scores


def unfold(T: np.ndarray, n: int) -> np.ndarray:
    """Mode-n unfolding, remaining indices row-major (last fastest)."""
    return np.moveaxis(np.asarray(T), n, 0).reshape(np.shape(T)[n], -1)


def cp_model(factors: Sequence[np.ndarray]) -> np.ndarray:
    """X_hat = sum_r a_1[:, r] o ... o a_N[:, r], by an explicit sum over r."""
    F = [np.asarray(A, dtype=np.float64) for A in factors]
    dims = tuple(A.shape[0] for A in F)
    R = F[0].shape[1]
    X = np.zeros(dims)
    for r in range(R):
        t = F[0][:, r]
        for A in F[1:]:
            t = np.multiply.outer(t, A[:, r])
        X += t
    return X


def cp_loss(X, factors, lam) -> float:
    """||X - X_hat||^2 + lam sum_n ||A^(n)||_F^2."""
    res = np.asarray(X, dtype=np.float64) - cp_model(factors)
    return float(np.sum(res * res) + lam * sum(np.sum(np.asarray(A, dtype=np.float64) ** 2)
                                               for A in factors))


def khatri_rao_rows(factors, n, idx) -> np.ndarray:
    """z_u = Hadamard_{k != n} A^(k)[j_k, :] for the multi-indices idx (list over k != n)."""
    others = [np.asarray(A, dtype=np.float64) for k, A in enumerate(factors) if k != n]
    z = None
    for A, j in zip(others, idx):
        a = A[np.asarray(j)]
        z = a.copy() if z is None else z * a
    return z


def khatri_rao(factors, n) -> np.ndarray:
    """The whole design Z_n (prod_{k != n} I_k x R), rows in row-major order."""
    others = [np.asarray(A, dtype=np.float64) for k, A in enumerate(factors) if k != n]
    grids = np.meshgrid(*[np.arange(A.shape[0]) for A in others], indexing="ij")
    return khatri_rao_rows(factors, n, [g.reshape(-1) for g in grids])


def cp_factor_update(X, factors, n, lam) -> np.ndarray:
    """The exact update of mode n: A^(n) = X_(n) Z_n (Z_n^T Z_n + lam I)^-1."""
    Z = khatri_rao(factors, n)
    Xn = unfold(np.asarray(X, dtype=np.float64), n)
    M = Z.T @ Z + lam * np.eye(Z.shape[1])
    return np.linalg.solve(M, (Xn @ Z).T).T


def cp_factor_update_from_rows(X, factors, n, lam, keys, w) -> np.ndarray:
    """The update on the rows `keys` of Z_n with weights w: A^(n) = Y M^-1,
    M = sum_u w_u z_u z_u^T + lam I, Y = sum_u w_u x_u z_u^T (x_u the mode-n fiber of
    X at row u, i.e. column keys_u of X_(n))."""
    dims = [int(v) for k, v in enumerate(np.shape(X)) if k != n]
    keys = np.asarray(keys, dtype=np.uint64)
    z = khatri_rao_rows(factors, n, S.decode_keys(keys, dims))
    Xn = unfold(np.asarray(X, dtype=np.float64), n)[:, keys.astype(np.int64)]
    wz = np.asarray(w, dtype=np.float64)[:, None] * z
    M = wz.T @ z + lam * np.eye(z.shape[1])
    return np.linalg.solve(M, (Xn @ wz).T).T


def cp_sample_key(sweep: int, n: int) -> int:
    """Philox key word 1 of the mode-n factor sampler (as the sketched Tucker factor update)."""
    return int(sweep) + ((int(n) + 1) << 32)


def sketched_cp_factor_update(X, factors, n, lam, m, seed, sweep=0):
    """m draws from the product of the leverage scores of A^(k), k != n, dedupe,
    w = c / (m p), and the weighted normal equations of cp_factor_update_from_rows."""
    others = [np.asarray(A, dtype=np.float64) for k, A in enumerate(factors) if k != n]
    dims = [int(v) for k, v in enumerate(np.shape(X)) if k != n]
    lev = [leverage_scores(A)[0] for A in others]
    keys, T = S.sample_keys(lev, dims, m, seed, cp_sample_key(sweep, n))
    ku, cu = S.dedupe(keys)
    p = S.row_probabilities(ku, lev, dims, S.REG_EXACT, 0)
    w = S.sample_weights(cu, p, T)
    A = cp_factor_update_from_rows(X, factors, n, lam, ku, w)
    return {"A": A, "keys": ku, "counts": cu, "prob": p, "w": w}


def cp_als_sweep(X, factors, lam, m: int = 0, seed: int = 0, sweep: int = 0):
    """One pass of regularised CP-ALS: factor updates n = 1..N in turn, each exact
    (m = 0) or sketched with m draws."""
    F = [np.asarray(A, dtype=np.float64).copy() for A in factors]
    for n in range(len(F)):
        F[n] = (sketched_cp_factor_update(X, F, n, lam, m, seed, sweep)["A"] if m > 0
                else cp_factor_update(X, F, n, lam))
    return F
