"""Core-tensor update of regularised Tucker ALS, exact and sketched (FP64).

Oracle module: test infrastructure.  Only tests/, __graft_entry__.smoke() and
bench.py's cpu_baseline / reference leg may import anything under oracle/.

  * exact update: Alg. 2 (core line): argmin_g ||K g - vec(X)||^2 + lam ||g||^2
    with K = A^(1) (x) ... (x) A^(N); two routes: the explicit normal equations
    (brute force) and the eigendecomposition of K^T K + lam I = (x V_n)(x S_n^2
    + lam)(x V_n)^T from the proof of Lemma 4.1 (Appendix B), with K^T vec(X)
    computed as the n-mode product chain X x_n A^(n)T (Sec. 2);
  * sketched update: Alg. 3 -> Alg. 1: rows of K sampled from the factored
    leverage distribution, weighted by c/(T p); the normal equations
    (SK)^T SK and (SK)^T S vec(X) as sums of outer products (Appendix B,
    proof of Thm 4.2); solved by Cholesky.  lam I is exact (REG_EXACT) or the
    sampled regulariser rows of the augmented matrix of Eq. problem_def
    (REG_AUGMENTED).
Row-major vec everywhere (the last index varies fastest), which is the order in
which K = A^(1) (x) ... (x) A^(N) indexes its rows and columns.
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np

from . import sampling as S
from .leverage import leverage_scores


def mode_product(T: np.ndarray, M: np.ndarray, n: int) -> np.ndarray:
    """T x_n M: (T x_n M)[.., j, ..] = sum_i T[.., i, ..] M[j, i]  (Sec. 2)."""
    out = np.tensordot(M, T, axes=([1], [n]))        # j first
    return np.moveaxis(out, 0, n)


def kron_matrix(factors: Sequence[np.ndarray]) -> np.ndarray:
    """Explicit K = A^(1) (x) ... (x) A^(N) (tiny inputs only)."""
    K = np.ones((1, 1))
    for A in factors:
        K = np.kron(K, np.asarray(A, dtype=np.float64))
    return K


def kron_rows(factors: Sequence[np.ndarray], idx: Sequence[np.ndarray]) -> np.ndarray:
    """Rows (i_1..i_N) of K: k[r_1..r_N] = prod_n A^(n)[i_n, r_n] (Lemma 4.1 indexing)."""
    rows = np.asarray(factors[0], dtype=np.float64)[idx[0]]
    for A, i in zip(factors[1:], idx[1:]):
        a = np.asarray(A, dtype=np.float64)[i]
        rows = (rows[:, :, None] * a[:, None, :]).reshape(rows.shape[0], -1)
    return rows


def sampled_rows_apply(factors: Sequence[np.ndarray], idx: Sequence[np.ndarray], g: np.ndarray,
                       chunk: int = 2048) -> np.ndarray:
    """z = K_S g for the sampled rows idx (z_u = k_u . g, the implicit design
    matrix of Alg. 3 applied to a vector), built from explicit row chunks."""
    n = len(idx[0])
    z = np.empty(n)
    g = np.asarray(g, dtype=np.float64)
    for s in range(0, n, chunk):
        z[s:s + chunk] = kron_rows(factors, [i[s:s + chunk] for i in idx]) @ g
    return z


def sampled_rows_apply_t(factors: Sequence[np.ndarray], idx: Sequence[np.ndarray],
                         c: np.ndarray, chunk: int = 2048) -> np.ndarray:
    """K_S^T c = sum_u c_u k_u over the sampled rows, from explicit row chunks."""
    n = len(idx[0])
    c = np.asarray(c, dtype=np.float64)
    out = None
    for s in range(0, n, chunk):
        part = kron_rows(factors, [i[s:s + chunk] for i in idx]).T @ c[s:s + chunk]
        out = part if out is None else out + part
    return out


def kron_gram_apply(factors: Sequence[np.ndarray], g: np.ndarray) -> np.ndarray:
    """(K^T K) vec(g) = vec(g x_n (A^(n)T A^(n)))  (mixed-product property)."""
    t = np.asarray(g, dtype=np.float64).reshape([A.shape[1] for A in factors])
    for n, A in enumerate(factors):
        A = np.asarray(A, dtype=np.float64)
        t = mode_product(t, A.T @ A, n)
    return t.reshape(-1)


def kt_x(X: np.ndarray, factors: Sequence[np.ndarray]) -> np.ndarray:
    """K^T vec(X) = vec(X x_1 A^(1)T ... x_N A^(N)T)  (n-mode product chain)."""
    t = np.asarray(X, dtype=np.float64)
    for n in range(len(factors) - 1, -1, -1):
        t = mode_product(t, np.asarray(factors[n], dtype=np.float64).T, n)
    return t.reshape(-1)


def ridge_loss_dense(X, factors, g, lam, xx: Optional[float] = None, ktx=None) -> float:
    """||K g - vec X||^2 + lam ||g||^2 via ||x||^2 - 2 g.K^T x + g.(K^T K) g + lam g.g."""
    g = np.asarray(g, dtype=np.float64).reshape(-1)
    if xx is None:
        x = np.asarray(X, dtype=np.float64).reshape(-1)
        xx = float(x @ x)
    if ktx is None:
        ktx = kt_x(X, factors)
    return float(xx - 2.0 * (g @ ktx) + g @ kron_gram_apply(factors, g) + lam * (g @ g))


def ridge_loss_rows(keys, vals, dims, factors, g, lam, chunk: int = 1 << 14) -> float:
    """sum over the given rows of (k_i^T g - x_i)^2 + lam ||g||^2 (missing-entry loss)."""
    g = np.asarray(g, dtype=np.float64).reshape(-1)
    tot = 0.0
    for s in range(0, len(keys), chunk):
        idx = S.decode_keys(keys[s:s + chunk], dims)
        r = kron_rows(factors, idx) @ g - np.asarray(vals[s:s + chunk], dtype=np.float64)
        tot += float(r @ r)
    return tot + lam * float(g @ g)


# ---------------------------------------------------------------- exact update

def exact_core_bruteforce(X, factors, lam) -> np.ndarray:
    """Solve (K^T K + lam I) g = K^T vec(X) with K formed explicitly (tiny only)."""
    K = kron_matrix(factors)
    x = np.asarray(X, dtype=np.float64).reshape(-1)
    return np.linalg.solve(K.T @ K + lam * np.eye(K.shape[1]), K.T @ x)


def exact_core_kron_eig(X, factors, lam, ktx=None) -> np.ndarray:
    """Exact core via K^T K + lam I = (x V)(x S^2 + lam)(x V)^T (Appendix B, Lemma 4.1 proof).

    y = K^T vec X by the n-mode product chain, z = y x_n V_n^T,
    z /= (S_1^2 (x) ... (x) S_N^2 + lam), g = z x_n V_n.
    """
    R = [A.shape[1] for A in factors]
    y = (kt_x(X, factors) if ktx is None else np.asarray(ktx, dtype=np.float64)).reshape(R)
    evals, evecs = [], []
    for A in factors:
        A = np.asarray(A, dtype=np.float64)
        e, V = np.linalg.eigh(A.T @ A)
        evals.append(e)
        evecs.append(V)
    z = y
    for n, V in enumerate(evecs):
        z = mode_product(z, V.T, n)
    lam_k = np.ones(1)
    for e in evals:
        lam_k = np.multiply.outer(lam_k, e).reshape(-1)
    z = z / (lam_k.reshape(R) + lam)
    for n, V in enumerate(evecs):
        z = mode_product(z, V, n)
    return z.reshape(-1)


def exact_core_rows(keys, vals, dims, factors, lam, chunk: int = 1 << 13) -> np.ndarray:
    """Exact core with only the rows `keys` of K (missing entries): explicit normal
    equations sum_i k_i k_i^T and sum_i x_i k_i over the observed rows."""
    d = int(np.prod([A.shape[1] for A in factors]))
    G = np.zeros((d, d))
    h = np.zeros(d)
    for s in range(0, len(keys), chunk):
        idx = S.decode_keys(keys[s:s + chunk], dims)
        Kr = kron_rows(factors, idx)
        G += Kr.T @ Kr
        h += Kr.T @ np.asarray(vals[s:s + chunk], dtype=np.float64)
    return np.linalg.solve(G + lam * np.eye(d), h)


# -------------------------------------------------------------- sketched update

def sketch(factors, dims, m, seed, sweep, reg=S.REG_EXACT, observed_keys=None,
           max_draws=0, lev_list=None):
    """Alg. 3 lines 1-3 and the sampling loop of Alg. 1: unique keys, counts,
    probabilities, weights, T."""
    d = int(np.prod([A.shape[1] for A in factors]))
    if lev_list is None:
        lev_list = [leverage_scores(A)[0] for A in factors]
    keys, T = S.sample_keys(lev_list, dims, m, seed, sweep, reg, d, observed_keys, max_draws)
    ku, cu = S.dedupe(keys)
    p = S.row_probabilities(ku, lev_list, dims, reg, d)
    w = S.sample_weights(cu, p, T)
    return {"keys": ku, "counts": cu, "prob": p, "w": w, "T": T, "lev": lev_list}


def gather_dense(X, keys_u, dims) -> np.ndarray:
    """b entries vec(X)[key]; 0 for augmented rows (b-bar = [b; 0], Eq. problem_def)."""
    x = np.asarray(X).reshape(-1)
    total = int(np.prod([int(v) for v in dims]))
    keys_u = np.asarray(keys_u, dtype=np.uint64)
    real = keys_u < np.uint64(total)
    out = np.zeros(keys_u.shape, dtype=np.float64)
    out[real] = x[keys_u[real].astype(np.int64)]
    return out


def gather_observed(obs_keys, obs_vals, keys_u) -> np.ndarray:
    """b entries of observed rows looked up by key (missing-entry case); 0 for
    augmented rows."""
    obs_keys = np.asarray(obs_keys, dtype=np.uint64)
    keys_u = np.asarray(keys_u, dtype=np.uint64)
    pos = np.searchsorted(obs_keys, keys_u)
    ok = (pos < obs_keys.size) & (obs_keys[np.minimum(pos, obs_keys.size - 1)] == keys_u)
    out = np.zeros(keys_u.shape, dtype=np.float64)
    out[ok] = np.asarray(obs_vals, dtype=np.float64)[pos[ok]]
    return out


def sketched_normal_equations(factors, dims, keys_u, w, x, chunk: int = 1 << 12):
    """G = sum_u w_u k_u k_u^T, h = sum_u w_u x_u k_u over real rows; D_j = sum of
    w_u over augmented rows j (the sampled lam rows of Eq. problem_def)."""
    d = int(np.prod([A.shape[1] for A in factors]))
    total = np.uint64(int(np.prod([int(v) for v in dims])))
    keys_u = np.asarray(keys_u, dtype=np.uint64)
    aug = keys_u >= total
    D = np.zeros(d)
    np.add.at(D, (keys_u[aug] - total).astype(np.int64), np.asarray(w)[aug])
    real = np.flatnonzero(~aug)
    G = np.zeros((d, d))
    h = np.zeros(d)
    for s in range(0, real.size, chunk):
        sel = real[s:s + chunk]
        Kr = kron_rows(factors, S.decode_keys(keys_u[sel], dims))
        ws = np.asarray(w, dtype=np.float64)[sel]
        G += Kr.T @ (Kr * ws[:, None])
        h += Kr.T @ (ws * np.asarray(x, dtype=np.float64)[sel])
    return G, h, D


def regularised_matrix(G, D, lam, reg):
    """G + lam I (REG_EXACT) or G + lam diag(D) (REG_AUGMENTED)."""
    if reg == S.REG_EXACT:
        return G + lam * np.eye(G.shape[0])
    return G + lam * np.diag(D)


def cholesky_solve(M, h):
    """Solve M g = h by the Cholesky factorisation M = L L^T (raises if M is not SPD)."""
    L = np.linalg.cholesky(M)
    y = np.linalg.solve(L, h)
    return np.linalg.solve(L.T, y)


def sketched_core(X, factors, lam, m, seed, sweep=0, reg=S.REG_EXACT, observed=None,
                  max_draws=0):
    """FastCoreTensorUpdate (Alg. 3) with sample count m.

    observed: None (dense X) or (keys, vals) of the observed entries, in which
    case X is ignored.
    """
    dims = tuple(int(v) for v in (X.shape if observed is None else observed[2]))
    obs_keys = None if observed is None else observed[0]
    sk = sketch(factors, dims, m, seed, sweep, reg, obs_keys, max_draws)
    if observed is None:
        x = gather_dense(X, sk["keys"], dims)
    else:
        x = gather_observed(observed[0], observed[1], sk["keys"])
    G, h, D = sketched_normal_equations(factors, dims, sk["keys"], sk["w"], x)
    g = cholesky_solve(regularised_matrix(G, D, lam, reg), h)
    sk.update({"x": x, "G": G, "h": h, "D": D, "g": g})
    return sk
