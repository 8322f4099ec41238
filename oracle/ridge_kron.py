"""Ridge leverage scores of the Kronecker design matrix, the constants that set
the sample count, and an exact sampler of the ridge leverage distribution of K.

Oracle module: test infrastructure.  Only tests/, __graft_entry__.smoke() and
bench.py's cpu_baseline / reference leg may import anything under oracle/.

Restated from the paper:
  * Lemma 4.1 for lam > 0: with A^(n) = U^(n) Sigma^(n) V^(n)T,
        l^lam_{(i),(j)}(K) = sum_t c_t prod_n u^(n)_{i_n t_n} u^(n)_{j_n t_n},
        c_t = P_t / (P_t + lam),  P_t = prod_n sigma^2_{t_n}(A^(n));
  * d_eff(K) = sum_i l^lam_i(K)  (Eq. d_eff_def), which is sum_t c_t because
    every column of U^(n) has unit norm;
  * Cor. leverage_score_overestimate: the classical scores are a
    (d_eff / rank)-overestimate of the lam-ridge scores;
  * Eq. beta_prime (Lemma beta_overestimate) and its lower bound used by
    Alg. 1 line 2, beta' = min{beta, 1} / (1 + min{1, d - d'_eff});
  * missing entries (Sec. 4.2, after Lemma 4.4): the ridge scores of A are a
    beta-overestimate for those of the observed rows with
    1/beta = 1 + 1/(1 - lambda_max(L_{S-bar,S-bar})), and the corollary to
    Thm 4.3 bounds 1/(1 - lambda_max) by 1 + prod_n ||A^(n)||_2^2 / lam;
    lambda_max from the observed rows' Gram as a generalized eigenvalue, and
    the sample count of the observed-entry sampler composed from beta and the
    factor by which classical scores of K bound its ridge scores.

The exact sampler is this library's design, not the paper's (the paper draws
from the product of the classical factor scores): by Lemma 4.1,
l^lam(K) / d_eff(K) is a mixture over t, with weights c_t / d_eff(K), of the
product distributions prod_n (u^(n)_{. t_n})^2 (unit-norm columns), so a draw
picks a component t and then one row index per mode.

Readings (listed in the design notes):
  * Lemma 4.1's sum runs over t_n in [min(I_n, R_n)] (the thin SVD); the
    printed index set [I_1] x ... x [I_N] only adds terms with sigma = 0;
  * a squared singular value at or below leverage.pinv_tol x the largest one
    of its factor counts as zero (the pseudo-inverse rule), so at lam = 0
    every c_t is 0 or 1;
  * sampler arithmetic as in sampling.py: fixed-point weights
    floor(clamp(x, 0, 1) 2^32), inclusive prefix sums, and
    min{i : C_i > floor(u Q / 2^64)}; the component (row-major over t) is
    chosen by word 0 of Philox stream 3, the row indices by the words the
    product sampler uses (word n % 4 of stream n // 4).
"""
from __future__ import annotations

from typing import Sequence

import numpy as np

from . import sampling as S
from . import core_update as CU
from .leverage import cross_ridge_leverage_scores, pinv_tol
from .philox import philox4x64_10, mulhi64

U64 = np.uint64


# ------------------------------------------------------------- Lemma 4.1, lam > 0

def factor_svds(factors: Sequence[np.ndarray]):
    """Per factor the thin SVD's U^(n) and sigma^2(A^(n)), squared singular
    values under the pseudo-inverse cutoff set to zero."""
    out = []
    for A in factors:
        A = np.asarray(A, dtype=np.float64)
        U, s, _ = np.linalg.svd(A, full_matrices=False)
        s2 = s ** 2
        top = float(s2.max()) if s2.size else 0.0
        out.append((U, np.where(s2 > pinv_tol(*A.shape) * top, s2, 0.0)))
    return out


def ridge_weights(factors: Sequence[np.ndarray], lam: float):
    """(c, [U^(n)]): c_t = P_t / (P_t + lam) on the grid of t (Lemma 4.1),
    P_t = prod_n sigma^2_{t_n}; c_t = 0 where P_t = 0."""
    svds = factor_svds(factors)
    P = np.ones(())
    for _, s2 in svds:
        P = np.multiply.outer(P, s2)
    c = np.zeros(P.shape)
    pos = P > 0
    c[pos] = P[pos] / (P[pos] + lam)
    return c, [U for U, _ in svds]


def kron_cross_ridge_leverage(factors: Sequence[np.ndarray], lam: float,
                              idx_i: Sequence[np.ndarray], idx_j: Sequence[np.ndarray]):
    """l^lam_{(i),(j)}(K) for row pairs given as per-mode index arrays (Lemma 4.1):
    sum_t c_t prod_n u^(n)_{i_n t_n} u^(n)_{j_n t_n}, contracted one mode at a time."""
    c, Us = ridge_weights(factors, lam)
    rows = len(idx_i[0])
    W = np.broadcast_to(c, (rows,) + c.shape)
    for n, U in enumerate(Us):
        e = U[np.asarray(idx_i[n])] * U[np.asarray(idx_j[n])]     # [rows, k_n]
        W = np.einsum("kt,kt...->k...", e, W)
    return W


def kron_ridge_leverage_scores(factors: Sequence[np.ndarray], lam: float,
                               idx: Sequence[np.ndarray]):
    """l^lam_i(K) for rows idx (Lemma 4.1 with i = j)."""
    return kron_cross_ridge_leverage(factors, lam, idx, idx)


def kron_effective_dimension(factors: Sequence[np.ndarray], lam: float) -> float:
    """d_eff(K) = sum_i l^lam_i(K) (Eq. d_eff_def) = sum_t c_t."""
    c, _ = ridge_weights(factors, lam)
    return float(c.sum())


def kron_rank(factors: Sequence[np.ndarray]) -> int:
    """rank(K) = prod_n rank(A^(n)) (Kronecker product of the singular values)."""
    r = 1
    for _, s2 in factor_svds(factors):
        r *= int(np.count_nonzero(s2))
    return r


def classical_overestimate_beta(factors: Sequence[np.ndarray], lam: float) -> float:
    """beta with which the classical scores of K overestimate its lam-ridge
    scores: d_eff(K) / rank(K)  (Cor. leverage_score_overestimate)."""
    return kron_effective_dimension(factors, lam) / kron_rank(factors)


# ------------------------------------------------------------ sample-count constants

def augmented_pmf(lhat: np.ndarray, d: int, d_eff_lower: float) -> np.ndarray:
    """Probability vector of D(l-hat, d'_eff) over [n + d] (the augmented
    distribution of Sec. 3): proportional to l-hat_i on the rows of A and to
    min{1, d - d'_eff} on each of the d regulariser rows."""
    lhat = np.asarray(lhat, dtype=np.float64)
    extra = min(1.0, d - d_eff_lower)
    mass = np.concatenate([lhat, np.full(d, extra)])
    return mass / mass.sum()


def lemma_beta_prime(beta: float, d: int, d_eff: float, d_eff_lower: float,
                     lhat_l1: float) -> float:
    """Eq. beta_prime: min{(1 + d min{1, d - d'_eff} / ||l-hat||_1)^-1 beta d / d_eff,
    (||l-hat||_1 / d + min{1, d - d'_eff})^-1}."""
    mlt = min(1.0, d - d_eff_lower)
    a = beta * d / d_eff / (1.0 + d * mlt / lhat_l1)
    b = 1.0 / (lhat_l1 / d + mlt)
    return min(a, b)


def alg1_beta_prime(beta: float, d: int, d_eff_lower: float) -> float:
    """beta' = min{beta, 1} / (1 + min{1, d - d'_eff})  (Alg. 1 line 2)."""
    return min(beta, 1.0) / (1.0 + min(1.0, d - d_eff_lower))


def missing_ridge_beta(factors: Sequence[np.ndarray], lam: float, observed_keys,
                       dims: Sequence[int]) -> float:
    """Exact beta for observed rows S of a small K (Sec. 4.2 after Lemma 4.4):
    1/beta = 1 + 1/(1 - lambda_max(L_{S-bar,S-bar})), L the cross lam-ridge
    score matrix of K (explicit); beta = 1 when no row is missing."""
    K = CU.kron_matrix(factors)
    n = K.shape[0]
    miss = np.setdiff1d(np.arange(n), np.asarray(observed_keys, dtype=np.int64))
    if miss.size == 0:
        return 1.0
    L = cross_ridge_leverage_scores(K, lam)
    lmax = float(np.linalg.eigvalsh(L[np.ix_(miss, miss)]).max())
    return 1.0 / (1.0 + 1.0 / (1.0 - lmax))


def missing_ridge_beta_bound(factors: Sequence[np.ndarray], lam: float) -> float:
    """Lower bound of that beta from the corollary to Thm 4.3:
    1/(1 - lambda_max) <= 1 + prod_n ||A^(n)||_2^2 / lam, so
    beta >= 1 / (2 + prod_n ||A^(n)||_2^2 / lam)."""
    p = 1.0
    for A in factors:
        p *= float(np.linalg.norm(np.asarray(A, dtype=np.float64), 2)) ** 2
    return 1.0 / (2.0 + p / lam)


def missing_ridge_beta_from_gram(factors: Sequence[np.ndarray], lam: float,
                                 G_obs: np.ndarray) -> tuple[float, float]:
    """(beta, lambda_max) of Sec. 4.2 from the Gram of the observed rows,
    G_obs = K_S^T K_S.  The nonzero eigenvalues of
    L_{S-bar,S-bar} = K_{S-bar} (K^T K + lam I)^-1 K_{S-bar}^T are those of the
    pencil (K_{S-bar}^T K_{S-bar}, K^T K + lam I), and
    K_{S-bar}^T K_{S-bar} = K^T K - G_obs, so lambda_max = 1 - nu_min with nu_min
    the smallest eigenvalue of the pencil (G_obs + lam I, K^T K + lam I)."""
    K = CU.kron_matrix(factors)
    d = K.shape[1]
    from scipy.linalg import eigh
    nu = eigh(G_obs + lam * np.eye(d), K.T @ K + lam * np.eye(d), eigvals_only=True)
    lmax = max(0.0, 1.0 - float(nu.min()))
    return 1.0 / (1.0 + 1.0 / (1.0 - lmax)), lmax


def classical_ridge_ratio_min(factors: Sequence[np.ndarray], lam: float) -> float:
    """c_min = min_t c_t over the components with P_t > 0.  By Lemma 4.1 at lam
    and at 0, l^lam_i(K) = sum_t c_t w_it and l_i(K) = sum_{t: P_t > 0} w_it with
    the same w_it = prod_n (u^(n)_{i_n t_n})^2 >= 0, so every classical score of
    K is at most l^lam_i(K) / c_min."""
    c, _ = ridge_weights(factors, lam)
    return float(c[c > 0].min())


def missing_overestimate_beta(factors: Sequence[np.ndarray], lam: float,
                              beta_miss: float) -> float:
    """beta for the sampler of observed entries (classical product scores of K,
    draws outside S rejected, so the distribution on S is l(K)_i / l(K)(S)) as
    an overestimate of the ridge scores of K_S:
    l_i / l(S) >= l^lam_i(K) / l(S) >= (l^lam(K)(S) / l(S)) beta_miss l^lam_i(K_S) / d_eff(K_S),
    and l^lam(K)(S) / l(S) >= c_min, so beta = c_min beta_miss."""
    return classical_ridge_ratio_min(factors, lam) * beta_miss


def missing_sample_count(factors: Sequence[np.ndarray], lam: float, eps: float, delta: float,
                         beta_miss: float) -> int:
    """Alg. 1 line 3's s for the observed-entry sampler: beta' of Alg. 1 line 2
    with d'_eff = 0 and beta = c_min beta_miss."""
    d = int(np.prod([np.asarray(A).shape[1] for A in factors]))
    beta = missing_overestimate_beta(factors, lam, beta_miss)
    return S.paper_sample_count(d, eps, delta, alg1_beta_prime(beta, d, 0.0))


def ridge_sample_count(factors: Sequence[np.ndarray], lam: float, eps: float,
                       delta: float) -> int:
    """Sample count for rows drawn from the exact lam-ridge scores of K: Alg. 1
    line 3's s with beta' from Eq. beta_prime, taking the scores themselves as
    the overestimate (beta = 1, ||l-hat||_1 = d_eff(K)) and d_eff(K) as the
    lower bound d'_eff."""
    d = int(np.prod([np.asarray(A).shape[1] for A in factors]))
    d_eff = kron_effective_dimension(factors, lam)
    bp = lemma_beta_prime(1.0, d, d_eff, d_eff, d_eff)
    return S.paper_sample_count(d, eps, delta, bp)


# ------------------------------------------- exact sampler of l^lam(K) / d_eff(K)

def ridge_mixture_tables(factors: Sequence[np.ndarray], lam: float):
    """Fixed-point tables: the component CDF over t (row-major, weights c_t)
    and, per mode n and column t_n, the CDF of (u^(n)_{i t_n})^2 over i."""
    c, Us = ridge_weights(factors, lam)
    _, Cc, _ = S.fixed_point_scores(c.reshape(-1))
    if Cc.size == 0 or Cc[-1] == 0:
        raise ValueError("all ridge weights are zero")
    cols = [[S.fixed_point_scores(U[:, t] ** 2)[1] for t in range(U.shape[1])] for U in Us]
    return {"shape": c.shape, "Cc": Cc, "cols": cols}


def draw_rows_ridge(tables, dims: Sequence[int], t: np.ndarray, seed: int, sweep: int):
    """Keys of draws t: component from word 0 of stream 3, then row index i_n
    from the CDF of column t_n of U^(n) with the product sampler's word for
    mode n."""
    N = len(dims)
    t = np.asarray(t, dtype=U64)
    w0 = philox4x64_10(t, U64(3), U64(0), U64(0), U64(seed), U64(sweep))[0]
    Cc = tables["Cc"]
    comp = np.searchsorted(Cc, mulhi64(w0, Cc[-1]), side="right")
    tn = np.unravel_index(comp, tables["shape"])
    words = []
    for s in range((N + 3) // 4):
        words.extend(philox4x64_10(t, U64(s), U64(0), U64(0), U64(seed), U64(sweep)))
    key = np.zeros(t.shape, dtype=U64)
    for n in range(N):
        i = np.zeros(t.shape, dtype=U64)
        for col in np.unique(tn[n]):
            sel = tn[n] == col
            C = tables["cols"][n][col]
            i[sel] = np.searchsorted(C, mulhi64(words[n][sel], C[-1]), side="right")
        key = key * U64(dims[n]) + i
    return key


def ridge_row_probabilities(tables, keys_u: np.ndarray, dims: Sequence[int]) -> np.ndarray:
    """Pr(row) of the sampler: sum over components t (row-major) of
    (q^c_t / Q^c) prod_n (q^(n, t_n)_{i_n} / Q^(n, t_n)), multiplied in mode
    order and summed in component order."""
    idx = S.decode_keys(keys_u, dims)
    Cc = tables["Cc"]
    qc = np.diff(np.concatenate([np.zeros(1, dtype=U64), Cc]))
    Qc = float(Cc[-1])
    p = np.zeros(len(idx[0]))
    for flat in range(qc.size):
        if qc[flat] == 0:
            continue
        tn = np.unravel_index(flat, tables["shape"])
        f = np.full(len(idx[0]), float(qc[flat]) / Qc)
        for n in range(len(dims)):
            C = tables["cols"][n][tn[n]]
            q = np.diff(np.concatenate([np.zeros(1, dtype=U64), C]))
            f = f * (q[idx[n]].astype(np.float64) / float(C[-1]))
        p = p + f
    return p


def sketch_ridge(factors: Sequence[np.ndarray], dims: Sequence[int], lam: float, m: int,
                 seed: int, sweep: int = 0):
    """m draws of the exact ridge sampler, deduplicated, with w = c / (m p)
    (the row scale of Alg. 1 line 6); lam I stays exact in the solve."""
    tables = ridge_mixture_tables(factors, lam)
    keys = draw_rows_ridge(tables, dims, np.arange(m, dtype=U64), seed, sweep)
    ku, cu = S.dedupe(keys)
    p = ridge_row_probabilities(tables, ku, dims)
    return {"keys": ku, "counts": cu, "prob": p, "w": S.sample_weights(cu, p, m), "T": m}


def sketched_core_ridge(X: np.ndarray, factors: Sequence[np.ndarray], lam: float, m: int,
                        seed: int, sweep: int = 0):
    """Sketched core update (Alg. 3's steps) with rows drawn from l^lam(K) / d_eff(K):
    the normal equations of the sample plus lam I, solved by Cholesky."""
    dims = tuple(int(v) for v in X.shape)
    sk = sketch_ridge(factors, dims, lam, m, seed, sweep)
    x = CU.gather_dense(X, sk["keys"], dims)
    G, h, _ = CU.sketched_normal_equations(factors, dims, sk["keys"], sk["w"], x)
    sk.update({"x": x, "G": G, "h": h,
               "g": CU.cholesky_solve(G + lam * np.eye(G.shape[0]), h)})
    return sk
