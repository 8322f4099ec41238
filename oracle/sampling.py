"""Product-distribution row sampling of the Kronecker design matrix, dedupe, weights.

Oracle module: test infrastructure.  Only tests/, __graft_entry__.smoke() and
bench.py's cpu_baseline / reference leg may import anything under oracle/.

Follows Alg. 3 lines 1-3 (factor leverage scores; a sampler for l(K) built from
the factored scores of Lemma 4.1; one inverse-CDF search per mode, Appendix B
proof of Thm 4.2) and Alg. 1 lines 4-7 (s i.i.d. draws with replacement from
the augmented distribution D(l, d'_eff) of Sec. 3, row scale 1/sqrt(Pr(j) s)).

Readings where the paper is silent (each one is listed in the design notes):
  * sampling arithmetic: q_i = floor(clamp(l_i, 0, 1) * 2^32) (uint64), C the
    inclusive prefix sum, Q = C[-1]; a 64-bit uniform u picks
    i = min{i : C_i > floor(u * Q / 2^64)}; p_i = q_i / Q exactly;
  * random numbers: Philox4x64-10, key (seed, sweep), counter (t, stream, 0, 0);
    mode n of draw t uses word n % 4 of stream n // 4; the augmented coin is
    the top bit of word 0 of stream 2 (0 = a row of K), the augmented row
    index is floor(u * d / 2^64) with u word 1 of stream 2;
  * augmented mode with d'_eff = 0 (Alg. 3 line 4): half the mass on rows of K
    (classical scores normalised to sum d), half on the d regulariser rows;
  * missing entries: draws from the full product distribution are accepted in
    counter order while their key is observed, until m are accepted; T = the
    number of draws used; regulariser rows are always accepted.
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence

import numpy as np

from .philox import philox4x64_10, mulhi64

U64 = np.uint64
TWO32 = 4294967296.0

REG_EXACT = 0
REG_AUGMENTED = 1


class DrawLimitError(RuntimeError):
    """Missing-entry sampling used max_draws draws before m were accepted."""


def fixed_point_scores(lev: np.ndarray):
    """(q, C, Q): q_i = floor(clamp(l_i,0,1) * 2^32), C = inclusive prefix sum, Q = C[-1]."""
    lev = np.asarray(lev, dtype=np.float64)
    q = np.floor(np.clip(lev, 0.0, 1.0) * TWO32).astype(U64)
    C = np.cumsum(q, dtype=U64)
    Q = U64(C[-1]) if C.size else U64(0)
    return q, C, Q


def paper_sample_count(d: int, eps: float, delta: float, beta_prime: float = 0.5) -> int:
    """s = ceil(4d/beta' * max{420 ln(4d/delta), 1/(delta eps)})  (Alg. 1 line 3).

    With classical leverage scores of K and d'_eff = 0, Cor. 3.3 gives
    beta' >= 1/2, which is the value used.
    """
    return int(math.ceil(4.0 * d / beta_prime *
                         max(420.0 * math.log(4.0 * d / delta), 1.0 / (delta * eps))))


def inverse_cdf(C: np.ndarray, u: np.ndarray) -> np.ndarray:
    """min{i : C_i > floor(u * Q / 2^64)}, Q = C[-1]: the row a 64-bit uniform
    word u selects from fixed-point weights with inclusive prefix sums C."""
    return np.searchsorted(C, mulhi64(u, C[-1]), side="right")


def _mode_words(t: np.ndarray, n_modes: int, seed: int, sweep: int):
    """Uniform 64-bit words, one per mode, for draws t (list of N arrays)."""
    words = []
    for s in range((n_modes + 3) // 4):
        w = philox4x64_10(t, U64(s), U64(0), U64(0), U64(seed), U64(sweep))
        words.extend(w)
    return words[:n_modes]


def draw_rows(C_list: Sequence[np.ndarray], dims: Sequence[int], t: np.ndarray,
              seed: int, sweep: int, reg: int = REG_EXACT, d: int = 0):
    """Keys of draws t (row-major linear row index of K, or prod(I)+j for an
    augmented regulariser row j).  One upper-bound search per mode."""
    N = len(dims)
    t = np.asarray(t, dtype=U64)
    words = _mode_words(t, N, seed, sweep)
    key = np.zeros(t.shape, dtype=U64)
    for n in range(N):
        i = inverse_cdf(C_list[n], words[n]).astype(U64)
        key = key * U64(dims[n]) + i
    if reg == REG_AUGMENTED:
        w0, w1, _, _ = philox4x64_10(t, U64(2), U64(0), U64(0), U64(seed), U64(sweep))
        aug = (w0 >> U64(63)) == U64(1)
        j = mulhi64(w1, U64(d))
        total = U64(int(np.prod([int(x) for x in dims])))
        key = np.where(aug, total + j, key)
    return key


def sample_keys(lev_list: Sequence[np.ndarray], dims: Sequence[int], m: int, seed: int,
                sweep: int, reg: int = REG_EXACT, d: int = 0,
                observed_keys: Optional[np.ndarray] = None, max_draws: int = 0,
                batch: int = 1 << 20):
    """(keys of the m accepted draws in counter order, T = draws used)."""
    C_list = [fixed_point_scores(l)[1] for l in lev_list]
    for C in C_list:
        if C.size == 0 or C[-1] == 0:
            raise ValueError("a factor has zero total leverage")
    if observed_keys is None:
        t = np.arange(m, dtype=U64)
        return draw_rows(C_list, dims, t, seed, sweep, reg, d), m
    total = U64(int(np.prod([int(x) for x in dims])))
    obs = np.asarray(observed_keys, dtype=U64)
    acc: List[np.ndarray] = []
    n_acc = 0
    t0 = 0
    limit = max_draws if max_draws > 0 else 1 << 62
    while n_acc < m:
        if t0 >= limit:
            raise DrawLimitError(f"{n_acc} of {m} accepted after {t0} draws")
        nb = min(batch, limit - t0)
        t = np.arange(t0, t0 + nb, dtype=U64)
        k = draw_rows(C_list, dims, t, seed, sweep, reg, d)
        pos = np.searchsorted(obs, k)
        hit = (k >= total) | ((pos < obs.size) & (obs[np.minimum(pos, obs.size - 1)] == k))
        idx = np.flatnonzero(hit)
        need = m - n_acc
        if idx.size >= need:
            acc.append(k[idx[:need]])
            return np.concatenate(acc), t0 + int(idx[need - 1]) + 1
        acc.append(k[idx])
        n_acc += idx.size
        t0 += nb
    return np.concatenate(acc), t0


def dedupe(keys: np.ndarray):
    """Sorted unique keys and their multiplicities (equal sampled rows merge)."""
    return np.unique(np.asarray(keys, dtype=U64), return_counts=True)


def decode_keys(keys: np.ndarray, dims: Sequence[int]):
    """Row-major multi-index (i_1..i_N) of real-row keys (list of int64 arrays)."""
    rem = np.asarray(keys, dtype=U64).copy()
    out = []
    for n in range(len(dims) - 1, -1, -1):
        out.append((rem % U64(dims[n])).astype(np.int64))
        rem = rem // U64(dims[n])
    return out[::-1]


def row_probabilities(keys_u: np.ndarray, lev_list: Sequence[np.ndarray], dims: Sequence[int],
                      reg: int = REG_EXACT, d: int = 0) -> np.ndarray:
    """Pr(row) under the sampling distribution: prod_n q_{i_n}/Q_n (Lemma 4.1 at
    lam=0), halved in augmented mode; an augmented row has 1/(2d).

    Evaluated in the fixed order p = q_1/Q_1; p = p * (q_n/Q_n) for n = 2..N;
    then p = 0.5 * p in augmented mode.
    """
    keys_u = np.asarray(keys_u, dtype=U64)
    total = U64(int(np.prod([int(x) for x in dims])))
    aug = keys_u >= total
    idx = decode_keys(np.where(aug, U64(0), keys_u), dims)
    p = None
    for n, lev in enumerate(lev_list):
        q, _, Q = fixed_point_scores(lev)
        f = q[idx[n]].astype(np.float64) / float(Q)
        p = f if p is None else p * f
    if reg == REG_AUGMENTED:
        p = 0.5 * p
        p = np.where(aug, 0.5 / float(d), p)
    return p


def sample_weights(counts: np.ndarray, p: np.ndarray, T: int) -> np.ndarray:
    """w_u = c_u / (T * p_u): the squared row scale 1/(Pr(j) s) of Alg. 1 line 6,
    summed over the c_u copies of a row."""
    return np.asarray(counts, dtype=np.float64) / (float(T) * np.asarray(p, dtype=np.float64))
