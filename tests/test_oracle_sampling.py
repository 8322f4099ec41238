"""Pins of the oracle's factored sampler, dedupe and weights.

* inverse CDF: against a linear scan with Python-integer arithmetic;
* distribution: chi-square fit of 2^20 draws to the product of the factor
  distributions (Lemma 4.1 at lam = 0);
* augmented distribution D(l, 0) of Sec. 3: coin and regulariser-row index;
* missing entries: accepted keys are observed, counter order, T, draw limit;
* Alg. 1 sample count (line 3) at d = 8 against the value derived by hand;
* weights: sum_u w_u = sum over draws of 1/(T p) (each draw's squared scale).
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import sampling as S
from oracle.philox import philox4x64_10


def test_fixed_point_scores_exact_values():
    q, C, Q = S.fixed_point_scores(np.array([0.5, 1.0, 0.0, -1e-17, 1.0 + 1e-12, 2.0 ** -33]))
    assert [int(v) for v in q] == [2 ** 31, 2 ** 32, 0, 0, 2 ** 32, 0]
    assert int(Q) == 2 ** 31 + 2 ** 33 and int(C[1]) == 2 ** 31 + 2 ** 32


def test_inverse_cdf_against_linear_scan():
    g = np.random.default_rng(11)
    lev = g.random(37)
    lev[[3, 4, 20]] = 0.0                          # zero-mass rows
    q, C, Q = S.fixed_point_scores(lev)
    dims = (37,)
    t = np.arange(5000, dtype=np.uint64)
    keys = S.draw_rows([C], dims, t, seed=99, sweep=4)
    w = philox4x64_10(t, np.uint64(0), np.uint64(0), np.uint64(0), np.uint64(99), np.uint64(4))[0]
    Cs = [int(c) for c in C]
    for u, k in zip(w, keys):
        target = (int(u) * int(Q)) >> 64
        i = next(j for j, c in enumerate(Cs) if c > target)
        assert i == int(k)
    assert not np.isin(keys, [3, 4, 20]).any()


def test_inverse_cdf_boundary_convention():
    """At the exact bucket edges: a target of C_i - 1 selects row i, a target of
    C_i the next row with mass (min{i : C_i > floor(u Q / 2^64)}); the words u
    that give those targets are found with Python integers."""
    q = np.array([3, 0, 5, 1, 7], dtype=np.uint64) * np.uint64(2 ** 29)
    C = np.cumsum(q, dtype=np.uint64)
    Q = int(C[-1])
    targets = sorted({t for c in C for t in (int(c) - 1, int(c)) if 0 <= t < Q})
    us = [-(-(t << 64) // Q) for t in targets]          # least u with floor(u Q / 2^64) = t
    for u, t in zip(us, targets):
        assert u < 2 ** 64 and (u * Q) >> 64 == t
    got = S.inverse_cdf(C, np.array(us, dtype=np.uint64))
    expect = [next(j for j in range(C.size) if int(C[j]) > t) for t in targets]
    assert [int(v) for v in got] == expect
    assert 1 not in expect                              # the zero-mass row is never selected


def test_product_distribution_chi_square():
    g = np.random.default_rng(12)
    dims = (5, 3, 4)
    levs = [g.random(n) + 0.05 for n in dims]
    Cs = [S.fixed_point_scores(l)[1] for l in levs]
    n = 1 << 20
    keys = S.draw_rows(Cs, dims, np.arange(n, dtype=np.uint64), seed=5, sweep=0)
    obs = np.bincount(keys.astype(np.int64), minlength=60)
    p = np.ones(1)
    for l in levs:
        q, _, Q = S.fixed_point_scores(l)
        p = np.multiply.outer(p, q / float(Q)).reshape(-1)
    chi = stats.chisquare(obs, p * n)
    assert chi.pvalue > 1e-4
    # the probability formula used for the weights is the same product
    pr = S.row_probabilities(np.arange(60, dtype=np.uint64), levs, dims)
    assert np.allclose(pr, p, rtol=1e-15, atol=0)


def test_augmented_coin_and_index():
    dims = (6, 5)
    levs = [np.full(6, 1 / 3), np.full(5, 0.4)]
    Cs = [S.fixed_point_scores(l)[1] for l in levs]
    d = 6
    n = 1 << 18
    keys = S.draw_rows(Cs, dims, np.arange(n, dtype=np.uint64), 3, 1, S.REG_AUGMENTED, d)
    aug = keys >= 30
    assert abs(aug.mean() - 0.5) < 5 * math.sqrt(0.25 / n)
    j = (keys[aug] - 30).astype(np.int64)
    assert j.min() == 0 and j.max() == d - 1
    assert stats.chisquare(np.bincount(j, minlength=d)).pvalue > 1e-4
    p = S.row_probabilities(np.array([0, 29, 30, 35], dtype=np.uint64), levs, dims,
                            S.REG_AUGMENTED, d)
    assert p[2] == p[3] == 0.5 / d
    assert abs(p[0] + 0.0 - 0.5 * (1 / 6) * (1 / 5)) < 1e-9   # fixed-point rounding only


def test_missing_entry_acceptance():
    g = np.random.default_rng(13)
    dims = (8, 9, 7)
    total = 8 * 9 * 7
    obs = np.sort(g.choice(total, size=50, replace=False)).astype(np.uint64)
    levs = [g.random(n) + 0.1 for n in dims]
    keys, T = S.sample_keys(levs, dims, 300, seed=21, sweep=2, observed_keys=obs, batch=97)
    assert keys.size == 300 and np.isin(keys, obs).all()
    # counter order: the same accepted keys as filtering one long run of draws
    Cs = [S.fixed_point_scores(l)[1] for l in levs]
    allk = S.draw_rows(Cs, dims, np.arange(T, dtype=np.uint64), 21, 2)
    hit = np.isin(allk, obs)
    assert np.array_equal(allk[hit], keys) and hit[-1]
    # all entries observed: identical to the dense sampler with T = m
    full = np.arange(total, dtype=np.uint64)
    k2, T2 = S.sample_keys(levs, dims, 300, 21, 2, observed_keys=full)
    k3, T3 = S.sample_keys(levs, dims, 300, 21, 2)
    assert T2 == T3 == 300 and np.array_equal(k2, k3)
    with pytest.raises(S.DrawLimitError):
        S.sample_keys(levs, dims, 300, 21, 2, observed_keys=obs, max_draws=500)


def test_paper_sample_count_d8():
    # Alg. 1 line 3 with beta' = 1/2, eps = delta = 0.1, d = 8:
    # 4d/beta' = 64; 420 ln(320) = 2422.689...; 64 * 2422.689... = 155052.1 -> 155053
    assert S.paper_sample_count(8, 0.1, 0.1) == 155053
    # the 1/(delta eps) branch wins for tiny delta*eps
    assert S.paper_sample_count(1, 1e-3, 1e-3) == math.ceil(8 * 1e6)


def test_dedupe_and_weights_consistent():
    g = np.random.default_rng(14)
    dims = (3, 4)
    levs = [g.random(3) + 0.2, g.random(4) + 0.2]
    keys, T = S.sample_keys(levs, dims, 5000, 1, 0)
    ku, cu = S.dedupe(keys)
    assert cu.sum() == 5000 and np.all(np.diff(ku.astype(np.int64)) > 0)
    p_u = S.row_probabilities(ku, levs, dims)
    w = S.sample_weights(cu, p_u, T)
    p_all = S.row_probabilities(keys, levs, dims)
    assert abs(w.sum() - np.sum(1.0 / (T * p_all))) < 1e-9 * w.sum()
