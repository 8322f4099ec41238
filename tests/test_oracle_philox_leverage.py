"""Pins of the oracle's generator and leverage scores against independent facts.

Philox4x64-10 is checked against numpy's own Philox bit generator (a library
implementation of the same published generator); the 128-bit product against
Python integers.  Leverage scores are checked against the SVD form
(Eq. ridge_leverage_score_svd_def, computed by LAPACK's SVD rather than the
Gram pseudo-inverse the oracle uses), sum = rank (Eq. d_eff_def at lam = 0),
0 <= l <= 1, l^lam <= l, Lemma 3.1, Lemma 4.1 on an explicit Kronecker
product, Lemma 4.4, Thm 4.3's exact update formula and bound, and the
corollary's lambda_max bound (Appendix B).
"""
import numpy as np
import pytest

from oracle import philox, leverage as LV
from oracle.core_update import kron_matrix


def test_philox_matches_numpy_bitgenerator():
    g = np.random.default_rng(7)
    for _ in range(50):
        c = [int(v) for v in g.integers(0, 2**63, size=4, dtype=np.int64)]
        c[0] |= 1                      # numpy pre-increments the counter: avoid borrow
        k = [int(v) for v in g.integers(0, 2**63, size=2, dtype=np.int64)]
        ctr = c[0] + (c[1] << 64) + (c[2] << 128) + (c[3] << 192)
        bg = np.random.Philox(key=k[0] + (k[1] << 64), counter=ctr - 1)
        ref = bg.random_raw(4)
        out = philox.philox4x64_10(c[0], c[1], c[2], c[3], k[0], k[1])
        assert [int(x) for x in out] == [int(x) for x in ref]


def test_philox_counter_zero_and_carry():
    # counter 0 (numpy wraps its all-ones counter to 0 before generating)
    bg = np.random.Philox(key=0, counter=(1 << 256) - 1)
    assert [int(x) for x in philox.philox4x64_10(0, 0, 0, 0, 0, 0)] == \
        [int(x) for x in bg.random_raw(4)]
    # counter word 0 = 0 with word 1 = 3 (the carry path of numpy's increment)
    bg = np.random.Philox(key=11, counter=(3 << 64) - 1)
    assert [int(x) for x in philox.philox4x64_10(0, 3, 0, 0, 11, 0)] == \
        [int(x) for x in bg.random_raw(4)]


def test_mulhilo64_against_python_ints():
    g = np.random.default_rng(3)
    a = g.integers(0, 2**64 - 1, size=1000, dtype=np.uint64, endpoint=True)
    b = g.integers(0, 2**64 - 1, size=1000, dtype=np.uint64, endpoint=True)
    a[:3] = [0, 2**64 - 1, 2**64 - 1]
    b[:3] = [2**64 - 1, 2**64 - 1, 1]
    hi, lo = philox.mulhilo64(a, b)
    for x, y, h, l in zip(a, b, hi, lo):
        p = int(x) * int(y)
        assert int(h) == p >> 64 and int(l) == p & (2**64 - 1)


def _rank_deficient(n, r, k, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal((n, k)) @ g.standard_normal((k, r))


@pytest.mark.parametrize("shape,k", [((40, 5), 5), ((40, 6), 3), ((7, 7), 7), ((9, 4), 1)])
def test_leverage_sum_is_rank_and_bounded(shape, k):
    A = _rank_deficient(shape[0], shape[1], k, 1)
    lev, rank = LV.leverage_scores(A)
    assert rank == k
    # the Gram route squares the condition number: allow kappa^2 * eps
    s = np.linalg.svd(A, compute_uv=False)[:k]
    tol = 1e-13 + 50 * (s[0] / s[-1]) ** 2 * np.finfo(float).eps
    assert abs(lev.sum() - k) < tol
    assert lev.min() > -tol and lev.max() < 1 + tol


def test_leverage_equals_svd_form():
    A = np.random.default_rng(2).standard_normal((30, 6))
    U, s, _ = np.linalg.svd(A, full_matrices=False)
    lam = 0.7
    ref0 = np.sum(U ** 2, axis=1)
    refl = np.sum(U ** 2 * (s ** 2 / (s ** 2 + lam)), axis=1)
    assert np.allclose(LV.leverage_scores(A)[0], ref0, rtol=0, atol=1e-13)
    assert np.allclose(LV.ridge_leverage_scores(A, lam), refl, rtol=0, atol=1e-13)
    # ridge scores never exceed classical scores; d_eff = sum s^2/(s^2+lam) <= r
    assert np.all(LV.ridge_leverage_scores(A, lam) <= ref0 + 1e-14)
    assert abs(LV.effective_dimension(A, lam) - np.sum(s ** 2 / (s ** 2 + lam))) < 1e-12


def test_lemma_3_1_augmented_matrix():
    A = np.random.default_rng(4).standard_normal((25, 5))
    lam = 2.5
    Abar = np.vstack([A, np.sqrt(lam) * np.eye(5)])
    assert np.allclose(LV.ridge_leverage_scores(A, lam), LV.leverage_scores(Abar)[0][:25],
                       rtol=0, atol=1e-13)


def test_lemma_4_1_kronecker_scores():
    g = np.random.default_rng(5)
    F = [g.standard_normal((4, 3)), g.standard_normal((5, 2)), g.standard_normal((3, 2))]
    K = kron_matrix(F)
    # lam = 0: scores and cross scores of K factor into products over the modes
    lk = LV.leverage_scores(K)[0]
    prod = np.ones(1)
    for A in F:
        prod = np.multiply.outer(prod, LV.leverage_scores(A)[0]).reshape(-1)
    assert np.allclose(lk, prod, rtol=0, atol=1e-12)
    L = LV.cross_ridge_leverage_scores(K)
    Lp = np.ones((1, 1))
    for A in F:
        Lp = np.kron(Lp, LV.cross_ridge_leverage_scores(A))
    assert np.allclose(L, Lp, rtol=0, atol=1e-12)
    # lam > 0: the SVD formula of Lemma 4.1
    lam = 0.3
    svds = [np.linalg.svd(A, full_matrices=False) for A in F]
    Ukr = kron_matrix([u for u, _, _ in svds])
    s2 = np.ones(1)
    for _, s, _ in svds:
        s2 = np.multiply.outer(s2, s ** 2).reshape(-1)
    lam_k = (Ukr * (s2 / (s2 + lam))) @ Ukr.T
    assert np.allclose(LV.cross_ridge_leverage_scores(K, lam), lam_k, rtol=0, atol=1e-12)


@pytest.mark.parametrize("lam", [0.0, 0.5, 4.0])
def test_lemma_4_4_sum_of_squared_cross_scores(lam):
    A = np.random.default_rng(6).standard_normal((20, 4))
    L = LV.cross_ridge_leverage_scores(A, lam)
    lhs = np.sum(L ** 2, axis=1)
    li = np.diag(L)
    if lam == 0.0:
        assert np.allclose(lhs, li, rtol=0, atol=1e-13)
    else:
        assert np.all(lhs < li)


def test_theorem_4_3_row_removal_formula_and_bound():
    g = np.random.default_rng(8)
    A = g.standard_normal((18, 4))
    lam = 0.8
    missing = np.array([1, 4, 5, 11, 17])
    keep = np.setdiff1d(np.arange(18), missing)
    L = LV.cross_ridge_leverage_scores(A, lam)
    Lss = L[np.ix_(missing, missing)]
    after = LV.ridge_leverage_scores(A[keep], lam)
    inv = np.linalg.inv(np.eye(missing.size) - Lss)
    lmax = np.linalg.eigvalsh(Lss).max()
    for pos, i in enumerate(keep):
        li_s = L[i, missing]
        exact = L[i, i] + li_s @ inv @ li_s            # Eq. ridge_score_update_formula
        assert abs(after[pos] - exact) < 1e-12
        bound = L[i, i] + np.sum(li_s ** 2) / (1 - lmax)
        assert after[pos] <= bound + 1e-12
    # corollary: 1/(1 - lmax(L_SS)) <= 1 + prod ||A^(n)||_2^2 / lam (here N = 1)
    assert 1 / (1 - lmax) <= 1 + np.linalg.norm(A, 2) ** 2 / lam + 1e-12
