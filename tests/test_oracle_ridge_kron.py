"""Pins of oracle.ridge_kron: the lam-ridge leverage scores of K = A^(1) (x) ... (x) A^(N)
by Lemma 4.1, d_eff(K), the overestimate constants that set the sample count
(Cor. leverage_score_overestimate, Eq. beta_prime, Alg. 1 line 2, the missing-entry
beta of Sec. 4.2 and its corollary bound), and the exact mixture sampler of
l^lam(K) / d_eff(K).

Each is checked against the explicit K (brute force through the pseudo-inverse
definition of Eq. ridge_leverage_score_def), against the definition of a
beta-overestimate, or statistically (chi-square, unbiasedness over seeds)."""
import numpy as np
import pytest
from scipy import stats
from scipy.linalg import eigh

from oracle import core_update as CU, leverage as LV, ridge_kron as RK, sampling as S


def _factors(seed, shapes, dup=None):
    g = np.random.default_rng(seed)
    F = [g.standard_normal(s) for s in shapes]
    if dup is not None:                  # rank-deficient factor: a repeated column
        n, a, b = dup
        F[n][:, b] = F[n][:, a]
    return F


def _all_rows(dims):
    keys = np.arange(int(np.prod(dims)), dtype=np.uint64)
    return keys, S.decode_keys(keys, dims)


SHAPES = [((4, 3), (5, 2), (3, 2)), ((6, 3), (2, 3), (4, 2))]   # the second has I_2 < R_2


@pytest.mark.parametrize("lam", [0.0, 0.3, 5.0])
@pytest.mark.parametrize("shapes,dup", [(SHAPES[0], None), (SHAPES[0], (0, 0, 2)),
                                        (SHAPES[1], None)])
def test_lemma_4_1_ridge_scores_equal_explicit_k(lam, shapes, dup):
    F = _factors(31, shapes, dup)
    dims = tuple(s[0] for s in shapes)
    K = CU.kron_matrix(F)
    _, idx = _all_rows(dims)
    got = RK.kron_ridge_leverage_scores(F, lam, idx)
    assert np.allclose(got, LV.ridge_leverage_scores(K, lam), rtol=0, atol=1e-12)
    # cross scores of random row pairs against the explicit cross-score matrix
    L = LV.cross_ridge_leverage_scores(K, lam)
    g = np.random.default_rng(32)
    a = g.integers(0, K.shape[0], 50)
    b = g.integers(0, K.shape[0], 50)
    ia = S.decode_keys(a.astype(np.uint64), dims)
    ib = S.decode_keys(b.astype(np.uint64), dims)
    assert np.allclose(RK.kron_cross_ridge_leverage(F, lam, ia, ib), L[a, b], rtol=0, atol=1e-12)


@pytest.mark.parametrize("dup", [None, (1, 0, 1)])
def test_effective_dimension_of_k(dup):
    F = _factors(33, SHAPES[0], dup)
    K = CU.kron_matrix(F)
    d = K.shape[1]
    rank = RK.kron_rank(F)
    assert rank == np.linalg.matrix_rank(K)
    assert abs(RK.kron_effective_dimension(F, 0.0) - rank) < 1e-12
    prev = float(rank)
    for lam in (1e-3, 0.1, 1.0, 10.0, 1e3):
        de = RK.kron_effective_dimension(F, lam)
        # the explicit route sees the numerically zero eigenvalues of K^T K (about
        # eps ||K||^2) as eps ||K||^2 / (eps ||K||^2 + lam): up to ~1e-11 at lam = 1e-3
        assert abs(de - LV.effective_dimension(K, lam)) < 1e-9
        assert 0 < de < prev <= d                    # shrinks as lam grows
        prev = de


@pytest.mark.parametrize("lam", [0.0, 0.5, 20.0])
def test_classical_scores_overestimate_ridge_scores(lam):
    F = _factors(34, SHAPES[0])
    K = CU.kron_matrix(F)
    beta = RK.classical_overestimate_beta(F, lam)
    lc = LV.leverage_scores(K)[0]
    lr = LV.ridge_leverage_scores(K, lam)
    assert 0 < beta <= 1 + 1e-15
    # Def. of a beta-overestimate: lhat_i / ||lhat||_1 >= beta l_i / ||l||_1 for every row
    assert np.all(lc / lc.sum() >= beta * lr / lr.sum() - 1e-15)
    if lam == 0.0:
        assert abs(beta - 1.0) < 1e-12


def test_alg1_beta_prime_special_cases():
    # classical scores of K with d'_eff = 0: beta' = 1/2 (the value the sampler's count uses)
    assert RK.alg1_beta_prime(1.0, 8, 0.0) == 0.5
    assert RK.alg1_beta_prime(2.0, 8, 8.0) == 1.0
    assert abs(RK.alg1_beta_prime(0.3, 8, 7.75) - 0.3 / 1.25) < 1e-15


@pytest.mark.parametrize("lam", [0.2, 3.0])
def test_lemma_beta_overestimate_on_augmented_matrix(lam):
    """Eq. beta_prime holds for D(lhat, d'_eff) against the leverage scores of
    A-bar = [A; sqrt(lam) I], and Alg. 1's beta' is a lower bound of it."""
    A = np.random.default_rng(35).standard_normal((20, 4))
    d = A.shape[1]
    Abar = np.vstack([A, np.sqrt(lam) * np.eye(d)])
    lbar = LV.leverage_scores(Abar)[0]
    target = lbar / lbar.sum()                              # ||l(A-bar)||_1 = d
    d_eff = LV.effective_dimension(A, lam)
    lc = LV.leverage_scores(A)[0]
    lhat = lc * d / lc.sum()                                # normalised to ||lhat||_1 = d
    beta = d_eff / d                                        # Cor. leverage_score_overestimate
    for d_low in (0.0, 0.5 * d_eff, d_eff):
        pmf = RK.augmented_pmf(lhat, d, d_low)
        bp = RK.lemma_beta_prime(beta, d, d_eff, d_low, lhat.sum())
        assert np.all(pmf >= bp * target - 1e-15)
        assert RK.alg1_beta_prime(beta, d, d_low) <= bp + 1e-15


def test_missing_entry_beta_and_bound():
    F = _factors(36, SHAPES[0])
    dims = (4, 5, 3)
    K = CU.kron_matrix(F)
    lam = 0.7
    g = np.random.default_rng(37)
    obs = np.sort(g.choice(K.shape[0], 42, replace=False))
    beta = RK.missing_ridge_beta(F, lam, obs, dims)
    assert 0 < beta <= 0.5 + 1e-15
    # the ridge scores of K on the observed rows are a beta-overestimate for the
    # ridge scores of the observed rows' matrix
    l_k = LV.ridge_leverage_scores(K, lam)[obs]
    l_obs = LV.ridge_leverage_scores(K[obs], lam)
    assert np.all(l_k / l_k.sum() >= beta * l_obs / l_obs.sum() - 1e-15)
    assert RK.missing_ridge_beta_bound(F, lam) <= beta + 1e-15
    # the formula itself, with lambda_max(L_{S-bar,S-bar}) by an independent route: the
    # generalized eigenproblem K_{S-bar}^T K_{S-bar} v = mu (K^T K + lam I) v has the same
    # nonzero eigenvalues as K_{S-bar} (K^T K + lam I)^-1 K_{S-bar}^T
    miss = np.setdiff1d(np.arange(K.shape[0]), obs)
    mu = eigh(K[miss].T @ K[miss], K.T @ K + lam * np.eye(K.shape[1]), eigvals_only=True).max()
    assert abs(1.0 / beta - (1.0 + 1.0 / (1.0 - mu))) < 1e-10 / beta
    assert RK.missing_ridge_beta(F, lam, np.arange(K.shape[0]), dims) == 1.0


@pytest.mark.parametrize("lam", [0.0, 0.4, 6.0])
def test_ridge_sampler_probabilities_are_the_ridge_distribution(lam):
    F = _factors(38, SHAPES[0])
    dims = (4, 5, 3)
    keys, idx = _all_rows(dims)
    tab = RK.ridge_mixture_tables(F, lam)
    p = RK.ridge_row_probabilities(tab, keys, dims)
    assert abs(p.sum() - 1.0) < 1e-12
    exact = RK.kron_ridge_leverage_scores(F, lam, idx) / RK.kron_effective_dimension(F, lam)
    # fixed-point weights: each q / Q is exact to about 2^-32 of its normaliser
    assert np.max(np.abs(p - exact)) < 1e-8
    if lam == 0.0:                      # reduces to the product of the classical scores
        levs = [LV.leverage_scores(A)[0] for A in F]
        assert np.max(np.abs(p - S.row_probabilities(keys, levs, dims))) < 1e-8


def test_ridge_sampler_chi_square_and_determinism():
    F = _factors(39, SHAPES[0])
    dims = (4, 5, 3)
    lam = 2.0
    keys_all, _ = _all_rows(dims)
    tab = RK.ridge_mixture_tables(F, lam)
    n = 1 << 18
    t = np.arange(n, dtype=np.uint64)
    keys = RK.draw_rows_ridge(tab, dims, t, seed=7, sweep=1)
    obs = np.bincount(keys.astype(np.int64), minlength=keys_all.size)
    p = RK.ridge_row_probabilities(tab, keys_all, dims)
    nz = p > 0
    assert obs[~nz].sum() == 0
    assert stats.chisquare(obs[nz], p[nz] * n).pvalue > 1e-4
    again = RK.draw_rows_ridge(tab, dims, t[:1000], seed=7, sweep=1)
    assert np.array_equal(again, keys[:1000])
    other = RK.draw_rows_ridge(tab, dims, t[:1000], seed=7, sweep=2)
    assert not np.array_equal(other, keys[:1000])


def test_ridge_sketch_gram_unbiased():
    F = _factors(40, ((5, 2), (4, 2), (3, 2)))
    dims = (5, 4, 3)
    K = CU.kron_matrix(F)
    KtK = K.T @ K
    acc = np.zeros_like(KtK)
    reps = 400
    for s in range(reps):
        sk = RK.sketch_ridge(F, dims, 1.5, 64, 2000 + s)
        G, _, _ = CU.sketched_normal_equations(F, dims, sk["keys"], sk["w"],
                                               np.zeros(sk["keys"].size))
        acc += G
    mean = acc / reps
    assert np.linalg.norm(mean - KtK) / np.linalg.norm(KtK) < 4 * np.sqrt(8 / 64 / reps)


def test_ridge_sketched_core_loss_ratio():
    g = np.random.default_rng(41)
    dims, ranks = (20, 18, 16), (2, 2, 2)
    F = [g.standard_normal((i, r)) for i, r in zip(dims, ranks)]
    core = g.standard_normal(ranks)
    X = core
    for n, A in enumerate(F):
        X = CU.mode_product(X, A, n)
    X = X + 0.5 * g.standard_normal(dims)
    lam = 5.0
    opt = CU.ridge_loss_dense(X, F, CU.exact_core_kron_eig(X, F, lam), lam)
    ratios = [CU.ridge_loss_dense(X, F, RK.sketched_core_ridge(X, F, lam, 800, s)["g"], lam) / opt
              for s in range(10)]
    assert 1.0 <= min(ratios) and float(np.median(ratios)) < 1 + 5 * 8 / 800


def test_ridge_sample_count_alg1_with_exact_ridge_scores():
    # Alg. 1 line 3 with beta' from Eq. beta_prime for the exact ridge scores of K
    # (beta = 1, ||l-hat||_1 = d_eff, d'_eff = d_eff): d_eff from the explicit K
    F = _factors(35, SHAPES[0])
    K = CU.kron_matrix(F)
    d = K.shape[1]
    prev = None
    for lam in (1e-2, 1.0, 10.0, 100.0):
        de = LV.effective_dimension(K, lam)                       # explicit, Eq. d_eff_def
        mlt = min(1.0, d - de)
        bp = d / (de + d * mlt)                                    # both terms of Eq. beta_prime
        s = RK.ridge_sample_count(F, lam, 0.1, 0.1)
        assert s == S.paper_sample_count(d, 0.1, 0.1, bp)
        assert 0.5 <= bp <= 1.0
        # once d - d_eff >= 1, beta' = d / (d_eff + d) grows as d_eff shrinks: fewer rows
        # (below that, min{1, d - d_eff} itself shrinks and beta' tends to 1 as d_eff -> d)
        if d - de >= 1.0:
            if prev is not None:
                assert s <= prev
            prev = s
    # lam -> 0 with full-rank factors: d_eff -> d, beta' -> 1, half the classical count
    s0 = RK.ridge_sample_count(F, 1e-12, 0.1, 0.1)
    assert s0 == S.paper_sample_count(d, 0.1, 0.1, 1.0)
    assert 2 * s0 in (S.paper_sample_count(d, 0.1, 0.1, 0.5), S.paper_sample_count(d, 0.1, 0.1, 0.5) + 1)


@pytest.mark.parametrize("lam", [0.05, 2.0, 40.0])
@pytest.mark.parametrize("dup", [None, (1, 0, 1)])
def test_classical_scores_bound_ridge_scores_pointwise(lam, dup):
    # c_min against an independent route: the nonzero eigenvalues mu of the explicit
    # K^T K are the products P_t, so c_min = min mu / (mu + lam); every row of the
    # explicit K then satisfies l^lam_i(K) >= c_min l_i(K), with equality on some row
    # when one component carries it alone
    F = _factors(41, SHAPES[0], dup)
    K = CU.kron_matrix(F)
    mu = np.linalg.eigvalsh(K.T @ K)
    mu = mu[mu > 1e-9 * mu.max()]
    cmin = RK.classical_ridge_ratio_min(F, lam)
    assert abs(cmin - float((mu / (mu + lam)).min())) <= 1e-12
    lr = LV.ridge_leverage_scores(K, lam)
    lc = LV.ridge_leverage_scores(K, 0.0)
    assert np.all(lr >= cmin * lc - 1e-13)
    assert np.all(lr <= lc + 1e-13)


@pytest.mark.parametrize("lam", [0.3, 3.0])
@pytest.mark.parametrize("frac", [0.3, 0.7])
def test_missing_overestimate_for_the_observed_entry_sampler(lam, frac):
    # the distribution the observed-entry sampler draws from on S (classical scores of K,
    # the rest rejected) is a (c_min beta_miss)-overestimate of the ridge scores of K_S,
    # by brute force on the explicit K, with beta_miss exact and from the corollary
    F = _factors(43, SHAPES[0])
    dims = (4, 5, 3)
    K = CU.kron_matrix(F)
    g = np.random.default_rng(44)
    obs = np.sort(g.choice(K.shape[0], int(frac * K.shape[0]), replace=False))
    q = LV.ridge_leverage_scores(K, 0.0)[obs]
    q = q / q.sum()
    l_obs = LV.ridge_leverage_scores(K[obs], lam)
    target = l_obs / l_obs.sum()
    for bm in (RK.missing_ridge_beta(F, lam, obs, dims), RK.missing_ridge_beta_bound(F, lam)):
        beta = RK.missing_overestimate_beta(F, lam, bm)
        assert np.all(q >= beta * target - 1e-15)


@pytest.mark.parametrize("lam", [0.1, 1.5])
def test_missing_beta_from_the_observed_gram(lam):
    # the pencil route equals the explicit L_{S-bar,S-bar} route; all rows observed
    # gives lambda_max = 0 (beta = 1/2 by the formula); the bound is below it
    F = _factors(45, SHAPES[1])
    dims = (6, 2, 4)
    K = CU.kron_matrix(F)
    g = np.random.default_rng(46)
    obs = np.sort(g.choice(K.shape[0], 30, replace=False))
    b, lmax = RK.missing_ridge_beta_from_gram(F, lam, K[obs].T @ K[obs])
    assert abs(b - RK.missing_ridge_beta(F, lam, obs, dims)) <= 1e-10
    L = LV.cross_ridge_leverage_scores(K, lam)
    miss = np.setdiff1d(np.arange(K.shape[0]), obs)
    assert abs(lmax - np.linalg.eigvalsh(L[np.ix_(miss, miss)]).max()) <= 1e-10
    assert RK.missing_ridge_beta_bound(F, lam) <= b + 1e-15
    b_all, l_all = RK.missing_ridge_beta_from_gram(F, lam, K.T @ K)
    assert l_all <= 1e-12 and abs(b_all - 0.5) <= 1e-12


def test_missing_sample_count_reduces_to_the_classical_count():
    # lam -> 0 with nothing missing (c_min -> 1, beta_miss = 1): beta' = 1/2, the count
    # Alg. 1 line 3 gives for classical scores; a smaller beta_miss needs more rows
    F = _factors(47, SHAPES[0])
    d = 12
    assert RK.missing_sample_count(F, 1e-14, 0.1, 0.1, 1.0) == S.paper_sample_count(d, 0.1, 0.1)
    s1 = RK.missing_sample_count(F, 1.0, 0.1, 0.1, 0.4)
    s2 = RK.missing_sample_count(F, 1.0, 0.1, 0.1, 0.1)
    assert s2 > s1 > S.paper_sample_count(d, 0.1, 0.1)
