"""Pins of the oracle's exact and sketched core updates, ALS and adjoint.

* exact core: explicit normal equations (brute force) = Kron-eig route
  (Appendix B, Lemma 4.1 proof) to 1e-12; noiseless recovery as lam -> 0;
  the rows-restricted (missing-entry) version with every row = the dense one;
* sketched core: the deduplicated count form equals Alg. 1's explicit sketch
  matrix S (duplicate rows, entries 1/sqrt(Pr(j) s)); the solve equals
  numpy.linalg.lstsq on S A-bar, S b-bar; E[(SK)^T SK] = K^T K (Thm A.3);
  the (1+eps) guarantee of Thm 3.4 with the paper's sample count;
* ALS (Alg. 2): factor update = explicit K_n; Tucker loss non-increasing;
  RMSE noise floor 0.10 for 1% of entries with N(0,1) noise (Sec. 5);
  exact and sketched ALS reach the same RMSE from the same start (Table 1);
* adjoint: central finite differences of the forward solve.
"""
import numpy as np
import pytest

from oracle import sampling as S, core_update as CU, als as ALS, adjoint as ADJ
from oracle.leverage import leverage_scores


def _problem(dims, ranks, sigma, seed):
    g = np.random.default_rng(seed)
    core = g.standard_normal(ranks)
    F = [g.standard_normal((i, r)) for i, r in zip(dims, ranks)]
    X = ALS.tucker_model(core, F) + sigma * g.standard_normal(dims)
    return X, core, F


@pytest.mark.parametrize("dims,ranks", [((5, 4, 6), (2, 3, 2)), ((3, 4, 3, 5), (2, 2, 1, 3))])
def test_exact_core_two_routes_agree(dims, ranks):
    X, _, F = _problem(dims, ranks, 0.3, 1)
    for lam in (1e-3, 0.5):
        a = CU.exact_core_bruteforce(X, F, lam)
        b = CU.exact_core_kron_eig(X, F, lam)
        assert np.max(np.abs(a - b)) < 1e-12 * max(1.0, np.max(np.abs(a)))


def test_exact_core_noiseless_recovery():
    X, core, F = _problem((12, 10, 9), (3, 2, 4), 0.0, 2)
    g = CU.exact_core_kron_eig(X, F, 1e-12)
    assert np.max(np.abs(g - core.reshape(-1))) < 1e-8


def test_exact_rows_all_observed_equals_dense():
    X, _, F = _problem((7, 6, 5), (2, 3, 2), 0.2, 3)
    keys = np.arange(X.size, dtype=np.uint64)
    a = CU.exact_core_rows(keys, X.reshape(-1), X.shape, F, 0.1)
    b = CU.exact_core_kron_eig(X, F, 0.1)
    assert np.max(np.abs(a - b)) < 1e-12


def test_ridge_loss_gram_identity_matches_residual():
    X, _, F = _problem((6, 7, 5), (2, 2, 3), 0.5, 4)
    g = np.random.default_rng(0).standard_normal(12)
    K = CU.kron_matrix(F)
    direct = np.sum((K @ g - X.reshape(-1)) ** 2) + 0.2 * g @ g
    assert abs(CU.ridge_loss_dense(X, F, g, 0.2) - direct) < 1e-10 * direct
    keys = np.arange(X.size, dtype=np.uint64)
    assert abs(CU.ridge_loss_rows(keys, X.reshape(-1), X.shape, F, g, 0.2) - direct) < 1e-10 * direct


@pytest.mark.parametrize("reg", [S.REG_EXACT, S.REG_AUGMENTED])
def test_count_form_equals_explicit_sketch_matrix(reg):
    X, _, F = _problem((6, 5, 4), (2, 2, 2), 0.3, 5)
    dims, d, lam, m = X.shape, 8, 0.4, 3000
    levs = [leverage_scores(A)[0] for A in F]
    keys, T = S.sample_keys(levs, dims, m, 17, 3, reg, d)
    sk = CU.sketch(F, dims, m, 17, 3, reg)
    x = CU.gather_dense(X, sk["keys"], dims)
    G, h, D = CU.sketched_normal_equations(F, dims, sk["keys"], sk["w"], x)
    # Alg. 1 lines 5-8: one row of S per draw, s_{t,j} = 1/sqrt(Pr(j) s)
    n = X.size
    Kfull = CU.kron_matrix(F)
    Abar = np.vstack([Kfull, np.sqrt(lam) * np.eye(d)])
    bbar = np.concatenate([X.reshape(-1), np.zeros(d)])
    p = S.row_probabilities(keys, levs, dims, reg, d)
    SA = Abar[keys.astype(np.int64)] / np.sqrt(p * T)[:, None]
    Sb = bbar[keys.astype(np.int64)] / np.sqrt(p * T)
    if reg == S.REG_EXACT:
        assert np.allclose(G, SA.T @ SA, rtol=1e-13, atol=1e-13 * np.abs(G).max())
    else:
        M = CU.regularised_matrix(G, D, lam, reg)
        assert np.allclose(M, SA.T @ SA, rtol=1e-13, atol=1e-13 * np.abs(M).max())
        g_ls = np.linalg.lstsq(SA, Sb, rcond=None)[0]           # Alg. 1 line 9
        assert np.allclose(CU.cholesky_solve(M, h), g_ls, rtol=1e-9, atol=1e-11)
    assert np.allclose(h, SA.T @ Sb, rtol=1e-13, atol=1e-13 * np.abs(h).max())
    assert n == int(np.prod(dims))


def test_sketched_gram_unbiased():
    _, _, F = _problem((5, 4, 3), (2, 2, 2), 0.0, 6)
    dims = (5, 4, 3)
    K = CU.kron_matrix(F)
    KtK = K.T @ K
    acc = np.zeros_like(KtK)
    reps = 400
    for s in range(reps):
        sk = CU.sketch(F, dims, 64, 1000 + s, 0)
        G, _, _ = CU.sketched_normal_equations(F, dims, sk["keys"], sk["w"],
                                               np.zeros(sk["keys"].size))
        acc += G
    mean = acc / reps
    # leverage sampling of a full-rank K: relative sd of one estimate <~ sqrt(d/m)
    assert np.linalg.norm(mean - KtK) / np.linalg.norm(KtK) < 4 * np.sqrt(8 / 64 / reps)


def test_theorem_3_4_guarantee_with_paper_sample_count():
    X, _, F = _problem((20, 18, 16), (2, 2, 2), 1.0, 7)
    lam, eps, delta = 1e-3, 0.1, 0.1
    s = S.paper_sample_count(8, eps, delta)
    opt = CU.ridge_loss_dense(X, F, CU.exact_core_kron_eig(X, F, lam), lam)
    ok = 0
    for seed in range(10):
        g = CU.sketched_core(X, F, lam, s, seed, 0, S.REG_AUGMENTED)["g"]
        ok += CU.ridge_loss_dense(X, F, g, lam) <= (1 + eps) * opt
    assert ok >= 9                                  # probability >= 1 - delta


def test_sketched_loss_ratio_scales_like_d_over_m():
    X, _, F = _problem((24, 24, 24), (2, 2, 2), 0.5, 8)
    lam = 1e-2
    opt = CU.ridge_loss_dense(X, F, CU.exact_core_kron_eig(X, F, lam), lam)
    ratios = [CU.ridge_loss_dense(X, F, CU.sketched_core(X, F, lam, 800, s)["g"], lam) / opt
              for s in range(20)]
    med = float(np.median(ratios)) - 1.0
    assert 0.0 <= med < 5 * 8 / 800


def test_missing_sketch_all_observed_equals_dense():
    X, _, F = _problem((6, 7, 5), (2, 2, 2), 0.2, 9)
    keys = np.arange(X.size, dtype=np.uint64)
    a = CU.sketched_core(X, F, 0.1, 500, 4, 1)
    b = CU.sketched_core(None, F, 0.1, 500, 4, 1, observed=(keys, X.reshape(-1), X.shape))
    assert np.array_equal(a["keys"], b["keys"]) and np.allclose(a["g"], b["g"], rtol=0, atol=0)


def test_factor_update_matches_explicit_kn():
    X, core, F = _problem((6, 5, 4), (2, 3, 2), 0.3, 10)
    for n in range(3):
        a = ALS.factor_update(X, core, F, n, 0.2)
        b = ALS.factor_update_bruteforce(X, core, F, n, 0.2)
        assert np.max(np.abs(a - b)) < 1e-11


def test_exact_als_loss_non_increasing():
    X, _, _ = _problem((14, 12, 10), (3, 3, 3), 0.1, 11)
    g = np.random.default_rng(1)
    core = g.standard_normal((2, 3, 2))
    F = [g.standard_normal((i, r)) for i, r in zip(X.shape, core.shape)]
    lam = 1e-3
    prev = ALS.tucker_loss(X, core, F, lam)
    for sweep in range(6):
        for n in range(3):
            F[n] = ALS.factor_update(X, core, F, n, lam)
            cur = ALS.tucker_loss(X, core, F, lam)
            assert cur <= prev * (1 + 1e-12)
            prev = cur
        core = CU.exact_core_kron_eig(X, F, lam).reshape(core.shape)
        cur = ALS.tucker_loss(X, core, F, lam)
        assert cur <= prev * (1 + 1e-12)
        prev = cur


def test_rmse_noise_floor_sec5(golden):
    # Sec. 5: N(0,1) noise on one percent of entries lower-bounds the RMSE at 0.10
    fx = golden("rmse_noise_floor.json")
    X, core, F = _problem((60, 60, 60), (2, 2, 2), 0.0, 12)
    g = np.random.default_rng(2)
    mask = g.random(X.shape) < fx["noise_fraction"]
    Y = X + mask * g.standard_normal(X.shape) * fx["noise_std"]
    assert abs(ALS.rmse(Y, core, F) - fx["rmse_floor"]) < 0.005


def test_als_and_sketched_als_same_rmse_table1():
    # Table 1: ALS and ALS-RS from the same start reach RMSEs equal to 3 decimals
    X, _, _ = _problem((30, 28, 26), (3, 3, 3), 0.1, 13)
    g = np.random.default_rng(3)
    core0 = g.standard_normal((3, 3, 3)) * 0.2
    F0 = [g.standard_normal((i, 3)) for i in X.shape]
    c1, f1 = core0, F0
    c2, f2 = core0, F0
    for sweep in range(4):
        c1, f1 = ALS.als_sweep(X, c1, f1, 1e-3)
        c2, f2 = ALS.als_sweep(X, c2, f2, 1e-3, sketched=True, m=20000, seed=5, sweep=sweep)
    assert abs(ALS.rmse(X, c1, f1) - ALS.rmse(X, c2, f2)) < 1e-3


@pytest.mark.parametrize("reg", [S.REG_EXACT, S.REG_AUGMENTED])
def test_adjoint_matches_central_differences(reg):
    X, _, F = _problem((7, 6, 5), (2, 2, 2), 0.3, 14)
    dims, lam = X.shape, 0.3
    sk = CU.sketch(F, dims, 400, 3, 0, reg)
    total = np.uint64(X.size)
    real = sk["keys"] < total
    keys, w = sk["keys"][real], sk["w"][real]
    D = np.ones(8)
    if reg == S.REG_AUGMENTED:
        D = np.zeros(8)
        np.add.at(D, (sk["keys"][~real] - total).astype(np.int64), sk["w"][~real])
        D += 1e-3                                           # keep M positive definite
    x = CU.gather_dense(X, keys, dims)
    gbar = np.random.default_rng(5).standard_normal(8)
    dA, dx = ADJ.backward(F, dims, keys, w, x, lam, D, gbar)
    h = 1e-6
    g = np.random.default_rng(6)
    for _ in range(8):
        dirs = [g.standard_normal(A.shape) for A in F]
        dirx = g.standard_normal(x.shape)
        fp = ADJ.forward([A + h * e for A, e in zip(F, dirs)], dims, keys, w, x + h * dirx, lam, D)
        fm = ADJ.forward([A - h * e for A, e in zip(F, dirs)], dims, keys, w, x - h * dirx, lam, D)
        fd = (fp - fm) @ gbar / (2 * h)
        an = sum(np.sum(a * e) for a, e in zip(dA, dirs)) + dx @ dirx
        assert abs(fd - an) < 1e-7 * max(1.0, abs(an))


@pytest.mark.parametrize("dims,ranks", [((40,), (3,)), ((8, 9), (3, 2)),
                                         ((5, 4, 3, 4), (2, 1, 2, 3))])
def test_adjoint_other_orders_match_central_differences(dims, ranks):
    """Orders 1, 2 and 4 (with a rank-1 mode): the contraction over the other
    modes is empty, a single product, or three products."""
    X, _, F = _problem(dims, ranks, 0.3, 15)
    d, lam = int(np.prod(ranks)), 0.2
    sk = CU.sketch(F, dims, 300, 4, 0, S.REG_EXACT)
    keys, w = sk["keys"], sk["w"]
    x = CU.gather_dense(X, keys, dims)
    gbar = np.random.default_rng(7).standard_normal(d)
    dA, dx = ADJ.backward(F, dims, keys, w, x, lam, np.ones(d), gbar)
    h = 1e-6
    g = np.random.default_rng(8)
    for _ in range(6):
        dirs = [g.standard_normal(A.shape) for A in F]
        dirx = g.standard_normal(x.shape)
        fp = ADJ.forward([A + h * e for A, e in zip(F, dirs)], dims, keys, w, x + h * dirx, lam,
                         np.ones(d))
        fm = ADJ.forward([A - h * e for A, e in zip(F, dirs)], dims, keys, w, x - h * dirx, lam,
                         np.ones(d))
        fd = (fp - fm) @ gbar / (2 * h)
        an = sum(np.sum(a * e) for a, e in zip(dA, dirs)) + dx @ dirx
        assert abs(fd - an) < 1e-7 * max(1.0, abs(an))


def test_sampled_row_products_equal_explicit_rows():
    """K_S g and K_S^T c against an explicit K indexed by the decoded keys."""
    g = np.random.default_rng(7)
    F = [g.standard_normal((5, 2)), g.standard_normal((4, 3)), g.standard_normal((3, 2))]
    dims = (5, 4, 3)
    keys = np.sort(g.choice(60, 25, replace=False)).astype(np.uint64)
    idx = S.decode_keys(keys, dims)
    K = CU.kron_matrix(F)[keys.astype(np.int64)]
    v = g.standard_normal(12)
    c = g.standard_normal(25)
    assert np.allclose(CU.sampled_rows_apply(F, idx, v, chunk=7), K @ v, rtol=1e-13, atol=1e-13)
    assert np.allclose(CU.sampled_rows_apply_t(F, idx, c, chunk=7), K.T @ c, rtol=1e-13, atol=1e-13)



def test_gram_regrouped_by_leading_index():
    """The sampled Gram regrouped by the leading index (the structure of the
    Kronecker rows, Sec. 4): with k_u = a_1(u) (x) b_u, b_u = a_2 (x) ... (x) a_N,
    sum_u w_u k_u k_u^T = sum_{i_1} (a_1 a_1^T) (x) M_{i_1},
    M_{i_1} = sum_{u: i_1(u) = i_1} w_u b_u b_u^T (row-major vec, r_1 outermost)."""
    g = np.random.default_rng(9)
    dims, ranks = (6, 5, 4), (3, 2, 2)
    F = [g.standard_normal((i, r)) for i, r in zip(dims, ranks)]
    keys = np.sort(g.choice(int(np.prod(dims)), 40, replace=False)).astype(np.uint64)
    w = g.random(keys.size) + 0.5
    idx = S.decode_keys(keys, dims)
    K = CU.kron_matrix(F)[keys.astype(np.int64)]
    G = K.T @ (K * w[:, None])
    d1 = ranks[1] * ranks[2]
    Gr = np.zeros_like(G)
    for i1 in np.unique(idx[0]):
        sel = idx[0] == i1
        B = np.stack([np.kron(F[1][a], F[2][b]) for a, b in zip(idx[1][sel], idx[2][sel])])
        M = B.T @ (B * w[sel][:, None])
        a1 = F[0][i1]
        Gr += np.kron(np.outer(a1, a1), M)
    assert M.shape == (d1, d1)
    assert np.allclose(Gr, G, rtol=1e-12, atol=1e-12)
