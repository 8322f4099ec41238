"""Pins of the oracle's sketched factor update (oracle.als): the restricted update on
every row of B_n with unit weights is Alg. 2's exact factor update; the design rows
are the columns of the explicit K_n = G_(n) W^T; the count form of the sketch equals
the explicit sampling matrix with repeated rows; the product of the other modes'
leverage scores is an (R_n / prod R_k)-overestimate of the leverage scores of B_n
(brute force on explicit B_n); the sketched Gram B_n^T S^T S B_n is unbiased over
seeds; and ALS with sketched factor and core updates reaches the noise floor of
exact ALS on a small noisy Tucker tensor."""
import numpy as np
import pytest

from oracle import als as ALS, core_update as CU, leverage as LV, sampling as S


def _problem(seed, dims=(9, 8, 7), ranks=(3, 2, 4), sigma=0.1):
    g = np.random.default_rng(seed)
    F = [g.standard_normal((i, r)) for i, r in zip(dims, ranks)]
    G = g.standard_normal(ranks)
    X = ALS.tucker_model(G, F) + sigma * g.standard_normal(dims)
    return X, G, F


@pytest.mark.parametrize("n", [0, 1, 2])
def test_all_rows_with_unit_weights_is_the_exact_update(n):
    X, G, F = _problem(1)
    dims = [d for k, d in enumerate(X.shape) if k != n]
    keys = np.arange(int(np.prod(dims)), dtype=np.uint64)
    A = ALS.factor_update_from_rows(X, G, F, n, 0.3, keys, np.ones(keys.size))
    assert np.allclose(A, ALS.factor_update_bruteforce(X, G, F, n, 0.3), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("n", [0, 2])
def test_design_rows_are_columns_of_explicit_kn(n):
    X, G, F = _problem(2)
    W = CU.kron_matrix([F[k] for k in range(3) if k != n])
    Kn = ALS.unfold(G, n) @ W.T                     # R_n x prod_{k != n} I_k
    dims = [d for k, d in enumerate(X.shape) if k != n]
    keys = np.array([0, 5, 17, int(np.prod(dims)) - 1], dtype=np.uint64)
    b = ALS.factor_design_rows(G, F, n, S.decode_keys(keys, dims))
    assert np.allclose(b, Kn[:, keys.astype(np.int64)].T, rtol=1e-12, atol=1e-13)


def test_count_form_equals_explicit_repeated_rows():
    X, G, F = _problem(3)
    n, lam, m = 1, 0.2, 400
    r = ALS.sketched_factor_update(X, G, F, n, lam, m, seed=7, sweep=2)
    # the explicit sketch: every accepted draw as its own row scaled by 1/sqrt(m p)
    dims = [d for k, d in enumerate(X.shape) if k != n]
    rep = np.repeat(r["keys"], r["counts"].astype(np.int64))
    p = np.repeat(r["prob"], r["counts"].astype(np.int64))
    W = CU.kron_matrix([F[k] for k in range(3) if k != n])
    B = (ALS.unfold(G, n) @ W.T).T[rep.astype(np.int64)] / np.sqrt(m * p)[:, None]
    Xr = ALS.unfold(X, n)[:, rep.astype(np.int64)] / np.sqrt(m * p)[None, :]
    A = np.linalg.solve(B.T @ B + lam * np.eye(B.shape[1]), B.T @ Xr.T).T
    assert np.allclose(r["A"], A, rtol=1e-10, atol=1e-12)
    assert r["counts"].sum() == m


@pytest.mark.parametrize("n", [0, 1, 2])
def test_product_scores_overestimate_the_design_scores(n):
    X, G, F = _problem(4)
    W = CU.kron_matrix([F[k] for k in range(3) if k != n])
    B = W @ ALS.unfold(G, n).T
    lB = LV.ridge_leverage_scores(B, 0.0)
    lW = LV.ridge_leverage_scores(W, 0.0)
    assert np.all(lW >= lB - 1e-12)                 # pointwise, so on the normalised scale:
    beta = G.shape[n] / np.prod([G.shape[k] for k in range(3) if k != n])
    assert np.all(lW / lW.sum() >= beta * lB / lB.sum() - 1e-15)


def test_sketched_factor_gram_is_unbiased():
    X, G, F = _problem(5)
    n, m = 0, 300
    W = CU.kron_matrix([F[k] for k in range(3) if k != n])
    B = W @ ALS.unfold(G, n).T
    exact = B.T @ B
    dims = [d for k, d in enumerate(X.shape) if k != n]
    acc = np.zeros_like(exact)
    reps = 300
    for s in range(reps):
        r = ALS.sketched_factor_update(X, G, F, n, 0.1, m, seed=s)
        b = ALS.factor_design_rows(G, F, n, S.decode_keys(r["keys"], dims))
        acc += (r["w"][:, None] * b).T @ b
    err = np.linalg.norm(acc / reps - exact) / np.linalg.norm(exact)
    assert err < 0.02, err


def test_sketched_als_reaches_the_exact_noise_floor():
    g = np.random.default_rng(6)
    dims, ranks, sigma, lam = (24, 22, 20), (3, 3, 3), 0.05, 1e-3
    Ft = [g.standard_normal((i, r)) for i, r in zip(dims, ranks)]
    X = ALS.tucker_model(g.standard_normal(ranks), Ft) + sigma * g.standard_normal(dims)
    F0 = [g.standard_normal((i, r)) for i, r in zip(dims, ranks)]
    G0 = g.standard_normal(ranks)
    out = {}
    for mf in (0, 1500):
        G, F = G0, F0
        for sw in range(8):
            G, F = ALS.als_sweep(X, G, F, lam, sketched=mf > 0, m=3000, seed=11, sweep=sw,
                                 m_factor=mf)
        out[mf] = ALS.rmse(X, G, F)
    assert out[0] < 1.2 * sigma
    assert out[1500] < 1.1 * out[0], out
