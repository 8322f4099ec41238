"""Pins of the CP-ALS oracle (oracle/cp.py): regularised CP-ALS with factor
updates on the Khatri-Rao design, exact and sketched by the product of the other
modes' leverage scores (Sec. 4's remark on Khatri-Rao designs; Sec. 6's
extension of leverage-score-sampled CP-ALS to L2 regularisation).

Each pin checks the oracle against something other than its own formulas:
element-by-element loops of the model and the design, the minimiser of the loss
itself (the loss cannot drop along any direction at the update), the Hadamard
Gram identity on the explicit design, leverage scores of the explicit design
against the product bound, the sketch on every row with unit weights against the
exact update, unbiasedness of the sampled Gram over seeds, monotone exact ALS and
the (1 + eps) ridge-loss bound of the sketch.  The last test plants mistakes and
checks that some pin fails."""
import itertools

import numpy as np
import pytest

from oracle import cp as CP, leverage as LV, sampling as S


def _problem(dims=(5, 6, 7), R=3, seed=0, noise=0.05):
    g = np.random.default_rng(seed)
    F = [g.standard_normal((i, R)) for i in dims]
    X = CP.cp_model(F) + noise * g.standard_normal(dims)
    return X, F


def pin_model_elementwise():
    X, F = _problem(noise=0.0)
    A, B, C = F
    for i, j, k in itertools.product(range(5), range(6), range(7)):
        v = sum(A[i, r] * B[j, r] * C[k, r] for r in range(3))
        assert abs(X[i, j, k] - v) <= 1e-12 * (1 + abs(v))


def pin_khatri_rao_rows_and_unfolding():
    _, F = _problem()
    A, B, C = F
    Z = CP.khatri_rao(F, 0)                      # rows (j, k), k fastest
    for j, k, r in itertools.product(range(6), range(7), range(3)):
        assert Z[j * 7 + k, r] == B[j, r] * C[k, r]
    Xh = CP.cp_model(F)
    for n in range(3):
        assert np.allclose(CP.unfold(Xh, n), F[n] @ CP.khatri_rao(F, n).T, atol=1e-12)


def pin_hadamard_gram():
    _, F = _problem(dims=(4, 5, 6, 3), R=4)
    for n in range(4):
        Z = CP.khatri_rao(F, n)
        H = np.ones((4, 4))
        for k, A in enumerate(F):
            if k != n:
                H *= A.T @ A
        assert np.allclose(Z.T @ Z, H, rtol=1e-12, atol=1e-12)


def pin_update_minimises_loss():
    X, F = _problem()
    lam = 0.3
    g = np.random.default_rng(5)
    for n in range(3):
        An = CP.cp_factor_update(X, F, n, lam)
        G = [A.copy() for A in F]
        G[n] = An
        base = CP.cp_loss(X, G, lam)
        for _ in range(8):
            E = g.standard_normal(An.shape)
            for h in (1e-3, -1e-3):
                H = [A.copy() for A in G]
                H[n] = An + h * E
                assert CP.cp_loss(X, H, lam) >= base - 1e-10 * base
        # central differences of the loss along random directions vanish at the minimiser
        E = g.standard_normal(An.shape)
        Hp, Hm = [A.copy() for A in G], [A.copy() for A in G]
        Hp[n], Hm[n] = An + 1e-5 * E, An - 1e-5 * E
        slope = (CP.cp_loss(X, Hp, lam) - CP.cp_loss(X, Hm, lam)) / 2e-5
        assert abs(slope) <= 1e-6 * base


def pin_leverage_product_bound():
    _, F = _problem(dims=(6, 5, 7), R=3, seed=2)
    for n in range(3):
        Z = CP.khatri_rao(F, n)
        lz = LV.leverage_scores(Z)[0]
        others = [A for k, A in enumerate(F) if k != n]
        prod = np.ones(1)
        for A in others:
            prod = np.multiply.outer(prod, LV.leverage_scores(A)[0]).reshape(-1)
        assert np.all(lz <= prod + 1e-12)
        assert abs(lz.sum() - 3) <= 1e-9                   # sum of scores = rank R
        assert abs(prod.sum() - 9) <= 1e-9                 # rank of the Kronecker product


def pin_all_rows_unit_weights_is_exact():
    X, F = _problem()
    for n in range(3):
        dims = [v for k, v in enumerate(X.shape) if k != n]
        keys = np.arange(int(np.prod(dims)), dtype=np.uint64)
        A1 = CP.cp_factor_update_from_rows(X, F, n, 0.2, keys, np.ones(keys.size))
        assert np.allclose(A1, CP.cp_factor_update(X, F, n, 0.2), rtol=1e-11, atol=1e-12)


def pin_sampled_gram_unbiased():
    X, F = _problem(dims=(4, 9, 8), R=3, seed=3)
    n = 0
    Z = CP.khatri_rao(F, n)
    ZtZ = Z.T @ Z
    acc = np.zeros_like(ZtZ)
    seeds = 200
    dims = [9, 8]
    for s in range(seeds):
        r = CP.sketched_cp_factor_update(X, F, n, 0.1, 60, s)
        z = CP.khatri_rao_rows(F, n, S.decode_keys(r["keys"], dims))
        acc += (r["w"][:, None] * z).T @ z
    assert np.linalg.norm(acc / seeds - ZtZ) <= 0.05 * np.linalg.norm(ZtZ)


def pin_exact_als_monotone():
    X, _ = _problem(dims=(6, 5, 7), R=3, seed=4, noise=0.2)
    g = np.random.default_rng(9)
    F = [g.standard_normal((i, 3)) for i in X.shape]
    lam = 0.05
    prev = CP.cp_loss(X, F, lam)
    for _ in range(6):
        F = CP.cp_als_sweep(X, F, lam)
        cur = CP.cp_loss(X, F, lam)
        assert cur <= prev * (1 + 1e-12)
        prev = cur


def pin_sketch_ridge_loss_bound():
    X, F = _problem(dims=(20, 24, 22), R=4, seed=6, noise=0.1)
    lam, n = 0.1, 1
    Z = CP.khatri_rao(F, n)
    Xn = CP.unfold(X, n)

    def obj(A):
        return float(np.sum((Xn - A @ Z.T) ** 2) + lam * np.sum(A * A))

    best = obj(CP.cp_factor_update(X, F, n, lam))
    ratios = [obj(CP.sketched_cp_factor_update(X, F, n, lam, 4000, s)["A"]) / best
              for s in range(5)]
    assert 1.0 <= min(ratios) and np.median(ratios) <= 1.01


PINS = [pin_model_elementwise, pin_khatri_rao_rows_and_unfolding, pin_hadamard_gram,
        pin_update_minimises_loss, pin_leverage_product_bound, pin_all_rows_unit_weights_is_exact,
        pin_sampled_gram_unbiased, pin_exact_als_monotone, pin_sketch_ridge_loss_bound]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    pin()


def _fails(mp):
    for pin in PINS:
        try:
            pin()
        except Exception:
            return True
    return False


@pytest.mark.parametrize("plant", ["kron_rows", "lambda_dropped", "fiber_transposed",
                                   "model_skips_first_component", "weights_without_m"])
def test_planted_mistakes_are_caught(monkeypatch, plant):
    if plant == "kron_rows":                 # Kronecker instead of Hadamard rows
        def bad(factors, n, idx):
            others = [np.asarray(A, dtype=np.float64) for k, A in enumerate(factors) if k != n]
            z = np.asarray(others[0])[np.asarray(idx[0])]
            for A, j in zip(others[1:], idx[1:]):
                a = A[np.asarray(j)]
                z = np.einsum("ua,ub->uab", z, a).reshape(z.shape[0], -1)[:, :a.shape[1]]
            return z
        monkeypatch.setattr(CP, "khatri_rao_rows", bad)
    elif plant == "lambda_dropped":
        orig = CP.cp_factor_update
        monkeypatch.setattr(CP, "cp_factor_update", lambda X, F, n, lam: orig(X, F, n, 0.0))
    elif plant == "fiber_transposed":        # rows decoded with the other modes' order reversed
        orig_dec = S.decode_keys
        monkeypatch.setattr(CP.S, "decode_keys", lambda k, d: orig_dec(k, d[::-1])[::-1])
    elif plant == "model_skips_first_component":   # off by one in the sum over r
        orig_m = CP.cp_model
        monkeypatch.setattr(CP, "cp_model", lambda F: orig_m([np.asarray(A)[:, 1:] for A in F]))
    elif plant == "weights_without_m":
        orig_w = S.sample_weights
        monkeypatch.setattr(CP.S, "sample_weights", lambda c, p, T: orig_w(c, p, 1))
    assert _fails(monkeypatch)
