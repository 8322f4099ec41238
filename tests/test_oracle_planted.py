"""Planted mistakes: a plausible error in the oracle (a dropped term or factor, a
wrong sign, index order or constant, an off-by-one) is planted on the CPU with
monkeypatch, and at least one of the oracle's pins must then fail.  This shows
that the pins constrain the oracle rather than restate it."""
import numpy as np
import pytest

from oracle import (adjoint as ADJ, als as ALS, core_update as CU, leverage as LV,
                    philox as PH, ridge_kron as RK, sampling as S)
from tests import test_oracle_core as TC
from tests import test_oracle_factor_sketch as TF
from tests import test_oracle_philox_leverage as TL
from tests import test_oracle_ridge_kron as TR
from tests import test_oracle_sampling as TS


def _fails(pins):
    for pin in pins:
        try:
            pin()
        except Exception:          # an assertion, or the pin's computation breaking down
            return True
    return False


def _kron_order_reversed(mp):
    orig = CU.kron_rows
    mp.setattr(CU, "kron_rows", lambda factors, idx: orig(list(factors)[::-1], list(idx)[::-1]))


def _exact_lambda_doubled(mp):
    orig = CU.exact_core_kron_eig
    mp.setattr(CU, "exact_core_kron_eig", lambda X, F, lam, ktx=None: orig(X, F, 2 * lam, ktx))


def _weights_without_T(mp):
    orig = S.sample_weights
    mp.setattr(S, "sample_weights", lambda c, p, T: orig(c, p, 1))


def _weights_doubled(mp):
    orig = S.sample_weights
    mp.setattr(S, "sample_weights", lambda c, p, T: 2.0 * orig(c, p, T))


def _augmented_half_dropped(mp):
    orig = S.row_probabilities
    mp.setattr(S, "row_probabilities",
               lambda keys, levs, dims, reg=S.REG_EXACT, d=0:
               orig(keys, levs, dims, S.REG_EXACT, d))


def _search_target_off_by_one(mp):
    orig = S.mulhi64
    mp.setattr(S, "mulhi64", lambda a, b: orig(a, b) + np.uint64(1))


def _search_lower_bound(mp):
    mp.setattr(S, "inverse_cdf",
               lambda C, u: np.searchsorted(C, S.mulhi64(u, C[-1]), side="left"))


def _ridge_term_ignored(mp):
    orig = LV.gram_pinv
    mp.setattr(LV, "gram_pinv", lambda A, lam=0.0: orig(A, 0.0))


def _philox_weyl_constant(mp):
    mp.setattr(PH, "PHILOX_W1", np.uint64(0xBB67AE8584CAA73A))


def _rhs_unweighted(mp):
    orig = CU.sketched_normal_equations

    def bad(factors, dims, keys_u, w, x, chunk=1 << 12):
        G, _, D = orig(factors, dims, keys_u, w, x, chunk)
        _, h, _ = orig(factors, dims, keys_u, np.ones_like(np.asarray(w, dtype=float)), x, chunk)
        return G, h, D
    mp.setattr(CU, "sketched_normal_equations", bad)


def _adjoint_dx_sign(mp):
    orig = ADJ.backward

    def bad(*a):
        dA, dx = orig(*a)
        return dA, -dx
    mp.setattr(ADJ, "backward", bad)


def _ridge_weight_lambda_doubled(mp):
    orig = RK.ridge_weights
    mp.setattr(RK, "ridge_weights", lambda F, lam: orig(F, 2 * lam))


def _factor_update_lambda_dropped(mp):
    orig = ALS.factor_update
    mp.setattr(ALS, "factor_update", lambda X, core, F, n, lam: orig(X, core, F, n, 0.0))


def _dedupe_counts_lost(mp):
    orig = S.dedupe

    def bad(keys):
        ku, cu = orig(keys)
        return ku, np.ones_like(cu)
    mp.setattr(S, "dedupe", bad)


def _decode_column_major(mp):
    def bad(keys, dims):
        rem = np.asarray(keys, dtype=np.uint64).copy()
        out = []
        for n in range(len(dims)):                      # first index fastest
            out.append((rem % np.uint64(dims[n])).astype(np.int64))
            rem = rem // np.uint64(dims[n])
        return out
    mp.setattr(S, "decode_keys", bad)


def _missing_beta_one_dropped(mp):
    orig = RK.missing_ridge_beta

    def bad(F, lam, obs, dims):
        b = orig(F, lam, obs, dims)
        return 1.0 / (1.0 / b - 1.0) if b < 1.0 else b   # 1/beta = 1/(1 - lmax) only
    mp.setattr(RK, "missing_ridge_beta", bad)


def _loss_lambda_dropped(mp):
    orig = CU.ridge_loss_dense
    mp.setattr(CU, "ridge_loss_dense",
               lambda X, F, g, lam, xx=None, ktx=None: orig(X, F, g, 0.0, xx, ktx))


def _observed_lookup_shifted(mp):
    orig = CU.gather_observed

    def bad(obs_keys, obs_vals, keys_u):
        v = np.asarray(obs_vals, dtype=np.float64)
        return orig(obs_keys, np.concatenate([v[1:], v[:1]]), keys_u)   # the next entry's value
    mp.setattr(CU, "gather_observed", bad)


def _exact_rows_lambda_dropped(mp):
    orig = CU.exact_core_rows
    mp.setattr(CU, "exact_core_rows",
               lambda keys, vals, dims, F, lam, chunk=1 << 13: orig(keys, vals, dims, F, 0.0, chunk))


def _adjoint_one_factor_scaled(mp):
    orig = ADJ.backward

    def bad(*a):
        dA, dx = orig(*a)
        return [2.0 * dA[0]] + list(dA[1:]), dx
    mp.setattr(ADJ, "backward", bad)


def _unobserved_accepted(mp):
    orig = S.sample_keys

    def bad(lev_list, dims, m, seed, sweep, reg=S.REG_EXACT, d=0, observed_keys=None,
            max_draws=0, batch=1 << 20):
        return orig(lev_list, dims, m, seed, sweep, reg, d, None, max_draws, batch)
    mp.setattr(S, "sample_keys", bad)


def _leverage_without_pinv(mp):
    def bad(A):
        A = np.asarray(A, dtype=np.float64)
        return np.einsum("ir,ir->i", A, A), np.linalg.matrix_rank(A)
    mp.setattr(LV, "leverage_scores", bad)


def _kron_matrix_reversed(mp):
    orig = CU.kron_matrix
    mp.setattr(CU, "kron_matrix", lambda factors: orig(list(factors)[::-1]))


def _augmented_reg_as_identity(mp):
    orig = CU.regularised_matrix
    mp.setattr(CU, "regularised_matrix",
               lambda G, D, lam, reg: orig(G, D, lam, S.REG_EXACT))


def _mixture_weight_dropped(mp):
    orig = RK.ridge_row_probabilities

    def bad(tables, keys_u, dims):
        flat = dict(tables)
        Cc = tables["Cc"]
        flat["Cc"] = np.arange(1, Cc.size + 1, dtype=np.uint64) * np.uint64(1 << 32)
        return orig(flat, keys_u, dims)                # every component weighted alike
    mp.setattr(RK, "ridge_row_probabilities", bad)


def _factor_rows_modes_swapped(mp):
    orig = ALS.factor_design_rows
    mp.setattr(ALS, "factor_design_rows",
               lambda core, factors, n, idx: orig(core, factors, n, list(idx)[::-1]))


def _factor_probabilities_uniform(mp):
    def bad(keys_u, lev_list, dims, reg=S.REG_EXACT, d=0):
        return np.full(np.asarray(keys_u).size, 1.0 / float(np.prod([int(v) for v in dims])))
    mp.setattr(S, "row_probabilities", bad)


PLANTS = {
    "kron_order_reversed": (_kron_order_reversed,
                            [TC.test_sampled_row_products_equal_explicit_rows]),
    "exact_lambda_doubled": (_exact_lambda_doubled,
                             [lambda: TC.test_exact_core_two_routes_agree((5, 4, 6), (2, 3, 2))]),
    "weights_without_T": (_weights_without_T, [TS.test_dedupe_and_weights_consistent]),
    "weights_doubled": (_weights_doubled, [TC.test_sketched_gram_unbiased]),
    "augmented_half_dropped": (_augmented_half_dropped, [TS.test_augmented_coin_and_index]),
    "search_target_off_by_one": (_search_target_off_by_one,
                                 [TS.test_inverse_cdf_boundary_convention]),
    "search_lower_bound": (_search_lower_bound, [TS.test_inverse_cdf_boundary_convention]),
    "ridge_term_ignored": (_ridge_term_ignored, [TL.test_lemma_3_1_augmented_matrix]),
    "philox_weyl_constant": (_philox_weyl_constant, [TL.test_philox_matches_numpy_bitgenerator]),
    "rhs_unweighted": (_rhs_unweighted,
                       [lambda: TC.test_count_form_equals_explicit_sketch_matrix(S.REG_EXACT)]),
    "adjoint_dx_sign": (_adjoint_dx_sign,
                        [lambda: TC.test_adjoint_matches_central_differences(S.REG_EXACT)]),
    "ridge_weight_lambda_doubled": (_ridge_weight_lambda_doubled,
                                    [lambda: TR.test_lemma_4_1_ridge_scores_equal_explicit_k(
                                        0.3, TR.SHAPES[0], None)]),
    "factor_update_lambda_dropped": (_factor_update_lambda_dropped,
                                     [TC.test_factor_update_matches_explicit_kn]),
    "dedupe_counts_lost": (_dedupe_counts_lost, [TS.test_dedupe_and_weights_consistent]),
    "decode_column_major": (_decode_column_major,
                            [TC.test_sampled_row_products_equal_explicit_rows]),
    "missing_beta_one_dropped": (_missing_beta_one_dropped,
                                 [TR.test_missing_entry_beta_and_bound]),
    "loss_lambda_dropped": (_loss_lambda_dropped,
                            [TC.test_ridge_loss_gram_identity_matches_residual]),
    "observed_lookup_shifted": (_observed_lookup_shifted,
                                [TC.test_missing_sketch_all_observed_equals_dense]),
    "exact_rows_lambda_dropped": (_exact_rows_lambda_dropped,
                                  [TC.test_exact_rows_all_observed_equals_dense]),
    "adjoint_one_factor_scaled": (_adjoint_one_factor_scaled,
                                  [lambda: TC.test_adjoint_matches_central_differences(
                                      S.REG_EXACT)]),
    "unobserved_accepted": (_unobserved_accepted, [TS.test_missing_entry_acceptance]),
    "leverage_without_pinv": (_leverage_without_pinv,
                              [lambda: TL.test_leverage_sum_is_rank_and_bounded((40, 5), 5)]),
    "kron_matrix_reversed": (_kron_matrix_reversed,
                             [TC.test_sampled_row_products_equal_explicit_rows]),
    "augmented_reg_as_identity": (_augmented_reg_as_identity,
                                  [lambda: TC.test_count_form_equals_explicit_sketch_matrix(
                                      S.REG_AUGMENTED)]),
    "factor_rows_modes_swapped": (_factor_rows_modes_swapped,
                                  [lambda: TF.test_design_rows_are_columns_of_explicit_kn(0)]),
    "factor_probabilities_uniform": (_factor_probabilities_uniform,
                                     [TF.test_sketched_factor_gram_is_unbiased]),
    "mixture_weight_dropped": (_mixture_weight_dropped,
                               [lambda: TR.test_ridge_sampler_probabilities_are_the_ridge_distribution(
                                   0.4)]),
}


@pytest.mark.parametrize("name", sorted(PLANTS))
def test_planted_mistake_is_caught(name, monkeypatch):
    plant, pins = PLANTS[name]
    assert not _fails(pins), "the pin fails without the planted mistake"
    plant(monkeypatch)
    assert _fails(pins), f"planted mistake {name!r} passes every pin"
