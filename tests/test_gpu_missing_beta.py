"""GPU parity of the missing-data overestimate factor (Sec. 4.2) and of the
sample count it sets for observed-entry tensors:

  * tucker_missing_beta's bound mode (the corollary to Thm 4.3) and c_min
    against the oracle's SVDs, and Alg. 1 line 3's count against the oracle's;
  * the exact mode (lambda_max(L_{S-bar,S-bar}) from the observed rows' Gram,
    whitened by the factor eigendecompositions, inverse iteration and a
    Cholesky certificate) against the oracle's explicit cross-score matrix:
    the GPU value must bound lambda_max from above and lie within the
    certificate's slack of it, for a uniform mask, a mask far from uniform,
    every entry observed, and a TF32 Gram;
  * m = 0 on a COO tensor draws the count of the bound mode (the same accepted
    draws and T as the oracle's sampler at that m, the same core), and a count
    of 2^31 or more is refused with EINVAL.
"""
import numpy as np
import pytest
import torch

from oracle import ridge_kron as RK, core_update as CU, sampling as S
from tests.gpu_common import dev, dev_keys, rel_err, handle  # noqa: F401
from paper_2107_10654_gb300 import tucker as T

pytestmark = pytest.mark.gpu


def _problem(dims, ranks, seed, frac=None, keys=None, orth=False):
    g = np.random.default_rng(seed)
    F = [g.standard_normal((i, r)) for i, r in zip(dims, ranks)]
    if orth:                                     # orthonormal columns: ||A||_2 = 1
        F = [np.linalg.qr(a)[0] for a in F]
    n = int(np.prod(dims))
    if keys is None:
        keys = np.sort(g.choice(n, int(frac * n), replace=False)).astype(np.uint64)
    vals = g.standard_normal(keys.size)
    return F, keys, vals


def _coo(keys, vals, dims, dtype=torch.float64):
    return T.CooTensor(dev_keys(keys), dev(vals).to(dtype), dims)


@pytest.mark.parametrize("lam", [0.5, 30.0])
def test_bound_mode_matches_oracle(handle, lam):
    dims, ranks = (12, 10, 9), (2, 3, 2)
    F, keys, vals = _problem(dims, ranks, 1, frac=0.4)
    info = T.tucker_missing_beta(handle, _coo(keys, vals, dims), [dev(a) for a in F], lam, "bound")
    bm = RK.missing_ridge_beta_bound(F, lam)
    assert abs(info["beta_miss"] - bm) <= 1e-12 * bm
    assert abs(info["c_min"] - RK.classical_ridge_ratio_min(F, lam)) <= 1e-12
    assert abs(info["beta"] - RK.missing_overestimate_beta(F, lam, bm)) <= 1e-12 * info["beta"]
    assert abs(info["s"] - RK.missing_sample_count(F, lam, 0.1, 0.1, bm)) <= 1.0
    # a dense tensor has nothing missing
    X = dev(np.zeros(dims))
    dn = T.tucker_missing_beta(handle, X, [dev(a) for a in F], lam, "bound")
    assert dn["beta_miss"] == 1.0 and dn["lambda_max"] == 0.0


def _exact_check(info, F, lam, keys, dims, slack):
    K = CU.kron_matrix(F)
    idx = keys.astype(np.int64)
    b_or, l_or = RK.missing_ridge_beta_from_gram(F, lam, K[idx].T @ K[idx])
    # an upper bound of lambda_max (for the Gram as formed), within the certificate's slack
    assert info["lambda_max"] >= l_or - 1e-10, (info["lambda_max"], l_or)
    assert info["lambda_max"] <= l_or + slack * (1.0 - l_or) + 1e-10, (info["lambda_max"], l_or)
    assert info["beta_miss"] <= b_or * (1 + 1e-10)
    assert info["nu_est"] >= (1.0 - l_or) * (1 - 1e-9)            # estimates are from above
    assert info["iters"] >= 1 and info["certify_tries"] >= 1
    return l_or


@pytest.mark.parametrize("lam", [0.2, 5.0])
def test_exact_mode_uniform_mask(handle, lam):
    dims, ranks = (12, 10, 9), (2, 3, 2)
    F, keys, vals = _problem(dims, ranks, 2, frac=0.4)
    info = T.tucker_missing_beta(handle, _coo(keys, vals, dims), [dev(a) for a in F], lam, "exact")
    _exact_check(info, F, lam, keys, dims, 1e-2)
    # the exact value is never below the corollary's bound
    assert info["beta_miss"] >= RK.missing_ridge_beta_bound(F, lam) * (1 - 1e-12)


def test_exact_mode_far_from_uniform_mask(handle):
    # only the slices i_1 < 3 observed: most of K's row space is missing
    dims, ranks, lam = (12, 10, 9), (3, 2, 2), 0.7
    n23 = dims[1] * dims[2]
    keys = np.arange(3 * n23, dtype=np.uint64)
    F, keys, vals = _problem(dims, ranks, 3, keys=keys)
    info = T.tucker_missing_beta(handle, _coo(keys, vals, dims), [dev(a) for a in F], lam, "exact")
    l_or = _exact_check(info, F, lam, keys, dims, 1e-2)
    assert l_or > 0.5


def test_exact_mode_all_observed(handle):
    dims, ranks, lam = (8, 7, 6), (2, 2, 3), 1.0
    keys = np.arange(int(np.prod(dims)), dtype=np.uint64)
    F, keys, vals = _problem(dims, ranks, 4, keys=keys)
    info = T.tucker_missing_beta(handle, _coo(keys, vals, dims), [dev(a) for a in F], lam, "exact")
    assert info["lambda_max"] <= 1e-3                      # nothing missing: the pencil is I
    assert abs(info["beta_miss"] - 0.5) <= 1e-3            # the formula's value at lambda_max = 0


def test_exact_mode_tf32_gram(handle):
    dims, ranks, lam = (30, 20, 20), (4, 8, 8), 2.0        # d = 256 on the tensor cores
    F, keys, vals = _problem(dims, ranks, 5, frac=0.3)
    F32 = [dev(a).float() for a in F]
    info = T.tucker_missing_beta(handle, _coo(keys, vals, dims, torch.float32), F32, lam,
                                 "exact", prec="tf32")
    Fr = [a.cpu().numpy().astype(np.float64) for a in F32]
    K = CU.kron_matrix(Fr)
    idx = keys.astype(np.int64)
    _, l_or = RK.missing_ridge_beta_from_gram(Fr, lam, K[idx].T @ K[idx])
    # the Gram is TF32-rounded (about 2^-10 relative per entry), so only close
    assert abs(info["lambda_max"] - l_or) <= 2e-2 * (1.0 - l_or) + 1e-3


def test_m_zero_on_observed_entries_draws_the_bound_count(handle):
    dims, ranks, lam = (20, 16, 12), (2, 2, 2), 1.0
    F, keys, vals = _problem(dims, ranks, 6, frac=0.5, orth=True)
    coo = _coo(keys, vals, dims)
    s = RK.missing_sample_count(F, lam, 0.1, 0.1, RK.missing_ridge_beta_bound(F, lam))
    assert s < (1 << 31)
    g, st = T.tucker_core_update_sketched(handle, coo, [dev(a) for a in F], lam, 0, 5, 0, "exact",
                                          "fp64", eps=0.1, delta=0.1, stats=True)
    ref = CU.sketched_core(None, F, lam, s, 5, 0, S.REG_EXACT, observed=(keys, vals, dims))
    assert st["n_draws"] == ref["T"] and st["n_unique"] == ref["keys"].size
    assert rel_err(g.cpu().numpy(), ref["g"]) <= 1e-8


def test_errors(handle):
    dims, ranks = (12, 10, 9), (2, 3, 2)
    F, keys, vals = _problem(dims, ranks, 7, frac=0.4)
    coo = _coo(keys, vals, dims)
    Fd = [dev(a) for a in F]
    with pytest.raises(T.TuckerError) as e:                 # Thm 4.3 needs lambda > 0
        T.tucker_missing_beta(handle, coo, Fd, 0.0, "bound")
    assert e.value.name == "EINVAL"
    # N(0,1) factors and a small lambda: the bound's count is far beyond any m
    with pytest.raises(T.TuckerError) as e:
        T.tucker_core_update_sketched(handle, coo, Fd, 1e-3, 0, 1, 0, "exact", "fp64",
                                      eps=0.1, delta=0.1)
    assert e.value.name == "EINVAL" and "missing-data bound" in str(e.value)
