"""GPU parity of lambda-ridge leverage sampling of K (Lemma 4.1 with lambda > 0):

  * tucker_ridge_tables against the oracle's thin SVDs: the squared columns
    of U^(n), the mixture weights c_t and d_eff(K);
  * tucker_sample_rows_ridge given the oracle's tables: keys, counts and
    probabilities bit-identical to the oracle's mixture sampler;
  * the sketched core update in ridge mode against the oracle's
    sketched_core_ridge (a frozen GPU sample: 1e-10 in FP64, 1e-6 for TF32;
    end to end from the GPU's own tables: the same sample, cores to 1e-8),
    and m = 0, which draws the sample count of Alg. 1 line 3 with beta' of
    Eq. beta_prime for the exact ridge scores.
"""
import numpy as np
import pytest
import torch

from oracle import ridge_kron as RK, sampling as S, core_update as CU
from tests.gpu_common import dev, dev_keys, host_keys, rel_err, handle  # noqa: F401
from paper_2107_10654_gb300 import tucker as T

pytestmark = pytest.mark.gpu


def _problem(shapes, seed, dtype=np.float64, dup=None):
    g = np.random.default_rng(seed)
    F = [g.standard_normal(s) for s in shapes]
    if dup is not None:                       # rank-deficient factor: a repeated column
        n, a, b = dup
        F[n][:, b] = F[n][:, a]
    dims = tuple(s[0] for s in shapes)
    X = g.standard_normal(dims)
    return [f.astype(dtype) for f in F], X.astype(dtype)


def _oracle_tables(F, lam):
    c, Us = RK.ridge_weights([np.asarray(a, dtype=np.float64) for a in F], lam)
    usq = [np.ascontiguousarray((U ** 2).T) for U in Us]         # K_n x I_n
    return usq, c.reshape(-1), list(c.shape)


CASES = [
    ([(40, 3), (30, 2), (20, 4)], 1e2, None),
    ([(64, 8), (48, 8), (50, 8)], 3e4, None),         # c_t spread over (0, 1)
    ([(3, 5), (20, 2), (10, 3)], 1.0, None),          # I_1 < R_1: K_1 = 3
    ([(25, 4), (18, 3), (30, 3)], 10.0, (0, 1, 3)),   # rank-deficient factor: cut columns
    ([(9, 2), (5, 1), (7, 3), (6, 2), (4, 2)], 0.5, None),   # order 5
]


@pytest.mark.parametrize("shapes,lam,dup", CASES)
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_ridge_tables_match_oracle(handle, shapes, lam, dup, dtype):
    F, _ = _problem(shapes, 3, dtype, dup)
    usq, c, K, deff = T.tucker_ridge_tables(handle, [dev(a) for a in F], lam)
    ref_u, ref_c, ref_K = _oracle_tables(F, lam)
    assert K == ref_K
    assert abs(deff - RK.kron_effective_dimension([np.asarray(a, np.float64) for a in F], lam)) \
        <= 1e-12 * max(1.0, deff)
    cg = c.cpu().numpy()
    assert np.max(np.abs(cg - ref_c)) <= 1e-12
    _, Us = RK.ridge_weights([np.asarray(a, np.float64) for a in F], lam)
    s2 = [s for _, s in RK.factor_svds([np.asarray(a, np.float64) for a in F])]
    for n in range(len(F)):
        got = usq[n].cpu().numpy()
        for t in range(K[n]):
            if s2[n][t] > 0:                           # columns of cut components are 0 here
                assert np.max(np.abs(got[t] - ref_u[n][t])) <= 1e-12, (n, t)
            else:
                assert np.all(got[t] == 0.0)


@pytest.mark.parametrize("shapes,lam,dup", CASES)
@pytest.mark.parametrize("m", [3000, 100000])
def test_ridge_sampler_bit_exact_given_oracle_tables(handle, shapes, lam, dup, m):
    F, _ = _problem(shapes, 4, np.float64, dup)
    dims = tuple(s[0] for s in shapes)
    usq, c, K = _oracle_tables(F, lam)
    smp = T.tucker_sample_rows_ridge(handle, dims, K, [dev(u) for u in usq], dev(c), m, 77, 2)
    tables = RK.ridge_mixture_tables(F, lam)
    keys = RK.draw_rows_ridge(tables, dims, np.arange(m, dtype=np.uint64), 77, 2)
    ku, cu = S.dedupe(keys)
    p = RK.ridge_row_probabilities(tables, ku, dims)
    assert smp.n_draws == m and smp.n_unique == ku.size
    assert np.array_equal(host_keys(smp.keys, smp.n_unique), ku)
    assert np.array_equal(smp.counts[:smp.n_unique].cpu().numpy().astype(np.int64), cu)
    assert np.array_equal(smp.prob[:smp.n_unique].cpu().numpy(), p)     # bit-identical


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("tf32", 1e-6)])
def test_ridge_core_update_frozen_sample(handle, prec, tol):
    shapes, lam = [(60, 4), (50, 4), (40, 4)], 2e3
    F, X = _problem(shapes, 5)
    dims = X.shape
    usq, c, K = _oracle_tables(F, lam)
    m = 8000
    smp = T.tucker_sample_rows_ridge(handle, dims, K, [dev(u) for u in usq], dev(c), m, 9, 0)
    g = T.tucker_core_update_sketched(handle, dev(X), [dev(a) for a in F], lam, 0, 0, 0,
                                      "ridge", prec, fixed=smp)
    ref = RK.sketched_core_ridge(X, F, lam, m, 9, 0)
    assert smp.n_unique == ref["keys"].size
    assert rel_err(g.cpu().numpy(), ref["g"]) <= tol


@pytest.mark.parametrize("solver", ["fp64", "kpcg"])
def test_ridge_core_update_end_to_end(solver):
    shapes, lam = [(60, 4), (50, 4), (40, 4)], 2e3
    F, X = _problem(shapes, 6)
    m = 8000
    with T.Handle(solver=solver) as h:
        g, st = T.tucker_core_update_sketched(h, dev(X), [dev(a) for a in F], lam, m, 11, 1,
                                              "ridge", "fp64" if solver == "fp64" else "tf32",
                                              stats=True)
        torch.cuda.synchronize()
    ref = RK.sketched_core_ridge(X, F, lam, m, 11, 1)
    assert st["n_draws"] == m and st["n_unique"] == ref["keys"].size
    # the GPU's tables agree with the oracle's SVD to ~1e-15; a fixed-point weight that
    # lands on the other side of a 2^-32 step moves a probability by ~1e-8 relative
    assert rel_err(g.cpu().numpy(), ref["g"]) <= (1e-6 if solver == "kpcg" else 1e-8)


def test_ridge_sample_count_when_m_is_zero(handle):
    shapes, lam = [(30, 2), (20, 2), (25, 2)], 3e2
    F, X = _problem(shapes, 7)
    s = RK.ridge_sample_count(F, lam, 0.1, 0.1)
    d = 8
    assert s < S.paper_sample_count(d, 0.1, 0.1)             # fewer rows than the classical count
    g, st = T.tucker_core_update_sketched(handle, dev(X), [dev(a) for a in F], lam, 0, 3, 0,
                                          "ridge", "fp64", eps=0.1, delta=0.1, stats=True)
    assert st["n_draws"] == s
    ref = RK.sketched_core_ridge(X, F, lam, s, 3, 0)
    assert st["n_unique"] == ref["keys"].size
    assert rel_err(g.cpu().numpy(), ref["g"]) <= 1e-8


def test_ridge_errors(handle):
    F, X = _problem([(10, 2), (9, 2), (8, 2)], 8)
    Fz = [np.zeros((10, 2))] + F[1:]
    with pytest.raises(T.TuckerError) as e:               # every c_t is 0
        T.tucker_core_update_sketched(handle, dev(X), [dev(a) for a in Fz], 1.0, 500, 1, 0,
                                      "ridge", "fp64")
    assert e.value.name == "ERANK"
    keys = np.arange(0, 720, 7, dtype=np.uint64)
    coo = T.CooTensor(dev_keys(keys), dev(np.ones(keys.size)), X.shape)
    with pytest.raises(T.TuckerError) as e:               # dense tensors only
        T.tucker_core_update_sketched(handle, coo, [dev(a) for a in F], 1.0, 500, 1, 0, "ridge",
                                      "fp64")
    assert e.value.name == "EINVAL"
    g = T.tucker_core_update_sketched(handle, dev(X), [dev(a) for a in F], 1.0, 500, 1, 0,
                                      "ridge", "fp64")
    assert torch.isfinite(g).all()
