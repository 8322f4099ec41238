"""GPU parity: leverage scores, the integer sampler and dedupe against the oracle.

Sampled keys, counts and probabilities must be bit-identical to the oracle's
given the same leverage scores (the oracle's own scores are fed to the GPU
sampler).  Leverage scores agree to 1e-10 relative; the fixed-point CDFs
built from GPU and oracle scores may differ by at most one unit per row.
"""
import numpy as np
import pytest
import torch

from oracle import leverage as LV, sampling as S, core_update as CU
from tests.gpu_common import dev, dev_keys, host_keys, handle  # noqa: F401
from paper_2107_10654_gb300 import tucker as T

pytestmark = pytest.mark.gpu


def _factors(shapes, seed, dtype=np.float64, rank_def=None):
    g = np.random.default_rng(seed)
    F = [g.standard_normal(s) for s in shapes]
    if rank_def is not None:
        n, k = rank_def
        i, r = shapes[n]
        F[n] = g.standard_normal((i, k)) @ g.standard_normal((k, r))
    return [f.astype(dtype) for f in F]


@pytest.mark.parametrize("shapes,rank_def", [
    ([(64, 4), (64, 4), (64, 4)], None),
    ([(1000, 7), (300, 3), (77, 16)], None),
    ([(513, 8), (40, 5)], (1, 2)),
    ([(128, 8)] * 4, None),
    ([(9, 2), (5, 1), (7, 3), (6, 2), (4, 2)], None),
])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_leverage_scores_match_oracle(handle, shapes, rank_def, dtype):
    F = _factors(shapes, 3, dtype, rank_def)
    lev, cdf, ranks = T.tucker_leverage_scores(handle, [dev(f) for f in F])
    for n, A in enumerate(F):
        ref, rk = LV.leverage_scores(A)
        assert ranks[n] == rk
        got = lev[n].cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-10 * max(1.0, np.max(np.abs(ref)))
        q_ref = S.fixed_point_scores(ref)[0].astype(np.int64)
        c = cdf[n].cpu().numpy()
        q_got = np.diff(np.concatenate([[0], c]))
        assert np.max(np.abs(q_got - q_ref)) <= 1


def _oracle_sample(levs, dims, m, seed, sweep, reg, d, obs=None, max_draws=0):
    keys, T_ = S.sample_keys(levs, dims, m, seed, sweep, reg, d, obs, max_draws)
    ku, cu = S.dedupe(keys)
    p = S.row_probabilities(ku, levs, dims, reg, d)
    return ku, cu, p, T_


@pytest.mark.parametrize("dims,ranks,m", [
    ((64, 64, 64), (4, 4, 4), 2000),
    ((100, 37, 250), (3, 5, 2), 4097),          # ragged sizes, m not a tile multiple
    ((16, 12, 10, 8), (2, 2, 2, 2), 30000),     # many duplicates
    ((9, 5, 7, 6, 4), (2, 1, 3, 2, 2), 999),    # order 5: second Philox stream
    ((512, 512, 512), (8, 8, 8), 50000),        # full-size dense 3-way sample
    ((512, 512, 512), (8, 8, 8), 100000),       # the 1.01x sample count: 16-CTA cluster sort
    ((30, 20, 10), (3, 2, 2), 131072),          # the 16-CTA sort at its largest, 6000 rows
    ((512, 512, 512), (8, 8, 8), 131073),       # one key past it: the multi-pass sort
    ((128, 128, 128, 128), (8, 8, 8, 8), 200000),   # full-size dense 4-way sample
])
@pytest.mark.parametrize("reg", ["exact", "augmented"])
def test_sampler_bit_exact(handle, dims, ranks, m, reg):
    F = _factors([(i, r) for i, r in zip(dims, ranks)], 5)
    levs = [LV.leverage_scores(A)[0] for A in F]
    d = int(np.prod(ranks))
    regc = S.REG_EXACT if reg == "exact" else S.REG_AUGMENTED
    ku, cu, p, T_ = _oracle_sample(levs, dims, m, 1234, 7, regc, d)
    out = T.tucker_sample_rows(handle, dims, ranks, [dev(l) for l in levs], m, 1234, 7, reg)
    assert out.n_unique == ku.size and out.n_draws == T_
    assert np.array_equal(host_keys(out.keys, out.n_unique), ku)
    assert np.array_equal(out.counts[:out.n_unique].cpu().numpy().astype(np.int64), cu)
    assert np.array_equal(out.prob[:out.n_unique].cpu().numpy(), p)      # bit-identical


@pytest.mark.parametrize("reg", ["exact", "augmented"])
def test_sampler_missing_entries_bit_exact(handle, reg):
    dims, ranks, m = (40, 30, 50), (3, 2, 4), 3000
    g = np.random.default_rng(9)
    total = int(np.prod(dims))
    obs = np.sort(g.choice(total, size=total // 10, replace=False)).astype(np.uint64)
    vals = g.standard_normal(obs.size)
    F = _factors([(i, r) for i, r in zip(dims, ranks)], 6)
    levs = [LV.leverage_scores(A)[0] for A in F]
    d = int(np.prod(ranks))
    regc = S.REG_EXACT if reg == "exact" else S.REG_AUGMENTED
    ku, cu, p, T_ = _oracle_sample(levs, dims, m, 77, 1, regc, d, obs)
    coo = T.CooTensor(dev_keys(obs), dev(vals), dims)
    out = T.tucker_sample_rows(handle, dims, ranks, [dev(l) for l in levs], m, 77, 1, reg,
                               observed=coo)
    assert out.n_draws == T_ and out.n_unique == ku.size
    assert np.array_equal(host_keys(out.keys, out.n_unique), ku)
    assert np.array_equal(out.counts[:out.n_unique].cpu().numpy().astype(np.int64), cu)
    assert np.array_equal(out.prob[:out.n_unique].cpu().numpy(), p)


def test_sampler_edge_cases(handle):
    dims, ranks = (7, 5), (2, 2)
    F = _factors([(7, 2), (5, 2)], 8)
    levs = [LV.leverage_scores(A)[0] for A in F]
    # m = 1
    out = T.tucker_sample_rows(handle, dims, ranks, [dev(l) for l in levs], 1, 5, 0)
    ku, cu, p, _ = _oracle_sample(levs, dims, 1, 5, 0, S.REG_EXACT, 4)
    assert out.n_unique == 1 and host_keys(out.keys, 1)[0] == ku[0]
    # zero-mass rows are never drawn
    l0 = levs[0].copy()
    l0[[1, 4]] = 0.0
    out = T.tucker_sample_rows(handle, dims, ranks, [dev(l0), dev(levs[1])], 5000, 5, 0)
    rows = host_keys(out.keys, out.n_unique) // 5
    assert not np.isin(rows, [1, 4]).any()
    # all-zero scores: ERANK, and the handle stays usable
    with pytest.raises(T.TuckerError) as e:
        T.tucker_sample_rows(handle, dims, ranks, [dev(np.zeros(7)), dev(levs[1])], 10, 5, 0)
    assert e.value.name == "ERANK"
    # draw limit in missing mode
    obs = np.array([3, 17], dtype=np.uint64)
    coo = T.CooTensor(dev_keys(obs), dev(np.ones(2)), dims)
    with pytest.raises(T.TuckerError) as e:
        T.tucker_sample_rows(handle, dims, ranks, [dev(l) for l in levs], 1000, 5, 0,
                             observed=coo, max_draws=2000)
    assert e.value.name == "EDRAWLIMIT"
    # capacity check and bad arguments
    with pytest.raises(T.TuckerError) as e:
        T.tucker_sample_rows(handle, dims, ranks, [dev(l) for l in levs], 10, 5, 0,
                             out=T.Samples.empty(5, "cuda"))
    assert e.value.name == "ECAPACITY"
    out = T.tucker_sample_rows(handle, dims, ranks, [dev(l) for l in levs], 100, 5, 0)
    assert out.n_unique > 0
