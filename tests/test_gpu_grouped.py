"""GPU parity of the tensor-core Gram grouped by the leading index (order >= 3):
sampled entries of G, h, and the FP64 residual of the refined core, against
the oracle (explicit sampled rows).

Wide M_{i_1} (d / R_1 >= 128): entries within the operand-rounding bound (BF16
2^-7, TF32 2^-9: the expansion by a_r1 a_r1' on the tensor cores rounds that
product to TF32 and keeps M exact as hi + lo), for R_1 = 2, 4, 8, 16, orders 3
and 4, and d / R_1 not a multiple of 16 or spanning two 256-wide tiles.

Narrow M_{i_1} (d / R_1 <= 64): every M_{i_1} from TF32 hi + lo operands and the
expansion in FP32, so the bound is an FP32 one, 2^-16 sum w |k_r| |k_c| (row
products, the dropped lo x lo term and FP32 sums of a few hundred terms), for
whichever tensor-core precision is asked; R_1 = 2, 4, 8, 16, orders 3 and 4,
d / R_1 from 8 to 64 and ragged (15), empty segments (values of i_1 that no
sampled row has) and segments of several 32-row chunks."""
import numpy as np
import pytest

from oracle import leverage as LV, sampling as S, core_update as CU
from tests.gpu_common import dev, host_keys, rel_err, handle  # noqa: F401
from tests.test_gpu_fullsize import _check_gram_entries, _check_residual, BF16_C, TF32_C
from paper_2107_10654_gb300 import tucker as T

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,ranks,prec", [
    ((48, 40, 40), (4, 16, 16), "bf16"),          # d = 1024, d / R_1 = 256
    ((30, 24, 20, 22), (8, 8, 4, 4), "bf16"),     # order 4, d / R_1 = 128
    ((64, 36, 36), (16, 8, 16), "tf32"),          # R_1 = 16, d / R_1 = 128
    ((40, 30, 25), (4, 12, 11), "tf32"),          # d / R_1 = 132: ragged 16-blocks
    ((24, 40, 40), (2, 16, 17), "bf16"),          # d / R_1 = 272: two 256-wide tiles of M
    ((70, 30, 30), (16, 16, 16), "tf32"),         # the 1024^3 ranks: R_1^2 = 256 pairs
])
def test_grouped_gram_and_solve(handle, dims, ranks, prec):
    g = np.random.default_rng(21)
    F = [g.standard_normal((i, r)).astype(np.float32) for i, r in zip(dims, ranks)]
    X = g.standard_normal(dims).astype(np.float32)
    Fd, Xd = [dev(a) for a in F], dev(X)
    m = 6000
    levs = [LV.leverage_scores(np.asarray(a, dtype=np.float64))[0] for a in F]
    smp = T.tucker_sample_rows(handle, dims, ranks, [dev(l) for l in levs], m, 5, 0)
    ku = host_keys(smp.keys, smp.n_unique)
    cnt = smp.counts[:smp.n_unique].cpu().numpy().astype(np.float64)
    w = S.sample_weights(cnt, smp.prob[:smp.n_unique].cpu().numpy(), smp.n_draws)
    G, h = T.tucker_sketched_gram(handle, Xd, Fd, prec, smp)
    Gh = G.cpu().numpy()
    assert np.array_equal(Gh, Gh.T)
    _check_gram_entries(F, dims, ku, w, Gh, n_pairs=160, seed=3,
                        c=BF16_C if prec == "bf16" else TF32_C)
    x = CU.gather_dense(X, ku, dims)
    hr = CU.sampled_rows_apply_t(F, S.decode_keys(ku, dims), w * x)
    assert rel_err(h.cpu().numpy(), hr) <= 1e-12
    core = T.tucker_core_update_sketched(handle, Xd, Fd, 0.1, 0, 0, 0, "exact", prec, fixed=smp)
    _check_residual(F, dims, ku, w, x, 0.1, core.cpu().numpy())


NARROW_C = 2.0 ** -16


@pytest.mark.parametrize("dims,ranks,m,prec", [
    ((96, 80, 72), (8, 8, 8), 6000, "tf32"),        # the 512^3 ranks: d' = 64, R_1 = 8
    ((96, 80, 72), (8, 8, 8), 6000, "bf16"),
    ((40, 44, 48), (16, 4, 16), 9000, "tf32"),      # R_1 = 16: 256 pairs, d' = 64
    ((300, 30, 30), (4, 3, 5), 4000, "tf32"),       # d' = 15 (ragged), many empty segments
    ((60, 30, 30), (2, 8, 8), 8000, "bf16"),        # R_1 = 2, about 130 rows per segment
    ((24, 20, 20, 20), (4, 4, 4, 4), 7000, "tf32"),  # order 4, d' = 64
    ((40, 30, 30), (16, 2, 4), 5000, "tf32"),       # R_1 = 16, d' = 8
])
def test_narrow_grouped_gram_and_solve(handle, dims, ranks, m, prec):
    g = np.random.default_rng(33)
    F = [g.standard_normal((i, r)).astype(np.float32) for i, r in zip(dims, ranks)]
    X = g.standard_normal(dims).astype(np.float32)
    Fd, Xd = [dev(a) for a in F], dev(X)
    levs = [LV.leverage_scores(np.asarray(a, dtype=np.float64))[0] for a in F]
    smp = T.tucker_sample_rows(handle, dims, ranks, [dev(l) for l in levs], m, 9, 0)
    ku = host_keys(smp.keys, smp.n_unique)
    cnt = smp.counts[:smp.n_unique].cpu().numpy().astype(np.float64)
    w = S.sample_weights(cnt, smp.prob[:smp.n_unique].cpu().numpy(), smp.n_draws)
    G, h = T.tucker_sketched_gram(handle, Xd, Fd, prec, smp)
    Gh = G.cpu().numpy()
    assert np.array_equal(Gh, Gh.T)
    _check_gram_entries(F, dims, ku, w, Gh, n_pairs=200, seed=4, c=NARROW_C)
    x = CU.gather_dense(X, ku, dims)
    hr = CU.sampled_rows_apply_t(F, S.decode_keys(ku, dims), w * x)
    assert rel_err(h.cpu().numpy(), hr) <= 1e-12
    core = T.tucker_core_update_sketched(handle, Xd, Fd, 0.1, 0, 0, 0, "exact", prec, fixed=smp)
    _check_residual(F, dims, ku, w, x, 0.1, core.cpu().numpy())


def test_narrow_grouped_gram_whole_matrix(handle):
    """Every entry of a small narrow grouped Gram against the explicit
    K_S^T W K_S (a transposed block, a wrong pair or a wrong mirror shows up as
    an O(1) error in some entry that sampled pairs could miss)."""
    dims, ranks, m = (50, 20, 24), (4, 4, 4), 3000
    g = np.random.default_rng(35)
    F = [g.standard_normal((i, r)).astype(np.float32) for i, r in zip(dims, ranks)]
    X = g.standard_normal(dims).astype(np.float32)
    levs = [LV.leverage_scores(np.asarray(a, dtype=np.float64))[0] for a in F]
    smp = T.tucker_sample_rows(handle, dims, ranks, [dev(l) for l in levs], m, 2, 0)
    ku = host_keys(smp.keys, smp.n_unique)
    cnt = smp.counts[:smp.n_unique].cpu().numpy().astype(np.float64)
    w = S.sample_weights(cnt, smp.prob[:smp.n_unique].cpu().numpy(), smp.n_draws)
    G, _ = T.tucker_sketched_gram(handle, dev(X), [dev(a) for a in F], "tf32", smp)
    K = CU.kron_rows([np.asarray(a, dtype=np.float64) for a in F], S.decode_keys(ku, dims))
    Gr = K.T @ (K * w[:, None])
    absG = np.abs(K).T @ (np.abs(K) * w[:, None])
    err = np.abs(G.cpu().numpy() - Gr)
    assert (err <= NARROW_C * absG + 1e-12 * np.max(absG)).all(), float(np.max(err / absG))
