"""GPU parity of the sketched normal equations G = sum w k k^T, h = sum w x k.

FP64 Gram: relative 1e-12 of the oracle.  Tensor-core Grams (BF16 / TF32
operands, FP32 accumulation): every entry within a bound set by operand
rounding, |dG_ij| <= c * sum_u w_u |k_ui| |k_uj| with c = 2^-7 (BF16: two
operands each rounded to 8 significant bits) or 2^-9 (TF32: 11 bits), which
catches any tile, swizzle or descriptor error (those give O(1) errors).
Shapes cover one partial tile, several 128 x 256 tiles with and without the
diagonal, ragged d, orders 2 to 4.
"""
import numpy as np
import pytest
import torch

from oracle import leverage as LV, sampling as S, core_update as CU, als as ALS
from tests.gpu_common import dev, host_keys, handle  # noqa: F401
from paper_2107_10654_gb300 import tucker as T

pytestmark = pytest.mark.gpu

SHAPES = [
    ((96, 80, 72), (8, 8, 8), 6000),          # d = 512: 3 upper tiles
    ((40, 36, 48, 44), (4, 4, 4, 4), 5000),   # d = 256, order 4
    ((50, 60, 70), (3, 5, 7), 3000),          # d = 105: one ragged tile
    ((64, 90), (16, 20), 4000),               # order 2, d = 320, ragged
    ((40, 44, 48), (8, 8, 16), 9000),         # d = 1024, d / R_1 = 128: grouped by i_1
    ((40, 44, 48), (16, 4, 16), 9000),        # d = 1024, d / R_1 = 64: full width, 10 tiles
]


def _problem(dims, ranks, seed):
    g = np.random.default_rng(seed)
    core = g.standard_normal(ranks)
    F = [g.standard_normal((i, r)) for i, r in zip(dims, ranks)]
    X = ALS.tucker_model(core, F) + 0.1 * g.standard_normal(dims)
    return X.astype(np.float32), [f.astype(np.float32) for f in F]


def _oracle_normal_eq(X, F, smp):
    dims = X.shape
    keys = host_keys(smp.keys, smp.n_unique)
    levs = [LV.leverage_scores(A)[0] for A in F]
    p = S.row_probabilities(keys, levs, dims)
    w = S.sample_weights(smp.counts[:smp.n_unique].cpu().numpy().astype(np.float64), p,
                         smp.n_draws)
    x = CU.gather_dense(X, keys, dims)
    G, h, _ = CU.sketched_normal_equations(F, dims, keys, w, x)
    K = np.abs(CU.kron_rows(F, S.decode_keys(keys, dims)))
    absG = K.T @ (K * w[:, None])
    return G, h, absG, levs


@pytest.mark.parametrize("dims,ranks,m", SHAPES)
@pytest.mark.parametrize("prec", ["fp64", "bf16", "tf32"])
def test_sketched_gram_matches_oracle(handle, dims, ranks, m, prec):
    X, F = _problem(dims, ranks, 11)
    levs = [LV.leverage_scores(A)[0] for A in F]
    smp = T.tucker_sample_rows(handle, dims, ranks, [dev(l) for l in levs], m, 17, 0)
    G, h = T.tucker_sketched_gram(handle, dev(X), [dev(a) for a in F], prec, smp)
    Gr, hr, absG, _ = _oracle_normal_eq(X, F, smp)
    G = G.cpu().numpy()
    assert np.array_equal(G, G.T)
    assert np.max(np.abs(h.cpu().numpy() - hr)) <= 1e-12 * np.max(np.abs(hr))
    if prec == "fp64":
        assert np.max(np.abs(G - Gr)) <= 1e-12 * np.max(np.abs(Gr))
    else:
        c = 2.0 ** -7 if prec == "bf16" else 2.0 ** -9
        err = np.abs(G - Gr)
        bound = c * absG + 1e-6 * np.max(absG)
        bad = err > bound
        assert not bad.any(), (np.argwhere(bad)[:5], err[bad][:5], bound[bad][:5])
        # and it is not trivially loose: the typical error is far below the bound
        assert np.median(err / (absG + 1e-300)) < c / 4
