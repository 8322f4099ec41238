"""GPU parity of paths the other files reach only in part:

  * the exact observed-entry update (Alg. 2 core line restricted to the
    observed rows of Sec. 4.2) on the tensor-core Gram grouped by the leading
    index, BF16 and TF32 with FP64 refinement, against the oracle's explicit
    normal equations over every observed row;
  * a sketched update with m = 0, which draws the paper's sample count s of
    Alg. 1 line 3 (beta' = 1/2, eps = delta = 0.1), against the oracle's count
    and its sketched core at that count;
  * the torch.autograd.Function over the frozen-sketch solve: the gradients
    autograd hands back for the factors and for the dense tensor (scattered to
    the sampled entries) against the oracle's adjoint;
  * the two-level sorted-sample walks (runs of equal (i_1, i_2) long enough,
    prod_{n >= 3} R_n a multiple of 32): the right-hand side h = K_S^T W x and the
    FP64 residual of the refined core against the oracle's explicit rows, for
    orders 3 and 4 and both the TF32 and the FP64 Gram.
"""
import dataclasses

import numpy as np
import pytest
import torch

import synth
from oracle import leverage as LV, sampling as S, core_update as CU, adjoint as ADJ
from tests.gpu_common import dev, dev_keys, host_keys, rel_err, handle  # noqa: F401
from paper_2107_10654_gb300 import tucker as T

pytestmark = pytest.mark.gpu


def _grouped(N, d, R1, I1):
    """The library's predicate for the leading-index grouping of the tensor-core Gram."""
    if N < 3 or R1 > 16 or R1 & (R1 - 1) or d % R1:
        return False
    dp = d // R1
    tiles = (dp + 255) // 256
    return dp >= 128 and I1 * tiles * (tiles + 1) // 2 <= 8192 and I1 * R1 * 4 <= 200 * 1024


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("solver", ["fp64", "mixed"])
def test_exact_missing_on_grouped_tensor_core_gram(prec, solver):
    w = synth.WORKLOADS["missing3_1024_r16_f32"]
    w = dataclasses.replace(w, ranks=(4, 16, 16), lam=0.1)
    dims = (48, 40, 40)
    assert _grouped(3, w.d, w.ranks[0], dims[0])            # d / R_1 = 256: grouped
    O = synth.observed_entries(w, dims=dims, frac=0.1)
    ref = CU.exact_core_rows(O["keys"], O["vals"], O["dims"], O["factors"], w.lam)
    coo = T.CooTensor(dev_keys(O["keys"]), dev(O["vals"]), O["dims"])
    with T.Handle(solver=solver) as h:
        g = T.tucker_core_update_exact(h, coo, [dev(a) for a in O["factors"]], w.lam, prec)
        torch.cuda.synchronize()
    assert rel_err(g.cpu().numpy(), ref) <= 1e-6


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("bf16", 1e-6)])
def test_paper_sample_count_when_m_is_zero(handle, prec, tol):
    rng = np.random.default_rng(21)
    dims, ranks, lam = (30, 20, 25), (2, 2, 2), 0.05
    F = [rng.standard_normal((i, r)) for i, r in zip(dims, ranks)]
    X = rng.standard_normal(dims)
    d = int(np.prod(ranks))
    s = S.paper_sample_count(d, 0.1, 0.1)
    assert s == 155053                                     # the count Alg. 1 line 3 gives at d = 8
    g, st = T.tucker_core_update_sketched(handle, dev(X), [dev(a) for a in F], lam, 0, 7, 0,
                                          "exact", prec, eps=0.1, delta=0.1, stats=True)
    assert st["n_draws"] == s
    ref = CU.sketched_core(X, F, lam, s, 7, 0, S.REG_EXACT)
    assert st["n_unique"] == ref["keys"].size
    assert rel_err(g.cpu().numpy(), ref["g"]) <= tol


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("bf16", 1e-6)])
def test_autograd_function_matches_oracle_adjoint(handle, prec, tol):
    from paper_2107_10654_gb300 import SketchedCoreSolve
    rng = np.random.default_rng(22)
    dims, ranks, lam = (20, 18, 16), (2, 3, 2), 0.2
    F = [rng.standard_normal((i, r)) for i, r in zip(dims, ranks)]
    X = rng.standard_normal(dims)
    d = int(np.prod(ranks))
    levs = [LV.leverage_scores(a)[0] for a in F]
    smp = T.tucker_sample_rows(handle, dims, ranks, [dev(l) for l in levs], 1500, 9, 0)
    A = [dev(a).requires_grad_(True) for a in F]
    Xd = dev(X).requires_grad_(True)
    g = SketchedCoreSolve.apply(handle, Xd, smp, lam, "exact", prec, *A)
    c = np.linspace(-1.0, 1.0, d)
    (g * torch.from_numpy(c).cuda()).sum().backward()
    keys = host_keys(smp.keys, smp.n_unique)
    cnt = smp.counts[:smp.n_unique].cpu().numpy().astype(np.float64)
    p = S.row_probabilities(keys, levs, dims, S.REG_EXACT, d)
    wts = S.sample_weights(cnt, p, smp.n_draws)
    x = CU.gather_dense(X, keys, dims)
    rg = ADJ.forward(F, dims, keys, wts, x, lam, np.ones(d))
    assert rel_err(g.detach().cpu().numpy(), rg) <= tol
    rdA, rdx = ADJ.backward(F, dims, keys, wts, x, lam, np.ones(d), c)
    for a, b in zip(A, rdA):
        assert rel_err(a.grad.cpu().numpy(), b) <= tol
    # dL/dX: the oracle's dx at the sampled entries, zero everywhere else
    ref_dX = np.zeros(X.size)
    ref_dX[keys.astype(np.int64)] = rdx
    got = Xd.grad.cpu().numpy().reshape(-1)
    assert rel_err(got, ref_dX) <= tol
    assert np.all(got[np.setdiff1d(np.arange(X.size), keys.astype(np.int64))] == 0.0)


@pytest.mark.parametrize("dims,ranks,m,prec", [
    ((10, 12, 30, 30), (4, 8, 8, 8), 20000, "tf32"),   # order 4: W_2 of 64 entries
    ((10, 12, 30, 30), (4, 8, 8, 8), 20000, "fp64"),
    ((20, 30, 200), (2, 4, 32), 8000, "tf32"),         # order 3: W_2 of 32 entries
])
def test_two_level_walks(handle, dims, ranks, m, prec):
    from tests.test_gpu_fullsize import _check_residual
    g = np.random.default_rng(41)
    F = [g.standard_normal((i, r)).astype(np.float32) for i, r in zip(dims, ranks)]
    X = g.standard_normal(dims).astype(np.float32)
    Fd, Xd = [dev(a) for a in F], dev(X)
    assert m >= 4 * dims[0] * dims[1]                   # the library's test for two levels
    levs = [LV.leverage_scores(np.asarray(a, dtype=np.float64))[0] for a in F]
    smp = T.tucker_sample_rows(handle, dims, ranks, [dev(l) for l in levs], m, 13, 0)
    ku = host_keys(smp.keys, smp.n_unique)
    cnt = smp.counts[:smp.n_unique].cpu().numpy().astype(np.float64)
    w = S.sample_weights(cnt, smp.prob[:smp.n_unique].cpu().numpy(), smp.n_draws)
    _, h = T.tucker_sketched_gram(handle, Xd, Fd, prec, smp)
    x = CU.gather_dense(X, ku, dims)
    hr = CU.sampled_rows_apply_t(F, S.decode_keys(ku, dims), w * x)
    assert rel_err(h.cpu().numpy(), hr) <= 1e-12
    core = T.tucker_core_update_sketched(handle, Xd, Fd, 0.1, 0, 0, 0, "exact", prec, fixed=smp)
    _check_residual(F, dims, ku, w, x, 0.1, core.cpu().numpy())
