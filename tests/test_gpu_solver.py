"""GPU parity of the mixed ridge solver (FP32 Cholesky preconditioning an FP64
iterative refinement) against the FP64 oracle, at the same tolerances as the
FP64 Cholesky solver: FP64 Gram 1e-10, FP32 Gram 1e-5, tensor-core Grams 1e-6.
"""
import dataclasses

import numpy as np
import pytest
import torch

import synth
from oracle import sampling as S, core_update as CU
from tests.gpu_common import dev, dev_keys, rel_err, handle  # noqa: F401
from tests.test_gpu_core import CASES, TOL, _small, _ragged_problem
from paper_2107_10654_gb300 import tucker as T
from paper_2107_10654_gb300 import _lib as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mixed():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    h = T.Handle(solver="mixed")
    yield h
    h.close()


@pytest.mark.parametrize("name,dims,ranks,m,prec", CASES)
@pytest.mark.parametrize("reg", ["exact", "augmented"])
def test_mixed_sketched_core_matches_oracle(mixed, name, dims, ranks, m, prec, reg):
    w = _small(name, dims, m, ranks)
    P = synth.tucker_problem(w)
    X, F = P["X"], P["factors"]
    regc = S.REG_EXACT if reg == "exact" else S.REG_AUGMENTED
    ref = CU.sketched_core(X, F, w.lam, w.m, w.seed_sample, 0, regc)
    g, st = T.tucker_core_update_sketched(mixed, dev(X), [dev(a) for a in F], w.lam, w.m,
                                          w.seed_sample, 0, reg, prec, stats=True)
    assert st["n_unique"] == ref["keys"].size and st["n_draws"] == ref["T"]
    assert 1 <= st["refine_iters"] <= 12
    assert rel_err(g.cpu().numpy(), ref["g"]) <= TOL[prec]


@pytest.mark.parametrize("dims,ranks,dtype,prec", [
    ((37, 29, 23), (3, 5, 2), np.float64, "fp64"),        # d = 30: ragged 32/64 blocks
    ((20, 70, 9), (4, 7, 3), np.float32, "fp32"),         # d = 84
    ((11, 13), (5, 13), np.float64, "fp64"),              # order 2, d = 65
    ((200,), (9,), np.float64, "fp64"),                   # order 1, d = 9
])
def test_mixed_ragged(mixed, dims, ranks, dtype, prec):
    X, F = _ragged_problem(dims, ranks, dtype, 1)
    m = 3001
    ref = CU.sketched_core(X, F, 0.05, m, 99, 2, S.REG_EXACT)
    g = T.tucker_core_update_sketched(mixed, dev(X), [dev(a) for a in F], 0.05, m, 99, 2,
                                      "exact", prec)
    assert rel_err(g.cpu().numpy(), ref["g"]) <= TOL[prec]


def test_mixed_exact_missing(mixed):
    w = _small("missing3_1024_r16_f32", (40, 36, 30))
    w = dataclasses.replace(w, ranks=(3, 4, 2))
    O = synth.observed_entries(w)
    ref = CU.exact_core_rows(O["keys"], O["vals"], O["dims"], O["factors"], w.lam)
    coo = T.CooTensor(dev_keys(O["keys"]), dev(O["vals"]), O["dims"])
    g = T.tucker_core_update_exact(mixed, coo, [dev(a) for a in O["factors"]], w.lam, "fp64")
    assert rel_err(g.cpu().numpy(), ref) <= 1e-6       # FP32 values, FP64 arithmetic


def test_mixed_adjoint_matches_fp64_solver(mixed, handle):
    X, F = _ragged_problem((30, 26, 22), (3, 4, 2), np.float64, 7)
    levs = [CU.leverage_scores(A)[0] for A in F]
    smp = T.tucker_sample_rows(handle, X.shape, (3, 4, 2), [dev(l) for l in levs], 2500, 4, 0)
    Xd, Fd = dev(X), [dev(a) for a in F]
    gbar = dev(np.random.default_rng(3).standard_normal(24))
    out = []
    for h in (handle, mixed):
        g, st = T.tucker_core_update_sketched(h, Xd, Fd, 0.1, 0, 0, 0, "exact", "fp64",
                                              fixed=smp, stats=True)
        dA, dx = T.tucker_core_solve_adjoint(h, Xd, Fd, 0.1, "exact", "fp64", smp,
                                             st["solve_id"], g, gbar)
        out.append((g.cpu().numpy(), [a.cpu().numpy() for a in dA], dx.cpu().numpy()))
    assert rel_err(out[1][0], out[0][0]) <= 1e-12
    for a, b in zip(out[1][1], out[0][1]):
        assert rel_err(a, b) <= 1e-11
    assert rel_err(out[1][2], out[0][2]) <= 1e-11


def test_mixed_not_spd_and_bad_solver(mixed):
    X, F = _ragged_problem((10, 9, 8), (2, 2, 2), np.float64, 5)
    F_bad = [f.copy() for f in F]
    F_bad[1][:, 1] = 0.0
    with pytest.raises(T.TuckerError) as e:
        T.tucker_core_update_sketched(mixed, dev(X), [dev(a) for a in F_bad], 0.0, 500, 1, 0,
                                      "exact", "fp64")
    assert e.value.name == "ENOTSPD"
    st = L.load().tucker_set_solver(mixed.h, 7)
    assert st == L.EINVAL
    g = T.tucker_core_update_sketched(mixed, dev(X), [dev(a) for a in F], 0.1, 500, 1)
    assert torch.isfinite(g).all()
