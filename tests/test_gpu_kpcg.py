"""GPU parity of the Kronecker-preconditioned CG ridge solver
(TUCKER_SOLVER_KRON_PCG): conjugate gradients on the rounded Gram M~,
preconditioned by (x) V_n diag(s (x) ev_n + lbar) (x) V_n^T, inside the FP64
refinement, against the FP64 oracle at the tolerances of the other solvers
(FP32 Gram 1e-5, tensor-core Grams 1e-6).  Also: the observed-entry paths,
the adjoint, an observation mask far from uniform, and that the CG path is the
one that ran (stats inner_iters > 0)."""
import dataclasses

import numpy as np
import pytest
import torch

import synth
from oracle import leverage as LV, sampling as S, core_update as CU
from tests.gpu_common import dev, dev_keys, rel_err, handle  # noqa: F401
from tests.test_gpu_core import CASES, TOL, _small, _ragged_problem
from paper_2107_10654_gb300 import tucker as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kpcg():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    h = T.Handle(solver="kpcg")
    yield h
    h.close()


ROUNDED = [c for c in CASES if c[-1] != "fp64"]


@pytest.mark.parametrize("name,dims,ranks,m,prec", ROUNDED)
@pytest.mark.parametrize("reg", ["exact", "augmented"])
def test_kpcg_sketched_core_matches_oracle(kpcg, name, dims, ranks, m, prec, reg):
    w = _small(name, dims, m, ranks)
    P = synth.tucker_problem(w)
    X, F = P["X"], P["factors"]
    regc = S.REG_EXACT if reg == "exact" else S.REG_AUGMENTED
    ref = CU.sketched_core(X, F, w.lam, w.m, w.seed_sample, 0, regc)
    g, st = T.tucker_core_update_sketched(kpcg, dev(X), [dev(a) for a in F], w.lam, w.m,
                                          w.seed_sample, 0, reg, prec, stats=True)
    assert st["n_unique"] == ref["keys"].size and st["n_draws"] == ref["T"]
    assert st["inner_iters"] > 0                       # the CG path ran and met its target
    assert rel_err(g.cpu().numpy(), ref["g"]) <= TOL[prec]


@pytest.mark.parametrize("dims,ranks,prec", [
    ((37, 29, 23), (3, 5, 2), "fp32"),                    # d = 30: no 16-byte rows
    ((20, 70, 9), (4, 7, 3), "bf16"),                     # d = 84
    ((11, 13), (5, 13), "tf32"),                          # order 2, d = 65
    ((200,), (9,), "fp32"),                               # order 1, d = 9
    ((48, 40, 40), (4, 16, 16), "bf16"),                  # grouped Gram, d = 1024
])
def test_kpcg_ragged(kpcg, dims, ranks, prec):
    X, F = _ragged_problem(dims, ranks, np.float32, 1)
    m = 3001 if int(np.prod(ranks)) < 512 else 12000
    ref = CU.sketched_core(X, F, 0.05, m, 99, 2, S.REG_EXACT)
    g, st = T.tucker_core_update_sketched(kpcg, dev(X), [dev(a) for a in F], 0.05, m, 99, 2,
                                          "exact", prec, stats=True)
    assert st["inner_iters"] != 0
    assert rel_err(g.cpu().numpy(), ref["g"]) <= TOL[prec]


def test_kpcg_missing_sketched_and_exact(kpcg):
    w = _small("missing3_1024_r16_f32", (48, 40, 40))
    w = dataclasses.replace(w, ranks=(4, 8, 8), m=20000)
    O = synth.observed_entries(w, frac=0.1)
    coo = T.CooTensor(dev_keys(O["keys"]), dev(O["vals"]), O["dims"])
    Fd = [dev(a) for a in O["factors"]]
    ref = CU.sketched_core(None, O["factors"], w.lam, w.m, w.seed_sample, 0, S.REG_EXACT,
                           observed=(O["keys"], O["vals"], O["dims"]))
    g, st = T.tucker_core_update_sketched(kpcg, coo, Fd, w.lam, w.m, w.seed_sample, 0, "exact",
                                          "bf16", stats=True)
    assert st["n_draws"] == ref["T"] and st["inner_iters"] > 0
    assert rel_err(g.cpu().numpy(), ref["g"]) <= 1e-6
    ref_e = CU.exact_core_rows(O["keys"], O["vals"], O["dims"], O["factors"], w.lam)
    ge = T.tucker_core_update_exact(kpcg, coo, Fd, w.lam, "bf16")
    assert rel_err(ge.cpu().numpy(), ref_e) <= 1e-6


def test_kpcg_far_from_uniform_mask(kpcg):
    # only the slice i_1 = 0 observed: K_Omega^T K_Omega = (a a^T) (x) K_23^T K_23 is far
    # from any multiple of K^T K (the preconditioner), so CG needs many iterations or the
    # factor takes over; either way the result meets the tolerance
    rng = np.random.default_rng(3)
    dims, ranks, lam = (40, 30, 20), (3, 2, 2), 1e-3
    F = [rng.standard_normal((i, r)).astype(np.float32) for i, r in zip(dims, ranks)]
    inner = dims[1] * dims[2]
    keys = np.arange(inner, dtype=np.uint64)
    vals = rng.standard_normal(inner).astype(np.float32)
    coo = T.CooTensor(dev_keys(keys), dev(vals), dims)
    ref = CU.exact_core_rows(keys, vals, dims, F, lam)
    g = T.tucker_core_update_exact(kpcg, coo, [dev(a) for a in F], lam, "tf32")
    assert rel_err(g.cpu().numpy(), ref) <= 1e-6


def test_kpcg_adjoint_matches_fp64_solver(kpcg, handle):
    X, F = _ragged_problem((30, 26, 22), (3, 4, 2), np.float32, 7)
    levs = [LV.leverage_scores(np.asarray(A, dtype=np.float64))[0] for A in F]
    smp = T.tucker_sample_rows(handle, X.shape, (3, 4, 2), [dev(l) for l in levs], 2500, 4, 0)
    Xd, Fd = dev(X), [dev(a) for a in F]
    gbar = dev(np.random.default_rng(3).standard_normal(24))
    out = []
    for h in (handle, kpcg):
        g, st = T.tucker_core_update_sketched(h, Xd, Fd, 0.1, 0, 0, 0, "exact", "bf16",
                                              fixed=smp, stats=True)
        dA, dx = T.tucker_core_solve_adjoint(h, Xd, Fd, 0.1, "exact", "bf16", smp,
                                             st["solve_id"], g, gbar)
        out.append((g.cpu().numpy(), [a.cpu().numpy() for a in dA], dx.cpu().numpy()))
    assert rel_err(out[1][0], out[0][0]) <= 1e-7
    for a, b in zip(out[1][1], out[0][1]):
        assert rel_err(a, b) <= 1e-6
    assert rel_err(out[1][2], out[0][2]) <= 1e-6


def test_kpcg_bench_workload(kpcg):
    w = synth.WORKLOADS["dense3_512_r8_f32"]
    P = synth.tucker_problem(w)
    X, F = P["X"], P["factors"]
    g, st = T.tucker_core_update_sketched(kpcg, dev(X), [dev(a) for a in F], w.lam, w.m,
                                          w.seed_sample, 0, "exact", "bf16", stats=True)
    ref = CU.sketched_core(X, F, w.lam, w.m, w.seed_sample, 0, S.REG_EXACT)
    assert st["inner_iters"] > 0
    assert rel_err(g.cpu().numpy(), ref["g"]) <= 1e-6


@pytest.mark.parametrize("solver", ["kpcg", "mixed", "fp64"])
@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_rounded_gram_not_spd_falls_back_to_cuda_core_grams(solver, prec):
    # a nearly repeated column and lambda = 0: the tensor-core Gram of rounded rows is
    # PSD except for its FP32 accumulation (about 2^-24 ||G|| ~ 2.6e-3 here), which
    # exceeds the smallest eigenvalue (about 2.7e-5), so the rounded matrix has no
    # Cholesky factor, or its refinement stalls; the update rebuilds the Gram of the same
    # rows on the CUDA cores (FP32, then FP64) with an FP64 factor and still meets the
    # oracle (kappa ~ 1.6e9)
    rng = np.random.default_rng(31)
    dims, ranks, lam = (30, 25, 20), (3, 2, 2), 0.0
    F = [rng.standard_normal((i, r)) for i, r in zip(dims, ranks)]
    F[0][:, 2] = F[0][:, 0] + 1e-4 * rng.standard_normal(dims[0])
    X = rng.standard_normal(dims)
    levs = [LV.leverage_scores(a)[0] for a in F]
    with T.Handle(solver=solver) as h:
        smp = T.tucker_sample_rows(h, dims, ranks, [dev(l) for l in levs], 6000, 3, 0)
        g, st = T.tucker_core_update_sketched(h, dev(X), [dev(a) for a in F], lam, 0, 0, 0,
                                              "exact", prec, fixed=smp, stats=True)
        torch.cuda.synchronize()
    ref = CU.sketched_core(X, F, lam, 6000, 3, 0, S.REG_EXACT)
    assert smp.n_unique == ref["keys"].size
    if solver != "kpcg":
        # a factor of the rounded matrix fails or its refinement stalls: CUDA-core Grams
        assert st["gram_prec_used"] in (T.PREC["fp32"], T.PREC["fp64"]), st["gram_prec_used"]
    # (CG with the FP64 correction may still reach the target on the rounded Gram)
    assert rel_err(g.cpu().numpy(), ref["g"]) <= 1e-6
