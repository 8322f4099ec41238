"""GPU parity of the core updates, ALS sweeps, ridge loss and adjoint.

Tolerances (relative, 2-norm over the core): FP64 path 1e-10; FP32 data with
the FP32 Gram 1e-5; tensor-core Grams after FP64 refinement 1e-6.  Inputs are
the seeded synthetic workloads (scaled down where the oracle must finish in
seconds) and small ragged shapes.
"""
import dataclasses

import numpy as np
import pytest
import torch

import synth
from oracle import sampling as S, core_update as CU, als as ALS, adjoint as ADJ
from tests.gpu_common import dev, dev_keys, host_keys, rel_err, handle  # noqa: F401
from paper_2107_10654_gb300 import tucker as T

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5, "tf32": 1e-6, "bf16": 1e-6}


def _small(name, dims=None, m=None, ranks=None):
    w = synth.WORKLOADS[name]
    kw = {}
    if dims is not None:
        kw["dims"] = dims
    if m is not None:
        kw["m"] = m
    if ranks is not None:
        kw["ranks"] = ranks
    return dataclasses.replace(w, **kw) if kw else w


def _ragged_problem(dims, ranks, dtype, seed=0, sigma=0.1):
    g = np.random.default_rng(seed)
    core = g.standard_normal(ranks)
    F = [g.standard_normal((i, r)) for i, r in zip(dims, ranks)]
    X = ALS.tucker_model(core, F) + sigma * g.standard_normal(dims)
    return X.astype(dtype), [f.astype(dtype) for f in F]


# shapes keep I_n >> R_n like the workloads (well-conditioned factor Grams)
CASES = [
    ("dense3_64_r4_f64", None, None, None, "fp64"),
    ("dense3_512_r8_f32", (96, 80, 72), None, 6000, "fp32"),
    ("dense3_512_r8_f32", (96, 80, 72), None, 6000, "fp64"),
    ("dense4_128_r8_f32", (40, 36, 48, 44), (4, 4, 4, 4), 8000, "fp32"),
    ("dense3_512_r8_f32", (96, 80, 72), None, 6000, "bf16"),
    ("dense3_512_r8_f32", (96, 80, 72), None, 6000, "tf32"),
    ("dense4_128_r8_f32", (40, 36, 48, 44), (4, 4, 4, 4), 8000, "bf16"),
]


@pytest.mark.parametrize("name,dims,ranks,m,prec", CASES)
@pytest.mark.parametrize("reg", ["exact", "augmented"])
def test_sketched_core_matches_oracle(handle, name, dims, ranks, m, prec, reg):
    w = _small(name, dims, m, ranks)
    P = synth.tucker_problem(w)
    X, F = P["X"], P["factors"]
    regc = S.REG_EXACT if reg == "exact" else S.REG_AUGMENTED
    ref = CU.sketched_core(X, F, w.lam, w.m, w.seed_sample, 0, regc)
    g, st = T.tucker_core_update_sketched(handle, dev(X), [dev(a) for a in F], w.lam, w.m,
                                          w.seed_sample, 0, reg, prec, stats=True)
    assert st["n_unique"] == ref["keys"].size and st["n_draws"] == ref["T"]
    assert rel_err(g.cpu().numpy(), ref["g"]) <= TOL[prec]


@pytest.mark.parametrize("dims,ranks,dtype,prec", [
    ((37, 29, 23), (3, 5, 2), np.float64, "fp64"),        # d = 30: ragged 64-tiles
    ((20, 70, 9), (4, 7, 3), np.float32, "fp32"),         # d = 84
    ((11, 13), (5, 13), np.float64, "fp64"),              # order 2, d = 65
    ((200,), (9,), np.float64, "fp64"),                   # order 1
])
def test_sketched_core_ragged(handle, dims, ranks, dtype, prec):
    X, F = _ragged_problem(dims, ranks, dtype, 1)
    m = 3001
    ref = CU.sketched_core(X, F, 0.05, m, 99, 2, S.REG_EXACT)
    g = T.tucker_core_update_sketched(handle, dev(X), [dev(a) for a in F], 0.05, m, 99, 2,
                                      "exact", prec)
    assert rel_err(g.cpu().numpy(), ref["g"]) <= TOL[prec]


def test_sketched_core_missing_entries(handle):
    w = _small("missing3_1024_r16_f32", (48, 40, 36), 8000)
    w = dataclasses.replace(w, ranks=(4, 4, 4))
    O = synth.observed_entries(w)
    keys, vals, F = O["keys"], O["vals"], O["factors"]
    ref = CU.sketched_core(None, F, w.lam, w.m, w.seed_sample, 0, S.REG_EXACT,
                           observed=(keys, vals, O["dims"]))
    coo = T.CooTensor(dev_keys(keys), dev(vals), O["dims"])
    g, st = T.tucker_core_update_sketched(handle, coo, [dev(a) for a in F], w.lam, w.m,
                                          w.seed_sample, 0, "exact", "fp32", stats=True)
    assert st["n_draws"] == ref["T"] and st["n_unique"] == ref["keys"].size
    assert rel_err(g.cpu().numpy(), ref["g"]) <= TOL["fp32"]


def test_frozen_sketch_reuse(handle):
    X, F = _ragged_problem((30, 20, 25), (3, 2, 4), np.float64, 2)
    levs = [CU.leverage_scores(A)[0] for A in F]
    smp = T.tucker_sample_rows(handle, X.shape, (3, 2, 4), [dev(l) for l in levs], 2000, 5, 1)
    g1 = T.tucker_core_update_sketched(handle, dev(X), [dev(a) for a in F], 0.1, 2000, 5, 1)
    g2 = T.tucker_core_update_sketched(handle, dev(X), [dev(a) for a in F], 0.1, 0, 0, 0,
                                       fixed=smp)
    assert rel_err(g2.cpu().numpy(), g1.cpu().numpy()) <= 1e-12


@pytest.mark.parametrize("dims,ranks,dtype,prec,tol", [
    ((64, 64, 64), (4, 4, 4), np.float64, "fp64", 1e-10),
    ((96, 80, 72), (8, 8, 8), np.float32, "fp32", 1e-5),
    ((20, 18, 16, 14), (3, 4, 2, 5), np.float64, "fp64", 1e-10),
    ((33, 17), (5, 7), np.float32, "fp32", 1e-5),
])
def test_exact_core_dense(handle, dims, ranks, dtype, prec, tol):
    X, F = _ragged_problem(dims, ranks, dtype, 3)
    ref = CU.exact_core_kron_eig(X, F, 1e-2)
    g = T.tucker_core_update_exact(handle, dev(X), [dev(a) for a in F], 1e-2, prec)
    assert rel_err(g.cpu().numpy(), ref) <= tol


def test_exact_core_missing(handle):
    w = _small("missing3_1024_r16_f32", (40, 36, 30))
    w = dataclasses.replace(w, ranks=(3, 4, 2))
    O = synth.observed_entries(w)
    ref = CU.exact_core_rows(O["keys"], O["vals"], O["dims"], O["factors"], w.lam)
    coo = T.CooTensor(dev_keys(O["keys"]), dev(O["vals"]), O["dims"])
    g = T.tucker_core_update_exact(handle, coo, [dev(a) for a in O["factors"]], w.lam, "fp64")
    assert rel_err(g.cpu().numpy(), ref) <= 1e-6       # FP32 values, FP64 arithmetic


def test_ridge_loss(handle):
    X, F = _ragged_problem((30, 26, 22), (3, 4, 2), np.float64, 4)
    g = np.random.default_rng(0).standard_normal(24)
    ref = CU.ridge_loss_dense(X, F, g, 0.3)
    got = T.tucker_ridge_loss(handle, dev(X), [dev(a) for a in F], 0.3, dev(g))
    assert abs(got - ref) <= 1e-10 * abs(ref)
    keys = np.sort(np.random.default_rng(1).choice(X.size, 3000, replace=False)).astype(np.uint64)
    vals = X.reshape(-1)[keys.astype(np.int64)]
    ref = CU.ridge_loss_rows(keys, vals, X.shape, F, g, 0.3)
    coo = T.CooTensor(dev_keys(keys), dev(vals), X.shape)
    got = T.tucker_ridge_loss(handle, coo, [dev(a) for a in F], 0.3, dev(g))
    assert abs(got - ref) <= 1e-10 * abs(ref)


@pytest.mark.parametrize("sketched", [False, True])
def test_als_sweeps_match_oracle(handle, sketched):
    w = synth.WORKLOADS["dense3_64_r4_f64"]
    P = synth.tucker_problem(w)
    core0, F0 = synth.init_state(w)
    Xd = dev(P["X"])
    Fd = [dev(a) for a in F0]
    cd = dev(core0.reshape(-1).astype(np.float64))
    c, F = core0, F0
    for s in range(w.sweeps):
        loss, rmse = T.tucker_als_sweep(handle, Xd, Fd, cd, w.lam, sketched, w.m, w.seed_sample, s)
        c, F = ALS.als_sweep(P["X"], c, F, w.lam, sketched, w.m, w.seed_sample, s)
        ref_loss = ALS.tucker_loss(P["X"], c, F, w.lam)
        assert abs(loss - ref_loss) <= 1e-8 * ref_loss
        assert abs(rmse - ALS.rmse(P["X"], c, F)) <= 1e-8
    assert rel_err(cd.cpu().numpy(), c.reshape(-1)) <= 1e-8
    for a, b in zip(Fd, F):
        assert rel_err(a.cpu().numpy(), b) <= 1e-8


def test_solver_errors_are_reported(handle):
    X, F = _ragged_problem((10, 9, 8), (2, 2, 2), np.float64, 5)
    # lam = 0 with a rank-deficient sketch (m < d is impossible here: use a
    # zero factor column) -> G singular -> ENOTSPD, and the handle recovers
    F_bad = [f.copy() for f in F]
    F_bad[1][:, 1] = 0.0
    with pytest.raises(T.TuckerError) as e:
        T.tucker_core_update_sketched(handle, dev(X), [dev(a) for a in F_bad], 0.0, 500, 1, 0,
                                      "exact", "fp64")
    assert e.value.name == "ENOTSPD"
    with pytest.raises(T.TuckerError) as e:
        T.tucker_core_update_sketched(handle, dev(X), [dev(a) for a in F], -1.0, 500, 1)
    assert e.value.name == "EINVAL"
    with pytest.raises(T.TuckerError) as e:
        T.tucker_core_update_sketched(handle, dev(X), [dev(np.zeros((10, 2)))] + [dev(a) for a in F[1:]],
                                      0.1, 500, 1)
    assert e.value.name == "ERANK"
    g = T.tucker_core_update_sketched(handle, dev(X), [dev(a) for a in F], 0.1, 500, 1)
    assert torch.isfinite(g).all()


@pytest.mark.parametrize("reg", ["exact", "augmented"])
def test_adjoint_matches_oracle_and_fd(handle, reg):
    w = synth.WORKLOADS["dense3_256_r8_grad"]
    w = dataclasses.replace(w, dims=(48, 40, 36), ranks=(3, 4, 2), m=3000)
    P = synth.tucker_problem(w)
    X, F = P["X"], P["factors"]
    regc = S.REG_EXACT if reg == "exact" else S.REG_AUGMENTED
    levs = [CU.leverage_scores(A)[0] for A in F]
    smp = T.tucker_sample_rows(handle, w.dims, w.ranks, [dev(l) for l in levs], w.m, 3, 0, reg)
    Xd, Fd = dev(X), [dev(a) for a in F]
    g, st = T.tucker_core_update_sketched(handle, Xd, Fd, w.lam, 0, 0, 0, reg, "fp64", fixed=smp,
                                          stats=True)
    gbar = np.random.default_rng(1).standard_normal(24)
    dA, dx = T.tucker_core_solve_adjoint(handle, Xd, Fd, w.lam, reg, "fp64", smp, st["solve_id"],
                                         g, dev(gbar))
    # oracle: same frozen sample (real rows), regulariser diagonal
    keys = host_keys(smp.keys, smp.n_unique)
    cnt = smp.counts[:smp.n_unique].cpu().numpy().astype(np.float64)
    prob = smp.prob[:smp.n_unique].cpu().numpy()
    ref_p = S.row_probabilities(keys, levs, w.dims, regc, 24)
    assert np.array_equal(prob, ref_p)
    wts = S.sample_weights(cnt, ref_p, smp.n_draws)
    total = np.uint64(X.size)
    real = keys < total
    D = np.ones(24)
    if regc == S.REG_AUGMENTED:
        D = np.zeros(24)
        D[(keys[~real] - total).astype(np.int64)] = wts[~real]
    x = CU.gather_dense(X, keys[real], w.dims)
    ref_g = ADJ.forward(F, w.dims, keys[real], wts[real], x, w.lam, D)
    assert rel_err(g.cpu().numpy(), ref_g) <= 1e-10
    rdA, rdx = ADJ.backward(F, w.dims, keys[real], wts[real], x, w.lam, D, gbar)
    for a, b in zip(dA, rdA):
        assert rel_err(a.cpu().numpy(), b) <= 1e-9
    assert rel_err(dx.cpu().numpy()[real], rdx) <= 1e-9
    assert np.all(dx.cpu().numpy()[~real] == 0.0)
    # central finite differences of the GPU forward (FP64, h = 1e-6)
    rng = np.random.default_rng(2)
    hstep = 1e-6
    for _ in range(4):
        dirs = [rng.standard_normal(a.shape) for a in F]
        gp = T.tucker_core_update_sketched(handle, Xd, [dev(a + hstep * e) for a, e in zip(F, dirs)],
                                           w.lam, 0, 0, 0, reg, "fp64", fixed=smp).cpu().numpy()
        gm = T.tucker_core_update_sketched(handle, Xd, [dev(a - hstep * e) for a, e in zip(F, dirs)],
                                           w.lam, 0, 0, 0, reg, "fp64", fixed=smp).cpu().numpy()
        fd = (gp - gm) @ gbar / (2 * hstep)
        an = sum(float(np.sum(a.cpu().numpy() * e)) for a, e in zip(dA, dirs))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


@pytest.mark.parametrize("dims,ranks,dtype", [
    ((300,), (7,), np.float64),                           # order 1: dA = w (al v - be g)
    ((41, 37), (5, 3), np.float32),                       # order 2, R_1 > R_2
    ((23, 19, 17, 15), (2, 3, 1, 4), np.float64),         # order 4, a rank-1 mode
    ((9, 8, 7, 6, 5), (3, 2, 2, 3, 2), np.float64),       # order 5
    ((33, 29, 31), (1, 6, 5), np.float32),                # R_1 = 1: T1 is all of dk
])
def test_adjoint_orders_and_ranks(handle, dims, ranks, dtype):
    X, F = _ragged_problem(dims, ranks, dtype, 11)
    d = int(np.prod(ranks))
    levs = [CU.leverage_scores(np.asarray(A, dtype=np.float64))[0] for A in F]
    smp = T.tucker_sample_rows(handle, dims, ranks, [dev(l) for l in levs], 2000, 8, 0)
    Xd, Fd = dev(X), [dev(a) for a in F]
    g, st = T.tucker_core_update_sketched(handle, Xd, Fd, 0.05, 0, 0, 0, "exact", "fp64",
                                          fixed=smp, stats=True)
    gbar = np.random.default_rng(4).standard_normal(d)
    dA, dx = T.tucker_core_solve_adjoint(handle, Xd, Fd, 0.05, "exact", "fp64", smp,
                                         st["solve_id"], g, dev(gbar))
    keys = host_keys(smp.keys, smp.n_unique)
    cnt = smp.counts[:smp.n_unique].cpu().numpy().astype(np.float64)
    wts = S.sample_weights(cnt, smp.prob[:smp.n_unique].cpu().numpy(), smp.n_draws)
    Fo = [np.asarray(a, dtype=np.float64) for a in F]
    x = CU.gather_dense(np.asarray(X, dtype=np.float64), keys, dims)
    rdA, rdx = ADJ.backward(Fo, dims, keys, wts, x, 0.05, np.ones(d), gbar)
    for a, b in zip(dA, rdA):
        assert a.shape == b.shape
        assert rel_err(a.cpu().numpy(), b) <= 1e-9
    assert rel_err(dx.cpu().numpy(), rdx) <= 1e-9


def test_autograd_function(handle):
    from paper_2107_10654_gb300 import SketchedCoreSolve
    X, F = _ragged_problem((20, 18, 16), (2, 3, 2), np.float64, 6)
    levs = [CU.leverage_scores(A)[0] for A in F]
    smp = T.tucker_sample_rows(handle, X.shape, (2, 3, 2), [dev(l) for l in levs], 1500, 9, 0)
    A = [dev(a).requires_grad_(True) for a in F]
    g = SketchedCoreSolve.apply(handle, dev(X), smp, 0.2, "exact", "fp64", *A)
    c = torch.linspace(-1, 1, 12, dtype=torch.float64, device="cuda")
    (g * c).sum().backward()
    assert all(a.grad is not None and torch.isfinite(a.grad).all() for a in A)
