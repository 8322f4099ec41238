"""GPU parity at the full workload sizes, in the configuration the benchmark
times (BF16 tensor-core Gram, FP64 Cholesky, refinement), on outputs the
oracle can produce at that size:

  * 512^3, d = 512, m = 5e4: the whole sketched update against the oracle's
    (explicit sampled rows, FP64 Cholesky), the exact update, the loss ratio;
  * 128^4, d = 4096, m = 2e5 and 1024^3 at 10 % observed, d = 4096, m = 5e5:
    bit-exact samples, sampled Gram entries within the operand-rounding bound,
    sampled right-hand-side entries, and the FP64 residual of the returned
    core, h - (K_S^T W K_S + lambda I) g, evaluated by the oracle row by row;
  * 256^3 FP64, d = 512, m = 2e4: the adjoint against the oracle's gradient and
    FP64 central differences on 64 random directions;
  * 128^4 FP32: the exact dense update (Kronecker eigendecomposition form)
    against the oracle's;
  * 512^3: ten ALS sweeps (Alg. 2), exact and sketched, against the oracle's
    sweeps (FP64 data: the comparison is of the arithmetic, not of the
    storage precision).
"""
import dataclasses

import numpy as np
import pytest
import torch

import synth
from oracle import leverage as LV, sampling as S, core_update as CU, adjoint as ADJ, als as ALS
from tests.gpu_common import dev, dev_keys, host_keys, rel_err, handle  # noqa: F401
from paper_2107_10654_gb300 import tucker as T

pytestmark = pytest.mark.gpu

BF16_C = 2.0 ** -7          # two operands each rounded to 8 significant bits
TF32_C = 2.0 ** -9          # two TF32 operands (2^-11 each) and, grouped, the TF32 a_r1 a_r1'


def _levs(F):
    return [LV.leverage_scores(np.asarray(A, dtype=np.float64))[0] for A in F]


def _check_sample(handle, F, dims, ranks, m, seed, reg="exact", coo=None, obs_keys=None):
    """GPU sample from the oracle's scores equals the oracle's sample bit for bit."""
    levs = _levs(F)
    d = int(np.prod(ranks))
    regc = S.REG_EXACT if reg == "exact" else S.REG_AUGMENTED
    keys, T_ = S.sample_keys(levs, dims, m, seed, 0, regc, d, obs_keys)
    ku, cu = S.dedupe(keys)
    p = S.row_probabilities(ku, levs, dims, regc, d)
    smp = T.tucker_sample_rows(handle, dims, ranks, [dev(l) for l in levs], m, seed, 0, reg,
                               observed=coo)
    assert smp.n_draws == T_ and smp.n_unique == ku.size
    assert np.array_equal(host_keys(smp.keys, smp.n_unique), ku)
    assert np.array_equal(smp.counts[:smp.n_unique].cpu().numpy().astype(np.int64), cu)
    assert np.array_equal(smp.prob[:smp.n_unique].cpu().numpy(), p)
    return smp, ku, S.sample_weights(cu, p, T_), levs


def _check_gram_entries(F, dims, ku, w, G, n_pairs=96, seed=0, c=BF16_C):
    """Sampled entries of the tensor-core Gram within c * sum w |k_r| |k_c|."""
    R = [A.shape[1] for A in F]
    d = int(np.prod(R))
    idx = S.decode_keys(ku, dims)
    rows = [np.asarray(A, dtype=np.float64)[i] for A, i in zip(F, idx)]
    g = np.random.default_rng(seed)
    pairs = list(zip(g.integers(0, d, n_pairs), g.integers(0, d, n_pairs)))
    pairs += [(r, r) for r in g.integers(0, d, 16)]
    for ri, ci in pairs:
        rr, cc = np.unravel_index(ri, R), np.unravel_index(ci, R)
        kr = np.prod([rows[n][:, rr[n]] for n in range(len(R))], axis=0)
        kc = np.prod([rows[n][:, cc[n]] for n in range(len(R))], axis=0)
        ref = float(np.sum(w * kr * kc))
        bound = c * float(np.sum(w * np.abs(kr) * np.abs(kc)))
        assert abs(G[ri, ci] - ref) <= bound + 1e-12 * abs(ref), (ri, ci, G[ri, ci], ref, bound)


def _check_residual(F, dims, ku, w, x, lam, g, tol=1e-7):
    """||h - (K_S^T W K_S + lam I) g|| / ||h|| in FP64 by the oracle."""
    idx = S.decode_keys(ku, dims)
    h = CU.sampled_rows_apply_t(F, idx, w * x)
    z = CU.sampled_rows_apply(F, idx, g)
    r = h - CU.sampled_rows_apply_t(F, idx, w * z) - lam * g
    assert np.linalg.norm(r) <= tol * np.linalg.norm(h), np.linalg.norm(r) / np.linalg.norm(h)
    return h


# ------------------------------------------------------------------ 512^3, the bench workload
@pytest.fixture(scope="module")
def dense512():
    w = synth.WORKLOADS["dense3_512_r8_f32"]
    P = synth.tucker_problem(w)
    yield w, P["X"], P["factors"]


def test_bench_workload_sketched_and_exact_match_oracle(handle, dense512):
    w, X, F = dense512
    Xd, Fd = dev(X), [dev(a) for a in F]
    g, st = T.tucker_core_update_sketched(handle, Xd, Fd, w.lam, w.m, w.seed_sample, 0, "exact",
                                          "bf16", stats=True)
    ref = CU.sketched_core(X, F, w.lam, w.m, w.seed_sample, 0, S.REG_EXACT)
    assert st["n_unique"] == ref["keys"].size and st["n_draws"] == ref["T"]
    assert rel_err(g.cpu().numpy(), ref["g"]) <= 1e-6
    ge = T.tucker_core_update_exact(handle, Xd, Fd, w.lam, "fp64")
    ref_e = CU.exact_core_kron_eig(X, F, w.lam)
    assert rel_err(ge.cpu().numpy(), ref_e) <= 1e-5           # FP32 data, FP32 first product
    ratio = T.tucker_ridge_loss(handle, Xd, Fd, w.lam, g) / T.tucker_ridge_loss(handle, Xd, Fd,
                                                                                 w.lam, ge)
    assert 1.0 <= ratio <= 1.01


@pytest.mark.parametrize("sketched", [False, True])
def test_bench_workload_ten_als_sweeps(handle, dense512, sketched):
    w, X, _ = dense512
    X64 = X.astype(np.float64)
    core0, F0 = synth.init_state(w)
    Xd = dev(X64)
    Fd = [dev(a.astype(np.float64)) for a in F0]
    cd = dev(core0.reshape(-1).astype(np.float64))
    c, F = core0.astype(np.float64), [a.astype(np.float64) for a in F0]
    assert w.sweeps == 10
    for s in range(w.sweeps):
        loss, rmse = T.tucker_als_sweep(handle, Xd, Fd, cd, w.lam, sketched, w.m, w.seed_sample, s)
        c, F = ALS.als_sweep(X64, c, F, w.lam, sketched, w.m, w.seed_sample, s)
    ref_loss = ALS.tucker_loss(X64, c, F, w.lam)
    # Sketched sweeps resample from the current factors through the fixed-point
    # CDF q_i = floor(l_i 2^32): factors that agree to FP64 rounding can put a
    # score on either side of a quantisation step, which moves that row's p by
    # 1 / q_i (about 1.5e-8 here, l_i ~ R / I = 1/64).  The oracle alone shows it:
    # a 1e-13 perturbation of the initial state moves its sketched core by 1e-8
    # after one sweep and its exact core by 1e-11.  Hence 1e-6 for the state, the
    # loss and the RMSE of the sketched sweeps, 1e-8 for the state of the exact ones.
    # The library's loss is the Gram identity ||X||^2 - 2 g.K^T x + g.Hg, which here
    # cancels ||X||^2 = 6.9e10 down to a residual of 3.6e5 (a factor of 2e5): its
    # FP64 terms, sums of 512-long sequences, carry about 1e-13 relative error, so the
    # loss is good to about 2e-8 relative; 5e-8 for the loss of the exact sweeps.
    tol = 1e-6 if sketched else 1e-8
    ltol = 1e-6 if sketched else 5e-8
    assert abs(loss - ref_loss) <= ltol * ref_loss
    ref_rmse = ALS.rmse(X64, c, F)
    assert abs(rmse - ref_rmse) <= ltol * ref_rmse
    assert rel_err(cd.cpu().numpy(), c.reshape(-1)) <= tol
    for a, b in zip(Fd, F):
        assert rel_err(a.cpu().numpy(), b) <= tol
    del Xd


def test_bench_workload_sample_bit_exact(handle, dense512):
    w, X, F = dense512
    _check_sample(handle, F, w.dims, w.ranks, w.m, w.seed_sample)


# ------------------------------------------------------------------ 128^4, d = 4096
@pytest.fixture(scope="module")
def dense4():
    w = synth.WORKLOADS["dense4_128_r8_f32"]
    P = synth.tucker_problem(w)
    yield w, P["X"], P["factors"]


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_4way_full_size(handle, dense4, prec):
    w, X, F = dense4
    Xd, Fd = dev(X), [dev(a) for a in F]
    smp, ku, wts, _ = _check_sample(handle, F, w.dims, w.ranks, w.m, w.seed_sample)
    x = CU.gather_dense(X, ku, w.dims)
    if prec == "bf16":
        G, h = T.tucker_sketched_gram(handle, Xd, Fd, "bf16", smp)
        _check_gram_entries(F, w.dims, ku, wts, G.cpu().numpy())
        hr = CU.sampled_rows_apply_t(F, S.decode_keys(ku, w.dims), wts * x)
        assert rel_err(h.cpu().numpy(), hr) <= 1e-12
        del G
    g = T.tucker_core_update_sketched(handle, Xd, Fd, w.lam, 0, 0, 0, "exact", prec, fixed=smp)
    _check_residual(F, w.dims, ku, wts, x, w.lam, g.cpu().numpy())


def test_4way_exact_full_size(handle, dense4):
    w, X, F = dense4
    g = T.tucker_core_update_exact(handle, dev(X), [dev(a) for a in F], w.lam, "fp64")
    ref = CU.exact_core_kron_eig(X, F, w.lam)
    assert rel_err(g.cpu().numpy(), ref) <= 1e-5           # FP32 data, FP32 first product


# ------------------------------------------------------------------ 1024^3 at 10 %, d = 4096
@pytest.fixture(scope="module")
def missing1024():
    w = synth.WORKLOADS["missing3_1024_r16_f32"]
    O = synth.observed_entries(w)
    yield w, O


def test_missing_full_size(handle, missing1024):
    w, O = missing1024
    F = O["factors"]
    coo = T.CooTensor(dev_keys(O["keys"]), dev(O["vals"]), O["dims"])
    Fd = [dev(a) for a in F]
    smp, ku, wts, _ = _check_sample(handle, F, O["dims"], w.ranks, w.m, w.seed_sample, coo=coo,
                                    obs_keys=O["keys"])
    G, h = T.tucker_sketched_gram(handle, coo, Fd, "bf16", smp)
    _check_gram_entries(F, O["dims"], ku, wts, G.cpu().numpy())
    del G
    x = CU.gather_observed(O["keys"], O["vals"], ku)
    g = T.tucker_core_update_sketched(handle, coo, Fd, w.lam, 0, 0, 0, "exact", "bf16", fixed=smp)
    hr = _check_residual(F, O["dims"], ku, wts, x, w.lam, g.cpu().numpy())
    assert rel_err(h.cpu().numpy(), hr) <= 1e-12
    # the update the benchmark times draws the same sample from the GPU's own scores
    g2, st = T.tucker_core_update_sketched(handle, coo, Fd, w.lam, w.m, w.seed_sample, 0, "exact",
                                           "bf16", stats=True)
    assert st["n_draws"] == smp.n_draws and st["n_unique"] == smp.n_unique
    assert rel_err(g2.cpu().numpy(), g.cpu().numpy()) <= 1e-6


# ------------------------------------------------------------------ 256^3 FP64 adjoint
def test_adjoint_full_size_against_oracle_and_fd(handle):
    w = synth.WORKLOADS["dense3_256_r8_grad"]
    P = synth.tucker_problem(w)
    X, F = P["X"], P["factors"]
    Xd, Fd = dev(X), [dev(a) for a in F]
    smp, ku, wts, _ = _check_sample(handle, F, w.dims, w.ranks, w.m, w.seed_sample)
    g, st = T.tucker_core_update_sketched(handle, Xd, Fd, w.lam, 0, 0, 0, "exact", "fp64",
                                          fixed=smp, stats=True)
    d = w.d
    gbar = np.random.default_rng(5).standard_normal(d)
    dA, dx = T.tucker_core_solve_adjoint(handle, Xd, Fd, w.lam, "exact", "fp64", smp,
                                         st["solve_id"], g, dev(gbar))
    x = CU.gather_dense(X, ku, w.dims)
    ref_g = ADJ.forward(F, w.dims, ku, wts, x, w.lam, np.ones(d))
    assert rel_err(g.cpu().numpy(), ref_g) <= 1e-10
    rdA, rdx = ADJ.backward(F, w.dims, ku, wts, x, w.lam, np.ones(d), gbar)
    for a, b in zip(dA, rdA):
        assert rel_err(a.cpu().numpy(), b) <= 1e-9
    assert rel_err(dx.cpu().numpy(), rdx) <= 1e-9
    rng = np.random.default_rng(6)
    hstep = 1e-6
    errs = []
    for _ in range(64):
        dirs = [rng.standard_normal(a.shape) for a in F]
        nrm = np.sqrt(sum(float(np.sum(e * e)) for e in dirs))
        dirs = [e / nrm for e in dirs]
        gp = T.tucker_core_update_sketched(handle, Xd, [dev(a + hstep * e) for a, e in zip(F, dirs)],
                                           w.lam, 0, 0, 0, "exact", "fp64", fixed=smp).cpu().numpy()
        gm = T.tucker_core_update_sketched(handle, Xd, [dev(a - hstep * e) for a, e in zip(F, dirs)],
                                           w.lam, 0, 0, 0, "exact", "fp64", fixed=smp).cpu().numpy()
        fd = (gp - gm) @ gbar / (2 * hstep)
        an = sum(float(np.sum(a.cpu().numpy() * e)) for a, e in zip(dA, dirs))
        errs.append(abs(fd - an) / max(1.0, abs(an)))
    assert max(errs) <= 1e-6, max(errs)
