"""GPU parity of the sketched factor update (leverage sample of the mode-n factor
design B_n = (x)_{k != n} A^(k) G_(n)^T from the product of the other modes'
scores, mode-n fibers, weighted normal equations) against the oracle's
sketched_factor_update on the same draws (FP64 data 1e-10; FP32 data within a
bound derived from the FP32 sums and the conditioning of M), for every mode of
orders 2, 3 and 4, the most strided mode of the 512^3 workload, ALS sweeps
with sketched factor and core updates against the oracle's sweeps, and the
argument checks."""
import numpy as np
import pytest
import torch

import synth
from oracle import als as ALS, sampling as S
from tests.gpu_common import dev, dev_keys, rel_err, handle  # noqa: F401
from paper_2107_10654_gb300 import tucker as T

pytestmark = pytest.mark.gpu


def _problem(dims, ranks, seed, dtype=np.float64, sigma=0.1):
    g = np.random.default_rng(seed)
    F = [g.standard_normal((i, r)) for i, r in zip(dims, ranks)]
    G = g.standard_normal(ranks)
    X = ALS.tucker_model(G, F) + sigma * g.standard_normal(dims)
    # the update starts from perturbed factors and core
    F0 = [a + 0.3 * g.standard_normal(a.shape) for a in F]
    G0 = G + 0.3 * g.standard_normal(ranks)
    return X.astype(dtype), [a.astype(dtype) for a in F0], G0


CASES = [
    ((20, 18, 16), (3, 2, 4), 3000),
    ((40, 35), (5, 3), 500),                        # order 2: one other mode
    ((9, 8, 7, 6), (2, 3, 2, 2), 2500),             # order 4
    ((33, 130, 17), (4, 8, 3), 8000),               # I_n > 128: several row blocks
    ((50, 44, 46), (40, 8, 8), 6000),               # R_n > 32: over 48 KB of normal-equation tiles
]


def _fp32_bound(X, G, F, n, lam, r):
    """||dA||_F bound of the FP32 path: Y = sum_u x_u (w b_u)^T summed in FP32 (each
    entry off by about sqrt(n_u) 2^-24 sum_u |x_ui| |w b_u|_r, rounding errors taken
    as independent), and dA = dY M^-1 with M formed in FP64; times 4."""
    dims = [d for k, d in enumerate(X.shape) if k != n]
    b = ALS.factor_design_rows(G, F, n, S.decode_keys(r["keys"], dims))
    wb = r["w"][:, None] * b
    Xs = ALS.unfold(X.astype(np.float64), n)[:, r["keys"].astype(np.int64)]
    M = wb.T @ b + lam * np.eye(b.shape[1])
    dY = np.sqrt(r["keys"].size) * 2.0 ** -24 * (np.abs(Xs) @ np.abs(wb))
    return 4.0 * np.linalg.norm(dY) * np.linalg.norm(np.linalg.inv(M), 2)


@pytest.mark.parametrize("dims,ranks,m", CASES)
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_factor_update_matches_oracle(handle, dims, ranks, m, dtype):
    X, F, G = _problem(dims, ranks, 1, dtype)
    for n in range(len(dims)):
        Fd = [dev(a) for a in F]
        T.tucker_factor_update_sketched(handle, dev(X), Fd, dev(G.reshape(-1)), n, 0.05, m, 7, 3)
        F64 = [a.astype(np.float64) for a in F]
        r = ALS.sketched_factor_update(X.astype(np.float64), G, F64, n, 0.05, m, 7, 3)
        got = Fd[n].cpu().numpy().astype(np.float64)
        if dtype == np.float64:
            assert rel_err(got, r["A"]) <= 1e-10, n
        else:
            # FP32 sums, then the result rounded to FP32 (2^-24 relative per entry)
            bound = _fp32_bound(X, G, F64, n, 0.05, r) + 2.0 ** -24 * np.linalg.norm(r["A"])
            assert np.linalg.norm(got - r["A"]) <= bound, (n, np.linalg.norm(got - r["A"]), bound)
        for k in range(len(dims)):                  # the other factors are untouched
            if k != n:
                assert np.array_equal(Fd[k].cpu().numpy(), F[k])


def test_most_strided_mode_of_the_512_workload(handle):
    w = synth.WORKLOADS["dense3_512_r8_f32"]
    P = synth.tucker_problem(w)
    X, F = P["X"], P["factors"]
    g = np.random.default_rng(2)
    G = P["core"].reshape(w.ranks) + 0.1 * g.standard_normal(w.ranks)
    Fd = [dev(a) for a in F]
    T.tucker_factor_update_sketched(handle, dev(X), Fd, dev(G.reshape(-1)), 0, w.lam, 16384, 5, 0)
    F64 = [a.astype(np.float64) for a in F]
    r = ALS.sketched_factor_update(X, G, F64, 0, w.lam, 16384, 5, 0)
    got = Fd[0].cpu().numpy().astype(np.float64)
    bound = _fp32_bound(X, G, F64, 0, w.lam, r) + 2.0 ** -24 * np.linalg.norm(r["A"])
    assert np.linalg.norm(got - r["A"]) <= bound


def test_als_sweeps_with_sketched_factors_match_oracle():
    w = synth.WORKLOADS["dense3_64_r4_f64"]
    P = synth.tucker_problem(w)
    core0, F0 = synth.init_state(w)
    Xd = dev(P["X"])
    Fd = [dev(a) for a in F0]
    cd = dev(core0.reshape(-1).astype(np.float64))
    c, F = core0, F0
    mf = 1500
    with T.Handle() as h:
        T.tucker_set_factor_sketch(h, mf)
        for s in range(3):
            loss, rmse = T.tucker_als_sweep(h, Xd, Fd, cd, w.lam, True, w.m, w.seed_sample, s)
            c, F = ALS.als_sweep(P["X"], c, F, w.lam, True, w.m, w.seed_sample, s, m_factor=mf)
            ref_loss = ALS.tucker_loss(P["X"], c, F, w.lam)
            assert abs(loss - ref_loss) <= 1e-8 * ref_loss
            assert abs(rmse - ALS.rmse(P["X"], c, F)) <= 1e-8
        torch.cuda.synchronize()
    assert rel_err(cd.cpu().numpy(), c.reshape(-1)) <= 1e-8
    for a, b in zip(Fd, F):
        assert rel_err(a.cpu().numpy(), b) <= 1e-8


def test_errors(handle):
    X, F, G = _problem((10, 9, 8), (2, 2, 2), 3)
    Fd = [dev(a) for a in F]
    for n, m in ((3, 100), (-1, 100), (0, 0)):
        with pytest.raises(T.TuckerError) as e:
            T.tucker_factor_update_sketched(handle, dev(X), Fd, dev(G.reshape(-1)), n, 0.1, m, 1)
        assert e.value.name == "EINVAL"
    keys = np.arange(0, 720, 7, dtype=np.uint64)
    coo = T.CooTensor(dev_keys(keys), dev(np.ones(keys.size)), X.shape)
    with pytest.raises(T.TuckerError) as e:
        T.tucker_factor_update_sketched(handle, coo, Fd, dev(G.reshape(-1)), 0, 0.1, 100, 1)
    assert e.value.name == "EINVAL"
    with pytest.raises(T.TuckerError) as e:
        T.tucker_set_factor_sketch(handle, -1)
    assert e.value.name == "EINVAL"
