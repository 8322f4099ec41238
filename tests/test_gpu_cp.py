"""GPU parity of the CP-ALS variant (Sec. 6's extension of leverage-score CP-ALS
to L2 regularisation; the Khatri-Rao design overestimated by Kronecker scores,
Sec. 4): the sketched CP factor update against the oracle's
sketched_cp_factor_update on the same draws (FP64 data 1e-10; FP32 data within
a bound derived from the FP32 sums and the conditioning of M) for every mode of
orders 2, 3 and 4; sketched CP-ALS sweeps against the oracle's; and the argument
checks."""
import numpy as np
import pytest

from oracle import cp as CP, sampling as S
from tests.gpu_common import dev, rel_err, handle  # noqa: F401
from paper_2107_10654_gb300 import tucker as T

pytestmark = pytest.mark.gpu


def _problem(dims, R, seed, dtype=np.float64, sigma=0.1):
    g = np.random.default_rng(seed)
    F = [g.standard_normal((i, R)) for i in dims]
    X = CP.cp_model(F) + sigma * g.standard_normal(dims)
    F0 = [a + 0.3 * g.standard_normal(a.shape) for a in F]        # a perturbed start
    return X.astype(dtype), [a.astype(dtype) for a in F0]


CASES = [
    ((20, 18, 16), 4, 3000),
    ((40, 35), 5, 500),                             # order 2: one other mode
    ((9, 8, 7, 6), 3, 2500),                        # order 4
    ((33, 130, 17), 6, 8000),                       # I_n > 128: several row blocks
    ((50, 44, 46), 40, 6000),                       # R > 32: two entries per lane
]


def _fp32_bound(X, F, n, lam, r):
    """||dA||_F of the FP32 path: Y summed in FP32 (each entry off by about
    sqrt(n_u) 2^-24 sum_u |x_ui| |w z_u|_r), dA = dY M^-1 with M in FP64; times 4."""
    dims = [d for k, d in enumerate(X.shape) if k != n]
    z = CP.khatri_rao_rows(F, n, S.decode_keys(r["keys"], dims))
    wz = r["w"][:, None] * z
    Xs = CP.unfold(X.astype(np.float64), n)[:, r["keys"].astype(np.int64)]
    M = wz.T @ z + lam * np.eye(z.shape[1])
    dY = np.sqrt(r["keys"].size) * 2.0 ** -24 * (np.abs(Xs) @ np.abs(wz))
    return 4.0 * np.linalg.norm(dY) * np.linalg.norm(np.linalg.inv(M), 2)


@pytest.mark.parametrize("dims,R,m", CASES)
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_cp_factor_update_matches_oracle(handle, dims, R, m, dtype):
    X, F = _problem(dims, R, 1, dtype)
    for n in range(len(dims)):
        Fd = [dev(a) for a in F]
        T.tucker_cp_factor_update_sketched(handle, dev(X), Fd, n, 0.05, m, 7, 3)
        F64 = [a.astype(np.float64) for a in F]
        r = CP.sketched_cp_factor_update(X.astype(np.float64), F64, n, 0.05, m, 7, 3)
        got = Fd[n].cpu().numpy().astype(np.float64)
        if dtype == np.float64:
            assert rel_err(got, r["A"]) <= 1e-10, n
        else:
            bound = _fp32_bound(X, F64, n, 0.05, r) + 2.0 ** -24 * np.linalg.norm(r["A"])
            assert np.linalg.norm(got - r["A"]) <= bound, (n, np.linalg.norm(got - r["A"]), bound)
        for k in range(len(dims)):                  # the other factors are untouched
            if k != n:
                assert np.array_equal(Fd[k].cpu().numpy(), F[k])


def test_cp_als_sweeps_match_oracle(handle):
    """Five sketched CP-ALS sweeps from one start, FP64 data: factors within 1e-8 of
    the oracle's sweeps (each sweep resamples from the current factors through the
    fixed-point CDFs, so FP64 rounding in the scores can move a quantisation step),
    and the ridge loss falls from the start and ends near the oracle's."""
    dims, R, m, lam = (30, 26, 28), 4, 6000, 0.05
    X, F = _problem(dims, R, 4)
    Fd = [dev(a) for a in F]
    Fo = [a.copy() for a in F]
    for sw in range(5):
        T.tucker_cp_als_sweep(handle, dev(X), Fd, lam, m, 11, sw)
        Fo = CP.cp_als_sweep(X, Fo, lam, m, 11, sw)
    for a, b in zip(Fd, Fo):
        assert rel_err(a.cpu().numpy(), b) <= 1e-8
    got = [a.cpu().numpy() for a in Fd]
    assert CP.cp_loss(X, got, lam) < CP.cp_loss(X, F, lam)
    assert abs(CP.cp_loss(X, got, lam) - CP.cp_loss(X, Fo, lam)) <= 1e-8 * CP.cp_loss(X, Fo, lam)


def test_cp_argument_checks(handle):
    X, F = _problem((10, 9, 8), 3, 2)
    Fd = [dev(a) for a in F]
    with pytest.raises(T.TuckerError):
        T.tucker_cp_factor_update_sketched(handle, dev(X), Fd, 3, 0.1, 100, 1)      # bad mode
    with pytest.raises(T.TuckerError):
        T.tucker_cp_factor_update_sketched(handle, dev(X), Fd, 0, 0.1, 0, 1)        # m = 0
    with pytest.raises(T.TuckerError):
        T.tucker_cp_factor_update_sketched(handle, dev(X), Fd, 0, -1.0, 100, 1)     # lambda < 0
