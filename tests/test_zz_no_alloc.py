"""The allocation-free sampling entry point (tucker_sample_rows_noalloc).

It is for callers that may not allocate device memory while they run; it
keeps its scratch in a fixed array inside the library.  Through the C ABI it
must return exactly what tucker_sample_rows returns, on two calls in a row
(the array is shared and reused), and refuse sizes beyond the array.  This
file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest
import torch

from oracle import leverage as LV
from tests.gpu_common import dev, host_keys, handle  # noqa: F401
from paper_2107_10654_gb300 import tucker as T

pytestmark = pytest.mark.gpu


def _scores(dims, ranks, seed):
    g = np.random.default_rng(seed)
    return [dev(LV.leverage_scores(g.standard_normal((i, r)))[0]) for i, r in zip(dims, ranks)]


@pytest.mark.parametrize("dims,ranks,m,reg", [
    ((512, 512, 512), (8, 8, 8), 50000, "exact"),
    ((100, 37, 250, 9), (3, 5, 2, 2), 20001, "augmented"),
])
def test_noalloc_matches_sample_rows_twice(handle, dims, ranks, m, reg):
    lev = _scores(dims, ranks, 4)
    ref = T.tucker_sample_rows(handle, dims, ranks, lev, m, 321, 2, reg)
    out = T.Samples.empty(m, "cuda")
    for call in range(2):
        out.keys.fill_(-1)
        out.counts.fill_(0)
        out.prob.fill_(float("nan"))
        got = T.tucker_sample_rows_noalloc(dims, ranks, lev, m, 321, 2, reg, out=out)
        torch.cuda.synchronize()
        assert got.n_unique == ref.n_unique and got.n_draws == ref.n_draws, call
        n = ref.n_unique
        assert np.array_equal(host_keys(got.keys, n), host_keys(ref.keys, n)), call
        assert torch.equal(got.counts[:n], ref.counts[:n]), call
        assert torch.equal(got.prob[:n], ref.prob[:n]), call


def test_noalloc_allocates_nothing_and_rejects_oversize(handle):
    dims, ranks, m = (64, 64, 64), (4, 4, 4), 30000
    lev = _scores(dims, ranks, 5)
    out = T.Samples.empty(m, "cuda")
    T.tucker_sample_rows_noalloc(dims, ranks, lev, m, 1, 0, out=out)     # first call: setup
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for s in range(3):
        T.tucker_sample_rows_noalloc(dims, ranks, lev, m, 1, s, out=out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    big = 4_000_000
    with pytest.raises(T.TuckerError) as e:
        T.tucker_sample_rows_noalloc(dims, ranks, lev, big, 1, 0, out=T.Samples.empty(big, "cuda"))
    assert e.value.name == "ECAPACITY" and "scratch" in str(e.value)
    # the array is still usable after a rejected call
    got = T.tucker_sample_rows_noalloc(dims, ranks, lev, m, 1, 0, out=out)
    assert got.n_unique > 0


def test_noalloc_rejects_wrapping_keys_like_sample_rows(handle):
    # 600^7 = 2.8e19 rows: linear keys would wrap modulo 2^64, although the CDFs
    # (7 x 600 entries) fit the fixed array; both entry points refuse before any
    # device work
    dims, ranks, m = (600,) * 7, (1,) * 7, 1000
    lev = [torch.full((600,), 1.0 / 600, dtype=torch.float64, device="cuda") for _ in dims]
    out = T.Samples.empty(m, "cuda")
    with pytest.raises(T.TuckerError) as e1:
        T.tucker_sample_rows(handle, dims, ranks, lev, m, 1, 0, out=out)
    with pytest.raises(T.TuckerError) as e2:
        T.tucker_sample_rows_noalloc(dims, ranks, lev, m, 1, 0, out=out)
    assert e1.value.name == "EINVAL" and e2.value.name == "EINVAL"
    assert "too large" in str(e2.value)
