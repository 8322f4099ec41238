"""Seeded synthetic inputs for the sketched Tucker core update.

This module only draws random numbers and assembles the Tucker model
X = G x_1 A^(1) x_2 ... x_N A^(N) + noise that the experiments of Sec. 5
describe (a random Tucker tensor plus Gaussian noise).  It holds none of the
core-update arithmetic (leverage scores, sampling, Gram, solve): both the CUDA
path and the CPU oracle consume the arrays it returns.

Layout convention (used everywhere in this repository): tensors are row-major,
the last index varies fastest, so the linear index of (i_1, ..., i_N) is
((i_1 * I_2 + i_2) * I_3 + i_3) ...; factor A^(n) is an I_n x R_n row-major
matrix; the core is stored as vec(G) in the same row-major order.

Random numbers come from numpy's Philox bit generator, seeded per purpose:
data (core, factors, noise), ALS initial state, sampling, observation mask.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

__all__ = ["Workload", "WORKLOADS", "tucker_problem", "random_factors",
           "observed_entries", "rng"]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed)))


@dataclasses.dataclass(frozen=True)
class Workload:
    """One benchmark/parity workload: shape, ranks, noise, lambda, sample count."""
    name: str
    dims: tuple
    ranks: tuple
    sigma: float
    lam: float
    m: int
    dtype: str                  # "f32" or "f64" storage of X and the factors
    sweeps: int = 0             # ALS sweeps in the workload (0: core update only)
    observed: float = 1.0       # fraction of observed entries (1.0: dense)
    index: int = 0              # seeds are 1234 + index (+1000 init, +2000 sample, +3000 mask)

    @property
    def order(self) -> int:
        return len(self.dims)

    @property
    def d(self) -> int:
        return int(np.prod(self.ranks))

    @property
    def seed_data(self) -> int:
        return 1234 + self.index

    @property
    def seed_init(self) -> int:
        return 2234 + self.index

    @property
    def seed_sample(self) -> int:
        return 3234 + self.index

    @property
    def seed_mask(self) -> int:
        return 4234 + self.index

    @property
    def np_dtype(self):
        return np.float64 if self.dtype == "f64" else np.float32


# The five workloads: shapes and parameters of the dense 3-way experiments of
# Sec. 5 scaled to the sizes named for this path, a 4-way precision case, a
# missing-entry case and a differentiation case.
WORKLOADS = {
    "dense3_64_r4_f64": Workload("dense3_64_r4_f64", (64, 64, 64), (4, 4, 4), 0.1, 1e-3,
                                 2000, "f64", sweeps=5, index=0),
    "dense3_512_r8_f32": Workload("dense3_512_r8_f32", (512, 512, 512), (8, 8, 8), 0.05, 1e-2,
                                  50000, "f32", sweeps=10, index=1),
    "dense4_128_r8_f32": Workload("dense4_128_r8_f32", (128, 128, 128, 128), (8, 8, 8, 8), 0.05,
                                  1e-2, 200000, "f32", index=2),
    "missing3_1024_r16_f32": Workload("missing3_1024_r16_f32", (1024, 1024, 1024), (16, 16, 16),
                                      0.1, 1e-1, 500000, "f32", observed=0.1, index=3),
    "dense3_256_r8_grad": Workload("dense3_256_r8_grad", (256, 256, 256), (8, 8, 8), 0.05, 1e-2,
                                   20000, "f64", index=4),
}


def random_factors(dims: Sequence[int], ranks: Sequence[int], seed: int, dtype=np.float64):
    """N(0,1) core (R_1..R_N) and factors (I_n x R_n) from one seed."""
    g = rng(seed)
    core = g.standard_normal(tuple(ranks)).astype(dtype)
    factors = [g.standard_normal((int(i), int(r))).astype(dtype) for i, r in zip(dims, ranks)]
    return core, factors


def _trailing_model(core64: np.ndarray, factors64: List[np.ndarray]) -> np.ndarray:
    """core x_2 A^(2) ... x_N A^(N): shape (R_1, I_2, ..., I_N), FP64."""
    t = core64
    for n in range(len(factors64) - 1, 0, -1):
        t = np.tensordot(t, factors64[n], axes=([n], [1]))       # appends I_n at the end
        t = np.moveaxis(t, -1, n)
    return t


def tucker_problem(w: Workload, with_dense: bool = True):
    """Dense Tucker tensor X = G x_n A^(n) + sigma*N(0,1), returned with the truth.

    Returns dict(X, core, factors): X has dtype w.np_dtype and shape w.dims.
    """
    core, factors = random_factors(w.dims, w.ranks, w.seed_data, np.float64)
    out = {"core": core.astype(w.np_dtype), "factors": [a.astype(w.np_dtype) for a in factors]}
    if not with_dense:
        return out
    g = rng(w.seed_data + 77777)
    X = np.empty(w.dims, dtype=w.np_dtype)
    t = _trailing_model(core, factors)
    slab = max(1, (1 << 24) // max(1, int(np.prod(w.dims[1:]))))
    for i0 in range(0, w.dims[0], slab):
        i1 = min(w.dims[0], i0 + slab)
        blk = np.tensordot(factors[0][i0:i1], t, axes=([1], [0]))
        noise = g.standard_normal(blk.shape, dtype=np.float64 if w.dtype == "f64" else np.float32)
        X[i0:i1] = (blk + w.sigma * noise).astype(w.np_dtype)
    out["X"] = X
    return out


def observed_entries(w: Workload, dims: Optional[Sequence[int]] = None,
                     frac: Optional[float] = None):
    """Observed-entry COO of the Tucker tensor: Bernoulli(frac) mask per entry.

    Returns dict(keys=uint64 sorted unique row-major linear indices,
    vals=values (model + sigma*N(0,1)) in w.np_dtype, core, factors).
    """
    dims = tuple(dims) if dims is not None else w.dims
    frac = w.observed if frac is None else frac
    core, factors = random_factors(dims, w.ranks, w.seed_data, np.float64)
    gm = rng(w.seed_mask)
    gn = rng(w.seed_data + 77777)
    inner = int(np.prod(dims[1:]))
    keys, vals = [], []
    # contract modes 2..N once; per leading index the slab is one small product
    t2 = _trailing_model(core, factors).reshape(core.shape[0], inner)                          # R_1 x inner
    for i in range(dims[0]):
        sel = np.flatnonzero(gm.random(inner, dtype=np.float32) < np.float32(frac))
        model = factors[0][i] @ t2[:, sel]
        noise = gn.standard_normal(sel.size)
        keys.append(sel.astype(np.uint64) + np.uint64(i * inner))
        vals.append((model + w.sigma * noise).astype(w.np_dtype))
    return {"keys": np.concatenate(keys), "vals": np.concatenate(vals),
            "core": core.astype(w.np_dtype), "factors": [a.astype(w.np_dtype) for a in factors],
            "dims": dims}


def init_state(w: Workload, dims: Optional[Sequence[int]] = None):
    """Random ALS initial state (core and factors N(0,1)), the same for both methods."""
    dims = tuple(dims) if dims is not None else w.dims
    core, factors = random_factors(dims, w.ranks, w.seed_init, np.float64)
    # scale so the initial model has entries of order one
    s = 1.0 / math.sqrt(max(1, int(np.prod(w.ranks))))
    return (core * s).astype(w.np_dtype), [a.astype(w.np_dtype) for a in factors]
