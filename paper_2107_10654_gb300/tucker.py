"""Python binding of the C ABI (include/tucker.h) over torch CUDA tensors.

Argument marshalling only: every function passes device pointers of torch
tensors to the library of the same name and raises TuckerError on a non-OK
status.  All arithmetic of the path runs in libtucker's CUDA kernels.
Tensors must be contiguous CUDA tensors on the handle's device; factors share
the dtype of X (float32 or float64); cores are float64.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple, Union

import torch

from . import _lib as L

__all__ = ["TuckerError", "Handle", "Samples", "CooTensor", "tucker_leverage_scores",
           "tucker_sample_rows", "tucker_core_update_sketched", "tucker_core_update_exact",
           "tucker_als_sweep", "tucker_ridge_loss", "tucker_core_solve_adjoint",
           "tucker_sample_rows_noalloc", "tucker_sketched_gram", "tucker_set_solver",
           "tucker_ridge_tables", "tucker_sample_rows_ridge", "tucker_missing_beta",
           "tucker_factor_update_sketched", "tucker_set_factor_sketch"]

PREC = {"fp64": L.PREC_FP64, "fp32": L.PREC_FP32, "tf32": L.PREC_TF32, "bf16": L.PREC_BF16}
REG = {"exact": L.REG_EXACT, "augmented": L.REG_AUGMENTED, "ridge": L.REG_RIDGE}
SOLVER = {"fp64": L.SOLVER_FP64_CHOLESKY, "mixed": L.SOLVER_MIXED, "kpcg": L.SOLVER_KRON_PCG}


class TuckerError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        self.name = L.STATUS_NAMES[status] if 0 <= status < len(L.STATUS_NAMES) else str(status)
        super().__init__(f"{self.name}: {msg}")


@dataclass
class CooTensor:
    """Observed entries of a tensor: sorted unique row-major keys and values."""
    keys: torch.Tensor          # int64 (bit pattern of uint64 keys), CUDA
    vals: torch.Tensor          # float32 / float64, CUDA
    dims: Tuple[int, ...]


@dataclass
class Samples:
    """A deduplicated row sample (device arrays of capacity m)."""
    keys: torch.Tensor          # int64 view of uint64 keys
    counts: torch.Tensor        # int32 view of uint32 counts
    prob: torch.Tensor          # float64
    n_unique: int = 0
    n_draws: int = 0

    @staticmethod
    def empty(capacity: int, device) -> "Samples":
        return Samples(torch.empty(capacity, dtype=torch.int64, device=device),
                       torch.empty(capacity, dtype=torch.int32, device=device),
                       torch.empty(capacity, dtype=torch.float64, device=device))

    def _c(self) -> L.TuckerSamples:
        return L.TuckerSamples(self.keys.numel(), self.n_unique, self.n_draws,
                               self.keys.data_ptr(), self.counts.data_ptr(), self.prob.data_ptr())


def _check(h, st: int):
    if st != L.OK:
        raise TuckerError(st, L.load().tucker_last_error(h).decode(errors="replace"))


class Handle:
    """Owns a tucker_handle bound to a CUDA stream (default: torch's current stream)."""

    def __init__(self, stream: Optional[torch.cuda.Stream] = None, synchronous: bool = True,
                 solver: str = "fp64"):
        lib = L.load()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        hp = C.c_void_p()
        st = lib.tucker_create(C.byref(hp), C.c_void_p(self.stream.cuda_stream))
        if st != L.OK:
            raise TuckerError(st, "tucker_create failed (needs an sm_103 GPU)")
        self.h = hp
        _check(self.h, lib.tucker_set_sync(self.h, int(synchronous)))
        self.set_solver(solver)

    def set_sync(self, synchronous: bool):
        """Synchronous calls wait for their kernels and report device errors at once;
        asynchronous calls return after enqueueing (errors surface at sync())."""
        _check(self.h, L.load().tucker_set_sync(self.h, int(synchronous)))

    def set_solver(self, solver: str):
        """Ridge solver of later updates: "fp64" (FP64 Cholesky), "mixed"
        (FP32 Cholesky preconditioning an FP64 iterative refinement) or "kpcg"
        (Kronecker-preconditioned CG inside the same refinement)."""
        _check(self.h, L.load().tucker_set_solver(self.h, SOLVER[solver]))

    def close(self):
        if getattr(self, "h", None):
            L.load().tucker_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def sync(self):
        _check(self.h, L.load().tucker_sync(self.h))


def _dt(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return L.F32
    if t.dtype == torch.float64:
        return L.F64
    raise TypeError(f"unsupported dtype {t.dtype}")


def _need(t: torch.Tensor, name: str):
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA tensor")


def _tensor(X: Union[torch.Tensor, CooTensor]) -> L.TuckerTensor:
    tt = L.TuckerTensor()
    if isinstance(X, CooTensor):
        _need(X.keys, "keys")
        _need(X.vals, "vals")
        tt.order = len(X.dims)
        for i, v in enumerate(X.dims):
            tt.dims[i] = int(v)
        tt.dtype = _dt(X.vals)
        tt.nnz = X.keys.numel()
        tt.keys = X.keys.data_ptr()
        tt.vals = X.vals.data_ptr()
    else:
        _need(X, "X")
        tt.order = X.dim()
        for i, v in enumerate(X.shape):
            tt.dims[i] = int(v)
        tt.dtype = _dt(X)
        tt.dense = X.data_ptr()
    return tt


def _ranks(R: Sequence[int]):
    arr = (C.c_int * L.MAX_ORDER)()
    for i, r in enumerate(R):
        arr[i] = int(r)
    return arr


def _factors(A: Sequence[torch.Tensor]):
    for i, a in enumerate(A):
        _need(a, f"A[{i}]")
    return L.ptr_array([a.data_ptr() for a in A])


def tucker_leverage_scores(h: Handle, A: Sequence[torch.Tensor], with_cdf: bool = True):
    """(lev list FP64, cdf list int64-viewed uint64 or None, ranks list)."""
    lib = L.load()
    N = len(A)
    I = (C.c_int64 * L.MAX_ORDER)(*[a.shape[0] for a in A])
    R = _ranks([a.shape[1] for a in A])
    dev = A[0].device
    lev = [torch.empty(a.shape[0], dtype=torch.float64, device=dev) for a in A]
    cdf = [torch.empty(a.shape[0], dtype=torch.int64, device=dev) for a in A] if with_cdf else None
    rank = (C.c_int * L.MAX_ORDER)()
    _check(h.h, lib.tucker_leverage_scores(
        h.h, N, I, R, _dt(A[0]), _factors(A), L.ptr_array([t.data_ptr() for t in lev]),
        L.ptr_array([t.data_ptr() for t in cdf]) if cdf else None, rank))
    return lev, cdf, [rank[i] for i in range(N)]


def tucker_sample_rows(h: Handle, dims: Sequence[int], ranks: Sequence[int],
                       lev: Sequence[torch.Tensor], m: int, seed: int, sweep: int = 0,
                       reg: str = "exact", observed: Optional[CooTensor] = None,
                       max_draws: int = 0, out: Optional[Samples] = None) -> Samples:
    lib = L.load()
    N = len(dims)
    I = (C.c_int64 * L.MAX_ORDER)(*[int(v) for v in dims])
    out = out if out is not None else Samples.empty(m, lev[0].device)
    cs = out._c()
    obs = C.byref(_tensor(observed)) if observed is not None else None
    _check(h.h, lib.tucker_sample_rows(h.h, N, I, _ranks(ranks), L.ptr_array([t.data_ptr() for t in lev]),
                                       int(m), int(seed), int(sweep), REG[reg], obs, int(max_draws),
                                       C.byref(cs)))
    out.n_unique, out.n_draws = int(cs.n_unique), int(cs.n_draws)
    return out


def tucker_core_update_sketched(h: Handle, X, A: Sequence[torch.Tensor], lam: float, m: int,
                                seed: int, sweep: int = 0, reg: str = "exact",
                                prec: str = "fp64", fixed: Optional[Samples] = None,
                                eps: float = 0.1, delta: float = 0.1,
                                core_out: Optional[torch.Tensor] = None, stats: bool = False):
    """Sketched core (float64, length prod R_n); with stats=True also a dict of stats."""
    lib = L.load()
    d = 1
    for a in A:
        d *= a.shape[1]
    core = core_out if core_out is not None else torch.empty(d, dtype=torch.float64, device=A[0].device)
    st = L.TuckerStats() if stats else None
    fx = C.byref(fixed._c()) if fixed is not None else None
    _check(h.h, lib.tucker_core_update_sketched(
        h.h, C.byref(_tensor(X)), _ranks([a.shape[1] for a in A]), _factors(A), float(lam),
        int(m), float(eps), float(delta), int(seed), int(sweep), REG[reg], PREC[prec], fx,
        core.data_ptr(), C.byref(st) if st is not None else None))
    if stats:
        return core, {k: getattr(st, k) for k, _ in L.TuckerStats._fields_}
    return core


def tucker_core_update_exact(h: Handle, X, A: Sequence[torch.Tensor], lam: float,
                             prec: str = "fp64", core_out: Optional[torch.Tensor] = None):
    lib = L.load()
    d = 1
    for a in A:
        d *= a.shape[1]
    core = core_out if core_out is not None else torch.empty(d, dtype=torch.float64, device=A[0].device)
    _check(h.h, lib.tucker_core_update_exact(h.h, C.byref(_tensor(X)), _ranks([a.shape[1] for a in A]),
                                             _factors(A), float(lam), PREC[prec], core.data_ptr()))
    return core


def tucker_als_sweep(h: Handle, X: torch.Tensor, A: List[torch.Tensor], core: torch.Tensor,
                     lam: float, sketched: bool = False, m: int = 0, seed: int = 0,
                     sweep: int = 0, reg: str = "exact", prec: str = "fp64"):
    """One ALS pass updating A (list of tensors) and core (float64) in place; (loss, rmse)."""
    lib = L.load()
    _need(core, "core")
    loss, rmse = C.c_double(), C.c_double()
    _check(h.h, lib.tucker_als_sweep(h.h, C.byref(_tensor(X)), _ranks([a.shape[1] for a in A]),
                                     _factors(A), core.data_ptr(), float(lam), int(sketched), int(m),
                                     int(seed), int(sweep), REG[reg], PREC[prec], C.byref(loss),
                                     C.byref(rmse)))
    return loss.value, rmse.value


def tucker_ridge_loss(h: Handle, X, A: Sequence[torch.Tensor], lam: float, g: torch.Tensor) -> float:
    lib = L.load()
    _need(g, "g")
    out = C.c_double()
    _check(h.h, lib.tucker_ridge_loss(h.h, C.byref(_tensor(X)), _ranks([a.shape[1] for a in A]),
                                      _factors(A), float(lam), g.data_ptr(), C.byref(out)))
    return out.value


def tucker_sketched_gram(h: Handle, X, A: Sequence[torch.Tensor], prec: str, samples: Samples,
                         with_rhs: bool = True):
    """(G d x d FP64, h FP64 or None) of a frozen sample: sum_u w_u k_u k_u^T, sum_u w_u x_u k_u."""
    lib = L.load()
    d = 1
    for a in A:
        d *= a.shape[1]
    G = torch.empty((d, d), dtype=torch.float64, device=A[0].device)
    hv = torch.empty(d, dtype=torch.float64, device=A[0].device) if with_rhs else None
    _check(h.h, lib.tucker_sketched_gram(h.h, C.byref(_tensor(X)), _ranks([a.shape[1] for a in A]),
                                         _factors(A), PREC[prec], C.byref(samples._c()),
                                         G.data_ptr(), hv.data_ptr() if hv is not None else None))
    return G, hv


def tucker_core_solve_adjoint(h: Handle, X, A: Sequence[torch.Tensor], lam: float, reg: str,
                              prec: str, samples: Samples, solve_id: int, g: torch.Tensor,
                              gbar: torch.Tensor):
    """(dA list FP64, dx FP64 per distinct sampled row) for cotangent gbar."""
    lib = L.load()
    dA = [torch.empty(a.shape, dtype=torch.float64, device=a.device) for a in A]
    dx = torch.empty(samples.n_unique, dtype=torch.float64, device=A[0].device)
    _check(h.h, lib.tucker_core_solve_adjoint(
        h.h, C.byref(_tensor(X)), _ranks([a.shape[1] for a in A]), _factors(A), float(lam),
        REG[reg], PREC[prec], C.byref(samples._c()), int(solve_id), g.data_ptr(), gbar.data_ptr(),
        L.ptr_array([t.data_ptr() for t in dA]), dx.data_ptr()))
    return dA, dx


def tucker_ridge_tables(h: Handle, A: Sequence[torch.Tensor], lam: float):
    """Tables of the lambda-ridge leverage distribution of K (Lemma 4.1):
    (usq list of K_n x I_n FP64, c FP64 [prod K_n], K list, d_eff)."""
    lib = L.load()
    N = len(A)
    I = (C.c_int64 * L.MAX_ORDER)(*[a.shape[0] for a in A])
    K = [min(a.shape[0], a.shape[1]) for a in A]
    dev = A[0].device
    usq = [torch.empty((k, a.shape[0]), dtype=torch.float64, device=dev) for k, a in zip(K, A)]
    dK = 1
    for k in K:
        dK *= k
    c = torch.empty(dK, dtype=torch.float64, device=dev)
    Kout = (C.c_int * L.MAX_ORDER)()
    deff = C.c_double()
    _check(h.h, lib.tucker_ridge_tables(h.h, N, I, _ranks([a.shape[1] for a in A]), _dt(A[0]),
                                        _factors(A), float(lam),
                                        L.ptr_array([t.data_ptr() for t in usq]), c.data_ptr(),
                                        Kout, C.byref(deff)))
    return usq, c, [int(Kout[n]) for n in range(N)], float(deff.value)


def tucker_sample_rows_ridge(h: Handle, dims: Sequence[int], K: Sequence[int],
                             usq: Sequence[torch.Tensor], c: torch.Tensor, m: int, seed: int,
                             sweep: int = 0, out: Optional[Samples] = None) -> Samples:
    """m rows of K drawn from l^lam(K) / d_eff(K) given its tables, deduplicated."""
    lib = L.load()
    N = len(dims)
    I = (C.c_int64 * L.MAX_ORDER)(*[int(v) for v in dims])
    out = out if out is not None else Samples.empty(m, c.device)
    cs = out._c()
    _check(h.h, lib.tucker_sample_rows_ridge(h.h, N, I, _ranks(K),
                                             L.ptr_array([t.data_ptr() for t in usq]),
                                             c.data_ptr(), int(m), int(seed), int(sweep),
                                             C.byref(cs)))
    out.n_unique, out.n_draws = int(cs.n_unique), int(cs.n_draws)
    return out


def tucker_factor_update_sketched(h: Handle, X: torch.Tensor, A: List[torch.Tensor],
                                  core: torch.Tensor, n: int, lam: float, m: int, seed: int,
                                  sweep: int = 0) -> torch.Tensor:
    """Sketched factor update of mode n (leverage sample of the factor design from the other
    modes' scores, mode-n fibers); A[n] is overwritten and returned."""
    lib = L.load()
    _need(core, "core")
    _check(h.h, lib.tucker_factor_update_sketched(h.h, C.byref(_tensor(X)),
                                                  _ranks([a.shape[1] for a in A]), _factors(A),
                                                  core.data_ptr(), int(n), float(lam), int(m),
                                                  int(seed), int(sweep)))
    return A[n]


def tucker_cp_factor_update_sketched(h: Handle, X: torch.Tensor, A: List[torch.Tensor], n: int,
                                     lam: float, m: int, seed: int, sweep: int = 0) -> torch.Tensor:
    """Sketched CP factor update of mode n (Khatri-Rao design rows sampled by the other
    modes' leverage scores, mode-n fibers); A[n] is overwritten and returned."""
    lib = L.load()
    _check(h.h, lib.tucker_cp_factor_update_sketched(h.h, C.byref(_tensor(X)), int(A[0].shape[1]),
                                                     _factors(A), int(n), float(lam), int(m),
                                                     int(seed), int(sweep)))
    return A[n]


def tucker_cp_als_sweep(h: Handle, X: torch.Tensor, A: List[torch.Tensor], lam: float, m: int,
                        seed: int, sweep: int = 0) -> List[torch.Tensor]:
    """One regularised CP-ALS sweep of sketched factor updates; the factors A are updated
    in place and returned."""
    lib = L.load()
    _check(h.h, lib.tucker_cp_als_sweep(h.h, C.byref(_tensor(X)), int(A[0].shape[1]), _factors(A),
                                        float(lam), int(m), int(seed), int(sweep)))
    return A


def tucker_set_factor_sketch(h: Handle, m: int) -> None:
    """m > 0: later ALS sweeps on h sketch their factor updates with m draws each."""
    lib = L.load()
    _check(h.h, lib.tucker_set_factor_sketch(h.h, int(m)))


BETA_MODE = {"bound": 0, "exact": 1}


def tucker_missing_beta(h: Handle, X, A: Sequence[torch.Tensor], lam: float, mode: str = "bound",
                        prec: str = "fp64", eps: float = 0.1, delta: float = 0.1) -> dict:
    """Overestimate factor of the observed-entry sampler (Sec. 4.2): lambda_max of the
    missing rows' cross ridge scores (the corollary's bound or the certified exact value),
    beta_miss, c_min, beta = c_min beta_miss, beta' and Alg. 1 line 3's s."""
    lib = L.load()
    info = L.TuckerMissingBetaInfo()
    _check(h.h, lib.tucker_missing_beta(h.h, C.byref(_tensor(X)), _ranks([a.shape[1] for a in A]),
                                        _factors(A), float(lam), BETA_MODE[mode], PREC[prec],
                                        float(eps), float(delta), C.byref(info)))
    return {k: getattr(info, k) for k, _ in L.TuckerMissingBetaInfo._fields_}


def tucker_sample_rows_noalloc(dims: Sequence[int], ranks: Sequence[int],
                               lev: Sequence[torch.Tensor], m: int, seed: int, sweep: int = 0,
                               reg: str = "exact", out: Optional[Samples] = None,
                               stream: Optional[torch.cuda.Stream] = None) -> Samples:
    """tucker_sample_rows without a handle and without device allocation by the
    library: its scratch is a fixed array inside libtucker (dense tensors only).
    `out` must be preallocated by callers that cannot allocate."""
    lib = L.load()
    N = len(dims)
    I = (C.c_int64 * L.MAX_ORDER)(*[int(v) for v in dims])
    out = out if out is not None else Samples.empty(m, lev[0].device)
    cs = out._c()
    s = stream if stream is not None else torch.cuda.current_stream()
    err = C.create_string_buffer(256)
    st = lib.tucker_sample_rows_noalloc(C.c_void_p(s.cuda_stream), N, I, _ranks(ranks),
                                        L.ptr_array([t.data_ptr() for t in lev]), int(m), int(seed),
                                        int(sweep), REG[reg], C.byref(cs), err, 256)
    if st != L.OK:
        raise TuckerError(st, err.value.decode(errors="replace"))
    out.n_unique, out.n_draws = int(cs.n_unique), int(cs.n_draws)
    return out


def tucker_set_solver(h: Handle, solver: str) -> None:
    """tucker_set_solver: "fp64" (FP64 Cholesky, the default) or "mixed"."""
    h.set_solver(solver)
