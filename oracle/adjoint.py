"""Adjoint of the sketched core solve, with the sketch held fixed (FP64).

Oracle module: test infrastructure.  Only tests/, __graft_entry__.smoke() and
bench.py's cpu_baseline / reference leg may import anything under oracle/.

Forward (Alg. 1 normal equations, Appendix B proof of Thm 4.2):
    M = sum_u w_u k_u k_u^T + lam diag(r),   h = sum_u w_u x_u k_u,   g = M^-1 h,
with k_u = A^(1)[i_1] (x) ... (x) A^(N)[i_N] and r = 1 (REG_EXACT) or the
sampled regulariser weights D (REG_AUGMENTED).  The sampled keys, counts and
probabilities are discrete and treated as constants.  For a cotangent gbar:
    v = M^-1 gbar,
    dL/dx_u = w_u (k_u . v),
    dL/dk_u = w_u (x_u v - (k_u . g) v - (k_u . v) g),
and dL/dA^(n)[i_n, r_n] accumulates dL/dk_u[r] * prod_{m != n} A^(m)[i_m, r_m]
over the r with that r_n (the chain rule through the Kronecker row).
"""
from __future__ import annotations

from typing import Sequence

import numpy as np

from . import sampling as S
from .core_update import kron_rows


def forward(factors: Sequence[np.ndarray], dims, keys_u, w, x, lam, reg_diag):
    """g = M^-1 h for the frozen sketch (keys_u: real rows only)."""
    idx = S.decode_keys(keys_u, dims)
    Kr = kron_rows(factors, idx)
    w = np.asarray(w, dtype=np.float64)
    M = Kr.T @ (Kr * w[:, None]) + lam * np.diag(np.asarray(reg_diag, dtype=np.float64))
    h = Kr.T @ (w * np.asarray(x, dtype=np.float64))
    return np.linalg.solve(M, h)


def backward(factors: Sequence[np.ndarray], dims, keys_u, w, x, lam, reg_diag, gbar):
    """(dA list, dx) for cotangent gbar of the frozen-sketch solve."""
    idx = S.decode_keys(keys_u, dims)
    Kr = kron_rows(factors, idx)
    w = np.asarray(w, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    M = Kr.T @ (Kr * w[:, None]) + lam * np.diag(np.asarray(reg_diag, dtype=np.float64))
    g = np.linalg.solve(M, Kr.T @ (w * x))
    v = np.linalg.solve(M, np.asarray(gbar, dtype=np.float64))
    zg = Kr @ g
    zv = Kr @ v
    dx = w * zv
    dK = w[:, None] * ((x - zg)[:, None] * v[None, :] - zv[:, None] * g[None, :])
    R = [A.shape[1] for A in factors]
    dK = dK.reshape([-1] + R)
    rows = [np.asarray(A, dtype=np.float64)[i] for A, i in zip(factors, idx)]
    letters = "abcdefgh"[:len(R)]
    dA = []
    for n, A in enumerate(factors):
        rest = [k for k in range(len(R)) if k != n]
        spec = ",".join(["u" + letters] + ["u" + letters[k] for k in rest]) + "->u" + letters[n]
        contrib = np.einsum(spec, dK, *[rows[k] for k in rest])
        out = np.zeros(np.asarray(A).shape)
        np.add.at(out, idx[n], contrib)
        dA.append(out)
    return dA, dx
