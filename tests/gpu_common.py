"""Helpers for the GPU parity tests: device upload and the library handle.

Inputs come from `synth` (or small seeded numpy draws) and are fed, as the
same arrays, to the CUDA path (through the C ABI binding) and to the oracle.
"""
import numpy as np
import pytest
import torch

from paper_2107_10654_gb300 import tucker as T


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def dev_keys(k):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(k, dtype=np.uint64).view(np.int64))).cuda()


def host_keys(t, n=None):
    a = t.cpu().numpy().view(np.uint64)
    return a if n is None else a[:n]


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def handle():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    h = T.Handle()
    yield h
    h.close()
