"""Host-side checks of the C ABI: the library builds for sm_103a, loads without a
GPU, and exports every entry point that include/tucker.h declares, with the
struct layouts the binding assumes."""
import ctypes
import os
import re

import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "tucker.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tucker_[a-z_]+)\s*\(", text)))


def test_header_declares_the_five_paper_entry_points():
    names = declared_functions()
    for n in ("tucker_leverage_scores", "tucker_sample_rows", "tucker_core_update_sketched",
              "tucker_core_update_exact", "tucker_als_sweep"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2107_10654_gb300 import _lib
    lib = _lib.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(_lib.SIGNATURES) <= set(declared_functions())


def test_struct_layouts_match_c():
    from paper_2107_10654_gb300 import _lib
    # tucker_tensor: int, pad, int64[8], int, pad, ptr, int64, ptr, ptr
    assert ctypes.sizeof(_lib.TuckerTensor) == 8 + 64 + 8 + 8 + 8 + 8 + 8
    assert ctypes.sizeof(_lib.TuckerSamples) == 6 * 8
    assert ctypes.sizeof(_lib.TuckerStats) == 7 * 8 + 3 * 8 + 8 + 8 + 8 + 8 + 2 * 8 + 2 * 8 + 8
    # tucker_missing_beta_info: seven doubles, two ints
    assert ctypes.sizeof(_lib.TuckerMissingBetaInfo) == 7 * 8 + 2 * 4


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2107_10654_gb300 import _lib
    lib = _lib.load()
    h = ctypes.c_void_p()
    st = lib.tucker_create(ctypes.byref(h), None)
    assert st in (_lib.ECUDA, _lib.ENOTSUP) and not h.value


def test_null_handle_and_bad_arguments_fail_before_any_device_work():
    """Every entry point that takes a handle returns EINVAL for a NULL handle, and
    the allocation-free sampler rejects bad arguments with its message, without a
    GPU (the checks come before any CUDA call)."""
    from paper_2107_10654_gb300 import _lib
    lib = _lib.load()
    assert lib.tucker_last_error(None) == b"null handle"
    zero = {ctypes.c_int: 0, ctypes.c_int64: 0, ctypes.c_uint64: 0, ctypes.c_uint32: 0,
            ctypes.c_double: 0.0, ctypes.c_size_t: 0}
    for name, (_, argtypes) in _lib.SIGNATURES.items():
        if name in ("tucker_create", "tucker_last_error", "tucker_sample_rows_noalloc"):
            continue
        args = [zero.get(t) for t in argtypes]
        assert getattr(lib, name)(*args) == _lib.EINVAL, name
    err = ctypes.create_string_buffer(256)
    dims = (ctypes.c_int64 * 8)(*([4] * 8))
    ranks = (ctypes.c_int * 8)(*([2] * 8))
    out = _lib.TuckerSamples()
    st = lib.tucker_sample_rows_noalloc(None, 3, dims, ranks, None, 10, 0, 0, 0,
                                        ctypes.byref(out), err, 256)
    assert st == _lib.EINVAL and b"null" in err.value
    lev = _lib.ptr_array([1, 1, 1])                 # never dereferenced: rejected first
    out.keys = out.counts = out.prob = 1
    out.capacity = 10
    for N, m in ((0, 10), (9, 10), (3, 0), (3, 1 << 31)):
        st = lib.tucker_sample_rows_noalloc(None, N, dims, ranks, lev, m, 0, 0, 0,
                                            ctypes.byref(out), err, 256)
        assert st == _lib.EINVAL and err.value, (N, m)
