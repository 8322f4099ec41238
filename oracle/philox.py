"""Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11).

Oracle module: test infrastructure.  Only tests/, __graft_entry__.smoke() and
bench.py's cpu_baseline / reference leg may import anything under oracle/.

Written from the published definition: the state is four 64-bit counter words
and two 64-bit key words; one round multiplies counter words 0 and 2 by the
two Philox multipliers, producing 128-bit products whose high halves are
XOR-ed with the other counter words and the key, and whose low halves are
carried over; between rounds the key is bumped by the two Weyl constants.
Ten rounds are applied.  Vectorised over numpy uint64 arrays.
"""
from __future__ import annotations

import numpy as np

U64 = np.uint64
_MASK32 = U64(0xFFFFFFFF)
_S32 = U64(32)

PHILOX_M0 = U64(0xD2E7470EE14C6C93)
PHILOX_M1 = U64(0xCA5A826395121157)
PHILOX_W0 = U64(0x9E3779B97F4A7C15)
PHILOX_W1 = U64(0xBB67AE8584CAA73B)


def mulhilo64(a, b):
    """(hi, lo) 64-bit halves of the 128-bit product a*b for uint64 arrays."""
    a = np.asarray(a, dtype=U64)
    b = np.asarray(b, dtype=U64)
    a_lo, a_hi = a & _MASK32, a >> _S32
    b_lo, b_hi = b & _MASK32, b >> _S32
    with np.errstate(over="ignore"):
        p0 = a_lo * b_lo
        p1 = a_lo * b_hi
        p2 = a_hi * b_lo
        p3 = a_hi * b_hi
        mid = (p0 >> _S32) + (p1 & _MASK32) + (p2 & _MASK32)
        lo = (p0 & _MASK32) | (mid << _S32)
        hi = p3 + (p1 >> _S32) + (p2 >> _S32) + (mid >> _S32)
    return hi, lo


def mulhi64(a, b):
    """floor(a*b / 2^64) for uint64 arrays."""
    return mulhilo64(a, b)[0]


def philox4x64_10(c0, c1, c2, c3, k0, k1):
    """Philox4x64 with 10 rounds on counter (c0,c1,c2,c3) and key (k0,k1).

    Every argument is a uint64 scalar or array (broadcast).  Returns four
    uint64 arrays, the output words 0..3.
    """
    c0 = np.asarray(c0, dtype=U64)
    c1 = np.asarray(c1, dtype=U64)
    c2 = np.asarray(c2, dtype=U64)
    c3 = np.asarray(c3, dtype=U64)
    k0 = U64(k0)
    k1 = U64(k1)
    with np.errstate(over="ignore"):
        for r in range(10):
            if r:
                k0 = U64(k0 + PHILOX_W0)
                k1 = U64(k1 + PHILOX_W1)
            hi0, lo0 = mulhilo64(PHILOX_M0, c0)
            hi1, lo1 = mulhilo64(PHILOX_M1, c2)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3
