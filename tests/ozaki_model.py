"""A numpy model of an FP64 product computed from BF16 slices with FP32
accumulation (the Ozaki splitting), test infrastructure for a tensor-core
product.

A (m x K) is scaled row by row and B (K x n) column by column by powers of
two so that every entry lies in (-1, 1).  Each scaled entry is then cut into
s slices: slice k is an integer multiple of 2^(-8k) with magnitude below
2^(-8(k-1)), so it has at most 8 significant bits and is exact in BF16.
The product of slice k of A and slice l of B is an integer times 2^(-8(k+l))
below 2^16 in magnitude, exact in FP32, and a sum of up to 256 of them stays
below 2^24, so it is exact in an FP32 accumulator too: K is cut into chunks
of at most 256 and the chunk sums are added in FP64.  Keeping the slice
pairs with k + l <= s + 1 drops terms of relative size about 2^(-8s).

Every partial sum of the model is exact, so a kernel that computes the same
slices and the same chunk sums on tensor cores must reproduce it bit for bit
whatever its accumulation order inside a chunk.
"""
from __future__ import annotations

import numpy as np

SLICE_BITS = 8
CHUNK = 256


def _scale_exponents(X, axis):
    """Per row (axis=1) or column (axis=0): e with max |x| < 2^e."""
    mx = np.max(np.abs(X), axis=axis)
    e = np.zeros_like(mx, dtype=np.int64)
    nz = mx > 0
    e[nz] = np.frexp(mx[nz])[1]            # mx = f 2^e, 0.5 <= f < 1
    return e


def split(X, s, axis):
    """(slices, e): X = 2^e * sum_k slices[k] (row scaling for axis=1,
    column scaling for axis=0) up to the residual below 2^(-8s); every slice
    entry is an integer multiple of 2^(-8(k+1)) of magnitude < 2^(-8k)."""
    e = _scale_exponents(X, axis)
    sc = np.ldexp(1.0, -e)
    R = X * (sc[:, None] if axis == 1 else sc[None, :])   # exact: powers of two
    out = []
    for k in range(1, s + 1):
        q = np.ldexp(np.trunc(np.ldexp(R, SLICE_BITS * k)), -SLICE_BITS * k)
        out.append(q)
        R = R - q                           # exact: q holds leading bits of R
    return out, e


def bf16_exact(x):
    """True where x is representable in BF16 (8 significant bits)."""
    m, _ = np.frexp(x)
    return np.all(np.ldexp(m, 8) == np.trunc(np.ldexp(m, 8)))


def product(A, B, s):
    """The emulated A @ B from s slices per operand."""
    As, ea = split(A, s, axis=1)
    Bs, eb = split(B, s, axis=0)
    m, K = A.shape
    n = B.shape[1]
    acc = np.zeros((m, n))
    for k in range(s):
        for l in range(s):
            if k + l > s - 1:               # slice pairs k + l <= s + 1 (1-based)
                continue
            a32 = As[k].astype(np.float32)
            b32 = Bs[l].astype(np.float32)
            for c0 in range(0, K, CHUNK):
                part = a32[:, c0:c0 + CHUNK] @ b32[c0:c0 + CHUNK, :]   # FP32, exact
                acc += part.astype(np.float64)
    return np.ldexp(acc, ea[:, None] + eb[None, :])
