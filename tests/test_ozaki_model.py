"""The slice arithmetic that a tensor-core FP64 product would use
(tests/ozaki_model.py), checked on the CPU: the slices are exact in BF16,
every FP32 chunk sum is exact (equal to integer arithmetic), and the
emulated product is as accurate as FP64 with 7 slices and at least as
accurate as FP32 products with 4 (3 slices fall short of FP32 by a factor of
a few on these operands).
These are the numbers behind the planned tensor-core form of the update
products; no product code uses this model.
"""
import numpy as np
import pytest

import ozaki_model as oz


def _operands(m, K, n, seed, spread=8.0):
    # rows / columns of very different size, like the factors of the sweep
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, K)) * 10.0 ** rng.uniform(-spread, 0, size=(m, 1))
    B = rng.standard_normal((K, n)) * 10.0 ** rng.uniform(-spread, 0, size=(1, n))
    B[:, 0] *= 10.0 ** -rng.uniform(0, 4, size=K)      # a column with wide dynamic range
    return A, B


@pytest.mark.parametrize("s", [3, 7])
def test_slices_are_bf16_and_rebuild_the_operand(s):
    A, _ = _operands(64, 300, 8, 1)
    sl, e = oz.split(A, s, axis=1)
    for k, q in enumerate(sl, start=1):
        assert oz.bf16_exact(q)
        assert np.all(np.abs(q) < 2.0 ** (-8 * (k - 1)))
        assert np.all(np.ldexp(q, 8 * k) == np.trunc(np.ldexp(q, 8 * k)))
    rebuilt = np.ldexp(sum(sl), e[:, None])
    bound = np.ldexp(np.ones(A.shape[0]), e - 8 * s)[:, None]       # residual below 2^(e - 8s)
    assert np.all(np.abs(rebuilt - A) < bound)


def test_fp32_chunk_sums_are_exact():
    A, B = _operands(32, 256, 16, 2)
    As, _ = oz.split(A, 3, axis=1)
    Bs, _ = oz.split(B, 3, axis=0)
    for k in range(3):
        for l in range(3):
            f32 = As[k].astype(np.float32) @ Bs[l].astype(np.float32)
            ia = np.ldexp(As[k], 8 * (k + 1)).astype(np.int64)        # integers below 2^8
            ib = np.ldexp(Bs[l], 8 * (l + 1)).astype(np.int64)
            exact = ia @ ib                                           # integer arithmetic
            assert np.all(np.abs(exact) < 2 ** 24)
            assert np.array_equal(np.ldexp(f32.astype(np.float64), 8 * (k + l + 2)),
                                  exact.astype(np.float64))


def _exact_product(A, B):
    return np.dot(A.astype(np.longdouble), B.astype(np.longdouble))


@pytest.mark.parametrize("m,K,n", [(64, 700, 48), (64, 64, 32)])
def test_accuracy_with_7_and_3_slices(m, K, n):
    if np.finfo(np.longdouble).eps > 1e-18:
        pytest.skip("needs an extended-precision long double for the reference")
    A, B = _operands(m, K, n, 3)
    ref = _exact_product(A, B)
    scale = np.dot(np.abs(A), np.abs(B))                              # |A| |B|
    err64 = np.max(np.abs((A @ B) - ref) / scale)
    prod32 = (A.astype(np.float32) @ B.astype(np.float32)).astype(np.float64)
    err32 = np.max(np.abs(prod32 - ref) / scale)
    err = {s: np.max(np.abs(oz.product(A, B, s) - ref) / scale) for s in (3, 4, 7)}
    assert err[7] <= max(4.0 * err64, 2.0 ** -52)                    # 7 slices: FP64-class
    assert err[4] <= err32                                            # 4 slices: FP32 or better
    assert err32 < err[3] <= 8.0 * err32                              # 3 slices: below FP32
