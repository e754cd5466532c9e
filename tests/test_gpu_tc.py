"""The tensor-core tile product of the mixed forms (tcgen05.mma, BF16
slices, FP32 accumulation in tensor memory) through the C ABI, against the
plain product of the same slices.

Every operand value a is rounded to FP32 and split into s BF16 slices,
a_0 = bf16(a), a_1 = bf16(a - a_0), ...; the device forms
sum_{p + q < s} A_p B_q with FP32 accumulation.  The reference below builds
the slices with numpy (FP32 rounding to nearest even, BF16 by rounding the
upper half of the FP32 bit pattern to nearest even) and multiplies them in
FP64.  The only difference allowed is the FP32 accumulation:
|C - C_ref| <= K 2^-23 (|A_s| |B_s|) elementwise.  A misplaced core matrix, a
wrong descriptor offset or a lost chunk gives errors of the size of C itself.
The shapes cover one tile, ragged tiles in M, N and K, several M and N tiles,
K = 0, and many CTAs resident at once (tensor-memory allocation under
contention); both staging orders of both operands.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _bf16(x32):
    b = x32.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def _slices(x, s):
    a = x.astype(np.float32)
    out = []
    for _ in range(s):
        h = _bf16(a)
        out.append(h.astype(np.float64))
        a = (a - h).astype(np.float32)
    return out


def _reference(A, B, s):
    As, Bs = _slices(A, s), _slices(B, s)
    C = np.zeros((A.shape[0], B.shape[1]))
    mag = np.zeros_like(C)
    for p in range(s):
        for q in range(s - p):
            C += As[p] @ Bs[q]
            mag += np.abs(As[p]) @ np.abs(Bs[q])
    return C, mag


SHAPES = [(128, 64, 64), (100, 70, 300), (17, 5, 1), (200, 130, 129), (64, 64, 0), (1, 1, 1000), (128, 8, 33)]


@pytest.fixture(scope="module")
def ctx():
    from paper_2104_07146_gb300 import hmle
    return hmle.Context()


@pytest.mark.parametrize("ns", [1, 2, 3])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "%dx%dx%d" % s)
def test_tc_product_matches_its_slices(ctx, ns, shape):
    M, N, K = shape
    rng = np.random.default_rng(M * 1000 + N * 10 + K + ns)
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-3, 3, (M, 1)))
    B = rng.standard_normal((K, N)) * np.exp(rng.uniform(-3, 3, (1, N)))
    Cref, mag = _reference(A, B, ns)
    for ak in (True, False):
        for bk in (True, False):
            C = ctx.tc_gemm(A, B, ns, ak, bk)[0]
            err = np.abs(C - Cref)
            assert np.all(err <= (max(K, 1) * 2.0 ** -23) * mag + 1e-300), (ns, ak, bk, err.max())


@pytest.mark.parametrize("ns", [1, 2, 3])
def test_tc_product_accuracy_per_slice_count(ctx, ns):
    """Against the exact FP64 product, relative to |A||B|: one slice is
    BF16-accurate (8 bits), two about 16 bits, three FP32-class (24-bit
    operands; with K = 500 the FP32 accumulation measured 1.0e-6, so the
    bound is 2^-18 = 3.8e-6, still 16 times below the two-slice bound)."""
    rng = np.random.default_rng(7 + ns)
    A = rng.standard_normal((96, 500))
    B = rng.standard_normal((500, 48))
    C = ctx.tc_gemm(A, B, ns)[0]
    rel = np.max(np.abs(C - A @ B) / (np.abs(A) @ np.abs(B)))
    bound = {1: 2.0 ** -8, 2: 2.0 ** -14, 3: 2.0 ** -18}[ns]
    assert rel <= bound, (ns, rel)


@pytest.mark.parametrize("ns", [1, 3])
def test_tc_product_many_ctas_agree(ctx, ns):
    rng = np.random.default_rng(11)
    A = rng.standard_normal((128, 256))
    B = rng.standard_normal((256, 64))
    C = ctx.tc_gemm(A, B, ns, copies=1200)
    assert np.array_equal(C, np.broadcast_to(C[0], C.shape))
    Cref, mag = _reference(A, B, ns)
    assert np.all(np.abs(C[0] - Cref) <= 256 * 2.0 ** -23 * mag)
