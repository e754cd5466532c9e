"""Mixed forms (Schur-update, Gram and panel-update products on the tensor
cores with BF16 slices and FP32 accumulation; FP64 recompression / POTRF /
log-det; quadratic form by PCG) through the C ABI, against the CPU oracle.

Two forms: HMLE_MIXED_FP32 (operands split into three BF16 slices, 24 bits)
and HMLE_MIXED_BF16 (two slices, 16 bits).  Stated bounds: the quadratic form
is won back by PCG to the FP64 bound |dq| / n <= 1e-6 in both; the
log-determinant carries the rounding of the Schur complements,
|d logdet| / n <= 5e-5 for the 24-bit form and <= 2e-3 for the 16-bit form,
and so does L.  The largest errors come from the smooth field (nu = 1.5 on
the blob mixture: 2.3e-5 and 7.0e-4 measured on GB300); on the rough fields
(nu = 1/2) the 24-bit form stays below 1e-6 and the 16-bit form near 1e-5.
"""
import pytest

import oracle
from paper_2104_07146_gb300 import synth

pytestmark = pytest.mark.gpu

# (precision, bound on |d logdet| / n and |dL| / n)
FORMS = [(1, 5e-5), (2, 2e-3)]


@pytest.fixture(params=FORMS, ids=["fp32", "bf16"])
def form(request):
    return request.param


@pytest.fixture(scope="module")
def ctx(hmle_lib):
    from paper_2104_07146_gb300 import hmle
    return hmle.Context()


def _tree(ctx, locs, **kw):
    from paper_2104_07146_gb300 import hmle
    return hmle.Tree(ctx, locs, **kw)


def _mixed_parity(ctx, form, locs, theta, leaf, eps, zseed, field=True, **kw):
    prec, bound = form
    n = locs.shape[0]
    Z = synth.normal(zseed, n)
    if field:
        Z = oracle.simulate(locs, theta, Z)
    t = _tree(ctx, locs, leaf_size=leaf, aca_eps=eps, precision=prec, **kw)
    ll, info = t.loglik(theta, Z)
    ref, ld, q = oracle.loglik_dense(locs, Z, theta)
    print("precision %d n %d: |dq|/n %.2e |dlogdet|/n %.2e |dL|/n %.2e pcg %d"
          % (prec, n, abs(info.quad - q) / n, abs(info.logdet - ld) / n, abs(ll - ref) / n, info.pcg_iters))
    assert info.pcg_iters >= 1 and info.pcg_relres <= 1e-10, (info.pcg_iters, info.pcg_relres)
    assert abs(info.quad - q) / n <= 1e-6, (info.quad, q)
    assert abs(info.logdet - ld) / n <= bound, (info.logdet, ld)
    assert abs(ll - ref) / n <= bound, (ll, ref)
    return info


def test_mixed_small_config(ctx, form):
    locs = synth.locations_uniform(2000, 2, seed=1000)
    _mixed_parity(ctx, form, locs, (0.1, 0.5, 1.0, 0.01), 32, 1e-8, 1001)


def test_mixed_white_noise_ragged(ctx, form):
    # white-noise Z on a smooth field (q ~ 43 n): the FP64 form needs its
    # factor truncated at 1e-10 for this quadratic form; the mixed factor
    # stays at its 1e-7 floor and the PCG on the ACA operator (eps 1e-10)
    # carries the quadratic form
    locs = synth.locations_uniform(3001, 2, seed=21)
    _mixed_parity(ctx, form, locs, (0.15, 1.3, 0.8, 0.02), 32, 1e-10, 22, field=False,
                  max_rank=48, oversample=16)


@pytest.mark.parametrize("nu,eps", [(0.5, 1e-6), (1.5, 1e-7)])
def test_mixed_blob_mixture_leaf64(ctx, form, nu, eps):
    locs = synth.locations_blobs(4096, 2, 0.3, 8, 0.03, seed=23)
    _mixed_parity(ctx, form, locs, (0.05, nu, 1.0, 1e-3), 64, eps, 24, max_rank=48, oversample=16)


def test_mixed_batch_matches_single(ctx, form):
    locs = synth.locations_uniform(2500, 2, seed=61)
    Z = synth.normal(62, 2500)
    t = _tree(ctx, locs, leaf_size=32, aca_eps=1e-8, precision=form[0])
    thetas = [(0.1, 0.5, 1.0, 0.01), (0.12, 0.6, 0.9, 0.02), (0.08, 0.7, 1.1, 0.01)]
    ll, st = t.loglik_batch(thetas, Z, concurrency=3)
    assert all(s == 0 for s in st), list(st)
    for th, v in zip(thetas, ll):
        assert v == t.loglik(th, Z)[0]


def test_pcg_not_converged_is_reported(ctx):
    from paper_2104_07146_gb300 import hmle
    locs = synth.locations_uniform(800, 2, seed=63)
    t = _tree(ctx, locs, leaf_size=32, aca_eps=1e-8, precision=1, pcg_tol=1e-30,
              pcg_max_iter=1)
    with pytest.raises(hmle.HmleError) as e:
        t.loglik((0.1, 0.5, 1.0, 0.01), synth.normal(64, 800))
    assert e.value.status == 7


@pytest.mark.slow
def test_mixed_medium_workload_subset_16384(ctx, form):
    # the medium workload's first 16,384 points at its theta (nu = 1/2, leaf 64,
    # eps 1e-6), Z = L xi from the dense oracle: the mixed form against the
    # oracle and against the FP64 form on the same tree geometry
    locs = synth.medium_locations(65536)[:16384]
    th = (0.05, 0.5, 1.0, 1e-3)
    info = _mixed_parity(ctx, form, locs, th, 64, 1e-6, 53)
    Z = oracle.simulate(locs, th, synth.normal(53, 16384))
    ll64, i64 = _tree(ctx, locs, leaf_size=64, aca_eps=1e-6).loglik(th, Z)
    assert abs(info.logdet - i64.logdet) / 16384 <= form[1]


def test_mixed_three_dimensional(ctx, form):
    locs = synth.locations_uniform(2500, 3, seed=25)
    _mixed_parity(ctx, form, locs, (0.2, 1.0, 1.0, 0.01), 32, 1e-7, 26, max_rank=48, oversample=16)
