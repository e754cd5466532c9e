"""a16 learned start on the GPU (through the C ABI) against the CPU oracle of
oracle/learned_start.py: the variogram features (bin decisions exact, values
to float32 rounding), the perceptron's forward pass, gradient and Adam step
(FP32 kernels vs the FP64 oracle), and training on simulated fields."""
import numpy as np
import pytest

from oracle import learned_start as ols
from paper_2104_07146_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(hmle_lib):
    from paper_2104_07146_gb300 import hmle
    return hmle.Context()


@pytest.mark.parametrize("n,d,seed", [(3000, 2, 81), (10007, 2, 82), (2500, 3, 83)])
def test_features_match_oracle(ctx, n, d, seed):
    # n = 10007 exercises the 4096-point subsample; d = 3 the third dimension
    from paper_2104_07146_gb300 import learned_start as ls
    if d == 2:
        locs = synth.locations_blobs(n, 2, 0.3, 8, 0.03, seed=seed)
    else:
        locs = synth.uniform(seed, n * 3).reshape(n, 3)
    Z = synth.normal(seed + 1, n) * 1.7 + 0.2
    f = ls.features(ctx, locs, Z)
    ref = ols.features(locs, Z)
    assert np.all(np.abs(f - ref) <= 2e-6 * np.maximum(1.0, np.abs(ref))), np.abs(f - ref).max()


def _model(ctx, seed):
    from paper_2104_07146_gb300 import learned_start as ls
    m = ls.LearnedStart(ctx, seed=seed)
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.25, ols.NPARAMS).astype(np.float32)
    mu = rng.normal(0, 1, 35).astype(np.float32)
    sd = rng.uniform(0.5, 2.0, 35).astype(np.float32)
    m.set(p, mu, sd)
    X = rng.normal(0, 2, (37, 35)).astype(np.float32)
    T = rng.normal(0, 1, (37, 4)).astype(np.float32)
    Xn = (X.astype(np.float64) - mu) / sd
    return m, p.astype(np.float64), X, Xn, T


def test_mlp_forward_matches_oracle(ctx):
    m, p, X, Xn, T = _model(ctx, 91)
    Y = m.forward(X)
    ref = ols.mlp_forward(p, Xn)[2]
    assert np.abs(Y - ref).max() <= 1e-4 * max(1.0, np.abs(ref).max())


def test_mlp_gradient_matches_oracle(ctx):
    m, p, X, Xn, T = _model(ctx, 92)
    g, loss = m.grad(X, T)
    gref = ols.mlp_grad(p, Xn, T.astype(np.float64))
    lref = ols.nll(ols.mlp_forward(p, Xn)[2], T.astype(np.float64))
    assert abs(loss - lref) <= 1e-4 * max(1.0, abs(lref))
    assert np.abs(g - gref).max() <= 1e-4 * max(1.0, np.abs(gref).max())


def test_adam_step_matches_oracle(ctx):
    m, p, X, Xn, T = _model(ctx, 93)
    g, _ = m.grad(X, T)
    m.adam_step(g, 1e-3)
    m.adam_step(g * 0.5, 1e-3)
    p1 = m.get()[0]
    q, mm, vv = ols.adam_step(p, np.zeros_like(p), np.zeros_like(p), g.astype(np.float64), 1, 1e-3)
    q, mm, vv = ols.adam_step(q, mm, vv, 0.5 * g.astype(np.float64), 2, 1e-3)
    assert np.abs(p1 - q).max() <= 1e-6


def test_training_on_simulated_fields_reduces_loss(ctx):
    from paper_2104_07146_gb300 import learned_start as ls
    F, T = ls.training_set(ctx, 32, seed=5, n_range=(300, 600))
    assert np.all(np.isfinite(F)) and np.all(np.isfinite(T))
    model = ls.LearnedStart(ctx, seed=3)
    l0, l1 = model.train(F, T, epochs=150, batch=16, lr=3e-3, seed=9)
    assert l1 < l0
    th0, steps, fb = model.start(*ls.field(ctx, 6, 0, 500)[:2])
    assert len(th0) == 4 and len(steps) == 4
    assert all(0.05 <= s <= 2.0 for s in steps) or fb
