"""a16 learned start on the GPU (through the C ABI) against the CPU oracle of
oracle/learned_start.py: the variogram features (bin decisions exact, values
to float32 rounding), the 35-256-256-256-8 perceptron's forward pass,
gradient and Adam step (tensor-core products with BF16 operands and FP32
accumulation, against the FP64 oracle whose product operands are rounded to
BF16 the same way), training on simulated fields, and what the trained
network gains over the default start."""
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
    p = rng.normal(0, 0.08, ols.NPARAMS).astype(np.float32)
    mu = rng.normal(0, 1, 35).astype(np.float32)
    sd = rng.uniform(0.5, 2.0, 35).astype(np.float32)
    m.set(p, mu, sd)
    X = rng.normal(0, 2, (37, 35)).astype(np.float32)
    T = rng.normal(0, 1, (37, 4)).astype(np.float32)
    Xn = (X.astype(np.float64) - mu) / sd
    return m, p.astype(np.float64), X, Xn, T


def _xn32(X, mu, sd):
    # the device standardises in FP32
    return ((X.astype(np.float32) - mu) / sd).astype(np.float64)


def test_mlp_forward_matches_oracle(ctx):
    m, p, X, Xn, T = _model(ctx, 91)
    mu, sd = m.get()[1], m.get()[2]
    Y = m.forward(X)
    ref = ols.mlp_forward(p, _xn32(X, mu, sd), bf16=True)[-1]
    assert np.abs(Y - ref).max() <= 1e-3 * max(1.0, np.abs(ref).max()), np.abs(Y - ref).max()
    # the BF16 operands are what the device multiplies: the FP64 network differs more
    full = ols.mlp_forward(p, Xn)[-1]
    assert np.abs(Y - full).max() > np.abs(Y - ref).max()


def test_mlp_gradient_matches_oracle(ctx):
    m, p, X, Xn, T = _model(ctx, 92)
    mu, sd = m.get()[1], m.get()[2]
    g, loss = m.grad(X, T)
    x32 = _xn32(X, mu, sd)
    gref = ols.mlp_grad(p, x32, T.astype(np.float64), bf16=True)
    lref = ols.nll(ols.mlp_forward(p, x32, bf16=True)[-1], T.astype(np.float64))
    assert abs(loss - lref) <= 1e-3 * max(1.0, abs(lref))
    assert np.abs(g - gref).max() <= 2e-3 * max(1.0, np.abs(gref).max()), np.abs(g - gref).max()


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
    assert F.shape == (32, 35)
    assert np.all(np.isfinite(F)) and np.all(np.isfinite(T))
    model = ls.LearnedStart(ctx, seed=3)
    l0, l1 = model.train(F, T, epochs=150, batch=16, lr=3e-3, seed=9)
    assert l1 < l0
    th0, steps, fb = model.start(*ls.field(ctx, 6, 0, 500)[:2])
    assert len(th0) == 4 and len(steps) == 4
    assert all(0.05 <= s <= 2.0 for s in steps) or fb


@pytest.mark.slow
def test_learned_start_needs_fewer_evaluations(ctx):
    """Trained on simulated fields, the network's start (theta and simplex
    steps) reaches the same maximum of L as the default start of Sec. 5 with
    fewer likelihood evaluations, summed over held-out fields."""
    from paper_2104_07146_gb300 import learned_start as ls
    F, T = ls.training_set(ctx, 240, seed=21, n_range=(800, 2000))
    model = ls.LearnedStart(ctx, seed=4)
    l0, l1 = model.train(F, T, epochs=120, batch=32, lr=1e-3, seed=5)
    assert l1 < l0
    fields = [ls.field(ctx, 977, i, 1500) for i in range(6)]
    rows, tot = ls.compare_starts(ctx, model, fields)
    for r in rows:
        n = r["n"]
        # the learned start's optimum is at least as likely (to 1e-6 per point)
        assert r["learned"]["L"] >= r["default"]["L"] - 1e-6 * n, r
    print("evaluations: default %d, learned %d" % (tot["default"]["evals"], tot["learned"]["evals"]))
    assert tot["learned"]["evals"] < tot["default"]["evals"], tot
