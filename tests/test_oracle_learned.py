"""Pins of the learned-start oracle (CPU): hand-computed variograms, the
backpropagated gradient against central finite differences, the closed form
of Adam's first step and of the loss at zero log-scales."""
import math

import numpy as np

from oracle import learned_start as ls


def test_variogram_unit_square_by_hand():
    # corners of the unit square, Z = 0, 1, 2, 3: S = 2, every pair has
    # h^2 >= e_31 = 1, so all six pairs land in bin 31:
    # (1 + 4 + 4 + 1 + 9 + 1) / 2 / 6 = 5/3
    locs = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    S, cnt, gam = ls.variogram(locs, np.array([0.0, 1.0, 2.0, 3.0]))
    assert S == 2.0
    assert cnt[31] == 6 and cnt.sum() == 6
    assert gam[31] == 5.0 / 3.0


def test_variogram_line_bins_by_hand():
    # x = 0, 1, 3 on a line: S = 9; h^2 = 1 -> 9 2^(k-32) <= 1 for k <= 28.83
    # (bin 28); h^2 = 4 -> bin 30; h^2 = 9 = S -> bin 31
    locs = np.array([[0.0, 0.0], [1.0, 0.0], [3.0, 0.0]])
    Z = np.array([1.0, 3.0, 4.0])
    S, cnt, gam = ls.variogram(locs, Z)
    assert S == 9.0
    assert cnt[28] == 1 and cnt[30] == 1 and cnt[31] == 1 and cnt.sum() == 3
    assert gam[28] == 2.0 and gam[30] == 0.5 and gam[31] == 4.5


def test_features_fill_rule_and_tail():
    locs = np.array([[0.0, 0.0], [1.0, 0.0], [3.0, 0.0]])
    f = ls.features(locs, np.array([1.0, 3.0, 4.0]))
    assert f.shape == (35,)
    # bins 0..28 take bin 28 (nearest non-empty above), bin 29 takes bin 30
    assert np.all(f[:29] == math.log(2.0)) and f[29] == math.log(0.5)
    assert f[30] == math.log(0.5) and f[31] == math.log(4.5)
    assert f[32] == math.log(3) and f[33] == 2.0 and f[34] == 0.5 * math.log(9.0)


def test_sample_indices_spread_over_the_input():
    assert list(ls.sample_indices(10, 4)) == [0, 2, 5, 7]
    assert list(ls.sample_indices(3, 4)) == [0, 1, 2]


def _params(seed):
    rng = np.random.default_rng(seed)
    return rng.normal(0, 0.1, ls.NPARAMS)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(5)
    p = _params(4)
    X = rng.normal(size=(7, ls.NF))
    T = rng.normal(size=(7, 4))
    g = ls.mlp_grad(p, X, T)
    for j in rng.choice(ls.NPARAMS, 40, replace=False):
        e = np.zeros_like(p)
        e[j] = 1e-6
        fd = (ls.nll(ls.mlp_forward(p + e, X)[-1], T) - ls.nll(ls.mlp_forward(p - e, X)[-1], T)) / 2e-6
        assert abs(fd - g[j]) <= 1e-6 * max(1.0, abs(fd)), (j, fd, g[j])


def test_nll_at_zero_log_scale_is_half_squared_error():
    Y = np.zeros((3, 8))
    Y[:, :4] = [[1, 2, 3, 4], [0, 0, 0, 0], [1, 1, 1, 1]]
    T = np.ones((3, 4))
    assert ls.nll(Y, T) == (0.5 * (0 + 1 + 4 + 9) + 0.5 * 4 + 0.0) / 3


def test_adam_first_step_is_lr_times_sign():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([3.0, -0.25, 1e-3])
    p1, m, v = ls.adam_step(p, np.zeros(3), np.zeros(3), g, 1, 0.01)
    # m_hat = g, v_hat = g^2: the step is lr g / (|g| + eps)
    assert np.allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_rounding_by_hand():
    # 8 significant bits: 1 + 2^-8 is a tie between 1 and 1 + 2^-7 and goes
    # to the even one (1); 1 + 3 2^-9 rounds up; the FP32 rounding comes first
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, 1.0 + 2.0 ** -7 + 2.0 ** -8, -3.0, 0.0,
                  1.0 + 2.0 ** -8 + 2.0 ** -30])
    r = ls.bf16(x)
    assert list(r) == [1.0, 1.0, 1.0 + 2.0 ** -7, 1.0 + 2.0 ** -6, -3.0, 0.0, 1.0]
    y = np.random.default_rng(3).normal(size=1000) * 10.0 ** np.random.default_rng(4).uniform(-5, 5, 1000)
    assert np.all(np.abs(ls.bf16(y) - y) <= (2.0 ** -8 + 2.0 ** -24) * np.abs(y))
    assert np.array_equal(ls.bf16(ls.bf16(y)), ls.bf16(y))


def test_bf16_products_only_round_the_operands():
    # with bf16=True the forward pass equals the FP64 pass of a network whose
    # every product operand was rounded: check the first layer by hand
    rng = np.random.default_rng(6)
    p = _params(7)
    X = rng.normal(size=(5, ls.NF))
    (W1, b1) = ls.unpack(p)[0]
    H1 = np.tanh(ls.bf16(X) @ ls.bf16(W1).T + b1)
    assert np.allclose(ls.mlp_forward(p, X, bf16=True)[0], H1, rtol=0, atol=1e-14)
    # and its gradient is the FP64 gradient up to the operand rounding
    T = rng.normal(size=(5, 4))
    g, gb = ls.mlp_grad(p, X, T), ls.mlp_grad(p, X, T, bf16=True)
    assert np.max(np.abs(g - gb)) <= 0.05 * np.max(np.abs(g))
    assert not np.array_equal(g, gb)
