"""CPU FP64 oracle of the learned start -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` and ``__graft_entry__.smoke()`` may import this module; the
GPU product path never imports it and shares no code with it.

The paper suggests precomputing the optimiser's initial guess (Sec. 7).
The learned start maps summary statistics of one field to an initial theta
and initial simplex steps.  This module is the plain definition of each
step:

* ``sample_indices`` / ``variogram`` / ``features`` -- the empirical
  semivariogram gamma(h) = mean over point pairs with |s_i - s_j| in bin k of
  (Z_i - Z_j)^2 / 2, on m = min(n, 4096) points taken at caller indices
  floor(i n / m).  Bins are in squared distance: with S = sum over dimensions
  of (max - min)^2 of the sampled points (the squared bounding-box diagonal),
  edges e_k = S 2^(k - 32), k = 0..32; bin k holds e_k <= h^2 < e_{k+1}
  (pairs below e_1 in bin 0, h^2 = S in bin 31).  h^2 is summed over
  dimensions in order.  Features (35): log gamma_k for the 32 bins (an
  empty bin takes the value of the nearest non-empty bin above it, else
  below), log n, d, log sqrt(S).
* ``mlp_forward`` / ``nll`` / ``mlp_grad`` / ``adam_step`` -- a
  35-256-256-256-8 perceptron with tanh hidden layers; outputs
  (mu_1..4, s_1..4) are the predicted transformed coordinates of Sec. 5 and
  log step scales, trained with the Gaussian negative log-likelihood
  sum_c [ exp(-2 s_c) (t_c - mu_c)^2 / 2 + s_c ] averaged over the batch,
  and Adam (beta1 0.9, beta2 0.999, eps 1e-8; Kingma & Ba 2015).  With
  ``bf16=True`` both operands of every matrix product are first rounded to
  BF16 (FP32 rounding to nearest even, then BF16 rounding to nearest even)
  and the product is taken in FP64: the arithmetic of products with BF16
  weights and activations, up to the accumulation.

Parameter layout (flat, 142856 values): W1 (256 x 35, row-major), b1 (256),
W2 (256 x 256), b2, W3 (256 x 256), b3, W4 (8 x 256), b4 (8).
"""
from __future__ import annotations

import math

import numpy as np

NF, NH, NO = 35, 256, 8
SIZES = (NF, NH, NH, NH, NO)       # layer widths, input to output
NBINS = 32
M_MAX = 4096


def sample_indices(n: int, m_max: int = M_MAX) -> np.ndarray:
    m = min(n, m_max)
    return np.array([(i * n) // m for i in range(m)], dtype=np.int64)


def variogram(locs, Z, m_max: int = M_MAX):
    """Returns (S, counts[32], gamma[32]) -- gamma is nan for empty bins."""
    locs = np.asarray(locs, dtype=np.float64)
    Z = np.asarray(Z, dtype=np.float64)
    idx = sample_indices(locs.shape[0], m_max)
    P = locs[idx]
    z = Z[idx]
    d = P.shape[1]
    S = 0.0
    for k in range(d):
        w = P[:, k].max() - P[:, k].min()
        S = S + w * w
    edges = np.array([math.ldexp(S, k - 32) for k in range(NBINS + 1)])
    cnt = np.zeros(NBINS)
    acc = np.zeros(NBINS)
    m = len(idx)
    for i in range(m - 1):
        h2 = np.zeros(m - i - 1)
        for k in range(d):
            dx = P[i, k] - P[i + 1:, k]
            h2 = h2 + dx * dx
        b = np.searchsorted(edges[1:NBINS], h2, side="right")
        dz = z[i] - z[i + 1:]
        np.add.at(cnt, b, 1.0)
        np.add.at(acc, b, 0.5 * dz * dz)
    with np.errstate(invalid="ignore", divide="ignore"):
        gam = np.where(cnt > 0, acc / np.maximum(cnt, 1), np.nan)
    return S, cnt, gam


def features(locs, Z, m_max: int = M_MAX) -> np.ndarray:
    locs = np.asarray(locs, dtype=np.float64)
    S, cnt, gam = variogram(locs, Z, m_max)
    f = np.zeros(NF)
    for k in range(NBINS):
        src = k
        if cnt[src] == 0:
            up = [j for j in range(k + 1, NBINS) if cnt[j] > 0]
            dn = [j for j in range(k - 1, -1, -1) if cnt[j] > 0]
            src = up[0] if up else (dn[0] if dn else -1)
        f[k] = math.log(gam[src]) if src >= 0 and gam[src] > 0 else 0.0
    f[32] = math.log(locs.shape[0])
    f[33] = float(locs.shape[1])
    f[34] = 0.5 * math.log(S) if S > 0 else 0.0
    return f


def unpack(p):
    """[(W_1, b_1), ..., (W_4, b_4)], W_l of shape (SIZES[l], SIZES[l - 1])."""
    p = np.asarray(p, dtype=np.float64)
    out, o = [], 0
    for a, b in zip(SIZES[:-1], SIZES[1:]):
        W = p[o:o + a * b].reshape(b, a); o += a * b
        c = p[o:o + b]; o += b
        out.append((W, c))
    assert o == p.size
    return out


NPARAMS = sum(a * b + b for a, b in zip(SIZES[:-1], SIZES[1:]))


def bf16(x):
    """Round to FP32 (nearest even), then to BF16 (nearest even on the upper
    16 bits of the FP32 pattern); returned as float64."""
    x32 = np.ascontiguousarray(x, dtype=np.float32)
    b = x32.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def _mm(A, B, lowp):
    return (bf16(A) @ bf16(B)) if lowp else (A @ B)


def mlp_forward(p, X, bf16=False):
    """X: B x 35 (already standardised).  Returns the activations
    [H_1, H_2, H_3, Y] (tanh hidden layers, linear output)."""
    layers = unpack(p)
    H, out = np.asarray(X, dtype=np.float64), []
    for l, (W, c) in enumerate(layers):
        A = _mm(H, W.T, bf16) + c
        H = A if l == len(layers) - 1 else np.tanh(A)
        out.append(H)
    return out


def nll(Y, T):
    mu, s = Y[:, :4], Y[:, 4:]
    return float(np.mean(np.sum(0.5 * np.exp(-2.0 * s) * (T - mu) ** 2 + s, axis=1)))


def mlp_grad(p, X, T, bf16=False):
    """Gradient of nll(mlp_forward(p, X)[-1], T) with respect to p (backprop):
    D_L = dloss/dY, D_l = (D_{l+1} W_{l+1}) (1 - H_l^2), dW_l = D_l^T H_{l-1},
    db_l = sum over the batch of D_l."""
    layers = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    acts = mlp_forward(p, X, bf16)
    B = X.shape[0]
    Y = acts[-1]
    mu, s = Y[:, :4], Y[:, 4:]
    e = np.exp(-2.0 * s)
    D = np.concatenate([-e * (T - mu), 1.0 - e * (T - mu) ** 2], axis=1) / B
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        Hin = X if l == 0 else acts[l - 1]
        grads[l] = (_mm(D.T, Hin, bf16), D.sum(0))
        if l > 0:
            D = _mm(D, layers[l][0], bf16) * (1.0 - acts[l - 1] ** 2)
    return np.concatenate([a.ravel() for gw, gb in grads for a in (gw, gb)])


def adam_step(p, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t = 1, 2, ...).  Returns (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
