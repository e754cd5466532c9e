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
* ``mlp_forward`` / ``nll`` / ``mlp_grad`` / ``adam_step`` -- a 35-64-64-8
  perceptron with tanh hidden layers; outputs (mu_1..4, s_1..4) are the
  predicted transformed coordinates of Sec. 5 and log step scales, trained
  with the Gaussian negative log-likelihood
  sum_c [ exp(-2 s_c) (t_c - mu_c)^2 / 2 + s_c ] averaged over the batch,
  and Adam (beta1 0.9, beta2 0.999, eps 1e-8; Kingma & Ba 2015).

Parameter layout (flat, 6984 values): W1 (64 x 35, row-major), b1 (64),
W2 (64 x 64), b2 (64), W3 (8 x 64), b3 (8).
"""
from __future__ import annotations

import math

import numpy as np

NF, NH, NO = 35, 64, 8
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
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + NH * NF].reshape(NH, NF); o += NH * NF
    b1 = p[o:o + NH]; o += NH
    W2 = p[o:o + NH * NH].reshape(NH, NH); o += NH * NH
    b2 = p[o:o + NH]; o += NH
    W3 = p[o:o + NO * NH].reshape(NO, NH); o += NO * NH
    b3 = p[o:o + NO]; o += NO
    assert o == p.size
    return W1, b1, W2, b2, W3, b3


NPARAMS = NH * NF + NH + NH * NH + NH + NO * NH + NO


def mlp_forward(p, X):
    """X: B x 35 (already standardised).  Returns (H1, H2, Y)."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    H1 = np.tanh(X @ W1.T + b1)
    H2 = np.tanh(H1 @ W2.T + b2)
    Y = H2 @ W3.T + b3
    return H1, H2, Y


def nll(Y, T):
    mu, s = Y[:, :4], Y[:, 4:]
    return float(np.mean(np.sum(0.5 * np.exp(-2.0 * s) * (T - mu) ** 2 + s, axis=1)))


def mlp_grad(p, X, T):
    """Gradient of nll(mlp_forward(p, X)[2], T) with respect to p (backprop)."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    H1, H2, Y = mlp_forward(p, X)
    B = X.shape[0]
    mu, s = Y[:, :4], Y[:, 4:]
    e = np.exp(-2.0 * s)
    D3 = np.concatenate([-e * (T - mu), 1.0 - e * (T - mu) ** 2], axis=1) / B
    D2 = (D3 @ W3) * (1.0 - H2 * H2)
    D1 = (D2 @ W2) * (1.0 - H1 * H1)
    g = [D1.T @ X, D1.sum(0), D2.T @ H1, D2.sum(0), D3.T @ H2, D3.sum(0)]
    return np.concatenate([a.ravel() for a in g])


def adam_step(p, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t = 1, 2, ...).  Returns (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
