"""Learned diagonal shift -- CPU oracle.  TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of bench.py may
import this module; it shares no code with the CUDA library.

Incomplete Cholesky of a matrix that is not an M-matrix can break down: a pivot
becomes zero or negative once fill is dropped.  Factoring B + alpha*diag(B)
instead makes the matrix more diagonally dominant and, for a large enough alpha,
restores positive pivots, at the price of a weaker preconditioner (more Krylov
iterations).  The plain remedy tries alpha = 0, then alpha0 and doubles alpha until
no breakdown occurs; a small network that predicts a good alpha from features of
the matrix saves the failed attempts.  This module states, in plain FP64 numpy:

  * ``features``: the 8 matrix features the predictor reads (definitions below);
  * the predictor: a 2-hidden-layer ReLU MLP on standardised features, its loss
    (half the mean squared error of log10 alpha), its analytic gradient and the
    Adam update;
  * ``retry_sequence``: the shift-doubling retry rule.

Every function is written from its definition; the tests pin them independently
(hand-derived features of small matrices, closed forms of the 5-point Laplacian,
central finite differences of the loss, the zero-weight network).
"""
from __future__ import annotations

import numpy as np

NFEAT = 8
FEATURE_NAMES = ("dd_min", "dd_mean", "rownorm_mean", "rownorm_max", "pos_offdiag_frac", "k", "log10_n", "nu")
DD_CAP = 1000.0  # diagonal dominance of a row without off-diagonal entries


def features(n, rowptr, colind, vals, k, nu=0.0):
    """Features of a symmetric matrix B with a positive diagonal (CSR, both triangles).

    For each row i, with d = B_ii, s = sum over j != i of |B_ij| and
    r = sqrt(sum over j of B_ij^2):
        dd_i = d / max(s, d / DD_CAP)    (diagonal dominance, at most DD_CAP)
        rn_i = r / d                      (row norm relative to the diagonal, >= 1)
    Features: min dd, mean dd, mean rn, max rn, the fraction of off-diagonal
    entries that are positive (0 when there are none), k, log10(n), nu (a material
    parameter supplied by the caller, 0 when none applies).
    """
    dd = np.empty(n)
    rn = np.empty(n)
    pos = 0
    off = 0
    for i in range(n):
        d = None
        s = 0.0
        sq = 0.0
        for e in range(rowptr[i], rowptr[i + 1]):
            j, v = int(colind[e]), float(vals[e])
            sq += v * v
            if j == i:
                d = v
            else:
                s += abs(v)
                off += 1
                pos += v > 0.0
        if d is None or not d > 0.0:
            raise ValueError(f"row {i}: diagonal missing or not positive")
        dd[i] = d / max(s, d / DD_CAP)
        rn[i] = np.sqrt(sq) / d
    return np.array([dd.min(), dd.mean(), rn.mean(), rn.max(), pos / off if off else 0.0, float(k),
                     np.log10(n), float(nu)])


# ---------------------------------------------------------------------- the MLP
# Flat parameter vector, in this order: W1 (NFEAT x H, row-major: W1[f, h]), b1 (H),
# W2 (H x H, row-major: W2[g, h], input g to unit h), b2 (H), w3 (H), b3 (1).


def n_params(hidden):
    return NFEAT * hidden + hidden + hidden * hidden + hidden + hidden + 1


def unpack(theta, hidden):
    H = hidden
    o = 0
    W1 = theta[o:o + NFEAT * H].reshape(NFEAT, H); o += NFEAT * H
    b1 = theta[o:o + H]; o += H
    W2 = theta[o:o + H * H].reshape(H, H); o += H * H
    b2 = theta[o:o + H]; o += H
    w3 = theta[o:o + H]; o += H
    b3 = theta[o]
    return W1, b1, W2, b2, w3, b3


def forward(theta, hidden, mean, std, X):
    """Predicted log10 alpha for each row of X (features), and the activations."""
    W1, b1, W2, b2, w3, b3 = unpack(np.asarray(theta, dtype=np.float64), hidden)
    Z = (np.asarray(X, dtype=np.float64) - mean) / std
    a1 = Z @ W1 + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2 + b2
    h2 = np.maximum(a2, 0.0)
    y = h2 @ w3 + b3
    return y, (Z, a1, h1, a2, h2)


def loss_and_grad(theta, hidden, mean, std, X, t):
    """L = (1 / 2N) sum (y_i - t_i)^2 and dL/dtheta by the chain rule, layer by layer."""
    theta = np.asarray(theta, dtype=np.float64)
    W1, b1, W2, b2, w3, b3 = unpack(theta, hidden)
    y, (Z, a1, h1, a2, h2) = forward(theta, hidden, mean, std, X)
    N = len(y)
    r = (y - np.asarray(t, dtype=np.float64)) / N      # dL/dy
    g_w3 = h2.T @ r
    g_b3 = r.sum()
    d2 = np.outer(r, w3) * (a2 > 0.0)                  # dL/da2
    g_W2 = h1.T @ d2
    g_b2 = d2.sum(axis=0)
    d1 = (d2 @ W2.T) * (a1 > 0.0)                      # dL/da1
    g_W1 = Z.T @ d1
    g_b1 = d1.sum(axis=0)
    L = 0.5 * float(np.sum((y - t) ** 2)) / N
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return L, g


def adam_step(theta, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


# ----------------------------------------------------------- the retry rule


def retry_sequence(alpha_first, alpha0=1e-3, max_tries=20):
    """Shifts tried in order: alpha_first, then twice the previous shift, where a
    zero shift is followed by alpha0; at most max_tries attempts."""
    seq = [float(alpha_first)]
    while len(seq) < max_tries:
        seq.append(2.0 * seq[-1] if seq[-1] > 0.0 else float(alpha0))
    return seq


def first_success(breaks, alpha_first, alpha0=1e-3, max_tries=20):
    """Runs the retry rule against breaks(alpha) -> bool (True on breakdown).
    Returns (alpha used, attempts), or (None, max_tries) when every attempt breaks."""
    for t, a in enumerate(retry_sequence(alpha_first, alpha0, max_tries)):
        if not breaks(a):
            return a, t + 1
    return None, max_tries
