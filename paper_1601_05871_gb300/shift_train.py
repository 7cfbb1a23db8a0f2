"""Training driver of the shift predictor: shift sweeps, labels, training, and the
learned-shift solve.  Every computation runs in libick.so's kernels (numeric
factorization, PCG, matrix features, the MLP's forward, gradient and Adam kernels);
this module only orders the calls.

A sweep factors one matrix with a grid of shifts alpha (B + alpha * diag(B)),
records which attempts break down and, for the others, how many PCG iterations
reach the tolerance.  The label is the largest shift whose iteration count is within
max(1, 2%) of the sweep's best: the cheapest preconditioner, with a margin above the
breakdown threshold.  The network learns log10 of that shift from the 8 matrix
features; at solve time its prediction is the first attempt of the shift-doubling
retry, which stays the fallback and has the last word (ic_numeric_shifted).
"""
from __future__ import annotations

import time

import numpy as np

from . import ick

ALPHA_FLOOR = 1e-4  # labels and predictions below this are taken as "no shift needed"


def sweep(h, values, b, x, alphas, tol=1e-8, maxit=5000, stop_ratio=1.5, stream=None):
    """Factor with each shift in ascending `alphas` and solve; returns a list of
    (alpha, iterations or None on breakdown).  Stops once the iteration count exceeds
    stop_ratio times the best seen (iterations grow with the shift past the optimum)."""
    out = []
    best = None
    for a in alphas:
        try:
            ick.ic_numeric_shifted(h, values, float(a), 1e-3, 1, stream)
        except ick.IckError as e:
            if e.status != ick.IC_ERR_BREAKDOWN:
                raise
            out.append((float(a), None))
            continue
        it, _ = ick.pcg_solve(h, values, b, x, tol, maxit, stream)
        out.append((float(a), int(it)))
        best = it if best is None else min(best, it)
        if it > stop_ratio * best:
            break
    return out


def label(sweep_result, slack=0.02):
    """log10 of the largest non-breaking shift within max(1, slack * best) iterations
    of the best; None when every attempt broke down."""
    ok = [(a, it) for a, it in sweep_result if it is not None]
    if not ok:
        return None
    best = min(it for _, it in ok)
    tol = max(1, int(np.ceil(slack * best)))
    a = max(a for a, it in ok if it <= best + tol)
    return float(np.log10(max(a, ALPHA_FLOOR)))


def train(X, y, steps=800, lr=1e-2, seed=0, hidden_init=None):
    """Trains a fresh network on features X (n x 8) and labels y (log10 alpha) with
    full-batch Adam on the GPU; returns (Mlp, final loss)."""
    import torch

    import synth

    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    mean = X.mean(axis=0)
    std = X.std(axis=0)
    std = np.where(std > 1e-12, std, 1.0)
    params = synth.mlp_init(32, seed) if hidden_init is None else hidden_init
    m = ick.Mlp(params.astype(np.float32))
    ick.ic_mlp_set_scaling(m, mean, std)
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    yd = torch.tensor(y, dtype=torch.float32, device="cuda")
    loss = None
    for s in range(steps):
        loss = ick.ic_mlp_train_step(m, Xd, yd, lr, want_loss=(s == steps - 1))
    return m, loss


def solve(h, values, b, x, *, mlp=None, nu=0.0, alpha0=1e-3, max_tries=20, tol=1e-8, maxit=5000, stream=None):
    """Factor (shift-doubling retry, first shift from the network when given, else 0)
    and solve with PCG.  Returns a dict: alpha, attempts, iterations, relres,
    seconds (wall time of the whole solve, synchronised)."""
    import torch

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    first = 0.0
    if mlp is not None:
        f = ick.ic_shift_features(h, values, nu, stream)
        first = ick.ic_mlp_predict_shift(mlp, f, stream)
        if first < ALPHA_FLOOR:
            first = 0.0
    a, tries = ick.ic_numeric_shifted(h, values, first, alpha0, max_tries, stream)
    it, rel = ick.pcg_solve(h, values, b, x, tol, maxit, stream)
    torch.cuda.synchronize()
    return {"alpha": a, "first": first, "attempts": tries, "iterations": int(it), "relres": float(rel),
            "seconds": time.perf_counter() - t0}
