"""Training data for the learned filter degree (chfsi_mlp_*, chfsi_set_degree_model).

The closed-form degree rule assumes that a degree-d Chebyshev filter reduces the residual of
a Ritz vector by rho^d, ln rho = acosh|t| with t = (theta - c)/e its position relative to
the filter interval.  From the solver's degree log (chfsi_degree_log_*), every column that
is still active in the next loop gives an observed per-degree log rate
y = ln(r_k / r_{k+1}) / d_k; the model learns z = ln(y / ln rho_k), the log of the factor by
which the observed rate differs from the closed form, from the features the solver
evaluates on the device: [ln rho, log10(r/tau), i/m, log10(max(gap/e, 1e-12))].
"""
from __future__ import annotations

import numpy as np

FIELDS = ("problem", "loop", "g", "i", "m", "theta", "r", "tau", "d", "c", "e", "gap")


def training_pairs(log: np.ndarray, zclip: float = 3.0):
    """(X [n, 4] float32, z [n] float32) from degree-log records [count, 12]."""
    log = np.asarray(log, dtype=np.float64)
    X, z = [], []
    if log.size == 0:
        return np.zeros((0, 4), np.float32), np.zeros(0, np.float32)
    nxt = {(int(p), int(k), int(g)): row for p, k, g, row in zip(log[:, 0], log[:, 1], log[:, 2], log)}
    for row in log:
        p, k, g, i, m, th, r, tau, d, c, e, gap = row
        after = nxt.get((int(p), int(k) + 1, int(g)))
        if after is None or not (e > 0):
            continue
        r2 = after[6]
        t = abs((th - c) / e)
        if t <= 1.0 or r <= tau or not (r2 > 0.0) or d < 1:
            continue
        lrho = float(np.log(t + np.sqrt(t * t - 1.0)))
        y = float(np.log(r / r2)) / d
        if not (y > 0.0) or not (lrho > 0.0):
            continue
        X.append([lrho, np.log10(r / tau), i / m, np.log10(max(gap / e, 1e-12))])
        z.append(float(np.clip(np.log(y / lrho), -zclip, zclip)))
    return np.asarray(X, np.float32).reshape(-1, 4), np.asarray(z, np.float32)
