"""Training data for the learned filter degree (chfsi_mlp_*, chfsi_set_degree_model).

The closed-form degree rule assumes that a degree-d Chebyshev filter reduces the residual of
a Ritz vector by rho^d, ln rho = acosh|t| with t = (theta - c)/e its position relative to
the filter interval.  Every record of the solver's degree log (chfsi_degree_log_*) holds a
vector's residual r before a loop, the degree d it was filtered with and the residual r_next
it had after the loop, so it gives an observed per-degree log rate
y = ln(r / r_next) / d; the model learns z = ln(y / ln rho), the log of the factor by which
the observed rate differs from the closed form, from the inputs the solver computed for that
vector (logged with the record, in the order of include/chfsi.h).
"""
from __future__ import annotations

import numpy as np

FIELDS = ("problem", "loop", "g", "i", "m", "theta", "r", "tau", "d", "c", "e", "r_next",
          "x0", "x1", "x2", "x3", "x4", "x5", "x6", "x7")
N_INPUTS = 8


def training_pairs(log: np.ndarray, zclip: float = 3.0):
    """(X [n, 8] float32, z [n] float32) from degree-log records [count, 20]: one pair per
    record of a vector outside the damped interval (|t| > 1) that was not yet below the
    locking threshold, was filtered (d >= 1) and whose residual fell."""
    log = np.asarray(log, dtype=np.float64)
    if log.size == 0:
        return np.zeros((0, N_INPUTS), np.float32), np.zeros(0, np.float32)
    log = log.reshape(-1, len(FIELDS))
    th, r, tau, d, c, e, r2 = (log[:, FIELDS.index(k)] for k in ("theta", "r", "tau", "d", "c", "e", "r_next"))
    X = log[:, FIELDS.index("x0"):]
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.abs((th - c) / e)
        lrho = np.log(t + np.sqrt(np.maximum(t * t - 1.0, 0.0)))
        y = np.log(r / r2) / d
        ok = (e > 0) & (t > 1.0) & (r > tau) & (r2 > 0.0) & (d >= 1) & (y > 0.0) & (lrho > 0.0)
        ok &= np.all(np.isfinite(X), axis=1)
        z = np.clip(np.log(y[ok] / lrho[ok]), -zclip, zclip)
    return np.asarray(X[ok], np.float32).reshape(-1, N_INPUTS), np.asarray(z, np.float32)
