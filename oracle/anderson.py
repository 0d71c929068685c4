"""Anderson mixing for IPT: the CPU statement (float64 numpy).

TEST INFRASTRUCTURE ONLY (like ipt_oracle): only tests/, __graft_entry__.smoke()
and bench.py's CPU legs use it; it shares no code with the CUDA library.

The paper (Section 5) points to acceleration of the fixed-point iteration; this
is Anderson mixing of depth one (Anderson 1965; in the form of Walker and Ni,
SIAM J. Numer. Anal. 49, 2011) applied to each column c of Alg. 2 on its own.
With g = F (Eq. dyn) and the column's fixed-point residual f_t = g(z_t) - z_t:

    gamma_t = <f_t - f_{t-1}, f_t> / ||f_t - f_{t-1}||^2      (0 if the norm is 0)
    z_{t+1} = g(z_t) - gamma_t (g(z_t) - g(z_{t-1}))

i.e. the combination of the last two map values whose linearised residual
(1 - gamma) f_t + gamma f_{t-1} is smallest.  The first step is a Picard step
(z_1 = g(z_0)).  Both map values are 1 at the unit entry i_c, so every iterate
keeps z_{i_c, c} = 1.  Safeguard: once a residual exceeds ten times the
smallest residual seen, every later step is a Picard step (gamma = 0).  The
stopping test, statuses and returned pair are those of ipt_solve: the tested Z
is returned, with Lambda from its evaluation.
"""

from __future__ import annotations

import numpy as np

from .ipt_oracle import (OK, MAXITER, DIVERGED, DEGENERATE_THETA, INVALID_ARG, partition,
                         unit_columns, inverse_gaps, ipt_map, initial_residual_norm,
                         _check_theta)


def anderson_gamma(f, f_prev):
    """Per-column mixing weight gamma = <f - f_prev, f> / ||f - f_prev||^2 (0 where
    the difference vanishes)."""
    df = f - f_prev
    num = np.sum(df * f, axis=0)
    den = np.sum(df * df, axis=0)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)


def anderson_update(g, g_prev, gamma):
    """The mixed iterate g - gamma (g - g_prev), column by column."""
    return g - gamma[None, :] * (g - g_prev)


def ipt_solve_anderson(M, theta=None, cols=None, tol=1e-12, max_iter=1000, stop="residual",
                       diverge_bound=1e8, history=False):
    """Alg. 2 with the depth-one Anderson update in place of Z <- F(Z)."""
    Delta, theta = partition(M, theta)
    n = len(theta)
    cols = np.arange(n) if cols is None else np.asarray(cols, dtype=np.int64)
    k = len(cols)
    out = {"status": INVALID_ARG, "iterations": 0, "Z": None, "lam": None,
           "increment": np.nan, "rho": np.nan, "inc_hist": [], "rho_hist": [], "gamma": []}
    if k == 0 or len(set(cols.tolist())) != k or cols.min() < 0 or cols.max() >= n:
        return out
    if not _check_theta(theta, cols):
        out["status"] = DEGENERATE_THETA
        return out
    G = inverse_gaps(theta, cols)
    r0 = initial_residual_norm(Delta, cols)
    Z = unit_columns(n, cols)
    Z_prev = g_prev = None
    best, fallback = np.inf, False
    for it in range(max_iter):
        F, P, d = ipt_map(Delta, theta, cols, Z, G=G)
        znorm = np.linalg.norm(Z)
        inc = np.linalg.norm(F - Z) / znorm
        lam = theta[cols] + d
        R = theta[:, None] * Z + P - Z * lam[None, :]
        rho = np.linalg.norm(R) / r0 if r0 > 0 else 0.0
        out.update(Z=Z, lam=lam, iterations=it + 1, increment=inc, rho=rho)
        if history:
            out["inc_hist"].append(inc)
            out["rho_hist"].append(rho)
        if not (np.isfinite(inc) and np.isfinite(rho)) or znorm > diverge_bound * np.sqrt(k):
            out["status"] = DIVERGED
            return out
        if (inc if stop == "increment" else rho) <= tol:
            out["status"] = OK
            return out
        if it + 1 == max_iter:
            out["status"] = MAXITER
            return out
        if it == 0 or rho < best:
            best = rho
        if it > 0 and rho > 10.0 * best:
            fallback = True
        if g_prev is None or fallback:
            gamma = np.zeros(k)
        else:
            gamma = anderson_gamma(F - Z, g_prev - Z_prev)
        if history:
            out["gamma"].append(gamma)
        Z_next = anderson_update(F, F if g_prev is None else g_prev, gamma)
        Z_prev, g_prev = Z, F
        Z = Z_next
    return out
