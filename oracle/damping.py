"""Learned damping for IPT: the CPU statement (float64 numpy).

TEST INFRASTRUCTURE ONLY (like ipt_oracle): only tests/, __graft_entry__.smoke()
and bench.py's CPU legs use it; it shares no code with the CUDA library.

The paper (Section 5) points to fixed-point acceleration for IPT; this is a
learned variant of the simplest one, a damped Picard step
    Z <- Z + alpha_c (F(Z) - Z)          (one alpha per column c)
with alpha_c = 2 sigmoid(y_c) in (0, 2) predicted by a small MLP from the
history of the column's increment norms and Rayleigh-quotient changes.

Model (weights rounded to FP16, arithmetic in float64 here):
    h1 = tanh(x W1 + b1)      x: 6 features, W1: 6 x 64
    h2 = tanh(h1 W2 + b2)     W2: 64 x 64
    y  = h2 W3 + b3           W3: 64 x 1
    alpha = 2 / (1 + exp(-y))

Features of column c at evaluation t (eps = 1e-30 guards logarithms):
    inc_t  = ||F(Z_t)_c - Z_t,c|| / ||Z_t,c||,   lam_t = theta_{i_c} + d_c(Z_t)
    x0 = log10(inc_t + eps)
    x1 = log10((inc_t + eps) / (inc_{t-1} + eps))
    x2 = log10((inc_{t-1} + eps) / (inc_{t-2} + eps))
    x3 = clip(q_t, -4, 4),   q_t = (lam_t - lam_{t-1}) / (lam_{t-1} - lam_{t-2})
         (0 when the denominator is 0)
    x4 = log10(|lam_{t-1} - lam_{t-2}| / (|lam_{t-1}| + eps) + eps)
    x5 = log10(|lam_t - lam_{t-1}| / (|lam_t| + eps) + eps)
Damping starts at the fourth evaluation (three histories needed); earlier
steps are plain Picard steps (alpha = 1), and so is every step after the
fallback trips (a residual above ten times the smallest residual seen).

Training target (supervision from two evaluations): with D1 = F(z) - z and
D2 = F(F(z)) - 2 F(z) + z, a linear model of F near its fixed point gives the
next residual of the damped step as D1 + alpha D2, smallest at
    alpha* = -<D1, D2> / ||D2||^2     (per column; clipped to [0.05, 2]).
"""

from __future__ import annotations

import numpy as np

from .ipt_oracle import (OK, MAXITER, DIVERGED, DEGENERATE_THETA, INVALID_ARG, partition,
                         unit_columns, inverse_gaps, ipt_map, initial_residual_norm,
                         _check_theta)

N_IN, N_HID = 6, 64
EPS = 1e-30
SHAPES = [("W1", (N_IN, N_HID)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_HID, 1)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(flat):
    """Flat parameter vector (order W1, b1, W2, b2, W3, b3; row-major) -> dict."""
    flat = np.asarray(flat, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = flat[o:o + size].reshape(shape)
        o += size
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1)
                           for name, _ in SHAPES])


def init_params(seed):
    """Seeded initial weights (uniform +-1/sqrt(fan_in)), rounded to FP16."""
    g = np.random.default_rng(seed)
    p = {}
    for name, shape in SHAPES:
        fan_in = shape[0] if name.startswith("W") else (N_IN if name == "b1" else N_HID)
        p[name] = g.uniform(-1.0, 1.0, size=shape) / np.sqrt(fan_in)
    return np.asarray(pack(p), dtype=np.float16)


def forward(flat16, X):
    """alpha and the cached activations for a batch X (B x 6)."""
    p = unpack(np.asarray(flat16, dtype=np.float16).astype(np.float64))
    X = np.asarray(X, dtype=np.float64)
    h1 = np.tanh(X @ p["W1"] + p["b1"])
    h2 = np.tanh(h1 @ p["W2"] + p["b2"])
    y = (h2 @ p["W3"] + p["b3"])[:, 0]
    alpha = 2.0 / (1.0 + np.exp(-y))
    return alpha, (X, h1, h2, y)


def loss_and_grad(flat16, X, target):
    """Mean squared error of alpha against target and its gradient (flat, float64)."""
    p = unpack(np.asarray(flat16, dtype=np.float16).astype(np.float64))
    alpha, (X, h1, h2, y) = forward(flat16, X)
    B = X.shape[0]
    r = alpha - np.asarray(target, dtype=np.float64)
    loss = float(np.mean(r * r))
    s = 1.0 / (1.0 + np.exp(-y))
    dy = (2.0 / B) * r * 2.0 * s * (1.0 - s)          # d loss / d y
    g = {"W3": h2.T @ dy[:, None], "b3": np.array([dy.sum()])}
    dh2 = dy[:, None] @ p["W3"].T
    da2 = dh2 * (1.0 - h2 * h2)
    g["W2"] = h1.T @ da2
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ p["W2"].T
    da1 = dh1 * (1.0 - h1 * h1)
    g["W1"] = X.T @ da1
    g["b1"] = da1.sum(axis=0)
    return loss, pack(g)


def features(inc_hist, lam_hist):
    """Feature rows (k x 6) from the last three increments and eigenvalues per column.

    inc_hist, lam_hist: arrays (3, k) ordered oldest .. newest (t-2, t-1, t)."""
    i2, i1, i0 = (np.asarray(inc_hist[j], dtype=np.float64) for j in range(3))
    l2, l1, l0 = (np.asarray(lam_hist[j], dtype=np.float64) for j in range(3))
    x0 = np.log10(i0 + EPS)
    x1 = np.log10((i0 + EPS) / (i1 + EPS))
    x2 = np.log10((i1 + EPS) / (i2 + EPS))
    num, den = l0 - l1, l1 - l2
    q = np.where(den != 0.0, num / np.where(den != 0.0, den, 1.0), 0.0)
    x3 = np.clip(q, -4.0, 4.0)
    x4 = np.log10(np.abs(den) / (np.abs(l1) + EPS) + EPS)
    x5 = np.log10(np.abs(num) / (np.abs(l0) + EPS) + EPS)
    return np.stack([x0, x1, x2, x3, x4, x5], axis=1)


def secant_alpha(D1, D2, lo=0.05, hi=2.0):
    """alpha* = -<D1, D2> / ||D2||^2 per column, clipped (1 where D2 = 0)."""
    num = -np.sum(D1 * D2, axis=0)
    den = np.sum(D2 * D2, axis=0)
    a = np.where(den > 0, num / np.where(den > 0, den, 1.0), 1.0)
    return np.clip(a, lo, hi)


def damped_solve(M, theta=None, cols=None, tol=1e-12, max_iter=1000, stop="residual",
                 diverge_bound=1e8, alpha_fn=None, history=False):
    """Alg. 2 with the damped update Z <- Z + alpha (F(Z) - Z) (alpha per column).

    ``alpha_fn(X)`` maps feature rows (k x 6) to k dampings; None = plain Picard
    (alpha = 1 always).  Damping applies from the fourth evaluation on.  The
    stopping test, statuses and returned pair are those of ipt_solve (the tested
    Z is returned, with Lambda from its evaluation)."""
    Delta, theta = partition(M, theta)
    n = len(theta)
    cols = np.arange(n) if cols is None else np.asarray(cols, dtype=np.int64)
    k = len(cols)
    out = {"status": INVALID_ARG, "iterations": 0, "Z": None, "lam": None,
           "increment": np.nan, "rho": np.nan, "inc_hist": [], "rho_hist": [], "alpha": []}
    if k == 0 or len(set(cols.tolist())) != k or cols.min() < 0 or cols.max() >= n:
        return out
    if not _check_theta(theta, cols):
        out["status"] = DEGENERATE_THETA
        return out
    G = inverse_gaps(theta, cols)
    r0 = initial_residual_norm(Delta, cols)
    Z = unit_columns(n, cols)
    incs, lams = [], []
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
        if len(incs) == 0 or rho < best:
            best = rho
        if len(incs) >= 3 and rho > 10.0 * best:
            fallback = True
        col_inc = np.linalg.norm(F - Z, axis=0) / np.linalg.norm(Z, axis=0)
        incs.append(col_inc)
        lams.append(lam)
        alpha = np.ones(k)
        if alpha_fn is not None and len(incs) >= 3 and not fallback:
            alpha = np.asarray(alpha_fn(features(incs[-3:], lams[-3:])), dtype=np.float64)
        if history:
            out["alpha"].append(alpha)
        Z = Z + alpha[None, :] * (F - Z)
    return out
