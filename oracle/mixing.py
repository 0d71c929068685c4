"""Learned damping and mixing for IPT: the CPU statement (float64 numpy).

TEST INFRASTRUCTURE ONLY (like ipt_oracle): only tests/, __graft_entry__.smoke()
and bench.py's CPU legs use it; it shares no code with the CUDA library.

The paper (Section 5) points to acceleration of the fixed-point iteration.  This
generalises the learned damping (oracle/damping.py) and depth-one Anderson
mixing (oracle/anderson.py): a small MLP proposes, per column c and step t, a
damping alpha_c and a mixing weight gamma_c for the update
    z_{t+1} = z_t + alpha f_t - gamma ((z_t - z_{t-1}) + alpha (f_t - f_{t-1}))
with f = F(z) - z the fixed-point residual of Eq. (dyn).  gamma = 0 is the
damped Picard step z + alpha f; alpha = 1 is Anderson mixing of depth one with
weight gamma, g_t - gamma (g_t - g_{t-1}), g = F(z).

Model (weights rounded to FP16, arithmetic in float64 here):
    h1 = tanh(x W1 + b1)      x: 7 features, W1: 7 x 64
    h2 = tanh(h1 W2 + b2)     W2: 64 x 64
    y  = h2 W3 + b3           W3: 64 x 2
    alpha = 2 / (1 + exp(-y0)),   gamma = 2 tanh(y1)
Features: the six of the damping model (increment-norm and eigenvalue history,
oracle/damping.features) and
    x6 = clip(gamma_ls, -4, 4),  gamma_ls = <f_t - f_{t-1}, f_t> / ||f_t - f_{t-1}||^2
(the least-squares Anderson weight; 0 where the difference vanishes).
The first three steps (no history yet) are Picard steps (alpha = 1, gamma = 0),
and so is every step after the fallback trips (a residual above ten times the
smallest residual seen).

Training targets (supervision from two extra evaluations per step): with
dz = z_t - z_{t-1}, df = f_t - f_{t-1} and a candidate weight gamma, the mixed
point y = z_t - gamma dz has the linearised residual r = f_t - gamma df, and the
step y + alpha r has the residual r + alpha J r, J r ~ f(y + r) - r.  The two
candidates are gamma = gamma_ls (Anderson) and gamma = 0 (Picard: y + r = F(z_t),
J r ~ F(F(z_t)) - 2 F(z_t) + z_t, the damping model's D2); per column the target
gamma* is the candidate whose point y + r has the smaller residual norm, and
    alpha* = -<r, J r> / ||J r||^2     (clipped to [0.05, 2]; 1 where J r = 0).
"""

from __future__ import annotations

import numpy as np

from .ipt_oracle import (OK, MAXITER, DIVERGED, DEGENERATE_THETA, INVALID_ARG, partition,
                         unit_columns, inverse_gaps, ipt_map, initial_residual_norm,
                         _check_theta)
from .damping import features as damping_features
from .anderson import anderson_gamma

N_IN, N_HID, N_OUT = 7, 64, 2
SHAPES = [("W1", (N_IN, N_HID)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_HID, N_OUT)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)
GAMMA_CLIP = 1.9


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
    """(alpha, gamma) and the cached activations for a batch X (B x 7)."""
    p = unpack(np.asarray(flat16, dtype=np.float16).astype(np.float64))
    X = np.asarray(X, dtype=np.float64)
    h1 = np.tanh(X @ p["W1"] + p["b1"])
    h2 = np.tanh(h1 @ p["W2"] + p["b2"])
    y = h2 @ p["W3"] + p["b3"]
    alpha = 2.0 / (1.0 + np.exp(-y[:, 0]))
    gamma = 2.0 * np.tanh(y[:, 1])
    return alpha, gamma, (X, h1, h2, y)


def loss_and_grad(flat16, X, target):
    """Mean over the batch of (alpha - t_alpha)^2 + (gamma - t_gamma)^2 (target: B x 2)
    and its gradient (flat, float64)."""
    p = unpack(np.asarray(flat16, dtype=np.float16).astype(np.float64))
    alpha, gamma, (X, h1, h2, y) = forward(flat16, X)
    B = X.shape[0]
    target = np.asarray(target, dtype=np.float64)
    ra, rg = alpha - target[:, 0], gamma - target[:, 1]
    loss = float(np.mean(ra * ra + rg * rg))
    s = 1.0 / (1.0 + np.exp(-y[:, 0]))
    t = np.tanh(y[:, 1])
    dy = np.stack([(2.0 / B) * ra * 2.0 * s * (1.0 - s),
                   (2.0 / B) * rg * 2.0 * (1.0 - t * t)], axis=1)   # d loss / d y
    g = {"W3": h2.T @ dy, "b3": dy.sum(axis=0)}
    dh2 = dy @ p["W3"].T
    da2 = dh2 * (1.0 - h2 * h2)
    g["W2"] = h1.T @ da2
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ p["W2"].T
    da1 = dh1 * (1.0 - h1 * h1)
    g["W1"] = X.T @ da1
    g["b1"] = da1.sum(axis=0)
    return loss, pack(g)


def features(inc_hist, lam_hist, gamma_ls):
    """Feature rows (k x 7): the damping model's six and clip(gamma_ls, -4, 4)."""
    x = damping_features(inc_hist, lam_hist)
    return np.concatenate([x, np.clip(np.asarray(gamma_ls, dtype=np.float64), -4.0, 4.0)
                           [:, None]], axis=1)


def mixed_update(z, f, z_prev, f_prev, alpha, gamma):
    """z + alpha f - gamma ((z - z_prev) + alpha (f - f_prev)), column by column."""
    a, g = np.asarray(alpha)[None, :], np.asarray(gamma)[None, :]
    return z + a * f - g * ((z - z_prev) + a * (f - f_prev))


def secant_alpha(r, Jr, lo=0.05, hi=2.0):
    """alpha* = -<r, J r> / ||J r||^2 per column, clipped (1 where J r = 0)."""
    num = -np.sum(r * Jr, axis=0)
    den = np.sum(Jr * Jr, axis=0)
    a = np.where(den > 0, num / np.where(den > 0, den, 1.0), 1.0)
    return np.clip(a, lo, hi)


def targets(z, f, z_prev, f_prev, f_at):
    """Training targets (alpha*, gamma*) per column (see the module docstring).

    f_at(x) returns the residual F(x) - x of the map at x (the two extra
    evaluations: at the Anderson point and at the Picard point)."""
    dz, df = z - z_prev, f - f_prev
    g_ls = np.clip(anderson_gamma(f, f_prev), -GAMMA_CLIP, GAMMA_CLIP)
    r_a = f - g_ls[None, :] * df
    y_a = z - g_ls[None, :] * dz
    fa = f_at(y_a + r_a)
    fp = f_at(z + f)
    use_a = np.linalg.norm(fa, axis=0) < np.linalg.norm(fp, axis=0)
    gamma = np.where(use_a, g_ls, 0.0)
    r = np.where(use_a[None, :], r_a, f)
    Jr = np.where(use_a[None, :], fa - r_a, fp - f)
    return secant_alpha(r, Jr), gamma


def mixed_solve(M, theta=None, cols=None, tol=1e-12, max_iter=1000, stop="residual",
                diverge_bound=1e8, model_fn=None, history=False):
    """Alg. 2 with the learned update in place of Z <- F(Z).

    ``model_fn(X)`` maps feature rows (k x 7) to (alpha, gamma) (k each); None =
    plain Picard.  The model applies from the fourth evaluation on (three
    histories needed), as long as the fallback has not tripped.  Statuses and
    the returned pair are those of ipt_solve (the tested Z, Lambda from its
    evaluation)."""
    Delta, theta = partition(M, theta)
    n = len(theta)
    cols = np.arange(n) if cols is None else np.asarray(cols, dtype=np.int64)
    k = len(cols)
    out = {"status": INVALID_ARG, "iterations": 0, "Z": None, "lam": None,
           "increment": np.nan, "rho": np.nan, "inc_hist": [], "rho_hist": [], "alpha": [],
           "gamma": []}
    if k == 0 or len(set(cols.tolist())) != k or cols.min() < 0 or cols.max() >= n:
        return out
    if not _check_theta(theta, cols):
        out["status"] = DEGENERATE_THETA
        return out
    G = inverse_gaps(theta, cols)
    r0 = initial_residual_norm(Delta, cols)
    Z = unit_columns(n, cols)
    Z_prev = f_prev = None
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
        f = F - Z
        incs.append(np.linalg.norm(f, axis=0) / np.linalg.norm(Z, axis=0))
        lams.append(lam)
        alpha, gamma = np.ones(k), np.zeros(k)
        if model_fn is not None and len(incs) >= 3 and not fallback:
            g_ls = anderson_gamma(f, f_prev)
            a, g = model_fn(features(incs[-3:], lams[-3:], g_ls))
            alpha, gamma = np.asarray(a, dtype=np.float64), np.asarray(g, dtype=np.float64)
        if history:
            out["alpha"].append(alpha)
            out["gamma"].append(gamma)
        Z_next = Z + alpha[None, :] * f if f_prev is None else \
            mixed_update(Z, f, Z_prev, f_prev, alpha, gamma)
        Z_prev, f_prev = Z, f
        Z = Z_next
    return out
