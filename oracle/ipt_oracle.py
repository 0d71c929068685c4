"""IPT oracle: a plain, slow, float64 CPU statement of the method.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this module: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` use it.  It shares no code,
constants or helpers with the CUDA library; it is written from the paper
(Kenmoe, Kriemann, Smerlak, Zadorin, "A fast iterative algorithm for
near-diagonal eigenvalue problems"), step by step and in its notation:

* partition M = D + Delta, D = diag(theta)          -- Alg. 1/2 step 1, Section 3
* inverse gaps G_jk = 1/(theta_j - theta_k), G_jj=0 -- Eq. (single_line_dyn)
* map F(Z) = I + G o (Z D(Delta Z) - Delta Z)        -- Eq. (dyn); for a column
  subset this is f_i of Eq. (single_line_dyn) applied column by column
* Picard iteration from Z = I with the stopping test
  ||Z - F(Z)|| / ||Z|| <= eta, eigenvalues D(M Z)     -- Alg. 1 and Alg. 2
* Rayleigh-Schroedinger corrections Z^[l]           -- Eq. (ARS-alpha), App. B
* the chart Jacobian of f_i whose multipliers the 3x3 polynomials of
  App. D.3 annihilate                               -- App. D.1
* Alternating Cyclic Extrapolation in place of the Picard update
  (IPT-ACX)                                         -- Alg. 3, Section 5

Everything is float64 and dense numpy (the sparse variant multiplies with
scipy's CSR product).  Library primitives (``@``, ``numpy.linalg``) serve as
single steps only; nothing is blocked, fused or reordered.

Readings of the paper this oracle takes (the paper is silent or garbled):

1. G follows Eq. (single_line_dyn): row j, column k holds
   1/(theta_j - theta_k); Alg. 2's "i != n" subscript is read as "i != j".
2. The norm of the stopping test is the Frobenius norm.
3. The loop returns the Z whose F(Z) passed the test (not F(Z)), with
   Lambda = D(M Z) = theta_cols + D(Delta Z) (Z_{i_c, c} = 1).
4. The relative residual is rho = ||M Z - Z Lambda||_F / ||M Z0 - Z0 Lambda0||_F
   with Z0 the unit columns e_{i_c}; the denominator is the Frobenius norm of
   the off-diagonal part of the requested columns of M (rho = 0 when that
   norm is 0).
5. ``iterations`` counts evaluations of F (products with Delta).  On MAXITER
   and DIVERGED the returned pair is the last Z at which F was evaluated.
6. Divergence: a non-finite increment or residual, or ||Z||_F > bound*sqrt(k).
7. theta must be pairwise distinct over the requested columns and every row
   (Section 3 requires simple unperturbed eigenvalues), else DEGENERATE_THETA.
8. Alg. 3 (ACX) as printed is garbled in three places; read as: the step
   length is sigma = |<D^p, D^(p-1)>| / ||D^p||^2 (squared norm: the update
   must not change under z -> scale); the update keeps the D^0 = z term,
   z <- z + 2 sigma D^1 + sigma^2 D^2 (p = 2) and
   z <- z + 3 sigma D^1 + 3 sigma^2 D^2 + sigma^3 D^3 (p = 3); the order
   index advances once per extrapolation, p = 3, 2, 3, 2, ...  For k
   columns each column has its own sigma (each column is its own fixed-point
   problem f_i of Alg. 1) unless a single global sigma is asked for; a column
   with D^p = 0 takes sigma = 1 (the update is then the plain iterate f^p(z)).
   ``iterations`` counts evaluations of F; the stopping test is made at the
   extrapolated points z only (Alg. 3's loop condition), and the returned pair
   is the last such z with Lambda from its evaluation.
"""

from __future__ import annotations

import numpy as np

# Status codes of the oracle's own solver (values chosen to read alongside
# the library's, but defined here independently).
OK, MAXITER, DIVERGED, DEGENERATE_THETA, INVALID_ARG = 0, 1, 2, 3, 4


def partition(M: np.ndarray, theta: np.ndarray | None = None):
    """Alg. 1/2 step 1: M = D + Delta with D = diag(theta); theta = diag(M) by default."""
    M = np.asarray(M, dtype=np.float64)
    theta = np.diag(M).copy() if theta is None else np.asarray(theta, dtype=np.float64)
    Delta = M - np.diag(theta)
    return Delta, theta


def unit_columns(n: int, cols: np.ndarray) -> np.ndarray:
    """E with E[:, c] = e_{cols[c]}: the starting point Z = I of Alg. 2 (Alg. 1: z = e_i)."""
    E = np.zeros((n, len(cols)))
    E[cols, np.arange(len(cols))] = 1.0
    return E


def inverse_gaps(theta: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """Columns cols of G: G[j, c] = 1/(theta_j - theta_{cols[c]}), 0 where j = cols[c].

    Eq. (single_line_dyn): (g_i)_j = (theta_j - theta_i)^{-1}, (g_i)_i = 0.
    """
    n, k = len(theta), len(cols)
    with np.errstate(divide="ignore"):
        G = 1.0 / (theta[:, None] - theta[cols][None, :])
    G[cols, np.arange(k)] = 0.0
    return G


def ipt_map(Delta, theta, cols, Z, G=None, product=None):
    """One evaluation of the IPT map, Eq. (dyn) restricted to the columns cols.

    Returns (F, P, d) with P = Delta Z, d_c = P[cols[c], c] (the diagonal
    D(Delta Z) of Eq. (dyn)) and F = E + G o (Z D(Delta Z) - Delta Z).
    ``product`` overrides the product Delta @ Z (the sparse oracle passes
    scipy's CSR product).
    """
    n, k = Z.shape
    if G is None:
        G = inverse_gaps(theta, cols)
    P = Delta @ Z if product is None else product(Z)
    d = P[cols, np.arange(k)]
    F = unit_columns(n, cols) + G * (Z * d[None, :] - P)
    return F, P, d


def residual(M, Z, lam):
    """M Z - Z Lambda for eigenpair columns (Z[:, c], lam[c])."""
    return M @ Z - Z * lam[None, :]


def initial_residual_norm(Delta, cols):
    """||M Z0 - Z0 Lambda0||_F at Z0 = unit columns: the off-diagonal part of Delta[:, cols]."""
    k = len(cols)
    Dc = Delta[:, cols]
    Dc = Dc.toarray() if hasattr(Dc, "toarray") else Dc
    R0 = np.array(Dc, dtype=np.float64, copy=True)
    R0[cols, np.arange(k)] = 0.0
    return float(np.linalg.norm(R0))


def _check_theta(theta, cols):
    """theta finite, and each theta_{cols[c]} occurs exactly once in theta."""
    if not np.all(np.isfinite(theta)):
        return False
    vals, counts = np.unique(theta, return_counts=True)
    return bool(np.all(counts[np.searchsorted(vals, theta[cols])] == 1))


def ipt_solve(M, theta=None, cols=None, tol=1e-12, max_iter=1000, stop="increment",
              diverge_bound=1e8, Z0=None, history=False, Delta=None, product=None):
    """Alg. 2 (full spectrum) / Alg. 1 applied to the columns ``cols`` (partial spectrum).

    Picard iteration Z <- F(Z) from Z = I (or ``Z0``) while the test fails.
    ``stop`` chooses the test: "increment" is Alg. 2's ||Z - F(Z)||_F/||Z||_F
    <= tol; "residual" is rho(Z) <= tol (reading 4 above).

    ``M`` may be None when ``Delta``, ``theta`` and ``product`` are given (the
    sparse oracle).  Returns a dict with Z, lam, status, iterations, increment,
    rho and (with ``history``) the per-evaluation increments and residuals.
    """
    if Delta is None:
        Delta, theta = partition(M, theta)
    theta = np.asarray(theta, dtype=np.float64)
    n = len(theta)
    cols = np.arange(n) if cols is None else np.asarray(cols, dtype=np.int64)
    k = len(cols)
    out = {"status": INVALID_ARG, "iterations": 0, "Z": None, "lam": None,
           "increment": np.nan, "rho": np.nan, "inc_hist": [], "rho_hist": []}
    if k == 0 or len(set(cols.tolist())) != k or cols.min() < 0 or cols.max() >= n:
        return out
    if max_iter < 1 or not (tol >= 0):
        return out
    if not _check_theta(theta, cols):
        out["status"] = DEGENERATE_THETA
        return out
    G = inverse_gaps(theta, cols)
    Z = unit_columns(n, cols) if Z0 is None else np.array(Z0, dtype=np.float64)
    r0 = initial_residual_norm(Delta, cols)
    for it in range(max_iter):
        F, P, d = ipt_map(Delta, theta, cols, Z, G=G, product=product)
        znorm = np.linalg.norm(Z)
        inc = np.linalg.norm(F - Z) / znorm
        lam = theta[cols] + d
        # M Z - Z Lambda with M = D + Delta: theta_j Z_jc + P_jc - Z_jc lam_c
        R = theta[:, None] * Z + P - Z * lam[None, :]
        rho = np.linalg.norm(R) / r0 if r0 > 0 else 0.0
        out.update(Z=Z, lam=lam, iterations=it + 1, increment=inc, rho=rho)
        if history:
            out["inc_hist"].append(inc)
            out["rho_hist"].append(rho)
        if not (np.isfinite(inc) and np.isfinite(rho)) or znorm > diverge_bound * np.sqrt(k):
            out["status"] = DIVERGED
            return out
        test = inc if stop == "increment" else rho
        if test <= tol:
            out["status"] = OK
            return out
        if it + 1 == max_iter:
            out["status"] = MAXITER
            return out
        Z = F
    return out


def ipt_solve_csr(rowptr, colind, vals, n, theta=None, cols=None, **kw):
    """The same iteration with a sparse M given in CSR (0-based, all entries of M).

    Delta = M - diag(theta), theta = diag(M) by default; the product Delta Z
    is scipy's CSR times dense product.
    """
    import scipy.sparse as sp

    M = sp.csr_matrix((np.asarray(vals, dtype=np.float64), np.asarray(colind),
                       np.asarray(rowptr)), shape=(n, n))
    if theta is None:
        theta = M.diagonal().astype(np.float64)
    theta = np.asarray(theta, dtype=np.float64)
    Delta = (M - sp.diags(theta)).tocsr()
    return ipt_solve(None, theta=theta, cols=cols, Delta=Delta,
                     product=lambda Z: np.asarray(Delta @ Z), **kw)


def ipt_solve_acx_csr(rowptr, colind, vals, n, theta=None, cols=None, **kw):
    """IPT-ACX (Alg. 3) for a sparse M given in CSR, as ipt_solve_csr does for
    Alg. 1/2: Delta = M - diag(theta) (theta = diag(M) by default) and the
    product Delta Z by scipy's CSR times dense product."""
    import scipy.sparse as sp

    M = sp.csr_matrix((np.asarray(vals, dtype=np.float64), np.asarray(colind),
                       np.asarray(rowptr)), shape=(n, n))
    if theta is None:
        theta = M.diagonal().astype(np.float64)
    theta = np.asarray(theta, dtype=np.float64)
    Delta = (M - sp.diags(theta)).tocsr()
    return ipt_solve_acx(None, theta=theta, cols=cols, Delta=Delta,
                         product=lambda Z: np.asarray(Delta @ Z), **kw)


def acx_differences(z, fs):
    """Alg. 3 lines 4-6 and 11: the differences of the iterates z, f(z), f^2(z), ...

    ``fs`` = [f(z), f^2(z), (f^3(z))]; returns [D^1, D^2, (D^3)] with
    D^1 = f(z) - z, D^2 = f^2(z) - 2 f(z) + z, D^3 = f^3(z) - 3 f^2(z) + 3 f(z) - z.
    """
    D = [fs[0] - z, fs[1] - 2.0 * fs[0] + z]
    if len(fs) >= 3:
        D.append(fs[2] - 3.0 * fs[1] + 3.0 * fs[0] - z)
    return D


def acx_sigma(Dp, Dq, per_column=True):
    """Alg. 3 lines 8 / 12 (reading 8): sigma = |<D^p, D^(p-1)>| / ||D^p||^2.

    Inner products over each column (per_column) or over the whole block;
    a zero ||D^p|| gives sigma = 1.  Returns a length-k array (global: repeated).
    """
    if per_column:
        num = np.abs(np.sum(Dp * Dq, axis=0))
        den = np.sum(Dp * Dp, axis=0)
    else:
        num = np.full(Dp.shape[1], abs(float(np.sum(Dp * Dq))))
        den = np.full(Dp.shape[1], float(np.sum(Dp * Dp)))
    safe = np.where(den > 0, den, 1.0)
    return np.where(den > 0, num / safe, 1.0)


def acx_update(z, fs, per_column=True):
    """Alg. 3 lines 7-14: the order-p extrapolation (p = len(fs)) from z, f(z), ..., f^p(z)."""
    D = acx_differences(z, fs)
    p = len(fs)
    if p == 2:
        s = acx_sigma(D[1], D[0], per_column)[None, :]
        return z + 2.0 * s * D[0] + s * s * D[1]
    if p == 3:
        s = acx_sigma(D[2], D[1], per_column)[None, :]
        return z + 3.0 * s * D[0] + 3.0 * s * s * D[1] + s * s * s * D[2]
    raise ValueError("ACX order must be 2 or 3")


def ipt_solve_acx(M, theta=None, cols=None, tol=1e-12, max_iter=1000, stop="increment",
                  diverge_bound=1e8, history=False, Delta=None, product=None,
                  sigma="column", orders=(3, 2)):
    """IPT-ACX: Alg. 1 / Alg. 2 with the Picard update replaced by Alg. 3.

    Each extrapolation evaluates F at z (where Alg. 3's test is made), at
    f(z) and, for order 3, at f^2(z), then moves z by acx_update.  Orders
    cycle through ``orders``.  Same arguments, statuses and result dict as
    ipt_solve (reading 8 for what ``iterations`` and the returned pair are).
    """
    if Delta is None:
        Delta, theta = partition(M, theta)
    theta = np.asarray(theta, dtype=np.float64)
    n = len(theta)
    cols = np.arange(n) if cols is None else np.asarray(cols, dtype=np.int64)
    k = len(cols)
    out = {"status": INVALID_ARG, "iterations": 0, "Z": None, "lam": None,
           "increment": np.nan, "rho": np.nan, "inc_hist": [], "rho_hist": []}
    if k == 0 or len(set(cols.tolist())) != k or cols.min() < 0 or cols.max() >= n:
        return out
    if max_iter < 1 or not (tol >= 0) or sigma not in ("column", "global"):
        return out
    if not _check_theta(theta, cols):
        out["status"] = DEGENERATE_THETA
        return out
    G = inverse_gaps(theta, cols)
    r0 = initial_residual_norm(Delta, cols)

    def evaluate(x):
        F, P, d = ipt_map(Delta, theta, cols, x, G=G, product=product)
        xnorm = np.linalg.norm(x)
        inc = np.linalg.norm(F - x) / xnorm
        lam = theta[cols] + d
        R = theta[:, None] * x + P - x * lam[None, :]
        rho = np.linalg.norm(R) / r0 if r0 > 0 else 0.0
        if history:
            out["inc_hist"].append(inc)
            out["rho_hist"].append(rho)
        bad = not (np.isfinite(inc) and np.isfinite(rho)) or xnorm > diverge_bound * np.sqrt(k)
        return F, lam, inc, rho, bad

    z = unit_columns(n, cols)
    evals, step = 0, 0
    while True:
        p = orders[step % len(orders)]
        F, lam, inc, rho, bad = evaluate(z)
        evals += 1
        out.update(Z=z, lam=lam, iterations=evals, increment=inc, rho=rho)
        if bad:
            out["status"] = DIVERGED
            return out
        if (inc if stop == "increment" else rho) <= tol:
            out["status"] = OK
            return out
        if evals == max_iter:
            out["status"] = MAXITER
            return out
        fs = [F]
        for _ in range(p - 1):
            Fq, _, _, _, bad = evaluate(fs[-1])
            evals += 1
            out["iterations"] = evals
            if bad:
                out["status"] = DIVERGED
                return out
            if evals == max_iter:
                out["status"] = MAXITER
                return out
            fs.append(Fq)
        z = acx_update(z, fs, per_column=(sigma == "column"))
        step += 1


def rs_corrections(Delta, theta, order):
    """Rayleigh-Schroedinger corrections Z^[0..order], Eq. (ARS-alpha) / App. B.

    Z^[0] = I and Z^[l] = G o (sum_{s=0}^{l-1} Z^[l-1-s] D(Delta Z^[s]) - Delta Z^[l-1]),
    full spectrum (k = n).
    """
    n = len(theta)
    G = inverse_gaps(theta, np.arange(n))
    Zs = [np.eye(n)]
    DZ = [Delta @ Zs[0]]
    for l in range(1, order + 1):
        acc = np.zeros((n, n))
        for s in range(l):
            acc += Zs[l - 1 - s] @ np.diag(np.diag(DZ[s]))
        Zl = G * (acc - DZ[l - 1])
        Zs.append(Zl)
        DZ.append(Delta @ Zl)
    return Zs


def chart_jacobian(Delta, theta, i, z):
    """Jacobian of f_i in the affine chart U_i (z_i = 1), App. D.1.

    f_i(z) = e_i + g_i o (z (Delta z)_i - Delta z), Eq. (single_line_dyn).
    d(f_i)_j / dz_s = (g_i)_j * (delta_js (Delta z)_i + z_j Delta_is - Delta_js),
    restricted to j, s != i: the (n-1) x (n-1) matrix whose eigenvalues are the
    multipliers of the fixed point.
    """
    n = len(theta)
    g = inverse_gaps(theta, np.array([i]))[:, 0]
    Dz = Delta @ z
    J = np.zeros((n, n))
    for j in range(n):
        for s in range(n):
            J[j, s] = g[j] * ((Dz[i] if j == s else 0.0) + z[j] * Delta[i, s] - Delta[j, s])
    keep = [j for j in range(n) if j != i]
    return J[np.ix_(keep, keep)]
