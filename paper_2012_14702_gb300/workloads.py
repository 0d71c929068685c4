"""Seeded synthetic near-diagonal eigenproblems (inputs only, no IPT arithmetic).

Both the CPU oracle (``oracle/``) and the CUDA path are fed from these
generators; nothing here evaluates the IPT map.  Every generator draws from
``numpy.random.Generator(PCG64(seed))`` in float64 on the host; callers cast.

Workload shapes follow the paper's test matrices:

* ``dense_symmetric``: M = diag(theta) + Delta with Delta symmetric,
  zero-diagonal, off-diagonal entries N(0,1)*scale.  With theta_i = i/8 and
  n = 8192 this is the dense full-spectrum workload; with theta_i = i,
  n = 256, scale 0.02 it is the small FP64 case.
* ``dense_paper``: the paper's own dense family of Section 6.2, Eq.
  (dense_matrix): M = diag(i) + eps * R, R ~ U[0,1] (non-symmetric), and
  its symmetrisation S = (M + M^T)/2.
* ``csr_banded``: the sparse partial-spectrum workload: n = 2^20 symmetric
  CSR, 8 distinct upper-triangle offsets per row drawn from {1..band},
  mirrored, values N(0,1)*scale, theta_i = i*1e-2 + U(0, 1e-3).
* ``morgan_tridiagonal``: the tridiagonal matrix of Section 6.1
  (M_ii = i, M_{i,i+1} = M_{i+1,i} = eps).
* ``two_by_two`` / ``three_by_three``: the worked examples of Eq. (2by2)
  (Section 4.3) and of Appendix D.3.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "rng",
    "dense_symmetric",
    "dense_paper",
    "csr_banded",
    "morgan_tridiagonal",
    "morgan_csr",
    "two_by_two",
    "three_by_three",
    "lowest_columns",
    "DENSE_CONFIGS",
    "CSR_CONFIGS",
    "batched_dense",
    "BATCHED_CONFIGS",
]


def rng(seed: int) -> np.random.Generator:
    """The one random source of every workload: PCG64 seeded with ``seed``."""
    return np.random.Generator(np.random.PCG64(seed))


def _sym_offdiag(n: int, scale: float, g: np.random.Generator) -> np.ndarray:
    """Symmetric n x n matrix, zero diagonal, strict upper triangle N(0,1)*scale."""
    r = g.standard_normal((n, n))
    a = np.triu(r, 1)
    del r
    a *= scale
    return a + a.T


def dense_symmetric(n: int, scale: float, seed: int, theta_step: float = 1.0,
                    symmetric: bool = True):
    """Return (M, theta): M = diag(theta) + Delta, theta_i = i * theta_step, i = 1..n.

    Delta has zero diagonal and off-diagonal N(0,1)*scale entries; with
    ``symmetric`` the strict upper triangle is drawn and mirrored, otherwise
    every off-diagonal entry is drawn independently.
    """
    g = rng(seed)
    theta = np.arange(1, n + 1, dtype=np.float64) * theta_step
    if symmetric:
        m = _sym_offdiag(n, scale, g)
    else:
        m = g.standard_normal((n, n)) * scale
        np.fill_diagonal(m, 0.0)
    m[np.diag_indices(n)] = theta
    return m, theta


def dense_paper(n: int, eps: float, seed: int, symmetric: bool = False):
    """The paper's dense test family, Eq. (dense_matrix): diag(i) + eps*U[0,1].

    Returns (M, theta) with theta = diag(M) (the paper's partition choice,
    Section 3: D is taken as the diagonal of M).  ``symmetric`` returns
    S = (M + M^T)/2 instead.
    """
    g = rng(seed)
    m = g.random((n, n)) * eps
    m[np.diag_indices(n)] += np.arange(1, n + 1, dtype=np.float64)
    if symmetric:
        m = 0.5 * (m + m.T)
    return m, np.diag(m).copy()


def morgan_tridiagonal(n: int, eps: float = 0.5):
    """Tridiagonal M_ii = i, M_{i,i+1} = M_{i+1,i} = eps (Section 6.1), dense."""
    m = np.zeros((n, n))
    idx = np.arange(n)
    m[idx, idx] = idx + 1.0
    m[idx[:-1], idx[:-1] + 1] = eps
    m[idx[:-1] + 1, idx[:-1]] = eps
    return m, np.diag(m).copy()


def morgan_csr(n: int, eps: float = 0.5):
    """The tridiagonal matrix of Section 6.1 in CSR form (rowptr int32, colind int32,
    vals float64, theta = diag): M_ii = i, M_{i,i+1} = M_{i+1,i} = eps, any n."""
    idx = np.arange(n, dtype=np.int64)
    rows = np.concatenate([idx, idx[:-1], idx[1:]])
    cols = np.concatenate([idx, idx[1:], idx[:-1]])
    vals = np.concatenate([idx + 1.0, np.full(n - 1, eps), np.full(n - 1, eps)])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.searchsorted(rows, np.arange(n + 1)).astype(np.int32)
    return rowptr, cols.astype(np.int32), vals, idx + 1.0


def two_by_two(eps: float):
    """The 2 x 2 example of Eq. (2by2): [[0, eps], [eps, 1]]."""
    m = np.array([[0.0, eps], [eps, 1.0]])
    return m, np.array([0.0, 1.0])


def three_by_three(eps: float):
    """The 3 x 3 example of Appendix D.3: diag(0, 1, 3) + eps*[[0,1,2],[1,0,3],[2,3,0]]."""
    d = np.diag([0.0, 1.0, 3.0])
    delta = np.array([[0.0, 1.0, 2.0], [1.0, 0.0, 3.0], [2.0, 3.0, 0.0]])
    return d + eps * delta, np.array([0.0, 1.0, 3.0])


def csr_banded(n: int, per_row: int, band: int, scale: float, seed: int,
               theta_step: float = 1e-2, theta_jitter: float = 1e-3,
               with_diagonal: bool = True):
    """Symmetric banded CSR near-diagonal matrix (the sparse workload).

    For every row i, ``per_row`` distinct offsets o in {1..band} are drawn and
    the pair (i, i+o) gets a N(0,1)*scale value, mirrored to (i+o, i); pairs
    past the last row are dropped.  The diagonal is theta_i = i*theta_step +
    U(0, theta_jitter), i = 1..n, stored in the CSR arrays as M_ii (unless
    ``with_diagonal`` is False) and also returned.  Returns (rowptr int32[n+1],
    colind int32[nnz], vals f64[nnz], theta f64[n]); column indices are
    sorted within each row.
    """
    g = rng(seed)
    offs = g.integers(1, band + 1, size=(n, per_row), dtype=np.int64)
    # redraw rows with repeated offsets until every row's offsets are distinct
    while True:
        s = np.sort(offs, axis=1)
        bad = np.nonzero((s[:, 1:] == s[:, :-1]).any(axis=1))[0]
        if bad.size == 0:
            break
        offs[bad] = g.integers(1, band + 1, size=(bad.size, per_row), dtype=np.int64)
    vals = g.standard_normal((n, per_row)) * scale
    theta = np.arange(1, n + 1, dtype=np.float64) * theta_step + g.random(n) * theta_jitter
    rows = np.repeat(np.arange(n, dtype=np.int64), per_row)
    cols = rows + offs.reshape(-1)
    v = vals.reshape(-1)
    keep = cols < n
    rows, cols, v = rows[keep], cols[keep], v[keep]
    diag = np.arange(n, dtype=np.int64) if with_diagonal else np.zeros(0, dtype=np.int64)
    r_all = np.concatenate([rows, cols, diag])
    c_all = np.concatenate([cols, rows, diag])
    v_all = np.concatenate([v, v, theta[diag]])
    order = np.lexsort((c_all, r_all))
    r_all, c_all, v_all = r_all[order], c_all[order], v_all[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, r_all + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr.astype(np.int32), c_all.astype(np.int32), v_all, theta


def batched_dense(count: int, nmin: int, nmax: int, scale: float, seed: int,
                  dtype=np.float32):
    """Many small dense problems packed back to back (the batched workload).

    Problem p has order n_p ~ U{nmin..nmax}, theta_i = i (i = 1..n_p) on the
    diagonal and a symmetric zero-diagonal perturbation with N(0,1)*scale/sqrt(n_p)
    entries.  Returns (sizes int64[count], M packed row-major in ``dtype``,
    theta packed float64): problem p starts at sum_{q<p} n_q^2 in M and at
    sum_{q<p} n_q in theta.
    """
    g = rng(seed)
    sizes = g.integers(nmin, nmax + 1, size=count).astype(np.int64)
    m = np.empty(int(np.sum(sizes * sizes)), dtype=dtype)
    th = np.empty(int(np.sum(sizes)), dtype=np.float64)
    mo = vo = 0
    for n in sizes:
        n = int(n)
        a = _sym_offdiag(n, scale / np.sqrt(n), g)
        t = np.arange(1, n + 1, dtype=np.float64)
        a[np.diag_indices(n)] = t
        m[mo:mo + n * n] = a.reshape(-1)
        th[vo:vo + n] = t
        mo += n * n
        vo += n
    return sizes, m, th


def lowest_columns(theta: np.ndarray, k: int) -> np.ndarray:
    """Indices of the k smallest theta, ascending (target choice of Section 6.1)."""
    return np.argsort(theta, kind="stable")[:k].astype(np.int32)


# The dense workloads by name: (n, theta_step, scale, seed).
DENSE_CONFIGS = {
    "dense_n256_fp64": (256, 1.0, 0.02, 1),
    "dense_n8192_eps1e-4": (8192, 0.125, 1e-4, 21),
    "dense_n8192_eps1e-3": (8192, 0.125, 1e-3, 22),
    "dense_n8192_eps3e-3": (8192, 0.125, 3e-3, 23),
    # beyond the Picard iteration's domain (it diverges), inside IPT-ACX's
    "dense_n4096_edge_sd6e-2": (4096, 0.25, 6e-2, 31),
}

# The sparse workloads by name: (n, per_row, band, scale, seed, k lowest).
CSR_CONFIGS = {
    "csr_n2p20_k64": (1 << 20, 8, 2048, 1e-3, 3, 64),
    "csr_n2p16_k64": (1 << 16, 8, 2048, 1e-3, 3, 64),
}

# The batched workloads by name: (count, nmin, nmax, scale, seed).
BATCHED_CONFIGS = {
    "batched_4096_n32_512": (4096, 32, 512, 1e-2, 4),
    "batched_512_n32_512": (512, 32, 512, 1e-2, 4),  # the same mix, small enough to profile
}
