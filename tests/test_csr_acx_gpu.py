"""GPU parity of IPT-ACX (Alg. 3) on the sparse path against the oracle.

FP64: the same evaluations and extrapolations as the oracle's IPT-ACX with the
CSR product, compared iterate by iterate (1e-11 of the largest entry of Z - E),
with and without the active window, per-column and global step lengths.  FP32:
the Morgan tridiagonal matrix of Section 6.1 at eps = 1, where the Picard
iteration diverges, converges to LAPACK's lowest eigenpairs with an FP64-verified
residual within tol.
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2012_14702_gb300 import workloads as w

pytestmark = pytest.mark.gpu


def cuda(x, dtype):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def morgan_csr(n, eps):
    """The Morgan matrix in CSR (diagonal i, off-diagonals eps)."""
    rows, cols, vals = [], [], []
    for j in range(n):
        for m in (j - 1, j, j + 1):
            if 0 <= m < n:
                rows.append(j)
                cols.append(m)
                vals.append(float(j + 1) if m == j else eps)
    rowptr = np.searchsorted(np.asarray(rows), np.arange(n + 1)).astype(np.int32)
    return rowptr, np.asarray(cols, dtype=np.int32), np.asarray(vals)


@pytest.mark.parametrize("window", [True, False])
@pytest.mark.parametrize("sigma", ["column", "global"])
def test_csr_acx_f64_iterates_match_oracle(ipt, window, sigma):
    """Stops at every position of the 3, 2, 3 extrapolation cycle."""
    n, k = 1500, 12
    rowptr, colind, vals, th = w.csr_banded(n, 4, 60, 2e-2, seed=31, theta_step=0.05)
    cols = w.lowest_columns(th, k)
    rp, ci, vv = cuda(rowptr, torch.int32), cuda(colind, torch.int32), cuda(vals, torch.float64)
    cg = cuda(cols, torch.int32)
    E = oracle.unit_columns(n, cols)
    for m in [1, 2, 3, 4, 5, 6, 8, 9, 14]:
        ref = oracle.ipt_solve_acx_csr(rowptr, colind, vals, n, cols=cols, tol=0.0,
                                       max_iter=m, stop="increment", sigma=sigma, history=True)
        lam, Z, info = ipt.Solver().solve_csr(rp, ci, vv, n, cols=cg, tol=0.0, max_iter=m,
                                              precision="f64", stop="increment",
                                              z_dtype=torch.float64, window=window,
                                              accel="acx", acx_sigma=sigma)
        assert info["status"] == "MAXITER" and info["iterations"] == m, (m, info["status"])
        scale = max(np.max(np.abs(ref["Z"] - E)), 1e-3)
        assert np.max(np.abs(Z.cpu().numpy() - ref["Z"])) <= 1e-11 * scale, m
        np.testing.assert_allclose(lam.cpu().numpy(), ref["lam"], rtol=1e-12)
        np.testing.assert_allclose(info["hist_increment"], ref["inc_hist"], rtol=1e-9)


@pytest.mark.parametrize("precision,vdt", [("f32", torch.float32), ("f64", torch.float64)])
@pytest.mark.parametrize("window", [True, False])
def test_csr_acx_morgan_beyond_picard(ipt, precision, vdt, window):
    """Section 6.1: the Morgan matrix at eps = 1 (n = 5000, the paper's size), the
    four lowest eigenpairs: Picard diverges, IPT-ACX converges to LAPACK's."""
    n, eps = 5000, 1.0
    rowptr, colind, vals = morgan_csr(n, eps)
    cols = np.arange(4, dtype=np.int32)
    rp, ci, vv = cuda(rowptr, torch.int32), cuda(colind, torch.int32), cuda(vals, vdt)
    cg = cuda(cols, torch.int32)
    s = ipt.Solver()
    _, _, plain = s.solve_csr(rp, ci, vv, n, cols=cg, tol=1e-6, max_iter=200,
                              precision=precision, window=window)
    assert plain["status"] in ("MAXITER", "DIVERGED"), plain["status"]
    lam, Z, info = s.solve_csr(rp, ci, vv, n, cols=cg, tol=1e-6, max_iter=400,
                               precision=precision, window=window, accel="acx",
                               verify_fp64=True)
    assert info["status"] == "OK", info
    assert info["rho_fp64"] <= 1e-6 and info["rho_fp64"] <= info["rho"] + info["rho_error"]
    # LAPACK on the lowest part: the band is tridiagonal, so a leading block holds the
    # lowest eigenvectors to rounding
    M, _ = w.morgan_tridiagonal(400, eps)
    ev, V = np.linalg.eigh(M)
    np.testing.assert_allclose(lam.cpu().numpy(), ev[:4], rtol=1e-6)
    Zh = Z.double().cpu().numpy()[:400]
    ref = V[:, :4] / V[cols, np.arange(4)][None, :]
    assert np.max(np.abs(Zh - ref)) <= 1e-4


def test_csr_acx_window_matches_all_rows(ipt):
    """The active window (widened by the band after every extrapolation) gives the
    all-rows iterates after 30 evaluations (up to the order of the step lengths'
    sums)."""
    n, k = 20000, 16
    rowptr, colind, vals, th = w.csr_banded(n, 6, 300, 1e-2, seed=8, theta_step=0.01)
    cols = w.lowest_columns(th, k)
    rp, ci, vv = cuda(rowptr, torch.int32), cuda(colind, torch.int32), cuda(vals, torch.float64)
    cg = cuda(cols, torch.int32)
    s = ipt.Solver()
    la, Za, ia = s.solve_csr(rp, ci, vv, n, cols=cg, tol=0.0, max_iter=30, precision="f64",
                             z_dtype=torch.float64, window=False, accel="acx")
    lw, Zw, iw = s.solve_csr(rp, ci, vv, n, cols=cg, tol=0.0, max_iter=30, precision="f64",
                             z_dtype=torch.float64, window=True, accel="acx")
    assert ia["status"] == iw["status"] == "MAXITER"
    assert ia["iterations"] == iw["iterations"] == 30
    assert ia["hist_rho"][-1] < 1e-4 * ia["hist_rho"][0]
    assert iw["rows_evaluated"] < ia["rows_evaluated"]
    assert torch.max(torch.abs(Za - Zw)).item() <= 1e-12
    assert torch.max(torch.abs(la - lw)).item() <= 1e-12 * torch.max(torch.abs(la)).item()


def test_csr_rejects_other_accelerations(ipt):
    rowptr, colind, vals = morgan_csr(50, 0.1)
    rp, ci, vv = cuda(rowptr, torch.int32), cuda(colind, torch.int32), cuda(vals, torch.float32)
    with pytest.raises(ValueError):
        ipt.Solver().solve_csr(rp, ci, vv, 50, accel="anderson")
