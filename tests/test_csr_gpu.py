"""GPU parity of the sparse path (ipt_solve_csr) against the CPU oracle.

Workloads are the banded symmetric CSR family of the sparse configuration
(theta_i = i*theta_step + U(0, 1e-3), N(0,1)*scale off-diagonal entries) and
the Morgan tridiagonal matrix of Section 6.1.  Tolerances: FP64 eigenvalues
1e-10 relative, FP32 1e-5 relative; eigenvectors to the converged oracle
within 1e-4 (relative to ||Z - E||) at rho <= 1e-6.
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2012_14702_gb300 import workloads as w

pytestmark = pytest.mark.gpu


def cuda(x, dtype):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def csr_on_gpu(rowptr, colind, vals, dtype=torch.float32):
    return cuda(rowptr, torch.int32), cuda(colind, torch.int32), cuda(vals, dtype)


@pytest.mark.parametrize("precision,vdt,lam_tol", [("f64", torch.float64, 1e-10),
                                                   ("f32", torch.float32, 1e-5)])
@pytest.mark.parametrize("k,permute", [(8, False), (37, True), (100, False)])
def test_csr_solve_matches_oracle(ipt, precision, vdt, lam_tol, k, permute):
    n = 3000
    rowptr, colind, vals, th = w.csr_banded(n, 4, 64, 1e-2, seed=3, theta_step=0.1)
    cols = w.lowest_columns(th, k)
    if permute:
        cols = w.rng(2).permutation(n)[:k].astype(np.int32)
    ref = oracle.ipt_solve_csr(rowptr, colind, vals, n, cols=cols, tol=1e-13, max_iter=200)
    assert ref["status"] == oracle.OK
    rp, ci, vv = csr_on_gpu(rowptr, colind, vals, vdt)
    lam, Z, info = ipt.Solver().solve_csr(rp, ci, vv, n, cols=cuda(cols, torch.int32),
                                          tol=1e-6 if precision == "f32" else 1e-12,
                                          max_iter=100, precision=precision,
                                          z_dtype=torch.float64)
    assert info["status"] == "OK", info
    lam = lam.cpu().numpy()
    assert np.max(np.abs(lam - ref["lam"]) / np.abs(ref["lam"])) <= lam_tol
    E = oracle.unit_columns(n, cols)
    err = np.linalg.norm(Z.cpu().numpy() - ref["Z"]) / np.linalg.norm(ref["Z"] - E)
    assert err <= (1e-4 if precision == "f32" else 1e-9), err


def test_csr_fixed_iterations_f64_match_oracle_iterates(ipt):
    """Same map, same iterates: max_iter evaluations in FP64 give the oracle's Z^(max_iter-1)."""
    n = 2000
    rowptr, colind, vals, th = w.csr_banded(n, 3, 40, 2e-2, seed=8, theta_step=0.05)
    cols = w.lowest_columns(th, 5)
    rp, ci, vv = csr_on_gpu(rowptr, colind, vals, torch.float64)
    for it in [1, 3]:
        ref = oracle.ipt_solve_csr(rowptr, colind, vals, n, cols=cols, tol=0.0, max_iter=it,
                                   history=True)
        lam, Z, info = ipt.Solver().solve_csr(rp, ci, vv, n, cols=cuda(cols, torch.int32),
                                              tol=0.0, max_iter=it, precision="f64",
                                              stop="increment", z_dtype=torch.float64)
        assert info["status"] == "MAXITER" and info["iterations"] == it
        assert np.max(np.abs(Z.cpu().numpy() - ref["Z"])) <= 1e-13
        assert np.max(np.abs(lam.cpu().numpy() - ref["lam"])) <= 1e-12
        np.testing.assert_allclose(info["hist_increment"], ref["inc_hist"], rtol=1e-10)


def test_csr_morgan_tridiagonal_lowest_eigenpair(ipt):
    """Section 6.1: tridiagonal M_ii = i, off-diagonal eps, lowest eigenpair (k = 1)."""
    n, eps = 5000, 0.3
    i = np.arange(n)
    rows = np.concatenate([i, i[:-1], i[1:]])
    cols = np.concatenate([i, i[1:], i[:-1]])
    vals = np.concatenate([i + 1.0, np.full(n - 1, eps), np.full(n - 1, eps)])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    ref = oracle.ipt_solve_csr(rowptr, cols, vals, n, cols=[0], tol=1e-12, max_iter=500,
                               stop="increment")
    rp, ci, vv = csr_on_gpu(rowptr, cols, vals, torch.float64)
    lam, Z, info = ipt.Solver().solve_csr(rp, ci, vv, n, cols=cuda([0], torch.int32), tol=1e-12,
                                          max_iter=500, precision="f64", stop="increment",
                                          z_dtype=torch.float64)
    assert info["status"] == "OK" and info["iterations"] == ref["iterations"]
    assert abs(lam.item() - ref["lam"][0]) <= 1e-12 * abs(ref["lam"][0])
    M = np.diag(i + 1.0) + eps * (np.eye(n, k=1) + np.eye(n, k=-1))
    assert abs(lam.item() - np.linalg.eigvalsh(M[:200, :200])[0]) < 1e-10


def test_csr_statuses(ipt):
    n = 500
    rowptr, colind, vals, th = w.csr_banded(n, 3, 20, 1e-2, seed=4, theta_step=0.1)
    rp, ci, vv = csr_on_gpu(rowptr, colind, vals)
    s = ipt.Solver()
    _, _, info = s.solve_csr(rp, ci, vv, n, cols=cuda([0, 0], torch.int32))
    assert info["status"] == "INVALID_ARG"
    _, _, info = s.solve_csr(rp, ci, vv, n, cols=cuda([3, n], torch.int32))
    assert info["status"] == "INVALID_ARG"
    _, _, info = s.solve_csr(rp, ci, vv, n, cols=cuda([1, 2], torch.int32), precision="bf16")
    assert info["status"] == "UNSUPPORTED"
    thd = th.copy()
    thd[7] = thd[3]
    _, _, info = s.solve_csr(rp, ci, vv, n, theta=cuda(thd, torch.float64),
                             cols=cuda([3], torch.int32))
    assert info["status"] == "DEGENERATE_THETA"
    _, _, info = s.solve_csr(rp, ci, vv, n, cols=cuda([3], torch.int32), precision="staged",
                             tol=1e-6)
    assert info["status"] == "OK" and info["hist_stage"][0] == "f32"
    # CSR structure errors are found on the device before any product reads Z
    bad = colind.copy()
    bad[len(bad) // 2] = n
    _, _, info = s.solve_csr(rp, cuda(bad, torch.int32), vv, n, cols=cuda([3], torch.int32))
    assert info["status"] == "INVALID_ARG"
    badp = rowptr.copy()
    badp[-1] -= 1
    _, _, info = s.solve_csr(cuda(badp, torch.int32), ci, vv, n, cols=cuda([3], torch.int32))
    assert info["status"] == "INVALID_ARG"
    _, _, info = s.solve_csr(rp, ci, vv, n, cols=cuda([3], torch.int32), tol=1e-6)
    assert info["status"] == "OK"


def _split_repeated(rowptr, colind, vals, dtype, seed):
    """The same matrix with repeated stored entries: on every 5th row the diagonal
    is stored as two or three pieces (first, middle and last of the row's
    entries), on every 7th row one off-diagonal entry as two; the pieces are
    values of `dtype`, and their sum is the matrix both sides solve."""
    g = w.rng(seed)
    rp, ci, vv = [0], [], []
    for i in range(len(rowptr) - 1):
        c = list(colind[rowptr[i]:rowptr[i + 1]])
        v = [float(x) for x in np.asarray(vals[rowptr[i]:rowptr[i + 1]]).astype(dtype)]
        if i % 5 == 0 and i in c:
            d = c.index(i)
            dv = v[d]
            p1 = float(np.asarray(dv * g.uniform(0.2, 0.8)).astype(dtype))
            pieces = [p1, float(np.asarray(dv - p1).astype(dtype))]
            if i % 10 == 0:
                p2 = float(np.asarray(pieces[1] * 0.5).astype(dtype))
                pieces = [p1, p2, float(np.asarray(pieces[1] - p2).astype(dtype))]
            del c[d], v[d]
            c = [i] + c + [i] * (len(pieces) - 1)
            v = [pieces[0]] + v + pieces[1:]
        if i % 7 == 0 and len(c) > 2:
            k = 1 if c[1] != i else 2
            half = float(np.asarray(v[k] * 0.5).astype(dtype))
            c.append(c[k])
            v.append(float(np.asarray(v[k] - half).astype(dtype)))
            v[k] = half
        ci += c
        vv += v
        rp.append(len(ci))
    return (np.asarray(rp, np.int32), np.asarray(ci, np.int32), np.asarray(vv, np.float64))


@pytest.mark.parametrize("vdt,npdt,lam_tol", [(torch.float32, np.float32, 1e-5),
                                              (torch.float64, np.float64, 1e-10)])
@pytest.mark.parametrize("theta_given", [False, True])
def test_csr_repeated_entries_add_up(ipt, vdt, npdt, lam_tol, theta_given):
    """Repeated stored entries add up, as in the oracle's scipy CSR matrix: the
    diagonal (theta = diag(M) and delta_j = M_jj - theta_j) and the product.
    Rows with a repeated FP32 diagonal take the row pass's out-of-line FP64 path."""
    n = 600
    rowptr, colind, vals, th = w.csr_banded(n, 3, 30, 1e-2, seed=5, theta_step=0.1)
    rp_, ci_, vv_ = _split_repeated(rowptr, colind, vals, npdt, seed=12)
    assert len(ci_) > len(colind)
    cols = w.lowest_columns(th, 8)
    theta = th if theta_given else None
    tol = 1e-6 if vdt == torch.float32 else 1e-12
    ref = oracle.ipt_solve_csr(rp_, ci_, vv_, n, theta=theta, cols=cols, tol=1e-13,
                               max_iter=200)
    assert ref["status"] == oracle.OK
    rp, ci, vv = csr_on_gpu(rp_, ci_, vv_, vdt)
    for window in (True, False):
        lam, Z, info = ipt.Solver().solve_csr(
            rp, ci, vv, n, theta=None if theta is None else cuda(theta, torch.float64),
            cols=cuda(cols, torch.int32), tol=tol, max_iter=100,
            precision="f32" if vdt == torch.float32 else "f64", window=window,
            z_dtype=torch.float64)
        assert info["status"] == "OK", info
        lam = lam.cpu().numpy()
        assert np.max(np.abs(lam - ref["lam"]) / np.abs(ref["lam"])) <= lam_tol


def test_csr_full_size_sampled_columns_match_oracle(ipt):
    """The sparse configuration at full size: n = 2^20, 8 offsets per row in
    {1..2048} mirrored, values N(0,1)*1e-3, theta_i = i*1e-2 + U(0,1e-3); the 64
    lowest eigenpairs in FP32 to rho <= 1e-6.  The oracle re-solves 8 of the 64
    columns (Alg. 1 per column, FP64) and they must match."""
    n = 1 << 20
    rowptr, colind, vals, th = w.csr_banded(n, 8, 2048, 1e-3, seed=3)
    cols = w.lowest_columns(th, 64)
    rp, ci, vv = csr_on_gpu(rowptr, colind, vals)
    lam, Z, info = ipt.Solver().solve_csr(rp, ci, vv, n, cols=cuda(cols, torch.int32),
                                          tol=1e-6, max_iter=50)
    assert info["status"] == "OK", info
    assert info["rho"] <= 1e-6
    pick = np.array([0, 9, 21, 33, 40, 51, 58, 63])
    ref = oracle.ipt_solve_csr(rowptr, colind, vals, n, cols=cols[pick], tol=1e-12,
                               max_iter=100)
    assert ref["status"] == oracle.OK
    assert np.max(np.abs(lam.cpu().numpy()[pick] - ref["lam"]) / np.abs(ref["lam"])) <= 1e-5
    Zs = Z[:, torch.as_tensor(pick, device="cuda")].double().cpu().numpy()
    E = oracle.unit_columns(n, cols[pick])
    err = np.linalg.norm(Zs - ref["Z"]) / np.linalg.norm(ref["Z"] - E)
    assert err <= 1e-4, err


def _random_pattern_csr(n, per_row, scale, seed):
    """Symmetric CSR with off-diagonal entries at uniformly random columns (no band)."""
    g = w.rng(seed)
    rows = np.repeat(np.arange(n), per_row)
    cols = g.integers(0, n, size=n * per_row)
    keep = rows != cols
    rows, cols = rows[keep], cols[keep]
    a = np.zeros((n, n))
    a[rows, cols] = g.standard_normal(rows.size) * scale
    a = np.triu(a, 1)
    a = a + a.T
    th = np.arange(1, n + 1) * 0.1
    a[np.arange(n), np.arange(n)] = th
    r, c = np.nonzero(a)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    return np.cumsum(rowptr).astype(np.int32), c.astype(np.int32), a[r, c], th


@pytest.mark.parametrize("precision,vdt", [("f32", torch.float32), ("f64", torch.float64)])
@pytest.mark.parametrize("case", ["banded_low", "banded_middle", "random_pattern", "tridiagonal"])
def test_csr_active_window_equals_all_rows(ipt, precision, vdt, case):
    """The active window (rows of the current iterate's support widened by the band)
    evaluates exactly the rows that can be nonzero: the same iterates, bit for bit,
    as evaluating every row."""
    n = 6000
    if case == "random_pattern":
        rowptr, colind, vals, th = _random_pattern_csr(n, 2, 1e-2, seed=12)
    elif case == "tridiagonal":
        i = np.arange(n)
        rows = np.concatenate([i, i[:-1], i[1:]])
        cc = np.concatenate([i, i[1:], i[:-1]])
        vv = np.concatenate([i + 1.0, np.full(n - 1, 0.3), np.full(n - 1, 0.3)])
        order = np.lexsort((cc, rows))
        rowptr = np.zeros(n + 1, dtype=np.int64)
        np.add.at(rowptr, rows[order] + 1, 1)
        rowptr, colind, vals, th = (np.cumsum(rowptr).astype(np.int32),
                                    cc[order].astype(np.int32), vv[order], i + 1.0)
    else:
        rowptr, colind, vals, th = w.csr_banded(n, 4, 100, 1e-3, seed=13, theta_step=0.05)
    k = 16
    if case == "banded_middle":
        cols = np.arange(3000, 3000 + k, dtype=np.int32)[::-1].copy()
    else:
        cols = w.lowest_columns(th, k)
    rp, ci, vv = csr_on_gpu(rowptr, colind, vals, vdt)
    cg = cuda(cols, torch.int32)
    out = {}
    for win in [True, False]:
        for it in [1, 2, 6]:
            lam, Z, info = ipt.Solver().solve_csr(rp, ci, vv, n, cols=cg, tol=0.0, max_iter=it,
                                                  precision=precision, stop="increment",
                                                  window=win, z_dtype=torch.float64)
            assert info["status"] == "MAXITER", info
            out[(win, it)] = (lam.cpu().numpy(), Z.cpu().numpy(), info["hist_increment"])
    for it in [1, 2, 6]:
        a, b = out[(True, it)], out[(False, it)]
        assert np.array_equal(a[1], b[1]), it
        assert np.array_equal(a[0], b[0])
        np.testing.assert_allclose(a[2], b[2], rtol=1e-12)
    # the window result also matches the oracle's iterate
    ref = oracle.ipt_solve_csr(rowptr, colind, vals, n, cols=cols, tol=0.0, max_iter=6,
                               stop="increment")
    E = oracle.unit_columns(n, cols)
    err = np.linalg.norm(out[(True, 6)][1] - ref["Z"]) / np.linalg.norm(ref["Z"] - E)
    assert err <= (1e-10 if precision == "f64" else 1e-4), err


def test_csr_handle_reuse_across_problems_and_dense(ipt):
    """One handle, several problems: the sparse path clears only the rows an
    earlier solve wrote, so results must not depend on what ran before."""
    n = 5000
    rowptr, colind, vals, th = w.csr_banded(n, 4, 60, 1e-3, seed=14, theta_step=0.05)
    rp, ci, vv = csr_on_gpu(rowptr, colind, vals)
    ca = cuda(np.arange(10, 30, dtype=np.int32), torch.int32)
    cb = cuda(np.arange(4000, 4012, dtype=np.int32), torch.int32)
    fresh = {}
    for name, cg in [("a", ca), ("b", cb)]:
        lam, Z, info = ipt.Solver().solve_csr(rp, ci, vv, n, cols=cg, tol=1e-6, max_iter=40)
        assert info["status"] == "OK"
        fresh[name] = Z.cpu().numpy()
    s = ipt.Solver()
    M, thd = w.dense_symmetric(512, 1e-3, seed=2, theta_step=0.5)
    for name, cg in [("a", ca), ("b", cb), ("a", ca), ("dense", None), ("b", cb),
                     ("window-off", None), ("a", ca)]:
        if name == "dense":
            s.solve_dense(cuda(M, torch.float32), theta=cuda(thd, torch.float64), tol=1e-6,
                          max_iter=30)
            continue
        if name == "window-off":
            s.solve_csr(rp, ci, vv, n, cols=cb, tol=1e-6, max_iter=40, window=False)
            continue
        lam, Z, info = s.solve_csr(rp, ci, vv, n, cols=cg, tol=1e-6, max_iter=40)
        assert info["status"] == "OK"
        assert np.array_equal(Z.cpu().numpy(), fresh[name]), name


@pytest.mark.parametrize("band,k,vdt", [(300, 64, torch.float32), (2048, 37, torch.float32),
                                        (2048, 64, torch.float64), (2600, 64, torch.float32)])
def test_csr_all_rows_equals_active_window_at_scale(ipt, band, k, vdt):
    """n = 40000 with bands up to 2600 and padded column chunks (k = 37): every row
    evaluated and the active window (a few thousand rows) sum the stored entries
    in the same order, so the iterates are identical; sampled columns match the
    oracle."""
    n = 40000
    rowptr, colind, vals, th = w.csr_banded(n, 6, band, 1e-3, seed=17, theta_step=0.01)
    cols = w.lowest_columns(th, k)
    rp = cuda(rowptr, torch.int32)
    ci = cuda(colind, torch.int32)
    vv = cuda(vals, vdt)
    cg = cuda(cols, torch.int32)
    s = ipt.Solver()
    lam_a, Z_a, ia = s.solve_csr(rp, ci, vv, n, cols=cg, tol=1e-6, max_iter=60, window=False)
    lam_w, Z_w, iw = s.solve_csr(rp, ci, vv, n, cols=cg, tol=1e-6, max_iter=60, window=True)
    assert ia["status"] == "OK" and iw["status"] == "OK", (ia, iw)
    assert ia["iterations"] == iw["iterations"]
    assert ia["rows_evaluated"] == ia["iterations"] * n
    assert torch.equal(Z_a, Z_w) and torch.equal(lam_a, lam_w)
    pick = np.array([0, 5, k // 2, k - 1])
    ref = oracle.ipt_solve_csr(rowptr, colind, vals, n, cols=cols[pick], tol=1e-12, max_iter=100)
    assert ref["status"] == oracle.OK
    np.testing.assert_allclose(lam_a.cpu().numpy()[pick], ref["lam"], rtol=1e-5)
    Zs = Z_a[:, torch.as_tensor(pick, device="cuda")].double().cpu().numpy()
    E = oracle.unit_columns(n, cols[pick])
    assert np.linalg.norm(Zs - ref["Z"]) / np.linalg.norm(ref["Z"] - E) <= 1e-4


@pytest.mark.parametrize("window,vdt", [(True, torch.float32), (False, torch.float32),
                                        (True, torch.float64)])
def test_csr_verify_fp64_matches_oracle_residual(ipt, window, vdt):
    """The sparse solve's FP64 verification (rho_fp64 * r0) equals the oracle's
    ||M Z - Z Lambda||_F (M from the CSR arrays, the values as the GPU sees them)
    on the GPU's own result, within both FP64 evaluations' rounding bounds."""
    sp = pytest.importorskip("scipy.sparse")
    n, k = 20000, 24
    rowptr, colind, vals, th = w.csr_banded(n, 6, 400, 1e-3, seed=21, theta_step=0.01)
    cols = w.lowest_columns(th, k)
    rp, ci, vv = csr_on_gpu(rowptr, colind, vals, vdt)
    lam, Z, info = ipt.Solver().solve_csr(rp, ci, vv, n, cols=cuda(cols, torch.int32),
                                          tol=1e-6, max_iter=40, window=window,
                                          verify_fp64=True)
    assert info["status"] == "OK", info
    v64 = vv.double().cpu().numpy()
    M = sp.csr_matrix((v64, colind, rowptr), shape=(n, n))
    Zh, lh = Z.double().cpu().numpy(), lam.cpu().numpy()
    ref = np.linalg.norm(M @ Zh - Zh * lh[None, :])
    u = 2.0 ** -53
    Ma = sp.csr_matrix((np.abs(v64), colind, rowptr), shape=(n, n))
    row_len = np.diff(rowptr).max() + 1
    bound = 2 * row_len * u * np.linalg.norm(Ma @ np.abs(Zh) + np.abs(Zh) * np.abs(lh)[None, :])
    got = info["rho_fp64"] * info["r0"]
    assert info["rho_fp64"] >= 0 and abs(got - ref) <= bound + 1e-12 * ref, (got, ref, bound)
    assert info["rho_fp64"] <= 1e-6
