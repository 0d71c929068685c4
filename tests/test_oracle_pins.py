"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed
forms (Section 4.3), textbook perturbation theory (App. B), the paper's
printed 3x3 multiplier polynomials (App. D.3, fixture in tests/golden/),
LAPACK and a brute-force Jacobi eigensolver, the convergence theorem of
Section 4.1, and invariants of the map.  Chosen so that a dropped term, a
wrong sign or index of G, or a transposed operand fails at least one.
"""

import os

import numpy as np
import pytest

import oracle
from paper_2012_14702_gb300 import workloads as w

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers
def jacobi_eigh(A, tol=1e-15, max_sweeps=50):
    """Cyclic Jacobi eigensolver for a symmetric matrix (textbook brute force)."""
    A = np.array(A, dtype=np.float64, copy=True)
    n = len(A)
    V = np.eye(n)
    for _ in range(max_sweeps):
        off = np.linalg.norm(A - np.diag(np.diag(A)))
        if off <= tol * np.linalg.norm(A):
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                if A[p, q] == 0.0:
                    continue
                th = (A[q, q] - A[p, p]) / (2.0 * A[p, q])
                t = np.sign(th) / (abs(th) + np.sqrt(th * th + 1.0)) if th != 0 else 1.0
                c = 1.0 / np.sqrt(t * t + 1.0)
                s = t * c
                cp, cq = A[:, p].copy(), A[:, q].copy()
                A[:, p], A[:, q] = c * cp - s * cq, s * cp + c * cq
                rp, rq = A[p, :].copy(), A[q, :].copy()
                A[p, :], A[q, :] = c * rp - s * rq, s * rp + c * rq
                vp, vq = V[:, p].copy(), V[:, q].copy()
                V[:, p], V[:, q] = c * vp - s * vq, s * vp + c * vq
    return np.diag(A).copy(), V


def match_eigvecs(V, cols):
    """For each requested index i_c, the eigenvector with the largest |V[i_c, :]|, scaled so z_{i_c} = 1."""
    Z = np.zeros((V.shape[0], len(cols)), dtype=V.dtype)
    idx = []
    for c, i in enumerate(cols):
        j = int(np.argmax(np.abs(V[i, :])))
        idx.append(j)
        Z[:, c] = V[:, j] / V[i, j]
    return Z, np.array(idx)


def load_polys():
    terms = {}
    with open(os.path.join(GOLDEN, "app_d3_multiplier_polynomials.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            z, c, a, b = line.split()
            terms.setdefault(z, []).append((int(c), int(a), int(b)))
    return terms


# ---------------------------------------------------------------- 2 x 2 closed form (Section 4.3)
@pytest.mark.parametrize("eps", [0.1, 0.3, 0.6, -0.45])
def test_2x2_iterates_match_closed_form(eps):
    """Z^(k) = [[1, -f^k(0)], [f^k(0), 1]] with f(x) = eps (x^2 - 1), Eq. (2by2)."""
    M, th = w.two_by_two(eps)
    Delta, th = oracle.partition(M, th)
    cols = np.arange(2)
    Z = np.eye(2)
    x = 0.0
    for _ in range(12):
        Z, _, _ = oracle.ipt_map(Delta, th, cols, Z)
        x = eps * (x * x - 1.0)
        np.testing.assert_allclose(Z, [[1.0, -x], [x, 1.0]], rtol=0, atol=1e-15)


@pytest.mark.parametrize("eps", [0.05, 0.3, 0.7, -0.8])
def test_2x2_eigenvalues_closed_form(eps):
    """Column 0 converges to lambda_- and column 1 to lambda_+ = (1 +- sqrt(1+4 eps^2))/2."""
    M, th = w.two_by_two(eps)
    r = oracle.ipt_solve(M, th, tol=1e-14, max_iter=5000)
    assert r["status"] == oracle.OK
    s = np.sqrt(1.0 + 4.0 * eps * eps)
    np.testing.assert_allclose(r["lam"], [(1 - s) / 2, (1 + s) / 2], rtol=0, atol=1e-12)


def test_2x2_flip_bifurcation():
    """Stable below |eps| = sqrt(3)/2, a 2-cycle above it; diverges far outside (Section 4.3)."""
    for eps, status in [(0.85, oracle.OK), (-0.85, oracle.OK), (0.87, oracle.MAXITER),
                        (-0.87, oracle.MAXITER), (3.0, oracle.DIVERGED)]:
        M, th = w.two_by_two(eps)
        r = oracle.ipt_solve(M, th, tol=1e-12, max_iter=4000)
        assert r["status"] == status, (eps, r["status"])
    # the 2-cycle: two successive iterates alternate
    M, th = w.two_by_two(0.87)
    Delta, th = oracle.partition(M, th)
    Z = np.eye(2)
    for _ in range(4000):
        Z, _, _ = oracle.ipt_map(Delta, th, np.arange(2), Z)
    Z1, _, _ = oracle.ipt_map(Delta, th, np.arange(2), Z)
    Z2, _, _ = oracle.ipt_map(Delta, th, np.arange(2), Z1)
    assert abs(Z1[1, 0] - Z[1, 0]) > 1e-2 and abs(Z2[1, 0] - Z[1, 0]) < 1e-8


# ---------------------------------------------------------------- 3 x 3 example (App. D.3)
@pytest.mark.parametrize("eps", [0.1, 0.3, -0.2])
@pytest.mark.parametrize("col", [0, 1, 2])
def test_3x3_multipliers_are_roots_of_printed_polynomials(eps, col):
    """The multipliers of the converged fixed point of f_i are zeros of the printed P(eps, mu)."""
    terms = load_polys()["z%d" % (col + 1)]
    M, th = w.three_by_three(eps)
    Delta, th = oracle.partition(M, th)
    r = oracle.ipt_solve(M, th, cols=[col], tol=1e-15, max_iter=5000)
    assert r["status"] == oracle.OK
    J = oracle.chart_jacobian(Delta, th, col, r["Z"][:, 0])
    for mu in np.linalg.eigvals(J):
        vals = [c * eps ** a * mu ** b for c, a, b in terms]
        assert abs(sum(vals)) <= 1e-12 * sum(abs(v) for v in vals)
    # the converged point is an eigenvector of M (intermediate normalisation)
    lam = r["lam"][0]
    z = r["Z"][:, 0]
    assert np.linalg.norm(M @ z - lam * z) < 1e-12


def test_3x3_z2_loses_stability_near_minus_049():
    """App. D.3: the z_2 fixed point continued from eps = 0 loses stability at eps ~ -0.49
    through a complex-conjugate pair of multipliers (Neimark-Sacker)."""
    def multipliers(eps):
        M, th = w.three_by_three(eps)
        Delta, _ = oracle.partition(M, th)
        ev, V = np.linalg.eig(M)
        j = int(np.argmax(np.abs(V[1, :])))
        z = (V[:, j] / V[1, j]).real
        return np.linalg.eigvals(oracle.chart_jacobian(Delta, th, 1, z))
    assert max(abs(multipliers(-0.45))) < 1.0
    assert max(abs(multipliers(-0.48))) < 1.0
    mu = multipliers(-0.50)
    assert max(abs(mu)) > 1.0
    assert abs(mu[0].imag) > 1e-3 and abs(mu[0] - np.conj(mu[1])) < 1e-12


# ---------------------------------------------------------------- textbook perturbation theory
def test_first_iterate_is_first_order_rs():
    """F(I) = I - G o Delta: the first-order RS eigenvector correction
    z_j = Delta_ji / (theta_i - theta_j); the second evaluation's eigenvalue is
    the second-order RS energy theta_i + Delta_ii + sum_j Delta_ij Delta_ji / (theta_i - theta_j)."""
    g = w.rng(5)
    n = 9
    th = np.sort(g.random(n) * 10)
    Delta = g.standard_normal((n, n)) * 0.05  # non-symmetric, non-zero diagonal
    M = np.diag(th) + Delta
    cols = np.arange(n)
    F, _, d = oracle.ipt_map(Delta, th, cols, np.eye(n))
    for i in range(n):
        for j in range(n):
            want = 1.0 if i == j else Delta[j, i] / (th[i] - th[j])
            assert abs(F[j, i] - want) < 1e-15
        assert abs(th[i] + d[i] - (th[i] + Delta[i, i])) < 1e-15  # first-order energy
    r = oracle.ipt_solve(M, th, tol=0.0, max_iter=2)
    assert r["status"] == oracle.MAXITER and r["iterations"] == 2
    for i in range(n):
        e2 = th[i] + Delta[i, i] + sum(Delta[i, j] * Delta[j, i] / (th[i] - th[j])
                                       for j in range(n) if j != i)
        assert abs(r["lam"][i] - e2) < 1e-13


def test_rs_corrections_sum_to_lapack_eigenvalues():
    """Eigenvalue corrections lambda^[l] = D(Delta Z^[l-1]) of App. B sum to the exact
    eigenvalues with an O(eps^(K+1)) remainder."""
    g = w.rng(7)
    n = 6
    th = np.arange(n, dtype=float)
    D0 = g.standard_normal((n, n))
    D0 = D0 + D0.T
    np.fill_diagonal(D0, 0.0)
    K = 4
    Zs = oracle.rs_corrections(D0, th, K)
    errs = []
    for eps in [0.02, 0.01]:
        lam = th.copy()
        for l in range(1, K + 1):
            lam = lam + eps ** l * np.diag(D0 @ Zs[l - 1])
        exact = np.linalg.eigvalsh(np.diag(th) + eps * D0)
        errs.append(np.max(np.abs(np.sort(lam) - exact)))
    slope = np.log2(errs[0] / errs[1])
    assert K + 0.6 < slope < K + 1.6, slope


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_ipt_contains_rs_series(k):
    """Z^(k) = sum_{l<=k} eps^l Z^[l] + O(eps^(k+1)) (Section 4.2, App. C).

    For k = 1 both sides are I - eps G o Delta exactly."""
    g = w.rng(11)
    n = 7
    th = np.arange(n, dtype=float) * 1.3
    D0 = g.standard_normal((n, n))  # non-symmetric on purpose
    np.fill_diagonal(D0, 0.0)
    Zs = oracle.rs_corrections(D0, th, k)
    errs = []
    for eps in [0.01, 0.005, 0.0025]:
        Delta = eps * D0
        Z = np.eye(n)
        for _ in range(k):
            Z, _, _ = oracle.ipt_map(Delta, th, np.arange(n), Z)
        rs = sum(eps ** l * Zs[l] for l in range(k + 1))
        errs.append(np.max(np.abs(Z - rs)))
    if k == 1:
        assert max(errs) < 1e-16
        return
    s1, s2 = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    assert k + 0.7 < s1 < k + 1.3 and k + 0.7 < s2 < k + 1.3, (s1, s2)


# ---------------------------------------------------------------- fixed points vs eigensolvers
@pytest.mark.parametrize("n", [8, 24, 64])
def test_fixed_point_matches_jacobi_bruteforce(n):
    M, th = w.dense_symmetric(n, 0.02, seed=100 + n)
    r = oracle.ipt_solve(M, th, tol=1e-14, max_iter=500)
    assert r["status"] == oracle.OK
    ev, V = jacobi_eigh(M)
    Zj, idx = match_eigvecs(V, np.arange(n))
    assert len(set(idx.tolist())) == n
    np.testing.assert_allclose(r["lam"], ev[idx], rtol=1e-13, atol=0)
    np.testing.assert_allclose(r["Z"], Zj, rtol=0, atol=1e-11)


def test_jacobi_helper_agrees_with_lapack():
    M, _ = w.dense_symmetric(20, 0.3, seed=3)
    ev, V = jacobi_eigh(M)
    np.testing.assert_allclose(np.sort(ev), np.linalg.eigvalsh(M), atol=1e-12)
    np.testing.assert_allclose(V.T @ V, np.eye(20), atol=1e-12)


def test_nonsymmetric_paper_family_matches_lapack_eig():
    """Eq. (dense_matrix) with eps = 1e-2 (non-symmetric, U[0,1] entries): IPT = eig."""
    M, th = w.dense_paper(120, 1e-2, seed=9)
    r = oracle.ipt_solve(M, th, tol=1e-13, max_iter=500)
    assert r["status"] == oracle.OK
    ev, V = np.linalg.eig(M)
    Zl, idx = match_eigvecs(V, np.arange(120))
    assert np.max(np.abs(ev.imag)) < 1e-12
    np.testing.assert_allclose(r["lam"], ev[idx].real, rtol=1e-12)
    np.testing.assert_allclose(r["Z"], Zl.real, atol=1e-10)


def test_partial_spectrum_with_permuted_columns():
    """Columns are independent (Alg. 1 per column): any column subset, any order."""
    M, th = w.dense_symmetric(40, 0.03, seed=4)
    cols = np.array([17, 3, 29, 0])
    r = oracle.ipt_solve(M, th, cols=cols, tol=1e-14, max_iter=500)
    assert r["status"] == oracle.OK
    ev, V = np.linalg.eigh(M)
    Zl, idx = match_eigvecs(V, cols)
    np.testing.assert_allclose(r["lam"], ev[idx], rtol=1e-13)
    np.testing.assert_allclose(r["Z"], Zl, atol=1e-11)
    full = oracle.ipt_solve(M, th, tol=1e-14, max_iter=500)
    np.testing.assert_allclose(r["Z"], full["Z"][:, cols], atol=1e-12)


# ---------------------------------------------------------------- convergence theorem (Section 4.1)
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_theorem_condition_implies_convergence_in_ball(seed):
    """||G|| ||Delta|| < 3 - 2 sqrt(2): convergence from I to a full-rank Z* in B_sqrt2(I)."""
    g = w.rng(seed)
    n = 30
    th = np.sort(g.random(n)) * n
    D0 = g.standard_normal((n, n))
    np.fill_diagonal(D0, 0.0)
    G = oracle.inverse_gaps(th, np.arange(n))
    scale = 0.16 / (np.linalg.norm(G, 2) * np.linalg.norm(D0, 2))
    Delta = scale * D0
    assert np.linalg.norm(G, 2) * np.linalg.norm(Delta, 2) < 3 - 2 * np.sqrt(2)
    r = oracle.ipt_solve(np.diag(th) + Delta, th, tol=1e-14, max_iter=2000)
    assert r["status"] == oracle.OK
    Zs = r["Z"]
    assert np.linalg.norm(Zs - np.eye(n), 2) <= np.sqrt(2)
    assert np.linalg.svd(Zs, compute_uv=False)[-1] > 1e-3


# ---------------------------------------------------------------- invariants and special cases
def test_diagonal_matrix_is_fixed_at_identity():
    th = np.array([3.0, -1.0, 2.5, 7.0])
    r = oracle.ipt_solve(np.diag(th), th, tol=1e-12)
    assert r["status"] == oracle.OK and r["iterations"] == 1
    np.testing.assert_array_equal(r["Z"], np.eye(4))
    np.testing.assert_array_equal(r["lam"], th)
    assert r["rho"] == 0.0


def test_intermediate_normalisation_and_residual_identity():
    """Z_{i_c, c} = 1 on every iterate, and for any such Z:
    (M Z - Z Lambda)_jc = (theta_j - theta_{i_c}) (Z - F(Z))_jc, j != i_c."""
    M, th = w.dense_symmetric(30, 0.05, seed=8)
    Delta, th = oracle.partition(M, th)
    cols = np.array([4, 11, 20])
    g = w.rng(8)
    Z = g.standard_normal((30, 3)) * 0.1
    Z[cols, np.arange(3)] = 1.0
    F, P, d = oracle.ipt_map(Delta, th, cols, Z)
    assert np.all(F[cols, np.arange(3)] == 1.0)
    lam = th[cols] + d
    R = oracle.residual(M, Z, lam)
    ident = (th[:, None] - th[cols][None, :]) * (Z - F)
    np.testing.assert_allclose(R, ident, atol=1e-15)
    assert np.all(np.abs(R[cols, np.arange(3)]) < 1e-15)


def test_rho_definition():
    M, th = w.dense_symmetric(50, 0.01, seed=2)
    r = oracle.ipt_solve(M, th, tol=0.0, max_iter=1)
    assert r["iterations"] == 1 and abs(r["rho"] - 1.0) < 1e-15
    Delta, _ = oracle.partition(M, th)
    r = oracle.ipt_solve(M, th, tol=1e-13, max_iter=100)
    R = oracle.residual(M, r["Z"], r["lam"])
    off = Delta - np.diag(np.diag(Delta))
    assert abs(r["rho"] - np.linalg.norm(R) / np.linalg.norm(off)) < 1e-12


def test_argument_errors():
    th = np.array([1.0, 2.0, 2.0, 4.0])
    M = np.diag(th) + 0.01
    assert oracle.ipt_solve(M, th)["status"] == oracle.DEGENERATE_THETA
    assert oracle.ipt_solve(M, th, cols=[0, 3])["status"] == oracle.OK
    assert oracle.ipt_solve(M, th, cols=[0, 0])["status"] == oracle.INVALID_ARG
    assert oracle.ipt_solve(M, th, cols=[])["status"] == oracle.INVALID_ARG
    assert oracle.ipt_solve(M, th, cols=[0], max_iter=0)["status"] == oracle.INVALID_ARG
    assert oracle.ipt_solve(M, np.array([1.0, np.nan, 3, 4]), cols=[0])["status"] == oracle.DEGENERATE_THETA
    Mn = M.copy()
    Mn[0, 3] = np.nan
    assert oracle.ipt_solve(Mn, th, cols=[3])["status"] == oracle.DIVERGED


# ---------------------------------------------------------------- sparse oracle and paper workloads
def test_csr_oracle_equals_dense_oracle():
    rowptr, colind, vals, th = w.csr_banded(400, 4, 30, 1e-2, seed=5, theta_step=0.1)
    import scipy.sparse as sp
    M = sp.csr_matrix((vals, colind, rowptr), shape=(400, 400)).toarray()
    assert np.allclose(M, M.T) and np.array_equal(np.diag(M), th)
    Ms = sp.csr_matrix(M)
    cols = w.lowest_columns(th, 8)
    rs = oracle.ipt_solve_csr(Ms.indptr, Ms.indices, Ms.data, 400, cols=cols, tol=1e-13)
    rd = oracle.ipt_solve(M, th, cols=cols, tol=1e-13)
    assert rs["status"] == rd["status"] == oracle.OK
    assert rs["iterations"] == rd["iterations"]
    np.testing.assert_allclose(rs["Z"], rd["Z"], atol=1e-14)
    np.testing.assert_allclose(rs["lam"], rd["lam"], rtol=1e-14)


def test_csr_generator_structure():
    n, per_row, band = 3000, 8, 64
    rowptr, colind, vals, th = w.csr_banded(n, per_row, band, 1e-3, seed=3)
    nnz = len(colind)
    assert rowptr[0] == 0 and rowptr[-1] == nnz
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    assert np.all(np.abs(colind - rows) <= band)
    on_diag = colind == rows
    assert on_diag.sum() == n and np.array_equal(vals[on_diag], th)
    assert 2 * per_row * n - 2 * band * per_row <= nnz - n <= 2 * per_row * n
    for i in range(0, n, 97):
        seg = colind[rowptr[i]:rowptr[i + 1]]
        assert np.all(np.diff(seg) > 0)
    assert np.all(np.diff(th) > 0)


def test_morgan_tridiagonal_threshold_qualitative():
    """Section 6.1: IPT converges for small off-diagonal eps and stops converging beyond ~0.5."""
    M, th = w.morgan_tridiagonal(400, 0.3)
    assert oracle.ipt_solve(M, th, cols=[0], tol=1e-10, max_iter=2000)["status"] == oracle.OK
    M, th = w.morgan_tridiagonal(400, 1.0)
    assert oracle.ipt_solve(M, th, cols=[0], tol=1e-10, max_iter=2000)["status"] != oracle.OK


# ------------------------------------------------------------------ ACX (Alg. 3)
@pytest.mark.parametrize("order", [2, 3])
def test_acx_solves_columnwise_affine_maps_in_one_extrapolation(order):
    """For a contraction f(x) = a x + b (a < 1, a scalar per column) the
    differences are D^q = (a - 1)^q (x - x*), the step is s = 1/(1 - a), and the
    order-p update of Alg. 3 (with the z term and the squared norm, reading 8)
    lands exactly on x* = b / (1 - a).  A dropped term, a wrong coefficient, a
    sign or an unsquared norm all miss x*."""
    g = np.random.default_rng(3)
    n, k = 40, 5
    a = np.array([0.9, -0.7, 0.3, 0.55, -0.2])
    b = g.standard_normal((n, k))
    x = g.standard_normal((n, k))
    f = lambda y: a[None, :] * y + b
    fs = [f(x)]
    for _ in range(order - 1):
        fs.append(f(fs[-1]))
    z = oracle.acx_update(x, fs, per_column=True)
    np.testing.assert_allclose(z, b / (1.0 - a[None, :]), rtol=1e-12, atol=1e-12)
    # one step length for the whole block is exact only when the factors agree
    z_glob = oracle.acx_update(x, fs, per_column=False)
    assert np.max(np.abs(z_glob - b / (1.0 - a[None, :]))) > 1e-3
    same = lambda y: 0.4 * y + b
    fs2 = [same(x)]
    for _ in range(order - 1):
        fs2.append(same(fs2[-1]))
    np.testing.assert_allclose(oracle.acx_update(x, fs2, per_column=False), b / 0.6,
                               rtol=1e-12, atol=1e-12)


def test_acx_differences_are_binomial_and_sigma_degenerate_column():
    """D^q are the forward differences of z, f(z), f^2(z), f^3(z); a column with
    D^p = 0 takes s = 1, so the update there is the plain iterate f^p(z)."""
    g = np.random.default_rng(4)
    z, f1, f2, f3 = (g.standard_normal((6, 3)) for _ in range(4))
    D = oracle.acx_differences(z, [f1, f2, f3])
    np.testing.assert_allclose(D[0], f1 - z)
    np.testing.assert_allclose(D[1], (f2 - f1) - (f1 - z))
    np.testing.assert_allclose(D[2], ((f3 - f2) - (f2 - f1)) - ((f2 - f1) - (f1 - z)))
    # column 0 sits at a fixed point (D^1 = D^2 = 0): s = 1 and z stays; column 1
    # moves by a constant (D^1 != 0, D^2 = 0): s = 1 and z -> f^2(z)
    zz = np.zeros((4, 2))
    c = np.ones(4)
    fs = [np.stack([c, c], 1), np.stack([c, 2 * c], 1)]
    zz[:, 0] = 1.0
    out = oracle.acx_update(zz, fs, per_column=True)
    np.testing.assert_allclose(out[:, 0], c)
    np.testing.assert_allclose(out[:, 1], 2 * c)


def test_acx_keeps_unit_entries_and_matches_plain_fixed_point():
    """f_i(z)_i = 1 for every z, so every difference vanishes at the unit entry
    and IPT-ACX keeps Z_{i_c, c} = 1 exactly; it converges to the same eigenpairs
    as the Picard iteration and LAPACK."""
    M, th = w.dense_symmetric(120, 0.01, seed=5, theta_step=0.5)
    cols = np.array([3, 50, 7, 99])
    r = oracle.ipt_solve_acx(M, th, cols=cols, tol=1e-13, max_iter=200)
    assert r["status"] == oracle.OK
    assert np.all(r["Z"][cols, np.arange(len(cols))] == 1.0)
    p = oracle.ipt_solve(M, th, cols=cols, tol=1e-13, max_iter=200)
    np.testing.assert_allclose(r["lam"], p["lam"], rtol=1e-12)
    np.testing.assert_allclose(r["Z"], p["Z"], atol=1e-11)
    ev, V = np.linalg.eigh(M)
    for c, i in enumerate(cols):
        j = np.argmin(np.abs(ev - r["lam"][c]))
        np.testing.assert_allclose(r["Z"][:, c], V[:, j] / V[i, j], atol=1e-10)


def test_acx_morgan_tridiagonal_domain_and_matvecs():
    """Section 5 / Fig. (morgan): on the tridiagonal M_ii = i, M_{i,i+-1} = eps,
    IPT-ACX needs far fewer matvecs than IPT at eps = 0.5, and converges where IPT
    no longer does (eps = 1, 5; IPT stops converging beyond eps ~ 0.5), to the
    lowest eigenpair."""
    n = 600
    M, th = w.morgan_tridiagonal(n, 0.5)
    plain = oracle.ipt_solve(M, th, cols=[0], tol=1e-10, max_iter=400)
    acx = oracle.ipt_solve_acx(M, th, cols=[0], tol=1e-10, max_iter=400)
    assert plain["status"] == acx["status"] == oracle.OK
    assert acx["iterations"] * 2 < plain["iterations"]
    ev = np.linalg.eigvalsh(M)[0]
    assert abs(acx["lam"][0] - ev) < 1e-9 and abs(plain["lam"][0] - ev) < 1e-9
    for eps in [1.0, 5.0]:
        M, th = w.morgan_tridiagonal(n, eps)
        plain = oracle.ipt_solve(M, th, cols=[0], tol=1e-10, max_iter=400)
        acx = oracle.ipt_solve_acx(M, th, cols=[0], tol=1e-10, max_iter=400)
        assert plain["status"] in (oracle.DIVERGED, oracle.MAXITER)
        assert acx["status"] == oracle.OK, (eps, acx["status"], acx["iterations"])
        assert abs(acx["lam"][0] - np.linalg.eigvalsh(M)[0]) < 1e-8 * max(1.0, eps)


@pytest.mark.parametrize("sigma", ["column", "global"])
def test_acx_full_spectrum_beyond_picard_domain(sigma):
    """Dense full spectrum at a perturbation where the Picard iteration no longer
    converges (n = 256, theta_i = i/8, Delta N(0,1)*0.03): IPT-ACX converges to
    all eigenvalues of LAPACK's eigvalsh."""
    M, th = w.dense_symmetric(256, 0.03, seed=7, theta_step=0.125)
    plain = oracle.ipt_solve(M, th, tol=1e-9, max_iter=150, stop="residual")
    assert plain["status"] == oracle.MAXITER
    r = oracle.ipt_solve_acx(M, th, tol=1e-9, max_iter=300, stop="residual", sigma=sigma)
    assert r["status"] == oracle.OK
    np.testing.assert_allclose(np.sort(r["lam"]), np.linalg.eigvalsh(M), atol=1e-9)


# ------------------------------------------------------------------ learned damping model
def test_damping_model_gradient_matches_finite_differences():
    """The backward pass of the damping perceptron against central differences of
    its own forward pass in float64 (the FP16 parameters perturbed in float64)."""
    from oracle import damping as dm
    g = np.random.default_rng(5)
    p16 = dm.init_params(3)
    X = g.standard_normal((40, 6))
    t = g.uniform(0.1, 1.9, 40)
    _, grad = dm.loss_and_grad(p16, X, t)
    base = p16.astype(np.float64)

    def loss_at(flat64):
        pp = dm.unpack(flat64)
        h1 = np.tanh(X @ pp["W1"] + pp["b1"])
        h2 = np.tanh(h1 @ pp["W2"] + pp["b2"])
        y = (h2 @ pp["W3"] + pp["b3"])[:, 0]
        a = 2.0 / (1.0 + np.exp(-y))
        return np.mean((a - t) ** 2)

    idx = g.choice(dm.N_PARAMS, 60, replace=False)
    for i in idx:
        e = np.zeros(dm.N_PARAMS)
        e[i] = 1e-6
        fd = (loss_at(base + e) - loss_at(base - e)) / 2e-6
        assert abs(fd - grad[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, grad[i])


def test_damping_features_and_secant_step():
    """Features of geometric histories, and the secant damping alpha* = 1/(1 - a)
    of a contraction f(x) = a x + b (which makes one damped step exact)."""
    from oracle import damping as dm
    a = 0.5
    inc = np.array([[1.0], [a], [a * a]])
    lam = np.array([[1.0], [1.0 + 0.1], [1.0 + 0.1 - 0.05]])
    X = dm.features(inc, lam)
    np.testing.assert_allclose(X[0, :3], [np.log10(a * a), np.log10(a), np.log10(a)],
                               atol=1e-12)
    np.testing.assert_allclose(X[0, 3], -0.5, atol=1e-12)  # (l0 - l1) / (l1 - l2)
    g = np.random.default_rng(6)
    for av in [0.9, -0.8, 0.2, -2.5]:
        b = g.standard_normal((7, 1))
        x = g.standard_normal((7, 1))
        f = lambda y: av * y + b
        D1 = f(x) - x
        D2 = f(f(x)) - 2 * f(x) + x
        alpha = dm.secant_alpha(D1, D2, lo=-1e9, hi=1e9)[0]
        np.testing.assert_allclose(alpha, 1.0 / (1.0 - av), rtol=1e-12)
        np.testing.assert_allclose(x + alpha * D1, b / (1.0 - av), atol=1e-12)


def test_damped_solve_with_unit_damping_is_picard():
    """alpha = 1 everywhere gives exactly the Picard iteration of Alg. 2."""
    from oracle import damping as dm
    M, th = w.dense_symmetric(90, 0.01, seed=8, theta_step=0.5)
    a = dm.damped_solve(M, th, tol=1e-12, max_iter=60, alpha_fn=lambda X: np.ones(len(X)))
    b = oracle.ipt_solve(M, th, tol=1e-12, max_iter=60, stop="residual")
    assert a["status"] == b["status"] == oracle.OK and a["iterations"] == b["iterations"]
    np.testing.assert_array_equal(a["Z"], b["Z"])


def test_damped_solve_secant_rule_extends_domain():
    """Damping each column by 1 / (1 - q) (q the Rayleigh-quotient change ratio,
    the secant rule the model is trained to imitate) converges on a matrix where
    the Picard iteration does not, to LAPACK's eigenvalues."""
    from oracle import damping as dm
    M, th = w.dense_symmetric(256, 0.03, seed=7, theta_step=0.125)
    plain = oracle.ipt_solve(M, th, tol=1e-8, max_iter=300, stop="residual")
    assert plain["status"] == oracle.MAXITER
    rule = lambda X: np.clip(1.0 / np.where(np.abs(1.0 - X[:, 3]) > 1e-12, 1.0 - X[:, 3],
                                            1e-12), 0.05, 2.0)
    r = dm.damped_solve(M, th, tol=1e-8, max_iter=400, alpha_fn=rule)
    assert r["status"] == oracle.OK
    np.testing.assert_allclose(np.sort(r["lam"]), np.linalg.eigvalsh(M), atol=1e-8)


# ---------------------------------------------------------------- Anderson mixing
def test_anderson_step_lands_on_fixed_point_of_scalar_multiplier_maps():
    """For g(z) = z* + a_c (z - z*) (one multiplier per column, contracting or not),
    a Picard step followed by one depth-one Anderson step gives z* exactly: both
    residuals are parallel to the first error, and the least-squares weight
    a/(a-1) cancels it.  A dropped term, a wrong sign or the two residuals swapped
    breaks this."""
    from oracle import anderson as an
    g = np.random.default_rng(7)
    n, a = 9, np.array([0.5, -0.8, 1.7, -2.5, 0.95, 3.0])
    zs = g.standard_normal((n, a.size))
    mapping = lambda z: zs + a[None, :] * (z - zs)
    z0 = g.standard_normal((n, a.size))
    g0 = mapping(z0)
    z1 = g0
    g1 = mapping(z1)
    gamma = an.anderson_gamma(g1 - z1, g0 - z0)
    np.testing.assert_allclose(gamma, a / (a - 1.0), rtol=1e-12)
    z2 = an.anderson_update(g1, g0, gamma)
    np.testing.assert_allclose(z2, zs, rtol=1e-10, atol=1e-12)
    # a vanishing residual difference gives a Picard step
    assert np.all(an.anderson_gamma(g1 - z1, g1 - z1) == 0.0)


def test_anderson_solve_first_step_is_picard_and_keeps_unit_entries():
    from oracle import anderson as an
    M, th = w.dense_symmetric(80, 0.05, 3, theta_step=0.25)
    cols = np.array([3, 17, 40, 79])
    for m in [1, 2]:
        a = an.ipt_solve_anderson(M, th, cols=cols, tol=0.0, max_iter=m, stop="increment")
        p = oracle.ipt_solve(M, th, cols=cols, tol=0.0, max_iter=m, stop="increment")
        np.testing.assert_array_equal(a["Z"], p["Z"])
    a = an.ipt_solve_anderson(M, th, cols=cols, tol=0.0, max_iter=7, stop="increment",
                              history=True)
    assert np.all(a["Z"][cols, np.arange(cols.size)] == 1.0)
    assert len(a["gamma"]) == 6 and np.all(a["gamma"][0] == 0.0)


def test_anderson_solve_converges_outside_picard_domain_to_eigh():
    """n = 128, theta_i = i/4, Delta N(0,1)*0.08: the Picard iteration does not reach
    rho <= 1e-10 in 300 evaluations; Anderson mixing does, and its eigenvalues are
    LAPACK's."""
    from oracle import anderson as an
    M, th = w.dense_symmetric(128, 0.08, 3, theta_step=0.25)
    p = oracle.ipt_solve(M, th, tol=1e-10, max_iter=300, stop="residual")
    assert p["status"] != oracle.OK
    a = an.ipt_solve_anderson(M, th, tol=1e-10, max_iter=300)
    assert a["status"] == oracle.OK
    np.testing.assert_allclose(np.sort(a["lam"]), np.linalg.eigvalsh(M), atol=1e-9)


def test_acx_csr_front_end_equals_dense_acx():
    """The sparse IPT-ACX entry (CSR product) takes the same steps as the dense
    one on the same matrix: the tridiagonal Morgan matrix of Section 6.1 at
    eps = 1, outside the Picard domain, and a banded random matrix."""
    import scipy.sparse as sp
    for M, th, cols in [(*w.morgan_tridiagonal(120, 1.0), [0, 1, 5]),
                        (*w.dense_symmetric(150, 0.05, seed=3, theta_step=0.25), [2, 40, 99])]:
        S = sp.csr_matrix(M)
        for sigma in ["column", "global"]:
            a = oracle.ipt_solve_acx(M, th, cols=cols, tol=1e-13, max_iter=300, sigma=sigma)
            b = oracle.ipt_solve_acx_csr(S.indptr, S.indices, S.data, M.shape[0], theta=th,
                                         cols=cols, tol=1e-13, max_iter=300, sigma=sigma)
            assert a["status"] == b["status"] == oracle.OK
            assert a["iterations"] == b["iterations"]
            np.testing.assert_allclose(b["lam"], a["lam"], rtol=1e-13)
            np.testing.assert_allclose(b["Z"], a["Z"], atol=1e-12)


# ------------------------------------------------------------------ learned damping + mixing
def test_mixing_model_gradient_matches_finite_differences():
    """The two-output backward pass against central differences of its own forward
    pass in float64 (FP16 parameters perturbed in float64), both outputs."""
    from oracle import mixing as mx
    g = np.random.default_rng(15)
    p16 = mx.init_params(4)
    X = g.standard_normal((40, 7))
    t = np.stack([g.uniform(0.1, 1.9, 40), g.uniform(-1.5, 1.5, 40)], axis=1)
    _, grad = mx.loss_and_grad(p16, X, t)
    base = p16.astype(np.float64)

    def loss_at(flat64):
        pp = mx.unpack(flat64)
        h1 = np.tanh(X @ pp["W1"] + pp["b1"])
        h2 = np.tanh(h1 @ pp["W2"] + pp["b2"])
        y = h2 @ pp["W3"] + pp["b3"]
        a = 2.0 / (1.0 + np.exp(-y[:, 0]))
        gm = 2.0 * np.tanh(y[:, 1])
        return np.mean((a - t[:, 0]) ** 2 + (gm - t[:, 1]) ** 2)

    idx = np.concatenate([g.choice(mx.N_PARAMS, 60, replace=False),
                          np.arange(mx.N_PARAMS - 130, mx.N_PARAMS)])  # all of W3, b3
    for i in idx:
        e = np.zeros(mx.N_PARAMS)
        e[i] = 1e-6
        fd = (loss_at(base + e) - loss_at(base - e)) / 2e-6
        assert abs(fd - grad[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, grad[i])


def test_mixed_update_special_cases_and_exact_targets():
    """gamma = 0 is the damped step and alpha = 1 Anderson mixing; on maps with one
    multiplier a per column (f(z) = (a - 1)(z - z*)) the targets land exactly:
    after a Picard step z_t = F(z_{t-1}) the Anderson candidate's point is z*
    (gamma* = gamma_ls = a / (a - 1))."""
    from oracle import anderson as an
    from oracle import mixing as mx
    g = np.random.default_rng(16)
    n, k = 9, 4
    zp, zs = (g.standard_normal((n, k)) for _ in range(2))
    a = np.array([0.5, -0.8, 2.5, -3.0])
    fz = lambda x: (a[None, :] - 1.0) * (x - zs)
    z = zp + fz(zp)  # z_t = F(z_{t-1}): a Picard step
    f, fp = fz(z), fz(zp)
    al, gm = g.uniform(0.3, 1.7, k), g.uniform(-1, 1, k)
    np.testing.assert_allclose(mx.mixed_update(z, f, zp, fp, al, np.zeros(k)),
                               z + al[None, :] * f, atol=1e-13)
    np.testing.assert_allclose(mx.mixed_update(z, f, zp, fp, np.ones(k), gm),
                               an.anderson_update(z + f, zp + fp, gm), atol=1e-12)
    alpha, gamma = mx.targets(z, f, zp, fp, fz)
    g_ls = np.clip(a / (a - 1.0), -mx.GAMMA_CLIP, mx.GAMMA_CLIP)
    np.testing.assert_allclose(gamma, np.where(np.abs(a / (a - 1.0)) <= mx.GAMMA_CLIP,
                                               g_ls, 0.0), atol=1e-9)
    # r = f - gamma* df vanishes there, so any alpha* lands on z*
    np.testing.assert_allclose(mx.mixed_update(z, f, zp, fp, alpha, gamma), zs, atol=1e-9)
    # the Picard candidate alone (z_{t-1} unrelated): its secant alpha* = 1 / (1 - a)
    # makes the damped step exact
    zq = g.standard_normal((n, k))
    fq = fz(zq)
    r, Jr = fq, fz(zq + fq) - fq
    np.testing.assert_allclose(mx.secant_alpha(r, Jr, lo=-1e9, hi=1e9), 1.0 / (1.0 - a),
                               rtol=1e-12)


def test_mixed_solve_reduces_to_picard_damping_and_anderson():
    """model = (1, 0) is Alg. 2's Picard iteration; model = (alpha, 0) the damped
    solve; model = (1, gamma_ls) depth-one Anderson after the first steps."""
    from oracle import damping as dm
    from oracle import mixing as mx
    M, th = w.dense_symmetric(90, 0.01, seed=8, theta_step=0.5)
    a = mx.mixed_solve(M, th, tol=1e-12, max_iter=60,
                       model_fn=lambda X: (np.ones(len(X)), np.zeros(len(X))))
    b = oracle.ipt_solve(M, th, tol=1e-12, max_iter=60, stop="residual")
    assert a["status"] == b["status"] == oracle.OK and a["iterations"] == b["iterations"]
    np.testing.assert_array_equal(a["Z"], b["Z"])
    rule = lambda X: np.clip(1.0 / np.where(np.abs(1.0 - X[:, 3]) > 1e-12, 1.0 - X[:, 3],
                                            1e-12), 0.05, 2.0)
    M, th = w.dense_symmetric(128, 0.03, seed=7, theta_step=0.125)
    c = mx.mixed_solve(M, th, tol=1e-9, max_iter=200, model_fn=lambda X: (rule(X[:, :6]),
                                                                          np.zeros(len(X))))
    d = dm.damped_solve(M, th, tol=1e-9, max_iter=200, alpha_fn=rule)
    assert c["status"] == d["status"] and c["iterations"] == d["iterations"]
    np.testing.assert_allclose(c["Z"], d["Z"], atol=1e-12)
    e = mx.mixed_solve(M, th, tol=1e-9, max_iter=200,
                       model_fn=lambda X: (np.ones(len(X)), X[:, 6]))
    assert e["status"] == oracle.OK
    np.testing.assert_allclose(np.sort(e["lam"]), np.linalg.eigvalsh(M), atol=1e-9)
