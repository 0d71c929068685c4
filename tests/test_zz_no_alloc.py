"""The allocation-free residual entry point (ipt_residual_dense_noalloc).

It serves callers that may not allocate device memory (processes whose device
memory belongs to another allocator, synchronisation-free loops).  Its result
must equal the FP64 residual that the solver's own verification reports,
||M Z - Z Lambda||_F = rho_fp64 * r0, on two calls in a row (the second call
reuses the static scratch the first one left behind), and the oracle's
residual of the same (M, Z, Lambda).  This file is collected last.
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2012_14702_gb300 import workloads as w

pytestmark = pytest.mark.gpu


def _solved(ipt, n, eps, seed, m_dtype):
    M, th = w.dense_symmetric(n, eps, seed=seed, theta_step=0.125)
    Mg = torch.as_tensor(M, dtype=m_dtype, device="cuda")
    lam, Z, info = ipt.Solver().solve_dense(Mg, theta=torch.as_tensor(th, device="cuda"),
                                            tol=1e-6, max_iter=40, verify_fp64=True)
    assert info["status"] == "OK"
    return Mg, lam, Z, info["rho_fp64"] * info["r0"]


def test_noalloc_residual_matches_solver_verification_twice(ipt):
    cases = [_solved(ipt, 300, 1e-3, 5, torch.float32), _solved(ipt, 1000, 2e-3, 6, torch.float64)]
    for _ in range(2):  # two calls in a row on each problem
        for Mg, lam, Z, ref in cases:
            st, out = ipt.residual_dense_noalloc(Mg, Z, lam)
            assert st == 0
            got = out.item()
            assert ref > 0 and abs(got - ref) <= 1e-9 * ref, (got, ref)


def _fp64_bound(M, Z, lam):
    """Bound on |fl(||M Z - Z Lambda||_F) - ||M Z - Z Lambda||_F| for one FP64 evaluation:
    each entry is a length-n dot product and one subtraction, so it errs by at most
    gamma_{n+1} (|M| |Z| + |Z| |Lambda|) (gamma_m = m u / (1 - m u), u = 2^-53)."""
    n = M.shape[0]
    u = 2.0 ** -53
    g = (n + 1) * u / (1 - (n + 1) * u)
    return g * np.linalg.norm(np.abs(M) @ np.abs(Z) + np.abs(Z) * np.abs(lam)[None, :])


@pytest.mark.parametrize("n,k", [(130, 130), (300, 77), (1000, 1000)])
def test_noalloc_exact_on_integer_inputs(ipt, n, k):
    """Integer M (non-symmetric), Z and Lambda: every product, sum and square is exact in
    FP64, so the C call must return exactly the oracle's ||M Z - Z Lambda||_F (any swap of
    row and column indexing of M or Z, or a dropped term, changes it)."""
    g = w.rng(90 + n)
    M = g.integers(-8, 9, size=(n, n)).astype(np.float64)
    Z = g.integers(-4, 5, size=(n, k)).astype(np.float64)
    lam = g.integers(-16, 17, size=k).astype(np.float64)
    ref = np.linalg.norm(oracle.residual(M, Z, lam))
    Mg = torch.as_tensor(M, dtype=torch.float32, device="cuda")
    Zg = torch.as_tensor(Z.T.copy(), dtype=torch.float32, device="cuda").t()
    lg = torch.as_tensor(lam, device="cuda")
    for _ in range(2):
        st, out = ipt.residual_dense_noalloc(Mg, Zg, lg)
        assert st == 0 and out.item() == ref, (out.item(), ref)
    ref_t = np.linalg.norm(oracle.residual(M.T, Z, lam))
    st, out = ipt.residual_dense_noalloc(Mg.t().contiguous(), Zg, lg)
    assert st == 0 and out.item() == ref_t != ref


@pytest.mark.parametrize("n", [130, 300, 1000])
def test_noalloc_residual_matches_oracle_residual(ipt, n):
    """Against the oracle's M Z - Z Lambda (float64 numpy) on the GPU's own solved
    (Z, Lambda) of the paper's non-symmetric dense family diag(i) + 0.01 U[0,1]
    (Section 6.2), within the sum of both FP64 evaluations' rounding bounds."""
    M, th = w.dense_paper(n, 0.01, seed=40 + n)
    Mg = torch.as_tensor(M, dtype=torch.float32, device="cuda")
    lam, Z, info = ipt.Solver().solve_dense(Mg, theta=torch.as_tensor(th, device="cuda"),
                                            tol=1e-6, max_iter=40)
    assert info["status"] == "OK"
    M32, Zh, lh = Mg.double().cpu().numpy(), Z.double().cpu().numpy(), lam.cpu().numpy()
    ref = np.linalg.norm(oracle.residual(M32, Zh, lh))
    bound = 2 * _fp64_bound(M32, Zh, lh)
    assert bound < 0.05 * ref
    for _ in range(2):
        st, out = ipt.residual_dense_noalloc(Mg, Z, lam)
        assert st == 0
        assert abs(out.item() - ref) <= bound, (out.item(), ref, bound)


def test_noalloc_binding_rejects_layouts_it_would_misread(ipt):
    n = 64
    M = torch.eye(n, dtype=torch.float32, device="cuda")
    Z = torch.eye(n, dtype=torch.float32, device="cuda").t()
    lam = torch.ones(n, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        ipt.residual_dense_noalloc(M.t(), Z, lam)  # column-major M
    with pytest.raises(ValueError):
        ipt.residual_dense_noalloc(M, Z, lam.float())  # FP32 eigenvalues
    with pytest.raises(ValueError):
        ipt.residual_dense_noalloc(M, Z.t().contiguous().t().contiguous(), lam)  # row-major Z
    with pytest.raises(ValueError):
        ipt.residual_dense_noalloc(M, Z, lam, out=torch.empty(1, device="cuda"))  # FP32 out
    st, out = ipt.residual_dense_noalloc(M, Z, lam)
    assert st == 0 and out.item() == 0.0


def test_noalloc_rejects_sizes_beyond_its_scratch(ipt):
    n = 8256  # ceil(8256/64)^2 = 129^2 > 16384 partial sums
    M = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    Z = torch.zeros((n, n), dtype=torch.float32, device="cuda").t()
    lam = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, _ = ipt.residual_dense_noalloc(M, Z, lam)
    assert st == 7  # IPT_UNSUPPORTED, nothing launched
