"""The next operand written by the product's epilogue (ipt_options.epilogue_operand).

In a staged solve each tensor-core product's epilogue holds F and writes the
next evaluation's operand (the 16-bit split of F - Z_b at one power-of-two
scale for all columns) and adds d_c = Delta_{cols[c], .} F_.c; the next
pre-pass only hands them over.  Checks:
  - the solve with it agrees with the solve whose pre-pass writes every
    operand (per-column scales): same status and evaluation count, FP64
    residual within tol for both, eigenvalues within 1e-8 relative and
    eigenvectors within 1e-5 (both converge to rho <= 1e-6; the eigenvalue
    error is second order in the residual);
  - it is used (epilogue_operands > 0) where a product follows a product;
  - d handed over from the epilogue: at a fixed evaluation count the returned
    Lambda - theta_cols equals (Delta Z)_{cols[c], c} of the returned Z, computed
    in FP64 on the host, to 2e-6 of sum_j |Delta_{cols[c], j} Z_jc| (FP32
    products, FP32 sums over 32 rows, FP64 sums of those), also for a
    non-symmetric Delta (row, not column, of Delta).
"""

import numpy as np
import pytest
import torch

from paper_2012_14702_gb300 import workloads as w

pytestmark = pytest.mark.gpu


def cuda(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


@pytest.mark.parametrize("n,k,bf16", [(1000, 1000, False), (1000, 300, False),
                                      (2500, 2500, False), (1000, 1000, True)])
def test_epilogue_operand_matches_prepass_operand(ipt, n, k, bf16):
    M, th = w.dense_symmetric(n, 3e-3, seed=n + k, theta_step=0.125)
    g = w.rng(11)
    cols = np.arange(n, dtype=np.int32) if k == n else np.sort(g.permutation(n)[:k]).astype(
        np.int32)
    Mg, tg, cg = cuda(M, torch.float32), cuda(th), cuda(cols, torch.int32)
    s = ipt.Solver()
    out = {}
    for epi in (True, False):
        lam, Z, info = s.solve_dense(Mg, theta=tg, cols=None if k == n else cg, tol=1e-6,
                                     max_iter=60, staged_bf16=bf16, verify_fp64=True,
                                     epilogue_operand=epi)
        assert info["status"] == "OK", (epi, info["status"])
        assert info["rho_fp64"] <= 1e-6, (epi, info["rho_fp64"])
        out[epi] = (lam.cpu().numpy(), Z.float().cpu().numpy(), info)
    (l1, z1, i1), (l2, z2, i2) = out[True], out[False]
    assert i1["iterations"] == i2["iterations"]
    assert i1["epilogue_operands"] >= 1 and i2["epilogue_operands"] == 0
    assert i1["epilogue_operands"] <= i1["iterations"] - 2  # not the first two evaluations
    assert np.max(np.abs(l1 - l2) / np.abs(l2)) <= 1e-8
    assert np.max(np.abs(z1 - z2)) <= 1e-5


@pytest.mark.parametrize("symmetric", [True, False])
@pytest.mark.parametrize("m", [3, 4, 5, 6])
def test_epilogue_d_matches_returned_iterate(ipt, symmetric, m):
    n, k = 777, 777
    M, th = w.dense_symmetric(n, 4e-3, seed=21, theta_step=0.125, symmetric=symmetric)
    Mg, tg = cuda(M, torch.float32), cuda(th)
    lam, Z, info = ipt.Solver().solve_dense(Mg, theta=tg, tol=0.0, max_iter=m)
    assert info["status"] == "MAXITER" and info["iterations"] == m
    assert info["epilogue_operands"] >= m - 2
    Zh = Z.double().cpu().numpy()
    # Delta as the solver forms it: M in FP32, theta in FP64, difference in FP64
    D = M.astype(np.float32).astype(np.float64) - np.diag(th)
    terms = D * Zh.T  # row c: Delta_{c, j} Z_{j, c}  (cols = identity)
    d_ref = terms.sum(axis=1)
    bound = 2e-6 * np.abs(terms).sum(axis=1) + 1e-12
    err = np.abs(lam.cpu().numpy() - th - d_ref)
    assert np.all(err <= bound), float(np.max(err / bound))
