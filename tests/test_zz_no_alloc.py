"""The allocation-free residual entry point (ipt_residual_dense_noalloc).

It serves callers that may not allocate device memory (stream capture,
foreign allocators, synchronisation-free loops).  Its result must equal the
FP64 residual that the solver's own verification reports, ||M Z - Z Lambda||_F
= rho_fp64 * r0, on two calls in a row (the second call reuses the static
scratch the first one left behind).  This file is collected last.
"""

import numpy as np
import pytest
import torch

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


def test_noalloc_rejects_sizes_beyond_its_scratch(ipt):
    n = 8256  # ceil(8256/64)^2 = 129^2 > 16384 partial sums
    M = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    Z = torch.zeros((n, n), dtype=torch.float32, device="cuda").t()
    lam = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, _ = ipt.residual_dense_noalloc(M, Z, lam)
    assert st == 7  # IPT_UNSUPPORTED, nothing launched
