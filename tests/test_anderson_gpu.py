"""GPU parity of depth-one Anderson mixing (accel="anderson") against the oracle.

FP64: the iterates, eigenvalues and per-evaluation increments of a fixed number
of evaluations equal the oracle's ipt_solve_anderson (1e-11 of the largest entry
of Z - E; the weights come from FP64 sums in a different order).  FP32 and
tensor-core precisions: converged results outside the Picard domain against
the oracle's converged result (eigenvalues 1e-6 relative, eigenvectors 1e-4 of
||Z - E||).
"""

import numpy as np
import pytest
import torch

import oracle
from oracle import anderson as an
from paper_2012_14702_gb300 import workloads as w

pytestmark = pytest.mark.gpu


def cuda(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


@pytest.mark.parametrize("n,k", [(200, 200), (300, 29)])
def test_anderson_f64_iterates_match_oracle(ipt, n, k):
    M, th = w.dense_symmetric(n, 0.07, seed=5, theta_step=0.25)
    cols = (np.arange(n) if k == n else w.rng(6).permutation(n)[:k]).astype(np.int32)
    Mg, tg, cg = cuda(M), cuda(th), cuda(cols, torch.int32)
    E = oracle.unit_columns(n, cols)
    for m in [1, 2, 3, 4, 6, 9]:
        ref = an.ipt_solve_anderson(M, th, cols=cols, tol=0.0, max_iter=m, stop="increment",
                                    history=True)
        lam, Z, info = ipt.Solver().solve_dense(Mg, theta=tg, cols=cg, tol=0.0, max_iter=m,
                                                precision="f64", stop="increment",
                                                accel="anderson", z_dtype=torch.float64)
        assert info["status"] == "MAXITER" and info["iterations"] == m, (m, info)
        Zg = Z.cpu().numpy()
        scale = max(np.max(np.abs(ref["Z"] - E)), 1e-3)
        assert np.max(np.abs(Zg - ref["Z"])) <= 1e-11 * scale, m
        np.testing.assert_allclose(lam.cpu().numpy(), ref["lam"], rtol=1e-12)
        np.testing.assert_allclose(info["hist_increment"], ref["inc_hist"], rtol=1e-9)
        assert np.all(Zg[cols, np.arange(k)] == 1.0)


@pytest.mark.parametrize("precision", ["f32", "fp16x3", "staged", "f64"])
def test_anderson_converges_outside_picard_domain(ipt, precision):
    """n = 512, theta_i = i/8, Delta N(0,1)*0.03: the Picard iteration does not
    converge in 150 evaluations; Anderson mixing reaches rho <= 1e-6 and matches the
    oracle's converged result."""
    n = 512
    M, th = w.dense_symmetric(n, 0.03, seed=7, theta_step=0.125)
    Mg = cuda(M, torch.float32 if precision != "f64" else torch.float64)
    tg = cuda(th)
    s = ipt.Solver()
    _, _, plain = s.solve_dense(Mg, theta=tg, tol=1e-6, max_iter=150, precision="f32")
    assert plain["status"] != "OK"
    lam, Z, info = s.solve_dense(Mg, theta=tg, tol=1e-6, max_iter=300, precision=precision,
                                 accel="anderson", verify_fp64=True)
    # OK only where the error model certifies the residual (see test_acx_gpu)
    assert info["status"] == "OK" or (info["status"] == "INACCURATE" and
                                       precision not in ("staged", "f64")), info
    assert info["rho_fp64"] <= info["rho"] + info["rho_error"], info
    if info["status"] != "OK":
        return
    assert info["rho_fp64"] <= 1e-6, info["rho_fp64"]
    ref = an.ipt_solve_anderson(M, th, tol=1e-12, max_iter=400)
    assert ref["status"] == oracle.OK
    np.testing.assert_allclose(lam.cpu().numpy(), ref["lam"], rtol=1e-6)
    E = np.eye(n)
    err = np.linalg.norm(Z.double().cpu().numpy() - ref["Z"]) / np.linalg.norm(ref["Z"] - E)
    assert err <= 1e-4, err


def test_anderson_stop_at_first_evaluation_and_host_entry(ipt):
    """A problem whose increment test passes at Z = E (rho(E) = 1 by definition, so
    the increment rule) returns the unit columns; the host-buffer entry point gives
    the device entry point's result."""
    M, th = w.dense_symmetric(96, 1e-9, seed=2, theta_step=1.0)
    s = ipt.Solver()
    lam, Z, info = s.solve_dense(cuda(M, torch.float32), theta=cuda(th), tol=1e-6,
                                 max_iter=20, accel="anderson", stop="increment")
    assert info["status"] == "OK" and info["iterations"] == 1
    assert torch.equal(Z.cpu(), torch.eye(96, dtype=torch.float32))
    M2, th2 = w.dense_symmetric(256, 0.05, seed=4, theta_step=0.25)
    lam_d, Z_d, i_d = s.solve_dense(cuda(M2, torch.float32), theta=cuda(th2), tol=1e-6,
                                    max_iter=200, accel="anderson")
    assert i_d["status"] == "OK"
    Mh = torch.as_tensor(M2, dtype=torch.float32)
    lam_h, Z_h, i_h = s.solve_dense_host(Mh, theta=torch.as_tensor(th2), tol=1e-6,
                                         max_iter=200, accel="anderson")
    assert i_h["status"] == "OK" and i_h["iterations"] == i_d["iterations"]
    np.testing.assert_array_equal(lam_h.numpy(), lam_d.cpu().numpy())
    np.testing.assert_array_equal(Z_h.numpy(), Z_d.cpu().numpy())
